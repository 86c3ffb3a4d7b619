"""The automatic gain ceiling of Corollary 1 (alpha_max = alpha*(|L0|, d_c) of Eq. 9 per shot,
clamped to [alpha_min, 1/eta]): pins of the oracle's per-shot plumbing (CPU) and the GPU
kernels against the oracle and against each other."""
import math

import numpy as np
import pytest

import oracle
from paper_2605_10433_gb300 import inputs as I

SAGMS_KW = dict(alpha_min=0.30, eta_unsat=1.10, max_iter=60)


def _ceiling(L0, dc, amin=0.30, eta=1.10):
    a = oracle.alpha_star(abs(L0), dc) if L0 != 0 else 0.0
    return min(max(a, amin), 1.0 / eta)


def _decode(code, syn, L0, flags=0, alpha_max=0.5):
    return oracle.decode_code(code, syn, np.asarray(L0, dtype=np.float64), mode=oracle.SAGMS,
                              alpha_max=alpha_max, flags=flags, **SAGMS_KW)


def _same(a, b):
    return all(np.array_equal(a[k], b[k]) for k in ("err", "conv", "iters"))


def test_ceiling_values_at_the_headline_priors():
    """Eq. 9 at d_c = 10 for p = 0.005 / 0.01 / 0.02 lies inside [alpha_min, 1/eta]: the
    ceiling is alpha* itself there (0.5850 / 0.5224 / 0.4383)."""
    for p, want in ((0.005, 0.5850), (0.01, 0.5224), (0.02, 0.4383)):
        L0 = math.log((1 - p) / p)
        assert abs(_ceiling(L0, 10) - want) < 5e-4
        assert _ceiling(L0, 10) == oracle.alpha_star(L0, 10)


@pytest.mark.parametrize("p", [0.01, 0.03])
def test_oracle_auto_equals_explicit_alpha_max_per_shot(p):
    """A batch with one prior: the flag gives exactly the decode with alpha_max set to the
    ceiling; with mixed priors each shot matches its own single-prior decode."""
    c = I.gb_code(127, 4)
    _, syn, L0, _ = I.workload(c, [p], 300, seed=41)
    dc = int(np.diff(c.row_ptr).max())
    auto = _decode(c, syn, L0, flags=oracle.FLAG_AUTO_CEILING)
    expl = _decode(c, syn, L0, alpha_max=_ceiling(float(L0[0]), dc))
    assert _same(auto, expl)
    assert not _same(auto, _decode(c, syn, L0, alpha_max=0.5)) or p == 0.01


def test_oracle_auto_mixed_priors_and_clamps():
    c = I.gb_code(63, 3)
    dc = int(np.diff(c.row_ptr).max())
    _, syn, _, _ = I.workload(c, [0.04], 240, seed=42)
    # per-shot priors: ordinary, very large (ceiling 1/eta), tiny (ceiling alpha_min), zero
    L0 = np.tile(np.array([3.2, 60.0, 0.05, 0.0, -2.5, 7.0]), 40)
    auto = _decode(c, syn, L0, flags=oracle.FLAG_AUTO_CEILING)
    for v in (3.2, 60.0, 0.05, 0.0, -2.5, 7.0):
        sel = np.nonzero(L0 == v)[0]
        one = _decode(c, syn[sel], L0[sel], alpha_max=_ceiling(v, dc))
        assert all(np.array_equal(auto[k][sel], one[k]) for k in ("err", "conv", "iters")), v
    assert _ceiling(60.0, dc) == pytest.approx(1 / 1.10)
    assert _ceiling(0.05, dc) == 0.30 and _ceiling(0.0, dc) == 0.30


# ----------------------------------------------------------------------------- GPU
@pytest.fixture(scope="module")
def S():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_10433_gb300 as S
    return S


@pytest.mark.gpu
@pytest.mark.parametrize("lw", [(255, 5), (1023, 5), (1024, 4)])
def test_gpu_auto_ceiling_parity_and_kernels(S, lw):
    from paper_2605_10433_gb300 import _native
    from tests import gpu_helpers as G
    c = I.gb_code(*lw)
    _, syn, L0, _ = I.workload(c, [0.005, 0.01, 0.02, 0.04], 1200, seed=43)
    L0 = L0.copy()
    L0[::97] = -L0[::97]
    p = S.Params(mode="sagms", alpha_min=0.30, alpha_max=0.5, eta_unsat=1.10, max_iter=80,
                 flags=S.FLAG_AUTO_CEILING)
    G.compare(c, S.DeviceCode.from_code(c), syn, L0, p)
    outs = []
    for kernel in (1, 2, 3, 4):
        dc = S.DeviceCode.from_code(c)
        _native.sagms_set_plan(dc.handle, kernel)
        outs.append(G.gpu_decode(dc, syn, L0, p))
    for o in outs[1:]:
        assert _same(o, outs[0])


@pytest.mark.gpu
def test_gpu_auto_ceiling_rejects_other_modes_and_per_qubit(S):
    from paper_2605_10433_gb300 import _native
    for p in (S.Params(mode="sms", flags=S.FLAG_AUTO_CEILING),
              S.Params(mode="sagms", flags=S.FLAG_AUTO_CEILING | S.FLAG_L0_PER_QUBIT),
              S.Params(mode="sagms", alpha_min=0.95, flags=S.FLAG_AUTO_CEILING)):
        assert _native.sagms_check_params(p.to_c()) == -4
