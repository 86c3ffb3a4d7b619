"""The layered-schedule kernel (SAGMS_FLAG_LAYERED) against the FP64 oracle's layered
schedule, element by element on the same seeded shots, with the acceptance of
tests/gpu_helpers.py (MS exact; SMS / SAGMS exact except for reported near-ties or
ill-conditioned shots; posterior traces within the normwise tolerance).  Codes cover both
block sizes (32 threads when no layer has more than 64 checks, else 128), irregular codes
with degree-0 and degree-1 checks, a random LDPC code and the full-size GB(1023, 5)."""
import numpy as np
import pytest
import torch

import paper_2605_10433_gb300 as S
from paper_2605_10433_gb300 import _native
from paper_2605_10433_gb300 import inputs as I
from tests import gpu_helpers as G
from tests.test_column_slots import _random_code

pytestmark = pytest.mark.gpu

LAY = S.FLAG_LAYERED
PARAMS = {
    "ms": S.Params(mode="ms", max_iter=60, flags=LAY),
    "sms": S.Params(mode="sms", alpha=0.75, max_iter=60, flags=LAY),
    "sagms": S.Params(mode="sagms", alpha_min=0.30, alpha_max=0.50, eta_unsat=1.10, max_iter=60, flags=LAY),
}


def _with(p, **kw):
    return S.Params(**{**p.__dict__, **kw})


@pytest.fixture(scope="module", autouse=True)
def dev_check():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _irregular(l, w):
    """GB(l, w) with rows emptied, cut to one edge or shortened (check degrees 2w .. 0)."""
    g = I.gb_code(l, w)
    rows = []
    for i in range(g.m):
        r = list(g.col_idx[g.row_ptr[i]:g.row_ptr[i + 1]])
        rows.append([] if i % 13 == 5 else r[:1] if i % 11 == 3 else r[:-1] if i % 7 == 0 else r)
    rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    return I.Code(m=g.m, n=g.n, row_ptr=rp, col_idx=np.array([c for r in rows for c in r], dtype=np.int32))


def _random(m, n, dv, dc, seed):
    rp, ci = _random_code(m, n, dv, dc, seed)
    return I.Code(m=m, n=n, row_ptr=rp, col_idx=ci)


CODES = {
    "gb63x3": lambda: I.gb_code(63, 3),
    "gb255x5": lambda: I.gb_code(255, 5),
    "gb255x8": lambda: I.gb_code(255, 8),
    "gb1023x3": lambda: I.gb_code(1023, 3),
    "irregular-gb255x5": lambda: _irregular(255, 5),
    "random-512x1024-(4,8)": lambda: _random(512, 1024, 4, 8, 31),
}


@pytest.mark.parametrize("mode", ["ms", "sms", "sagms"])
@pytest.mark.parametrize("key", list(CODES))
def test_layered_oracle_parity(key, mode):
    c = CODES[key]()
    dc = S.DeviceCode.from_code(c)
    _, syn, L0, _ = I.workload(c, [0.01, 0.03, 0.06], 401, seed=17)
    syn = syn.copy()
    L0 = L0.copy()
    syn[::9] = 0
    L0[4::13] = -L0[4::13]
    G.compare(c, dc, syn, L0, PARAMS[mode], min_frac=0.0)


def test_layered_full_size_gb1023_oracle_parity():
    c = I.gb_code(1023, 5)
    dc = S.DeviceCode.from_code(c)
    _, syn, L0, _ = I.workload(c, [0.005, 0.01, 0.02], 300, seed=18)
    G.compare(c, dc, syn, L0, PARAMS["sagms"], min_frac=0.0)


@pytest.mark.parametrize("key", ["gb63x3", "gb1023x3", "irregular-gb255x5"])
def test_layered_traces(key):
    c = CODES[key]()
    dc = S.DeviceCode.from_code(c)
    _, syn, L0, _ = I.workload(c, [0.02, 0.05], 24, seed=19)
    worst, _, _ = G.compare_traces(c, dc, syn, L0, _with(PARAMS["sagms"], max_iter=12, flags=LAY | S.FLAG_NO_EARLY_STOP))
    assert worst <= G.MSG_RTOL


def test_layered_per_qubit_priors_and_auto_ceiling():
    c = I.gb_code(255, 5)
    dc = S.DeviceCode.from_code(c)
    rng = np.random.default_rng(20)
    _, syn = I.sample(c, 0.03, 400, seed=21)
    L0q = I.llr_prior(rng.uniform(0.005, 0.08, size=c.n)).astype(np.float32)
    L0q[rng.choice(c.n, size=c.n // 50, replace=False)] *= -1.0
    G.compare(c, dc, syn, L0q, _with(PARAMS["sagms"], flags=LAY | S.FLAG_L0_PER_QUBIT), min_frac=0.0)
    _, syn, L0, _ = I.workload(c, [0.01, 0.04], 400, seed=22)
    G.compare(c, dc, syn, L0, _with(PARAMS["sagms"], flags=LAY | S.FLAG_AUTO_CEILING), min_frac=0.0)
    bad = L0q.copy()
    bad[7] = np.inf
    g = G.gpu_decode(dc, syn[:50], bad, _with(PARAMS["sagms"], flags=LAY | S.FLAG_L0_PER_QUBIT))
    assert (g["iters"] == -1).all() and (g["conv"] == 0).all() and not g["err"].any()


def test_layered_conv_matches_residual_at_full_size():
    """At the benchmark's size, on many shots: conv agrees with s XOR H e_hat = 0, every
    shot's iteration count is within budget, and layered decoding converges in fewer rounds
    than flooding on average (a later layer already uses the messages of an earlier one)."""
    c = I.gb_code(1023, 5)
    dc = S.DeviceCode.from_code(c)
    _, syn, L0, _ = I.workload(c, [0.005, 0.01, 0.02], 60000, seed=23)
    p = _with(PARAMS["sagms"], max_iter=100)
    g = G.gpu_decode(dc, syn, L0, p)
    ok = G.residual_ok(c, syn, g["err"])
    assert np.array_equal(ok, g["conv"].astype(bool))
    assert ((g["iters"] >= 0) & (g["iters"] <= 100)).all()
    f = G.gpu_decode(dc, syn, L0, _with(p, flags=0))
    assert g["iters"].mean() < f["iters"].mean()


def test_layered_rejects_bp_and_wide_checks():
    c = I.gb_code(63, 3)
    dc = S.DeviceCode.from_code(c)
    _, syn, L0, _ = I.workload(c, [0.05], 8, seed=1)
    with pytest.raises(_native.SagmsError):
        G.gpu_decode(dc, syn, L0, S.Params(mode="bp", max_iter=10, flags=LAY))
    rows = [list(range(k, k + 26)) for k in range(0, 40, 2)]          # check degree 26 > 24
    H = np.zeros((len(rows), 70), dtype=np.uint8)
    for i, r in enumerate(rows):
        H[i, r] = 1
    w = I.code_from_dense(H)
    dw = S.DeviceCode.from_code(w)
    _, syn, L0, _ = I.workload(w, [0.05], 8, seed=2)
    with pytest.raises(_native.SagmsError):
        G.gpu_decode(dw, syn, L0, PARAMS["ms"])
