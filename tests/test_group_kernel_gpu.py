"""The two-group kernels (two independent shot groups per CTA, one shot each; the general layout
and the column-indexed one for codes whose edges line up slot by slot) against the
one-shot-per-CTA kernel and the two-slot kernel, on the codes they cover (more than 512 and
at most 1024 checks, at most 2048 qubits).

All of them run each shot's arithmetic in the same order, so outputs and posterior traces
must agree bit for bit; parity of the one-shot-per-CTA kernel against the FP64 oracle is
covered in test_parity_gpu.py, and oracle comparisons here pin the group kernels directly."""
import numpy as np
import pytest
import torch

import paper_2605_10433_gb300 as S
from paper_2605_10433_gb300 import _native
from paper_2605_10433_gb300 import inputs as I
from tests import gpu_helpers as G

pytestmark = pytest.mark.gpu

KERNEL_GENERIC, KERNEL_SLOTS, KERNEL_GROUPS, KERNEL_QC = 1, 2, 3, 4
PARAMS = {
    "ms": S.Params(mode="ms", max_iter=60),
    "sms": S.Params(mode="sms", alpha=0.75, max_iter=60),
    "sagms": S.Params(mode="sagms", alpha_min=0.30, alpha_max=0.50, eta_unsat=1.10, max_iter=60),
}


def _with(p, **kw):
    return S.Params(**{**p.__dict__, **kw})


@pytest.fixture(scope="module")
def dev_check():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(scope="module")
def group_codes():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out = {}
    # GB(1023, 5): the benchmark code (no padded edges); GB(1024, 4): every check padded
    # from 8 to 10 edges and every qubit from 4 to 5; a random code with ragged degrees.
    for key in [(1023, 5), (1024, 4)]:
        c = I.gb_code(*key)
        out[key] = c
    rng = np.random.default_rng(2024)
    m, n = 700, 1500
    H = np.zeros((m, n), dtype=np.uint8)
    for i in range(m):
        H[i, rng.choice(n, size=int(rng.integers(1, 11)), replace=False)] = 1
    while H.sum(axis=0).max() > 5:
        j = int(np.argmax(H.sum(axis=0)))
        H[np.nonzero(H[:, j])[0][0], j] = 0
    out["ragged"] = I.code_from_dense(H)
    out["gb-truncated"] = _truncated_gb(1023, 5)
    return out


def _truncated_gb(l, w):
    """GB(l, w) with trailing edges dropped from some rows (rows keep polynomial-term order,
    so the column-indexed layout still applies): check degrees 2w, 2w - 1, 1 and 0, qubit
    degrees w and below."""
    g = I.gb_code(l, w)
    rows = []
    for i in range(g.m):
        r = list(g.col_idx[g.row_ptr[i]:g.row_ptr[i + 1]])
        if i % 13 == 5:
            r = []
        elif i % 11 == 3:
            r = r[:1]
        elif i % 7 == 0:
            r = r[:-1]
        rows.append(r)
    row_ptr = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    col_idx = np.concatenate([np.asarray(r, dtype=np.int32) for r in rows])
    return I.Code(m=g.m, n=g.n, row_ptr=row_ptr, col_idx=col_idx, name=f"truncated GB({l},{w})")


def _decode_with_kernel(code, kernel, syn, L0, p, trace=False):
    dc = S.DeviceCode.from_code(code)
    _native.sagms_set_plan(dc.handle, kernel)
    return G.gpu_decode(dc, syn, L0, p, trace=trace)


def _same(a, b):
    return all(np.array_equal(a[k], b[k]) for k in ("err", "conv", "iters"))


@pytest.mark.parametrize("mode", ["ms", "sms", "sagms"])
@pytest.mark.parametrize("key", [(1023, 5), (1024, 4), "ragged", "gb-truncated"])
def test_group_kernel_bitwise_identical_to_other_kernels(group_codes, mode, key):
    c = group_codes[key]
    _, syn, L0, _ = I.workload(c, [0.005, 0.02, 0.05], 3001, seed=71)
    p = PARAMS[mode]
    ref = _decode_with_kernel(c, KERNEL_GENERIC, syn, L0, p)
    for kernel in (KERNEL_SLOTS, KERNEL_GROUPS, KERNEL_QC):
        assert _same(_decode_with_kernel(c, kernel, syn, L0, p), ref), kernel
    tr = _decode_with_kernel(c, KERNEL_GENERIC, syn[:24], L0[:24], p, trace=True)["trace"]
    for kernel in (KERNEL_GROUPS, KERNEL_QC):
        tg = _decode_with_kernel(c, kernel, syn[:24], L0[:24], p, trace=True)["trace"]
        assert np.array_equal(np.nan_to_num(tr, nan=7.0), np.nan_to_num(tg, nan=7.0)), kernel


# Gains at the edges of what the parameter check accepts, and gain 1.
EXTREME_GAINS = {
    "sagms-floor": S.Params(mode="sagms", alpha_min=2.0 ** -20, alpha_max=0.9, eta_unsat=1.1, max_iter=40),
    "sagms-auto-floor": S.Params(mode="sagms", alpha_min=2.0 ** -20, eta_unsat=1.1, max_iter=40,
                                 flags=S.FLAG_AUTO_CEILING),
    "sms-subnormal": S.Params(mode="sms", alpha=float(np.nextafter(np.float32(0), np.float32(1))), max_iter=40),
    "sms-one": S.Params(mode="sms", alpha=1.0, max_iter=40),
}


@pytest.mark.parametrize("name", list(EXTREME_GAINS))
@pytest.mark.parametrize("lw", [(63, 3), (255, 4), (1023, 5)])
def test_check_node_output_at_gain_extremes(dev_check, lw, name):
    """The column-indexed kernel forms each edge's check-node output as an unsigned minimum
    over the other edges' sign-carrying scaled magnitudes, which needs a positive gain.  At
    the smallest gains the parameter check accepts it must still agree bit for bit with the
    one-shot-per-CTA kernel's smallest / second-smallest selection, posterior traces
    included.  The cases:
    - alpha_min = 2^-20, with every check unsatisfied in a third of the shots, which puts
      Eq. 7's gain at its floor;
    - the same with the automatic ceiling;
    - SMS with the smallest subnormal scale, where most scaled values underflow to zero;
    - gain 1."""
    c = I.gb_code(*lw)
    shots = 1500
    _, syn, L0, _ = I.workload(c, [0.01, 0.05], shots, seed=31 * lw[0] + lw[1])
    syn = syn.copy()
    rng = np.random.default_rng(lw[0] + 17 * len(name))
    k = shots // 3
    syn[:k] = rng.integers(0, 2 ** 32, size=(k, syn.shape[1]), dtype=np.uint64).astype(np.uint32)
    syn[-k:] = np.uint32(0xFFFFFFFF)
    if c.m % 32:
        syn[:, -1] &= np.uint32((1 << (c.m % 32)) - 1)
    p = EXTREME_GAINS[name]
    ref = _decode_with_kernel(c, KERNEL_GENERIC, syn, L0, p)
    assert _same(_decode_with_kernel(c, KERNEL_QC, syn, L0, p), ref)
    sel = np.r_[0:4, k:k + 4, shots - 4:shots]
    tr = _decode_with_kernel(c, KERNEL_GENERIC, syn[sel], L0[sel], p, trace=True)["trace"]
    tq = _decode_with_kernel(c, KERNEL_QC, syn[sel], L0[sel], p, trace=True)["trace"]
    assert np.array_equal(np.nan_to_num(tr, nan=7.0), np.nan_to_num(tq, nan=7.0))


@pytest.mark.parametrize("kernel", [KERNEL_GROUPS, KERNEL_QC])
@pytest.mark.parametrize("shots", [1, 2, 3, 5, 300, 305])
def test_group_kernel_small_and_ragged_batches(group_codes, shots, kernel):
    """Fewer shots than groups, one idle group, and batch tails that end mid-chunk."""
    c = group_codes[(1023, 5)]
    _, syn, L0, _ = I.workload(c, [0.03], shots, seed=shots)
    p = PARAMS["sagms"]
    assert _same(_decode_with_kernel(c, kernel, syn, L0, p),
                 _decode_with_kernel(c, KERNEL_GENERIC, syn, L0, p))


@pytest.mark.parametrize("kernel", [KERNEL_GROUPS, KERNEL_QC])
@pytest.mark.parametrize("key", [(1024, 4), "gb-truncated"])
def test_group_kernel_edge_inputs(group_codes, key, kernel):
    """Zero syndromes, negative and zero priors, invalid priors, max_iter = 0 and no early stop."""
    c = group_codes[key]
    _, syn, L0, _ = I.workload(c, [0.02], 400, seed=5)
    syn = syn.copy()
    L0 = L0.copy()
    syn[::7] = 0
    L0[5::11] = -L0[5::11]
    L0[9::13] = 0.0
    L0[[3, 50, 399]] = [np.nan, np.inf, -np.inf]
    for p in (PARAMS["sagms"], _with(PARAMS["sagms"], max_iter=0),
              _with(PARAMS["ms"], max_iter=9, flags=S.FLAG_NO_EARLY_STOP)):
        g = _decode_with_kernel(c, kernel, syn, L0, p)
        assert _same(g, _decode_with_kernel(c, KERNEL_GENERIC, syn, L0, p))
        assert (g["iters"][[3, 50, 399]] == -1).all()


@pytest.mark.parametrize("key,kernel", [("ragged", KERNEL_GROUPS), ("gb-truncated", KERNEL_QC),
                                        ((1023, 5), KERNEL_QC)])
def test_group_kernel_oracle_parity(group_codes, key, kernel):
    """The group kernels directly against the FP64 oracle (same acceptance as the other
    kernels: exact agreement except for shots traced to near-ties or ill-conditioning)."""
    c = group_codes[key]
    dc = S.DeviceCode.from_code(c)
    _native.sagms_set_plan(dc.handle, kernel)
    _, syn, L0, _ = I.workload(c, [0.01, 0.03], 400, seed=88)
    G.compare(c, dc, syn, L0, PARAMS["sagms"])


def test_group_kernel_falls_back_for_per_qubit_priors(group_codes):
    """Per-qubit priors on GB(1023, 5): the column-indexed kernel runs them itself; the
    two-group kernel's plan falls back to the two-slot kernel.  Identical results."""
    c = group_codes[(1023, 5)]
    _, syn = I.sample(c, 0.02, 500, seed=8)
    L0q = I.llr_prior(np.random.default_rng(3).uniform(0.005, 0.05, size=c.n)).astype(np.float32)
    p = _with(PARAMS["sagms"], flags=S.FLAG_L0_PER_QUBIT)
    for kernel in (KERNEL_GROUPS, KERNEL_QC):
        assert _same(_decode_with_kernel(c, kernel, syn, L0q, p),
                     _decode_with_kernel(c, KERNEL_GENERIC, syn, L0q, p))


@pytest.mark.parametrize("lw", [(63, 3), (127, 4), (255, 5), (255, 8), (511, 5), (1023, 5)])
def test_column_indexed_per_qubit_priors(dev_check, lw):
    """Per-qubit priors (LLR units, some negative) on every column-indexed shape: bitwise
    equal to the one-shot-per-CTA kernel, including zero syndromes (decision [L0 < 0]) and
    traces; a non-finite prior invalidates every shot."""
    c = I.gb_code(*lw)
    rng = np.random.default_rng(lw[0])
    _, syn = I.sample(c, 0.03, 1201, seed=lw[0] + 1)
    syn = syn.copy()
    syn[::11] = 0
    L0q = I.llr_prior(rng.uniform(0.005, 0.08, size=c.n)).astype(np.float32)
    L0q[rng.choice(c.n, size=max(1, c.n // 50), replace=False)] *= -1.0
    for mode in ("ms", "sagms"):
        p = _with(PARAMS[mode], flags=S.FLAG_L0_PER_QUBIT)
        assert _same(_decode_with_kernel(c, KERNEL_QC, syn, L0q, p), _decode_with_kernel(c, KERNEL_GENERIC, syn, L0q, p))
    p = _with(PARAMS["sagms"], flags=S.FLAG_L0_PER_QUBIT)
    tr = _decode_with_kernel(c, KERNEL_GENERIC, syn[:12], L0q, p, trace=True)["trace"]
    tq = _decode_with_kernel(c, KERNEL_QC, syn[:12], L0q, p, trace=True)["trace"]
    assert np.array_equal(np.nan_to_num(tr, nan=7.0), np.nan_to_num(tq, nan=7.0))
    bad = L0q.copy()
    bad[c.n // 2] = np.nan
    g = _decode_with_kernel(c, KERNEL_QC, syn[:40], bad, p)
    assert (g["iters"] == -1).all() and (g["conv"] == 0).all() and not g["err"].any()


def test_column_indexed_per_qubit_oracle_parity(dev_check):
    c = I.gb_code(255, 5)
    dc = S.DeviceCode.from_code(c)
    _native.sagms_set_plan(dc.handle, KERNEL_QC)
    _, syn = I.sample(c, 0.02, 500, seed=19)
    L0q = I.llr_prior(np.random.default_rng(19).uniform(0.005, 0.05, size=c.n)).astype(np.float32)
    G.compare(c, dc, syn, L0q, _with(PARAMS["sagms"], flags=S.FLAG_L0_PER_QUBIT))


def test_set_plan_rejects_unknown_bits(group_codes):
    dc = S.DeviceCode.from_code(group_codes[(1023, 5)])
    for bad in (1 << 4, 5, 7):
        with pytest.raises(_native.SagmsError):
            _native.sagms_set_plan(dc.handle, bad)
    _native.sagms_set_plan(dc.handle, KERNEL_QC | (1 << 16))


@pytest.mark.parametrize("lw", [(63, 3), (63, 4), (63, 5), (127, 3), (127, 4), (127, 5), (255, 3), (255, 4),
                                (255, 5), (255, 6), (255, 8), (511, 3), (511, 4), (511, 5), (1023, 3)])
def test_column_indexed_shapes_for_smaller_codes(dev_check, lw):
    """Every compiled column-indexed shape (n from 126 to 1022, warp-sized groups up to four
    256-thread groups) against the one-shot-per-CTA kernel, bit for bit, on mixed noise with
    zero syndromes, negative priors and an odd shot count."""
    c = I.gb_code(*lw)
    _, syn, L0, _ = I.workload(c, [0.005, 0.02, 0.06], 2501, seed=lw[0] + lw[1])
    syn = syn.copy()
    L0 = L0.copy()
    syn[::9] = 0
    L0[4::13] = -L0[4::13]
    for mode in ("ms", "sagms"):
        p = PARAMS[mode]
        assert _same(_decode_with_kernel(c, KERNEL_QC, syn, L0, p), _decode_with_kernel(c, KERNEL_GENERIC, syn, L0, p))
    tr = _decode_with_kernel(c, KERNEL_GENERIC, syn[:16], L0[:16], PARAMS["sagms"], trace=True)["trace"]
    tq = _decode_with_kernel(c, KERNEL_QC, syn[:16], L0[:16], PARAMS["sagms"], trace=True)["trace"]
    assert np.array_equal(np.nan_to_num(tr, nan=7.0), np.nan_to_num(tq, nan=7.0))


def test_small_truncated_code_oracle_parity(dev_check):
    """A truncated GB(255, 5) (check degrees 10, 9, 1, 0) on the n <= 512 shape against the
    FP64 oracle."""
    c = _truncated_gb(255, 5)
    dc = S.DeviceCode.from_code(c)
    _native.sagms_set_plan(dc.handle, KERNEL_QC)
    _, syn, L0, _ = I.workload(c, [0.01, 0.03], 600, seed=89)
    G.compare(c, dc, syn, L0, PARAMS["sagms"])
    assert _same(G.gpu_decode(dc, syn, L0, PARAMS["sagms"]),
                 _decode_with_kernel(c, KERNEL_GENERIC, syn, L0, PARAMS["sagms"]))


def test_bivariate_bicycle_code_on_the_column_indexed_kernel(dev_check):
    """A code of another family with the slot structure: the bivariate-bicycle [[144,12,12]]
    code runs on the column-indexed kernel, bit for bit as on the one-shot-per-CTA kernel."""
    from tests.test_mc import bb_code
    c = bb_code(12, 6, [("x", 3), ("y", 1), ("y", 2)], [("y", 3), ("x", 1), ("x", 2)])
    _, syn, L0, _ = I.workload(c, [0.01, 0.03, 0.05], 3000, seed=144)
    for mode in ("ms", "sagms"):
        assert _same(_decode_with_kernel(c, KERNEL_QC, syn, L0, PARAMS[mode]),
                     _decode_with_kernel(c, KERNEL_GENERIC, syn, L0, PARAMS[mode]))


def test_negative_zero_priors_decide_zero(dev_check):
    """Per-qubit priors of -0.0 (one of them on a qubit no check touches): the decision is
    [P < 0], so such a qubit decodes to 0 on every kernel and in the layered schedule, as in
    the oracle."""
    g = I.gb_code(63, 3)
    c = I.Code(m=g.m, n=g.n + 1, row_ptr=g.row_ptr, col_idx=g.col_idx)   # qubit 126: no check
    rng = np.random.default_rng(5)
    _, syn = I.sample(c, 0.04, 300, seed=6)
    L0q = I.llr_prior(rng.uniform(0.01, 0.06, size=c.n)).astype(np.float32)
    L0q[[3, 40, 126]] = -0.0
    for mode in ("ms", "sagms"):
        p = _with(PARAMS[mode], flags=S.FLAG_L0_PER_QUBIT)
        ref = _decode_with_kernel(c, KERNEL_GENERIC, syn, L0q, p)
        assert not (I.unpack_bits(ref["err"], c.n)[:, 126]).any()
        for kernel in (KERNEL_SLOTS, KERNEL_QC):
            assert _same(_decode_with_kernel(c, kernel, syn, L0q, p), ref), kernel
        dc = S.DeviceCode.from_code(c)
        G.compare(c, dc, syn, L0q, p)
        lay = _with(p, flags=S.FLAG_L0_PER_QUBIT | S.FLAG_LAYERED)
        G.compare(c, dc, syn, L0q, lay)
        assert not (I.unpack_bits(G.gpu_decode(dc, syn, L0q, lay)["err"], c.n)[:, 126]).any()


@pytest.mark.parametrize("lw", [(63, 3), (63, 5), (127, 4), (255, 5), (511, 5), (1023, 5), (1023, 3), (255, 3), (511, 4)])
def test_column_indexed_bp_bitwise_identical_to_one_shot_per_cta(dev_check, lw):
    """BP (Eq. 3, per-shot priors in LLR units) on the column-indexed kernel: the same slot
    order, phi function and prefix / suffix sums as the one-shot-per-CTA kernel, so outputs
    and posterior traces agree bit for bit (zero syndromes and negative priors included).
    For 129 to 512 and 1025 to 2048 qubits BP has shapes of its own (two checks per thread,
    groups of 64, 128 and 512 threads, every slot-degree class): they serve the default plan
    and plan 4; at 1022 qubits it keeps the code's own column-indexed shape under plan 4."""
    c = I.gb_code(*lw)
    _, syn, L0, _ = I.workload(c, [0.005, 0.02, 0.06], 1501, seed=lw[0] + 7)
    syn = syn.copy()
    L0 = L0.copy()
    syn[::9] = 0
    L0[4::13] = -L0[4::13]
    p = S.Params(mode="bp", max_iter=40)
    dc = S.DeviceCode.from_code(c)
    assert "two-group-qc" in dc.kernels
    assert ("two-group-qc-bp" in dc.kernels) == (128 < c.n <= 512 or c.n > 1024)
    ref = _decode_with_kernel(c, KERNEL_GENERIC, syn, L0, p)
    assert _same(_decode_with_kernel(c, KERNEL_QC, syn, L0, p), ref)
    assert _same(G.gpu_decode(dc, syn, L0, p), ref)   # the default plan
    tr = _decode_with_kernel(c, KERNEL_GENERIC, syn[:12], L0[:12], p, trace=True)["trace"]
    tq = _decode_with_kernel(c, KERNEL_QC, syn[:12], L0[:12], p, trace=True)["trace"]
    assert np.array_equal(np.nan_to_num(tr, nan=7.0), np.nan_to_num(tq, nan=7.0))


def test_column_indexed_bp_on_a_recoloured_code_and_oracle_parity(dev_check):
    """A random (5, 10) LDPC code (slots from the edge colouring, padded slots in the middle
    of checks after dropped repeats) and GB(255, 5): BP on the column-indexed kernel equals
    the one-shot-per-CTA kernel and meets the oracle acceptance."""
    from tests.test_column_slots import _random_code
    rp, ci = _random_code(1024, 2048, 5, 10, 41)
    r = I.Code(m=1024, n=2048, row_ptr=rp, col_idx=ci)
    _, syn, L0, _ = I.workload(r, [0.01, 0.03], 1001, seed=42)
    p = S.Params(mode="bp", max_iter=40)
    assert _same(_decode_with_kernel(r, KERNEL_QC, syn, L0, p), _decode_with_kernel(r, KERNEL_GENERIC, syn, L0, p))
    c = I.gb_code(255, 5)
    dc = S.DeviceCode.from_code(c)
    _native.sagms_set_plan(dc.handle, KERNEL_QC)
    _, syn, L0, _ = I.workload(c, [0.01, 0.03], 400, seed=43)
    G.compare(c, dc, syn, L0, S.Params(mode="bp", max_iter=60))
