"""GPU parity of the quaternary (GF(4)) decoder against the GF(4) FP64 oracle, on the paper's own
decoding setting (Sec. II, Sec. V): the overcomplete stabilizer matrix of a GB code with l = 63,
w = 5 (X-type rows of H_X over Z-type rows of H_Z: m = 126 rows, check and qubit degree 10),
depolarising noise at eps, prior L0 = ln((1 - eps0)/(eps0/3)) with eps0 = eps (matched) or
eps0 = 0.1 (the mismatch of Fig. 2b / Fig. 3).  Modes: BP4, SMS(0.5), SAGMS(0.30, 0.50, 1.10).

Per point: the GPU FER lies in the oracle's 95% Wilson interval (or the paired McNemar test
does not reject equal FERs at 1%, as in tests/gpu_helpers.py); per-shot outputs
(x bits, z bits, conv, iters) are identical except for a capped fraction of shots, each of
which must pass the GF(4) shadow replay (every round re-done in FP64 from the GPU's own
per-Pauli posteriors lands within the binary32 rounding bound, pinned in
tests/test_gf4_shadow.py) and is classified at its first differing decision (near-ties at most
0.01% of the shots); posterior traces agree to 1e-5 (normwise, LLR units) at every check
before the first differing decision within the first rounds.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2605_10433_gb300 as S
from oracle import gf4 as O4
from paper_2605_10433_gb300 import inputs as I
from paper_2605_10433_gb300.inputs import gf4 as I4
from paper_2605_10433_gb300.stats import wilson_interval
from tests import gpu_helpers as G

pytestmark = pytest.mark.gpu

MODES = {
    "bp": (S.Params(mode="bp", max_iter=100), oracle.BP),
    "sms": (S.Params(mode="sms", alpha=0.5, max_iter=100), oracle.SMS),
    "sagms": (S.Params(mode="sagms", alpha_min=0.30, alpha_max=0.50, eta_unsat=1.10, max_iter=100), oracle.SAGMS),
}
MISMATCH_CAP = 2e-3
# the column-indexed CSS kernel (the default for the CSS stack) and the generic kernel forced
KERNELS = {"css": 0, "generic": S.FLAG_GENERIC_KERNEL}


@pytest.fixture(scope="module")
def setting():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g = I4.css_code(I.gb_code(63, 5))
    dc = S.Gf4DeviceCode(g)
    assert dc.css_layout
    return g, dc


def _with_kernel(p, kernel):
    return S.Params(**{**p.__dict__, "flags": p.flags | KERNELS[kernel]})


def _run(g, dc, syn, L0, p, mode_o, trace=False, threads=16):
    d_syn = torch.from_numpy(np.ascontiguousarray(syn).view(np.int32)).cuda()
    d_L0 = torch.from_numpy(np.ascontiguousarray(L0, dtype=np.float32)).cuda()
    out = S.gf4_decode(dc, d_syn, d_L0, p, trace=trace)
    torch.cuda.synchronize()
    gres = {"ex": out[0][:, 0].cpu().numpy().view(np.uint32), "ez": out[0][:, 1].cpu().numpy().view(np.uint32),
            "conv": out[1].cpu().numpy(), "iters": out[2].cpu().numpy()}
    if trace:
        gres["trace"] = out[3].cpu().numpy()
    o = O4.decode(g, syn, L0.astype(np.float64), mode=mode_o, alpha=p.alpha, alpha_min=p.alpha_min,
                  alpha_max=p.alpha_max, eta_unsat=p.eta_unsat, max_iter=p.max_iter,
                  flags=p.flags & ~S.FLAG_GENERIC_KERNEL, trace=trace, threads=threads)
    return gres, o


def _same(a, b):
    return ((a["ex"] == b["ex"]).all(axis=1) & (a["ez"] == b["ez"]).all(axis=1) & (a["conv"] == b["conv"])
            & (a["iters"] == b["iters"]))


def _decisions(Lam):
    """Pauli decisions (0 I, 1 X, 2 Z, 3 Y) of per-Pauli LLRs [..., 3] (X, Z, Y), ties to I, X, Z, Y."""
    full = np.concatenate([np.zeros(Lam.shape[:-1] + (1,)), Lam], axis=-1)
    return np.array([0, 1, 2, 3])[np.argmin(full, axis=-1)]


def _check_mismatches(g, dc, syn, L0, p, mo, gr, o):
    """Every shot whose outputs differ: the traced GPU run reproduces the batch run and its outputs
    are the ones its trace implies; the GF(4) shadow replay (oracle.gf4.shadow) accepts the trace
    at every round; the first differing decision is classified as a near-tie (the oracle's two
    smallest Pauli LLRs, the identity's 0 included, within 1e-4) or amplified.  Returns
    (near-ties, amplified, worst shadow ratio)."""
    bad = np.nonzero(~_same(gr, o))[0]
    near, amp, worst = 0, 0, 0.0
    kw = dict(mode=mo, alpha=p.alpha, alpha_min=p.alpha_min, alpha_max=p.alpha_max, eta_unsat=p.eta_unsat)
    for c0 in range(0, len(bad), 64):
        idx = bad[c0:c0 + 64]
        gt, ot = _run(g, dc, syn[idx], L0[idx], p, mo, trace=True)
        for k, s in enumerate(idx):
            for key in ("ex", "ez", "conv", "iters"):
                assert np.array_equal(gt[key][k], gr[key][s]), f"shot {s}: traced run differs ({key})"
            rounds = int(gt["iters"][k])
            last = _decisions(gt["trace"][k, rounds].astype(np.float64))
            want = I.unpack_bits(gr["ex"][s:s + 1], g.n)[0] + 2 * I.unpack_bits(gr["ez"][s:s + 1], g.n)[0]
            assert np.array_equal(last, want), f"shot {s}: e_hat differs from its last traced decisions"
            dev, bnd, _ = O4.shadow(g, syn[s], L0[s:s + 1].astype(np.float64), gt["trace"][k], rounds, **kw)
            with np.errstate(divide="ignore", invalid="ignore"):
                ratio = float(np.max(np.where(dev == 0.0, 0.0, np.abs(dev) / bnd)))
            worst = max(worst, ratio)
            assert ratio <= 1.0, f"shot {s}: GPU posteriors at {ratio:.3g} of the binary32 rounding bound"
            for l in range(min(rounds, int(ot["iters"][k])) + 1):
                da = _decisions(gt["trace"][k, l].astype(np.float64))
                db = _decisions(ot["trace"][k, l])
                if (da != db).any():
                    b = np.concatenate([np.zeros((g.n, 1)), ot["trace"][k, l]], axis=1)[da != db]
                    srt = np.sort(b, axis=1)
                    if float((srt[:, 1] - srt[:, 0]).max()) < 1e-4:
                        near += 1
                    else:
                        amp += 1
                    break
    return near, amp, worst


@pytest.mark.parametrize("kernel", ["css", "generic"])
@pytest.mark.parametrize("eps,eps0", [(0.01, 0.01), (0.02, 0.02), (0.01, 0.1), (0.02, 0.1)])
@pytest.mark.parametrize("mode", ["bp", "sms", "sagms"])
def test_gf4_fer_parity(setting, mode, eps, eps0, kernel):
    g, dc = setting
    shots = 100_000
    _, _, syn = I4.depolarizing(g, eps, shots, seed=int(9000 + 1000 * eps + 100 * eps0))
    L0 = np.full(shots, I4.prior(eps0), dtype=np.float32)
    p, mo = MODES[mode]
    p = _with_kernel(p, kernel)
    gr, o = _run(g, dc, syn, L0, p, mo)
    same = _same(gr, o)
    bad = np.nonzero(~same)[0]
    fer_g, fer_o = 1 - gr["conv"].mean(), 1 - o["conv"].mean()
    lo, hi = wilson_interval(int(round(fer_o * shots)), shots)
    pm = G.mcnemar_p(gr["conv"], o["conv"])
    assert (lo - 1e-12 <= fer_g <= hi + 1e-12) or pm >= 0.01
    near, amp, worst = _check_mismatches(g, dc, syn, L0, p, mo, gr, o)
    assert near <= int(1e-4 * shots + 1e-6), f"{near} near-ties of {shots}"
    assert len(bad) <= MISMATCH_CAP * shots, f"{len(bad)} mismatching shots of {shots}"
    print(f"gf4 GB(63,5) CSS {kernel} kernel eps={eps} eps0={eps0} {mode}: FER gpu {fer_g:.3e} oracle {fer_o:.3e} "
          f"[{lo:.3e}, {hi:.3e}] McNemar p {pm:.3g}, mismatches {len(bad)} (near-tie {near}, amplified {amp}, "
          f"shadow worst {worst:.3g}), "
          f"mean iters {gr['iters'].mean():.2f}")


@pytest.mark.parametrize("kernel", ["css", "generic"])
@pytest.mark.parametrize("mode", ["bp", "sms", "sagms"])
def test_gf4_posterior_traces(setting, mode, kernel):
    g, dc = setting
    _, _, syn = I4.depolarizing(g, 0.03, 64, seed=321)
    L0 = np.full(64, I4.prior(0.03), dtype=np.float32)
    p, mo = MODES[mode]
    p = _with_kernel(S.Params(**{**p.__dict__, "max_iter": 30}), kernel)
    gt, ot = _run(g, dc, syn, L0, p, mo, trace=True)
    worst = 0.0
    for s in range(64):
        last = min(int(gt["iters"][s]), int(ot["iters"][s]), 3)
        for l in range(last + 1):
            a = gt["trace"][s, l].astype(np.float64)
            b = ot["trace"][s, l]
            da = np.argmin(np.concatenate([np.zeros((g.n, 1)), a], axis=1), axis=1)
            db = np.argmin(np.concatenate([np.zeros((g.n, 1)), b], axis=1), axis=1)
            e = float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), 1.0))
            worst = max(worst, e)
            assert e <= 1e-5, f"shot {s} check {l}: normwise error {e:.3g}"
            if (da != db).any():
                break
    print(f"gf4 traces {kernel} kernel {mode}: normwise error {worst:.2e} over the first rounds")


@pytest.mark.parametrize("kernel", ["css", "generic"])
def test_gf4_edge_cases(setting, kernel):
    g, dc = setting
    z = torch.zeros((50, g.mw), dtype=torch.int32, device="cuda")
    L0 = torch.full((50,), float(I4.prior(0.01)), dtype=torch.float32, device="cuda")
    L0[7] = float("nan")
    err, conv, iters = S.gf4_decode(dc, z, L0, _with_kernel(MODES["sagms"][0], kernel))
    torch.cuda.synchronize()
    assert not err.any()
    c, it = conv.cpu().numpy(), iters.cpu().numpy()
    assert it[7] == -1 and c[7] == 0
    keep = np.arange(50) != 7
    assert (c[keep] == 1).all() and (it[keep] == 0).all()
    e0, _, _ = S.gf4_decode(dc, torch.zeros((0, g.mw), dtype=torch.int32, device="cuda"),
                            torch.zeros((0,), dtype=torch.float32, device="cuda"), MODES["bp"][0])
    assert e0.shape[0] == 0


def _random_pauli_code(m, n, seed, max_dc=8, max_dv=6):
    """A random stabilizer-like matrix with X, Y and Z entries, irregular degrees (rows of 2..8
    entries, qubit degree capped), m not a multiple of 32.  Not a commuting stabilizer group:
    the decoder needs none, and the syndromes come from sampled errors."""
    rng = np.random.default_rng(seed)
    deg = np.zeros(n, dtype=int)
    rows, paulis = [], []
    for _ in range(m):
        k = int(rng.integers(2, max_dc + 1))
        free = np.nonzero(deg < max_dv)[0]
        cols = sorted(rng.choice(free, size=min(k, len(free)), replace=False).tolist())
        deg[cols] += 1
        rows.append(cols)
        paulis.append([int(rng.integers(1, 4)) for _ in cols])
    row_ptr = np.cumsum([0] + [len(r) for r in rows]).astype(np.int32)
    return I4.Gf4Code(m=m, n=n, row_ptr=row_ptr, col_idx=np.array([c for r in rows for c in r], dtype=np.int32),
                      pauli=np.array([p for r in paulis for p in r], dtype=np.uint8), name=f"random-pauli{seed}")


def _sample_paulis(g, eps, shots, seed):
    """Depolarising errors on any Pauli matrix (numpy's Philox generator keyed by the seed) and
    their syndromes as trace inner products."""
    rng = np.random.Generator(np.random.Philox(key=seed))
    hit = rng.random((shots, g.n)) < eps
    kind = np.where(hit, rng.integers(1, 4, size=(shots, g.n)), 0)
    x, z = kind & 1, kind >> 1
    s = np.zeros((shots, g.m), dtype=np.uint8)
    for i in range(g.m):
        for e in range(g.row_ptr[i], g.row_ptr[i + 1]):
            c, t = g.col_idx[e], int(g.pauli[e])
            s[:, i] ^= ((x[:, c] & (t >> 1)) ^ (z[:, c] & (t & 1))).astype(np.uint8)
    return I.pack_bits(s)


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("mode", ["bp", "sms", "sagms"])
def test_gf4_general_pauli_matrices(mode, seed):
    """Y entries, mixed entry types at a qubit, irregular degrees, m = 77 (not a multiple of 32):
    every branch of the per-Pauli sums and of the commute LLR, against the oracle."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g = _random_pauli_code(77, 90, seed)
    dc = S.Gf4DeviceCode(g)
    assert not dc.css_layout
    shots = 4000
    syn = _sample_paulis(g, 0.01, shots, seed=100 + seed)
    L0 = np.full(shots, I4.prior(0.01), dtype=np.float32)
    p, mo = MODES[mode]
    p = S.Params(**{**p.__dict__, "max_iter": 40})
    gr, o = _run(g, dc, syn, L0, p, mo)
    same = _same(gr, o)
    fails_g, fails_o = int((gr["conv"] == 0).sum()), int((o["conv"] == 0).sum())
    # these random matrices are poor codes (FER of a few percent): the non-converging shots
    # wander, so mismatches are bounded relative to them, and the FERs are compared paired
    assert int((~same).sum()) <= 2 * fails_o + int(0.002 * shots), f"{mode}: {int((~same).sum())} mismatches"
    assert G.mcnemar_p(gr["conv"], o["conv"]) >= 0.01
    _check_mismatches(g, dc, syn, L0, p, mo, gr, o)
    gt, ot = _run(g, dc, syn[:32], L0[:32], p, mo, trace=True)
    worst = 0.0
    for s in range(32):
        last = min(int(gt["iters"][s]), int(ot["iters"][s]), 3)
        for l in range(last + 1):
            a, b = gt["trace"][s, l].astype(np.float64), ot["trace"][s, l]
            fin = np.isfinite(b)
            e = float(np.max(np.abs(a[fin] - b[fin])) / max(float(np.max(np.abs(b[fin]))), 1.0))
            worst = max(worst, e)
            da = np.argmin(np.concatenate([np.zeros((g.n, 1)), a], axis=1), axis=1)
            db = np.argmin(np.concatenate([np.zeros((g.n, 1)), b], axis=1), axis=1)
            if (da != db).any():
                break
    assert worst <= 1e-5, worst
    print(f"gf4 random Pauli matrix {seed} {mode}: {same.mean() * 100:.2f}% identical, FER gpu {fails_g / shots:.4f} "
          f"oracle {fails_o / shots:.4f}, trace error {worst:.2e}")


def _random_css_code(m, n, seed, max_dc=10, max_dv=4):
    """A random CSS matrix: rows of one Pauli type each, X and Z rows interleaved at random, rows
    of 2..max_dc entries, at most max_dv edges of each type per qubit, m not a multiple of 32.  The
    CSR order rarely gives distinct slots, so the loader's edge colouring is exercised, and the
    irregular degrees leave padded check slots and unused message rows."""
    rng = np.random.default_rng(seed)
    deg = np.zeros((2, n), dtype=int)
    rows, paulis = [], []
    for _ in range(m):
        t = int(rng.integers(1, 3))
        k = int(rng.integers(2, max_dc + 1))
        free = np.nonzero(deg[t - 1] < max_dv)[0]
        cols = sorted(rng.choice(free, size=min(k, len(free)), replace=False).tolist())
        deg[t - 1][cols] += 1
        rows.append(cols)
        paulis.append([t] * len(cols))
    row_ptr = np.cumsum([0] + [len(r) for r in rows]).astype(np.int32)
    return I4.Gf4Code(m=m, n=n, row_ptr=row_ptr, col_idx=np.array([c for r in rows for c in r], dtype=np.int32),
                      pauli=np.array([p for r in paulis for p in r], dtype=np.uint8), name=f"random-css{seed}")


@pytest.mark.parametrize("seed", [11, 12])
@pytest.mark.parametrize("mode", ["bp", "sms", "sagms"])
def test_gf4_css_kernel_random_css_matrices(mode, seed):
    """The CSS kernel on irregular CSS matrices (interleaved X and Z rows, coloured slots, padded
    slots and message rows, m = 93): against the oracle as the general matrices are, and its
    first-round posteriors against the generic kernel's (the priors bit for bit; after round 1 the
    message sums differ only in their order)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g = _random_css_code(93, 100, seed)
    dc = S.Gf4DeviceCode(g)
    assert dc.css_layout
    shots = 4000
    syn = _sample_paulis(g, 0.01, shots, seed=200 + seed)
    L0 = np.full(shots, I4.prior(0.01), dtype=np.float32)
    p, mo = MODES[mode]
    p = S.Params(**{**p.__dict__, "max_iter": 40})
    gr, o = _run(g, dc, syn, L0, p, mo)
    same = _same(gr, o)
    fails_o = int((o["conv"] == 0).sum())
    assert int((~same).sum()) <= 2 * fails_o + int(0.002 * shots), f"{mode}: {int((~same).sum())} mismatches"
    assert G.mcnemar_p(gr["conv"], o["conv"]) >= 0.01
    _check_mismatches(g, dc, syn, L0, p, mo, gr, o)
    gt, _ = _run(g, dc, syn[:32], L0[:32], p, mo, trace=True)
    gg, _ = _run(g, dc, syn[:32], L0[:32], _with_kernel(p, "generic"), mo, trace=True)
    assert np.array_equal(gt["trace"][:, 0], gg["trace"][:, 0])
    ran = (gt["iters"] >= 1) & (gg["iters"] >= 1)   # rows past a shot's last check are not written
    assert ran.sum() >= 16
    # the same posteriors up to the order of each sum: normwise, as the traces against the oracle
    # (a value near zero may come out of terms near +-L0, where a reordering moves a few ulp of L0)
    a, b = gt["trace"][ran, 1].astype(np.float64), gg["trace"][ran, 1].astype(np.float64)
    assert float(np.max(np.abs(a - b))) <= 1e-5 * max(float(np.max(np.abs(b))), 1.0)
    print(f"gf4 random CSS matrix {seed} {mode}: {same.mean() * 100:.2f}% identical to the oracle, "
          f"FER gpu {float((gr['conv'] == 0).mean()):.4f} oracle {fails_o / shots:.4f}")


@pytest.mark.parametrize("lw,eps,shots", [((127, 4), 0.05, 4000), ((255, 5), 0.05, 2000)])
@pytest.mark.parametrize("mode", ["bp", "sagms"])
def test_gf4_css_kernel_larger_stacks(lw, eps, shots, mode):
    """The CSS kernel's other shapes and sizes: the CSS stacks of GB(127, 4) (m = 254, d_c = 8,
    four rows per type and qubit: the (8, 4) shape) and GB(255, 5) (m = 510, 512 threads per
    CTA, the largest block), against the oracle under the same acceptance."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g = I4.css_code(I.gb_code(*lw))
    dc = S.Gf4DeviceCode(g)
    assert dc.css_layout
    _, _, syn = I4.depolarizing(g, eps, shots, seed=lw[0] + 31)
    L0 = np.full(shots, I4.prior(eps), dtype=np.float32)
    p, mo = MODES[mode]
    p = S.Params(**{**p.__dict__, "max_iter": 50})
    gr, o = _run(g, dc, syn, L0, p, mo)
    same = _same(gr, o)
    bad = int((~same).sum())
    assert bad <= max(2, int(MISMATCH_CAP * shots)), f"{bad} mismatching shots of {shots}"
    assert G.mcnemar_p(gr["conv"], o["conv"]) >= 0.01
    near, amp, worst = _check_mismatches(g, dc, syn, L0, p, mo, gr, o)
    assert near <= max(1, int(1e-4 * shots))
    print(f"gf4 CSS stack GB{lw} (m={g.m}) {mode}: FER gpu {float((gr['conv'] == 0).mean()):.4f} "
          f"oracle {float((o['conv'] == 0).mean()):.4f}, mismatches {bad} (near-tie {near}, amplified {amp})")


@pytest.mark.parametrize("mode", ["bp", "sms", "sagms"])
def test_gf4_css_kernel_degenerate_rows(mode):
    """Rows the CSS layout must pad: two empty rows (typed as X rows, all slots padded), three
    rows of a single entry (degree-1 checks: no second minimum, BP's sum over no other edge) and
    a qubit in no row at all, among random CSS rows; both kernels against the oracle."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    base = _random_css_code(40, 50, 21, max_dc=6, max_dv=3)
    rows = [list(base.col_idx[base.row_ptr[i]:base.row_ptr[i + 1]]) for i in range(base.m)]
    paul = [list(base.pauli[base.row_ptr[i]:base.row_ptr[i + 1]]) for i in range(base.m)]
    rows = [[c for c in r if c != 49] for r in rows]   # qubit 49 in no row
    paul = [p[:len(r)] for p, r in zip(paul, rows)]
    rows[3], paul[3] = [], []
    rows[17], paul[17] = [], []
    for i, (c, t) in zip((5, 11, 30), ((7, 1), (8, 2), (9, 1))):
        rows[i], paul[i] = [c], [t]
    row_ptr = np.cumsum([0] + [len(r) for r in rows]).astype(np.int32)
    g = I4.Gf4Code(m=40, n=50, row_ptr=row_ptr, col_idx=np.array([c for r in rows for c in r], dtype=np.int32),
                   pauli=np.array([p for r in paul for p in r], dtype=np.uint8), name="css-degenerate")
    dc = S.Gf4DeviceCode(g)
    assert dc.css_layout
    shots = 3000
    syn = _sample_paulis(g, 0.02, shots, seed=77)
    L0 = np.full(shots, I4.prior(0.02), dtype=np.float32)
    p, mo = MODES[mode]
    p = S.Params(**{**p.__dict__, "max_iter": 30})
    for kernel in ("css", "generic"):
        gr, o = _run(g, dc, syn, L0, _with_kernel(p, kernel), mo)
        same = _same(gr, o)
        fails_o = int((o["conv"] == 0).sum())
        assert int((~same).sum()) <= 2 * fails_o + int(0.002 * shots), f"{kernel}: {int((~same).sum())} mismatches"
        _check_mismatches(g, dc, syn, L0, _with_kernel(p, kernel), mo, gr, o)
        print(f"gf4 degenerate CSS rows {mode} {kernel} kernel: {same.mean() * 100:.2f}% identical to the oracle")
