"""GPU parity: the CUDA decoder (through the C ABI) against the FP64 oracle on the same
seeded shots.  Marked gpu; they need a CUDA device and the built libsagms.so."""
import math

import numpy as np
import pytest
import torch

import paper_2605_10433_gb300 as S
from paper_2605_10433_gb300 import inputs as I
from tests import gpu_helpers as G

pytestmark = pytest.mark.gpu

MODES = {
    "ms": S.Params(mode="ms"),
    "sms": S.Params(mode="sms", alpha=0.75),
    "sagms": S.Params(mode="sagms", alpha_min=0.30, alpha_max=0.50, eta_unsat=1.10),
    "bp": S.Params(mode="bp"),
}


def _p(mode, **kw):
    return S.Params(**{**MODES[mode].__dict__, **kw})


@pytest.fixture(scope="module")
def codes():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out = {}
    for l, w in [(63, 3), (127, 4), (255, 3), (255, 4), (255, 5), (255, 6), (255, 8), (1023, 5)]:
        c = I.gb_code(l, w)
        out[(l, w)] = (c, S.DeviceCode.from_code(c))
    return out


# --------------------------------------------------------------------------- config 1
@pytest.mark.parametrize("mode", ["ms", "sms", "sagms", "bp"])
def test_config1_n126_per_shot_parity(codes, mode):
    """GB l=63 (n=126), iid Z flips p=0.05, L0=ln((1-p)/p), 1e4 shots, max_iter=50."""
    c, dc = codes[(63, 3)]
    _, syn, L0, _ = I.workload(c, [0.05], 10000, seed=101)
    r = G.compare(c, dc, syn, L0, _p(mode, max_iter=50))
    print(f"config1 {mode}: mismatches {r['mismatch']}/{r['shots']} (near-tie {r['near_tie']}, amplified "
          f"{r['amplified']}) FER gpu {r['fer_gpu']:.4f} oracle {r['fer_oracle']:.4f}")
    if mode == "ms":
        assert r["mismatch"] == 0   # MS is integer-valued in L0 units: exact on both sides


@pytest.mark.parametrize("mode", ["ms", "sms", "sagms", "bp"])
def test_config1_posterior_traces(codes, mode):
    c, dc = codes[(63, 3)]
    _, syn, L0, _ = I.workload(c, [0.05], 96, seed=102)
    w_in, w_all, hz = G.compare_traces(c, dc, syn, L0, _p(mode, max_iter=50))
    print(f"trace {mode}: normwise error {w_in:.2e} within horizons (mean {hz:.1f} checks), {w_all:.2e} overall")
    if mode == "ms":
        assert w_all == 0.0


# --------------------------------------------------------------------------- config 2
@pytest.mark.parametrize("p_dep", [0.01, 0.02, 0.04])
@pytest.mark.parametrize("mode", ["ms", "sms", "sagms", "bp"])
def test_config2_n254_fer_parity(codes, mode, p_dep):
    """GB l=127 (n=254), depolarising p marginalised to 2p/3, max_iter=100."""
    c, dc = codes[(127, 4)]
    q = float(I.depolarizing_to_z(p_dep))
    _, syn, L0, _ = I.workload(c, [q], 30000, seed=int(2000 + 1000 * p_dep))
    r = G.compare(c, dc, syn, L0, _p(mode, max_iter=100))
    (lo, hi), _ = G.fer_check(r, r["shots"])
    print(f"config2 {mode} p={p_dep}: mismatches {r['mismatch']} (near-tie {r['near_tie']}, amplified {r['amplified']}) FER gpu {r['fer_gpu']:.4f} oracle {r['fer_oracle']:.4f} [{lo:.4f},{hi:.4f}]")


@pytest.mark.parametrize("mode", ["sms", "sagms", "bp"])
def test_config2_posterior_traces(codes, mode):
    c, dc = codes[(127, 4)]
    _, syn, L0, _ = I.workload(c, [float(I.depolarizing_to_z(0.04))], 48, seed=203)
    w_in, w_all, hz = G.compare_traces(c, dc, syn, L0, _p(mode, max_iter=40))
    print(f"config2 trace {mode}: {w_in:.2e} within horizons (mean {hz:.1f}), {w_all:.2e} overall")


# --------------------------------------------------------------------------- config 3
@pytest.mark.parametrize("w", [3, 4, 5, 6, 8])
def test_config3_n510_mixed_degrees(codes, w):
    """GB l=255 (n=510), w in {3,4,5,6,8} (check degree 6..16), p=0.02, SAGMS max_iter=100."""
    c, dc = codes[(255, w)]
    _, syn, L0, _ = I.workload(c, [0.02], 3000, seed=300 + w)
    r = G.compare(c, dc, syn, L0, _p("sagms", max_iter=100))
    print(f"config3 w={w}: mismatches {r['mismatch']} FER gpu {r['fer_gpu']:.4f} oracle {r['fer_oracle']:.4f}")


# --------------------------------------------------------------------------- config 4
@pytest.mark.parametrize("p", [0.005, 0.01, 0.02])
@pytest.mark.parametrize("mode", ["ms", "sms", "sagms"])
def test_config4_n2046_sampled_parity(codes, mode, p):
    """GB l=1023 (n=2046, 10230 edges), iid Z flips, max_iter=100: a sample the oracle
    decodes shot by shot."""
    c, dc = codes[(1023, 5)]
    _, syn, L0, _ = I.workload(c, [p], 600, seed=int(4000 + 1e5 * p))
    r = G.compare(c, dc, syn, L0, _p(mode, max_iter=100))
    print(f"config4 {mode} p={p}: mismatches {r['mismatch']} FER gpu {r['fer_gpu']:.4f} oracle {r['fer_oracle']:.4f}")


def test_config4_full_launch_properties(codes):
    """At the benchmark's launch shape (one launch over an interleaved p in {0.005, 0.01, 0.02}
    batch), check properties that hold at any size: conv == [H e_hat == s], iters in range,
    converged shots' counts below max_iter, run-to-run bitwise determinism; and a strided
    sample against the oracle."""
    c, dc = codes[(1023, 5)]
    shots = 200000
    _, syn, L0, _ = I.workload(c, [0.005, 0.01, 0.02], shots, seed=777)
    p = _p("sagms", max_iter=100)
    g1 = G.gpu_decode(dc, syn, L0, p)
    g2 = G.gpu_decode(dc, syn, L0, p)
    for k in ("err", "conv", "iters"):
        assert np.array_equal(g1[k], g2[k])
    ok = G.residual_ok(c, syn, g1["err"])
    assert np.array_equal(ok, g1["conv"].astype(bool))
    assert g1["iters"].min() >= 0 and g1["iters"].max() <= 100
    assert (g1["iters"][g1["conv"] == 0] == 100).all()
    # a strided sample of this launch's outputs against the oracle, under the full acceptance
    idx = np.arange(0, shots, 97)
    r = G.compare(c, dc, syn[idx], L0[idx], p, gpu={k: g1[k][idx] for k in ("err", "conv", "iters")})
    print(f"config4 full launch, {len(idx)} sampled shots: mismatches {r['mismatch']} (near-tie {r['near_tie']}, "
          f"amplified {r['amplified']})")


# --------------------------------------------------------------------------- edge cases
def test_zero_shots_and_zero_syndromes(codes):
    c, dc = codes[(63, 3)]
    z = torch.zeros((0, c.mw), dtype=torch.int32, device="cuda")
    out = S.decode(dc, z, torch.zeros(0, dtype=torch.float32, device="cuda"))
    assert out[0].shape[0] == 0
    syn = np.zeros((77, c.mw), dtype=np.uint32)
    L0 = np.full(77, 3.0, dtype=np.float32)
    for mode in MODES:
        g = G.gpu_decode(dc, syn, L0, _p(mode))
        assert not g["err"].any() and (g["conv"] == 1).all() and (g["iters"] == 0).all()


def test_max_iter_zero_and_no_early_stop(codes):
    c, dc = codes[(127, 4)]
    _, syn, L0, _ = I.workload(c, [0.02], 500, seed=5)
    G.compare(c, dc, syn, L0, _p("sagms", max_iter=0))
    G.compare(c, dc, syn, L0, _p("sagms", max_iter=12, flags=S.FLAG_NO_EARLY_STOP))
    G.compare(c, dc, syn, L0, _p("bp", max_iter=12, flags=S.FLAG_NO_EARLY_STOP))


def test_invalid_prior_marks_shot(codes):
    c, dc = codes[(63, 3)]
    _, syn, L0, _ = I.workload(c, [0.05], 64, seed=6)
    L0 = L0.copy()
    L0[[3, 10]] = [np.nan, np.inf]
    r = G.compare(c, dc, syn, L0, _p("sagms", max_iter=30))
    assert r["gpu"]["iters"][3] == -1 and r["gpu"]["iters"][10] == -1


@pytest.mark.parametrize("mode", ["ms", "sagms", "bp"])
def test_per_qubit_priors(codes, mode):
    c, dc = codes[(127, 4)]
    rng = np.random.default_rng(7)
    qj = rng.uniform(0.005, 0.05, size=c.n)
    _, syn = I.sample(c, 0.02, 2000, seed=8)
    L0q = I.llr_prior(qj).astype(np.float32)
    r = G.compare(c, dc, syn, L0q, _p(mode, max_iter=60, flags=S.FLAG_L0_PER_QUBIT))
    print(f"per-qubit {mode}: mismatches {r['mismatch']}")


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("mode", ["ms", "sagms", "bp"])
def test_irregular_tree_codes_with_degree_one_checks(mode, seed):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = I.tree_code(40, seed, max_deg=5, deg1_prob=0.3)
    dc = S.DeviceCode.from_code(c)
    _, syn, L0, _ = I.workload(c, [0.1], 300, seed=seed)
    # Small symmetric trees have exact ties (P = 0 in exact arithmetic) by construction, so
    # near-tie mismatches are not budgeted here; each one is still traced to a near-tie.
    G.compare(c, dc, syn, L0, _p(mode, max_iter=40), min_frac=0.0)
    G.compare_traces(c, dc, syn[:16], L0[:16], _p(mode, max_iter=40))


def test_largest_supported_check_count():
    """m = 1024 checks (one full CTA of check threads), GB l = 1024 (w = 4: an odd weight gives
    k = 0 when l is a power of two)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = I.gb_code(1024, 4)
    dc = S.DeviceCode.from_code(c)
    _, syn, L0, _ = I.workload(c, [0.01], 300, seed=9)
    G.compare(c, dc, syn, L0, _p("sagms", max_iter=100))


def test_random_irregular_code_wide_degrees():
    """A random code with check degrees up to 20 and qubit degrees up to 9 (the widest variant)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rng = np.random.default_rng(10)
    m, n = 200, 300
    H = np.zeros((m, n), dtype=np.uint8)
    for i in range(m):
        d = int(rng.integers(3, 21))
        H[i, rng.choice(n, size=d, replace=False)] = 1
    while H.sum(axis=0).max() > 16:
        j = int(np.argmax(H.sum(axis=0)))
        H[np.nonzero(H[:, j])[0][0], j] = 0
    c = I.code_from_dense(H)
    dc = S.DeviceCode.from_code(c)
    _, syn, L0, _ = I.workload(c, [0.03], 400, seed=11)
    for mode in ("sagms", "bp"):
        G.compare(c, dc, syn, L0, _p(mode, max_iter=50))


def test_decode_host_matches_device_path(codes):
    c, dc = codes[(255, 4)]
    _, syn, L0, _ = I.workload(c, [0.02], 30000, seed=12)
    p = _p("sagms")
    g = G.gpu_decode(dc, syn, L0, p)
    err, conv, iters = S.decode_host(dc, syn, L0, p)
    assert np.array_equal(err, g["err"]) and np.array_equal(conv, g["conv"]) and np.array_equal(iters, g["iters"])


def test_concurrent_streams_share_a_code(codes):
    c, dc = codes[(255, 5)]
    _, syn, L0, _ = I.workload(c, [0.02], 20000, seed=13)
    p = _p("sagms")
    ref = G.gpu_decode(dc, syn, L0, p)
    d_syn = torch.from_numpy(syn.view(np.int32)).cuda()
    d_L0 = torch.from_numpy(L0).cuda()
    streams = [torch.cuda.Stream() for _ in range(3)]
    outs = []
    for s in streams:
        with torch.cuda.stream(s):
            outs.append(S.decode(dc, d_syn, d_L0, p, stream=s))
    torch.cuda.synchronize()
    for o in outs:
        assert np.array_equal(o[0].cpu().numpy().view(np.uint32), ref["err"])
        assert np.array_equal(o[2].cpu().numpy(), ref["iters"])


@pytest.mark.parametrize("mode", ["ms", "sms", "sagms"])
@pytest.mark.parametrize("lw", [(63, 3), (127, 4), (255, 8), (1023, 5)])
def test_two_slot_kernel_is_bitwise_identical_to_generic(codes, mode, lw):
    """The two-slot continuous-batching kernel and the one-shot-per-CTA kernel run the same
    arithmetic in the same order: outputs and posterior traces agree bit for bit."""
    c, dc = codes[lw]
    _, syn, L0, _ = I.workload(c, [0.01, 0.03, 0.06], 3001, seed=31 + lw[0])
    p = _p(mode, max_iter=60)
    pg = _p(mode, max_iter=60, flags=S.FLAG_GENERIC_KERNEL)
    a = G.gpu_decode(dc, syn, L0, p)
    b = G.gpu_decode(dc, syn, L0, pg)
    for k in ("err", "conv", "iters"):
        assert np.array_equal(a[k], b[k])
    ta = G.gpu_decode(dc, syn[:40], L0[:40], p, trace=True)["trace"]
    tb = G.gpu_decode(dc, syn[:40], L0[:40], pg, trace=True)["trace"]
    assert np.array_equal(np.nan_to_num(ta, nan=7.0), np.nan_to_num(tb, nan=7.0))
