"""Pins of the FP64 oracle against things other than itself.  CPU only.

Each test fixes a part of the oracle to an independent fact:
brute force over all error patterns on cycle-free Tanner graphs (BP = exact marginals,
MS = min-marginals), closed forms at the first iteration, reductions between the decoder
modes, the single-check ratio of Eq. 9 and its printed values, a hand-worked two-round
SAGMS example, and the zero-syndrome special case.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2605_10433_gb300 import inputs as I
from tests import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _dense_code(rows, n):
    H = np.zeros((len(rows), n), dtype=np.uint8)
    for i, r in enumerate(rows):
        H[i, r] = 1
    return H


def _run_tree_case(seed, mode):
    rng = np.random.default_rng(1000 + seed)
    c = I.tree_code(int(rng.integers(6, 13)), seed, max_deg=4)
    H = c.dense()
    L0 = rng.uniform(0.4, 3.0, size=c.n)
    e = (rng.random(c.n) < 0.3).astype(np.uint8)
    s = (H.astype(np.int64) @ e) % 2
    syn = I.pack_bits(s[None, :].astype(np.uint8))
    it = 2 * (c.n + c.m)
    r = oracle.decode_code(c, syn, L0, mode=mode, max_iter=it,
                           flags=oracle.FLAG_L0_PER_QUBIT | oracle.FLAG_NO_EARLY_STOP, trace=True)
    return c, H, s, L0, r, it


@pytest.mark.parametrize("seed", range(12))
def test_bp_on_trees_equals_exact_marginals(seed):
    """On a cycle-free Tanner graph BP (Eqs. 2, 3) computes exact posterior LLRs."""
    c, H, s, L0, r, it = _run_tree_case(seed, oracle.BP)
    post = r["trace"][0, it]
    ref = brute.exact_llr(H, s, L0)
    assert np.max(np.abs(post)) < oracle.BP_CLIP  # the clip never binds here
    np.testing.assert_allclose(post, ref, rtol=0, atol=1e-9)


@pytest.mark.parametrize("seed", range(12))
def test_ms_on_trees_equals_min_marginals(seed):
    """On a cycle-free Tanner graph MS (Eqs. 2, 4) computes min-marginal cost differences
    (max-product), and its hard decision is the unique minimum-cost pattern."""
    c, H, s, L0, r, it = _run_tree_case(seed, oracle.MS)
    post = r["trace"][0, it]
    ref = brute.min_marginal_diff(H, s, L0)
    np.testing.assert_allclose(post, ref, rtol=0, atol=1e-9)
    best, unique = brute.ml_pattern(H, s, L0)
    if unique:
        assert np.array_equal(I.unpack_bits(r["err"], c.n)[0], best)


def test_sms_scale_one_is_ms_bitwise():
    c = I.gb_code(63, 3)
    _, syn = I.sample(c, 0.05, 400, seed=5)
    L0 = I.llr_prior(np.full(400, 0.05))
    a = oracle.decode_code(c, syn, L0, mode=oracle.MS, max_iter=30, trace=True)
    b = oracle.decode_code(c, syn, L0, mode=oracle.SMS, alpha=1.0, max_iter=30, trace=True)
    for k in ("err", "conv", "iters", "trace"):
        assert np.array_equal(a[k], b[k])


def test_sagms_flat_gain_is_sms_bitwise():
    """alpha_min = alpha_max = alpha and eta = 1 makes Eq. 7 the constant alpha (SMS)."""
    c = I.gb_code(127, 4)
    _, syn = I.sample(c, 2 * 0.02 / 3, 300, seed=6)
    L0 = I.llr_prior(np.full(300, 2 * 0.02 / 3))
    a = oracle.decode_code(c, syn, L0, mode=oracle.SMS, alpha=0.625, max_iter=40, trace=True)
    b = oracle.decode_code(c, syn, L0, mode=oracle.SAGMS, alpha_min=0.625, alpha_max=0.625, eta_unsat=1.0,
                           max_iter=40, trace=True)
    for k in ("err", "conv", "iters", "trace"):
        assert np.array_equal(a[k], b[k])


@pytest.mark.parametrize("mode", [oracle.MS, oracle.SMS, oracle.SAGMS, oracle.BP])
def test_zero_syndrome_gives_zero_error_at_iteration_zero(mode):
    c = I.gb_code(63, 3)
    syn = np.zeros((5, c.mw), dtype=np.uint32)
    r = oracle.decode_code(c, syn, np.full(5, 2.9), mode=mode, max_iter=10)
    assert not r["err"].any()
    assert (r["conv"] == 1).all() and (r["iters"] == 0).all()


@pytest.mark.parametrize("mode", [oracle.MS, oracle.SMS, oracle.SAGMS, oracle.BP])
def test_zero_posterior_decides_no_flip(mode):
    """Reading of the binary hard decision: e_hat_j = 1 iff P_j < 0, so a posterior of exactly
    zero decides 0.  With a zero prior every posterior is zero at the first check: e_hat = 0
    and, on a zero syndrome, the decoder stops there; a qubit in no check with a zero prior
    keeps e_hat = 0 however the rest decodes."""
    c = I.gb_code(63, 3)
    syn = np.zeros((3, c.mw), dtype=np.uint32)
    r = oracle.decode_code(c, syn, np.zeros(3), mode=mode, max_iter=10)
    assert not r["err"].any() and (r["iters"] == 0).all() and (r["conv"] == 1).all()
    code = I.code_from_dense(_dense_code([[0, 1], [1, 2]], 4))   # qubit 3 is in no check
    syn = np.array([[0b01], [0b11]], dtype=np.uint32)
    r = oracle.decode_code(code, syn, np.array([2.0, 1.5, 2.5, 0.0]), mode=mode, max_iter=10,
                           flags=oracle.FLAG_L0_PER_QUBIT)
    assert not (r["err"][:, 0] >> 3 & 1).any()


@pytest.mark.parametrize("mode", [oracle.MS, oracle.SMS, oracle.SAGMS, oracle.BP])
def test_no_early_stop_runs_every_round_and_reports_convergence(mode):
    """SAGMS_FLAG_NO_EARLY_STOP: a zero syndrome still runs all max_iter rounds; the shot ends
    with iters = max_iter and conv = 1 (the residual is zero at return) and e_hat = 0."""
    c = I.gb_code(63, 3)
    syn = np.zeros((3, c.mw), dtype=np.uint32)
    r = oracle.decode_code(c, syn, np.full(3, 2.9), mode=mode, max_iter=7, flags=oracle.FLAG_NO_EARLY_STOP)
    assert not r["err"].any() and (r["iters"] == 7).all() and (r["conv"] == 1).all()


def test_negative_prior_decides_every_qubit_flipped():
    """A per-shot prior below zero (flip probability above one half) makes every qubit's first
    decision a flip: on a code with even check degrees the all-flipped pattern satisfies the
    zero syndrome, so the decoder stops at the first check with e_hat = all ones, in
    L0-normalised and in LLR units alike."""
    c = I.gb_code(63, 3)      # check degree 6
    syn = np.zeros((2, c.mw), dtype=np.uint32)
    for flags in (0, oracle.FLAG_NATURAL_UNITS):
        r = oracle.decode_code(c, syn, np.full(2, -2.9), mode=oracle.SAGMS, max_iter=10, flags=flags)
        bits = np.unpackbits(r["err"].view(np.uint8), axis=1, bitorder="little")[:, :c.n]
        assert bits.all() and (r["iters"] == 0).all() and (r["conv"] == 1).all()


def test_sagms_first_round_closed_form():
    """At l = 1 all CN inputs equal the prior, so Eq. 8 gives (-1)^{s_i} g_i with
    g_i = [a_max - (a_max - a_min) |s|/m] (eta if s_i else 1) (Eqs. 6, 7), and the
    posterior after one round is 1 + sum_{i in N(j)} (-1)^{s_i} g_i (normalised units)."""
    c = I.gb_code(63, 3)
    rng = np.random.default_rng(9)
    s = rng.integers(0, 2, size=(20, c.m)).astype(np.uint8)
    s[0] = 0
    s[0, 5] = 1
    syn = I.pack_bits(s)
    amin, amax, eta = 0.3, 0.5, 1.1
    r = oracle.decode_code(c, syn, np.full(20, 3.7), mode=oracle.SAGMS, alpha_min=amin, alpha_max=amax,
                           eta_unsat=eta, max_iter=1, flags=oracle.FLAG_NO_EARLY_STOP, trace=True)
    H = c.dense().astype(np.float64)
    for k in range(20):
        gamma = s[k].sum() / c.m
        g = (amax - (amax - amin) * gamma) * np.where(s[k] == 1, eta, 1.0)
        msg = np.where(s[k] == 1, -g, g)
        expect = 1.0 + H.T @ msg
        np.testing.assert_allclose(r["trace"][k, 1], expect, rtol=0, atol=1e-12)


def test_bp_first_round_matches_eq9_on_gb_code():
    """At l = 1 every BP CN output of a degree-d_c check has magnitude alpha*(L0, d_c) L0
    (Remark 1, Eq. 9): the posterior after one round is L0 + sum (-1)^{s_i} alpha* L0."""
    c = I.gb_code(127, 4)
    rng = np.random.default_rng(2)
    s = rng.integers(0, 2, size=(6, c.m)).astype(np.uint8)
    L0 = 4.3
    r = oracle.decode_code(c, I.pack_bits(s), np.full(6, L0), mode=oracle.BP, max_iter=1,
                           flags=oracle.FLAG_NO_EARLY_STOP, trace=True)
    astar = 2 * math.atanh(math.tanh(L0 / 2) ** (2 * c.w - 1)) / L0
    H = c.dense().astype(np.float64)
    for k in range(6):
        expect = L0 + H.T @ np.where(s[k] == 1, -astar * L0, astar * L0)
        np.testing.assert_allclose(r["trace"][k, 1], expect, rtol=0, atol=1e-12)


def _single_check_outputs(dc, L0, mode):
    rows = [list(range(dc))]
    c = I.code_from_dense(_dense_code(rows, dc))
    syn = np.zeros((1, 1), dtype=np.uint32)
    r = oracle.decode_code(c, syn, np.full(dc, L0), mode=mode, max_iter=1,
                           flags=oracle.FLAG_NO_EARLY_STOP | oracle.FLAG_L0_PER_QUBIT, trace=True)
    return r["trace"][0, 1] - L0     # the CN -> VN message of the one round


@pytest.mark.parametrize("L0", [1.0, math.log(27.0), 5.293])
def test_single_check_bp_to_ms_ratio_is_eq9_and_decreases_with_dc(L0):
    """Remark 1 / Proposition 1: one BP round over a single check with all inputs L0, divided
    by the MS output, is alpha*(L0, d_c) of Eq. 9 and strictly decreases in d_c."""
    prev = None
    for dc in range(2, 33):
        bp = _single_check_outputs(dc, L0, oracle.BP)
        ms = _single_check_outputs(dc, L0, oracle.MS)
        np.testing.assert_allclose(ms, L0, rtol=0, atol=1e-14)  # MS output = min = L0
        ratio = bp / ms
        exact = 2 * math.atanh(math.tanh(L0 / 2) ** (dc - 1)) / L0
        np.testing.assert_allclose(ratio, exact, rtol=0, atol=1e-12)
        assert abs(oracle.alpha_star(L0, dc) - exact) < 1e-12
        if prev is not None:
            assert ratio[0] < prev
        prev = ratio[0]


@pytest.mark.parametrize("dc", [3, 4, 6, 10])
def test_bp_transfer_function_bounded_by_ms(dc):
    """Eq. 5: T_BP4(kappa) = phi^{-1}((d_c-1) phi(kappa)) <= kappa = T_MS(kappa)."""
    for kappa in np.linspace(0.05, 3.0, 25):
        bp = _single_check_outputs(dc, kappa, oracle.BP)[0]
        t = math.tanh(kappa / 2) ** (dc - 1)
        assert abs(bp - math.log((1 + t) / (1 - t))) < 1e-12
        assert bp <= kappa + 1e-15


def test_paper_printed_alpha_star_values():
    g = json.load(open(os.path.join(GOLDEN, "paper_printed_values.json")))
    a = g["alpha_star_first_order"]
    for p in a["points"]:
        assert abs(oracle.alpha_star_approx(a["L0"], p["dc"]) - p["value"]) <= p["tol"]
    e = g["alpha_fixed_excess"]
    assert abs(e["alpha"] - oracle.alpha_star_approx(e["L0"], e["dc"]) - e["value"]) <= e["tol"]
    d = g["delta_alpha"]
    delta = oracle.alpha_star_approx(d["L0"], d["dc_ref"]) - oracle.alpha_star_approx(d["L0"], d["dc_new"])
    assert abs(delta - d["value"]) <= d["tol"]
    assert abs(delta - math.log((d["dc_new"] - 1) / (d["dc_ref"] - 1)) / d["L0"]) < 1e-12   # Eq. 10
    L = g["L0_mismatch"]
    assert abs(math.log((1 - L["eps0"]) / (L["eps0"] / 3)) - L["value"]) <= L["tol"]


def test_alpha_star_first_order_is_the_large_L0_limit():
    """Eq. 9's approximation uses phi(x) ~ 2 e^{-x}: the gap to the exact form shrinks with L0."""
    for dc in (4, 10, 16):
        gaps = [abs(oracle.alpha_star(L0, dc) - oracle.alpha_star_approx(L0, dc)) for L0 in (4.0, 8.0, 16.0)]
        assert gaps[0] > gaps[1] > gaps[2]
        assert gaps[2] < 1e-4


def test_hand_worked_two_round_sagms_example():
    g = json.load(open(os.path.join(GOLDEN, "hand_sagms_two_rounds.json")))
    H = _dense_code(g["rows"], g["n"])
    c = I.code_from_dense(H)
    syn = I.pack_bits(np.array([g["syndrome"]], dtype=np.uint8))
    r = oracle.decode_code(c, syn, np.array([g["L0"]]), mode=oracle.SAGMS, alpha_min=g["alpha_min"],
                           alpha_max=g["alpha_max"], eta_unsat=g["eta_unsat"], max_iter=g["max_iter"], trace=True)
    np.testing.assert_allclose(r["trace"][0], np.array(g["trace"]), rtol=0, atol=1e-12)
    assert list(I.unpack_bits(r["err"], g["n"])[0]) == g["err_bits"]
    assert r["conv"][0] == g["conv"] and r["iters"][0] == g["iters"]


def test_degree_one_check_saturates_at_the_clip():
    """A degree-1 check has an empty leave-one-out set: its output saturates at the clip
    with sign (-1)^{s_i} (reading of the paper's silence on degree-1 checks)."""
    H = _dense_code([[0], [0, 1]], 2)
    c = I.code_from_dense(H)
    syn = I.pack_bits(np.array([[1, 1]], dtype=np.uint8))
    for mode, clip in ((oracle.MS, oracle.MSFAM_CLIP), (oracle.BP, oracle.BP_CLIP)):
        r = oracle.decode_code(c, syn, np.array([2.0, 2.0]), mode=mode, max_iter=1,
                               flags=oracle.FLAG_NO_EARLY_STOP | oracle.FLAG_L0_PER_QUBIT, trace=True)
        # VN 0 hears -clip from check 0 and -(g * 2) or BP value from check 1
        other = -2.0 if mode == oracle.MS else -2 * math.atanh(math.tanh(1.0))
        assert abs(r["trace"][0, 1, 0] - (2.0 - clip + other)) < 1e-9


def test_normalised_units_change_no_decision():
    """MS/SMS/SAGMS are positively homogeneous of degree 1 in (L0, messages): running them
    in L0-normalised units gives the same decisions as LLR units, shot by shot, except
    where LLR-unit rounding breaks an exact tie."""
    c = I.gb_code(127, 4)
    _, syn = I.sample(c, 0.02, 300, seed=8)
    L0 = I.llr_prior(np.full(300, 0.02))
    for mode in (oracle.MS, oracle.SMS, oracle.SAGMS):
        a = oracle.decode_code(c, syn, L0, mode=mode, max_iter=30)
        b = oracle.decode_code(c, syn, L0, mode=mode, max_iter=30, flags=oracle.FLAG_NATURAL_UNITS)
        same = (a["err"] == b["err"]).all(axis=1) & (a["iters"] == b["iters"])
        assert same.mean() >= 0.97


def test_ml_agreement_rate_on_tiny_loopy_code_is_reported():
    """Loopy-code agreement with brute-force ML is reported, not asserted beyond sanity:
    on loopy graphs no decoder here is exact (parity of the whole decoder is unpinned
    beyond the structural pins above)."""
    rng = np.random.default_rng(4)
    n, m = 14, 8
    while True:
        H = (rng.random((m, n)) < 0.3).astype(np.uint8)
        if H.sum(axis=1).min() >= 2 and H.sum(axis=0).min() >= 1:
            break
    c = I.code_from_dense(H)
    agree = 0
    trials = 60
    L0 = math.log(0.9 / 0.1)
    for t in range(trials):
        e = (rng.random(n) < 0.1).astype(np.uint8)
        s = (H.astype(np.int64) @ e) % 2
        best, _ = brute.ml_pattern(H, s, np.full(n, L0))
        r = oracle.decode_code(c, I.pack_bits(s[None, :].astype(np.uint8)), np.array([L0]),
                               mode=oracle.SAGMS, max_iter=50)
        agree += int(np.array_equal(I.unpack_bits(r["err"], n)[0], best))
    print(f"SAGMS agreement with ML on a loopy n=14 code: {agree}/{trials}")
    assert agree > 0


def test_non_finite_prior_marks_shot_invalid():
    c = I.gb_code(63, 3)
    _, syn = I.sample(c, 0.05, 3, seed=1)
    r = oracle.decode_code(c, syn, np.array([np.nan, 2.0, np.inf]), mode=oracle.SAGMS, max_iter=10)
    assert list(r["iters"][[0, 2]]) == [-1, -1] and not r["conv"][[0, 2]].any()
    assert not r["err"][[0, 2]].any()
    assert r["iters"][1] >= 0


@pytest.mark.parametrize("mode,alpha", [(oracle.MS, 1.0), (oracle.SMS, 0.5)])
def test_exact_modes_are_invariant_under_relabelling(mode, alpha):
    """Algorithm 1 does not depend on how checks, qubits or the edges within a check are
    numbered.  MS in normalised units and SMS with a dyadic scale are exact in FP64, so a
    relabelled code (rows and columns permuted, each row's edges in a new order) must give the
    same decisions, convergence flags and iteration counts, mapped back: a mis-indexed edge,
    a transposed operand or a row/column mix-up anywhere in the oracle breaks this."""
    c = I.gb_code(127, 4)
    err, syn, L0, _ = I.workload(c, [0.06], 300, seed=61, want_err=True)
    r0 = oracle.decode_code(c, syn, L0.astype(np.float64), mode=mode, alpha=alpha, max_iter=30)
    rng = np.random.default_rng(62)
    rows = rng.permutation(c.m)        # old row i becomes row rows[i]
    cols = rng.permutation(c.n)        # old column j becomes column cols[j]
    new_rows = [None] * c.m
    for i in range(c.m):
        edges = cols[c.col_idx[c.row_ptr[i]:c.row_ptr[i + 1]]]
        new_rows[rows[i]] = list(rng.permutation(edges))
    rp = np.concatenate([[0], np.cumsum([len(r) for r in new_rows])]).astype(np.int32)
    ci = np.concatenate([np.asarray(r, dtype=np.int32) for r in new_rows])
    c2 = I.Code(m=c.m, n=c.n, row_ptr=rp, col_idx=ci, name="relabelled")
    s = I.unpack_bits(syn, c.m)
    s2 = np.zeros_like(s)
    s2[:, rows] = s
    r1 = oracle.decode_code(c2, I.pack_bits(s2), L0.astype(np.float64), mode=mode, alpha=alpha, max_iter=30)
    e1 = I.unpack_bits(r1["err"], c.n)[:, cols]
    assert np.array_equal(e1, I.unpack_bits(r0["err"], c.n))
    assert np.array_equal(r1["conv"], r0["conv"]) and np.array_equal(r1["iters"], r0["iters"])
    assert 0 < r0["conv"].sum() < 300          # both outcomes occur


@pytest.mark.parametrize("layered", [False, True])
def test_scale_trace_bounds_the_posterior(layered):
    """The acceptance helper of the GPU tests: the scale trace is |L0_j| + sum of |messages|,
    so it bounds |P_j| (triangle inequality) and equals |L0_j| before the first round."""
    c = I.gb_code(63, 3)
    _, syn, L0, _ = I.workload(c, [0.04, 0.08], 20, seed=12)
    r = oracle.decode_code(c, syn, L0, mode=oracle.SAGMS, max_iter=6, trace=True,
                           flags=oracle.FLAG_NO_EARLY_STOP | (oracle.FLAG_LAYERED if layered else 0))
    assert (r["scale"] >= np.abs(r["trace"]) - 1e-12).all()
    np.testing.assert_array_equal(r["scale"][:, 0, :], np.abs(r["trace"][:, 0, :]))


@pytest.mark.parametrize("lw,q,max_iter", [((63, 3), 0.05, 50), ((127, 4), 0.04 * 2 / 3, 100), ((255, 5), 0.02, 100)])
def test_clip_frequency_on_the_configs(lw, q, max_iter):
    """Readings 8 and 9 (the paper is silent on message overflow): the MS-family clip (1e6 in
    L0 units) never binds on a converging shot of these workloads, and here on none at all;
    the BP clip (ln 2e10) binds on some converging shots (strong priors saturate the rule).
    Both frequencies are reported."""
    c = I.gb_code(*lw)
    _, syn, L0, _ = I.workload(c, [q], 1500, seed=7)
    for mode in (oracle.MS, oracle.SMS, oracle.SAGMS, oracle.BP):
        r = oracle.decode_code(c, syn, L0.astype(np.float64), mode=mode, max_iter=max_iter, threads=4)
        conv = r["conv"] == 1
        fired = r["clips"] > 0
        print(f"GB{lw} mode {mode}: clip binds on {int(fired[conv].sum())}/{int(conv.sum())} converging and "
              f"{int(fired[~conv].sum())}/{int((~conv).sum())} failing shots")
        if mode != oracle.BP:
            assert not fired.any()


@pytest.mark.parametrize("mode", [oracle.MS, oracle.SMS, oracle.SAGMS, oracle.BP])
def test_per_qubit_priors_equal_to_the_shot_prior_decode_identically(mode):
    """The per-qubit prior path (SAGMS_FLAG_L0_PER_QUBIT, LLR units) with every qubit's prior
    set to the shot's L0 is the per-shot path in LLR units: same decisions, iteration counts
    and posterior traces, bit for bit, in every mode.  This ties the two prior plumbings to
    each other (a wrong prior index or a unit slip in either one breaks it)."""
    c = I.gb_code(127, 4)
    shots = 40
    _, syn = I.sample(c, 0.03, shots, seed=21)
    L0 = I.llr_prior(np.full(shots, 0.03))
    units = 0 if mode == oracle.BP else oracle.FLAG_NATURAL_UNITS
    a = oracle.decode_code(c, syn, L0, mode=mode, max_iter=25, flags=units, trace=True)
    for s in range(shots):
        b = oracle.decode_code(c, syn[s:s + 1], np.full(c.n, L0[s]), mode=mode, max_iter=25,
                               flags=oracle.FLAG_L0_PER_QUBIT, trace=True)
        assert np.array_equal(a["err"][s], b["err"][0]) and a["iters"][s] == b["iters"][0]
        assert np.array_equal(np.nan_to_num(a["trace"][s], nan=7.0), np.nan_to_num(b["trace"][0], nan=7.0))
