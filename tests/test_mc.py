"""Fused Monte Carlo engine: the logical basis (CPU), the on-device frame sampler against the
input generator (bit for bit), and the sample -> decode -> check pipeline against its parts,
the FP64 oracle and the rank test of the logical condition."""
import numpy as np
import pytest

import paper_2605_10433_gb300 as S
from paper_2605_10433_gb300 import _native
from paper_2605_10433_gb300 import inputs as I
from paper_2605_10433_gb300.stats import logical_ok


def _csr(rows, n):
    rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    ci = np.asarray([j for r in rows for j in r], dtype=np.int32)
    return rp, ci


def _bits(vec_words, n):
    return np.unpackbits(np.asarray(vec_words, dtype=np.uint32).view(np.uint8), bitorder="little")[:n]


def _rank(rows_bits):
    pivots = {}
    rank = 0
    for r in rows_bits:
        x = int("".join("1" if b else "0" for b in reversed(r.tolist())), 2) if len(r) else 0
        while x:
            top = x.bit_length() - 1
            if top in pivots:
                x ^= pivots[top]
            else:
                pivots[top] = x
                rank += 1
                break
    return rank


def _dense(rp, ci, n):
    H = np.zeros((len(rp) - 1, n), dtype=np.uint8)
    for i in range(len(rp) - 1):
        H[i, ci[rp[i]:rp[i + 1]]] = 1
    return H


# ----------------------------------------------------------------------------- CPU: logicals
def test_steane_code_has_one_logical_anticommuting_with_all_ones():
    """[[7,1,3]]: H_X = H_Z = the Hamming(7,4) checks; k = 1 and the X-logical has odd overlap
    with the all-ones Z-logical (they must anticommute)."""
    ham = [[3, 4, 5, 6], [1, 2, 5, 6], [0, 2, 4, 6]]
    rp, ci = _csr(ham, 7)
    L = _native.sagms_x_logicals(7, rp, ci, rp, ci)
    assert L.shape == (1, 1)
    x = _bits(L[0], 7)
    assert x.sum() % 2 == 1
    assert not (_dense(rp, ci, 7) @ x % 2).any()


@pytest.mark.parametrize("lw", [(63, 3), (127, 4), (255, 5)])
def test_gb_logicals_span_kernel_modulo_stabilizers(lw):
    c = I.gb_code(*lw)
    L = S.x_logicals(c)
    n = c.n
    hz_rows = [[j for j in range(n) if (r >> j) & 1] for r in c.hz_rows]
    hz_rp, hz_ci = _csr(hz_rows, n)
    HX = _dense(c.row_ptr, c.col_idx, n)
    HZ = _dense(hz_rp, hz_ci, n)
    rx, rz = _rank(list(HX)), _rank(list(HZ))
    assert L.shape[0] == n - rx - rz == c.k
    X = np.array([_bits(v, n) for v in L])
    assert not (HZ.astype(np.int64) @ X.T % 2).any()          # every logical is in ker H_Z
    assert _rank(list(HX) + list(X)) == rx + L.shape[0]       # independent modulo rowspace H_X


def _nullspace(H, n):
    """Basis of {x : H x = 0 over GF(2)} by row reduction (test-side, dense)."""
    A = (np.array(H, dtype=np.uint8).reshape(-1, n) & 1).copy()
    piv, r = [], 0
    for c in range(n):
        rows = [i for i in range(r, A.shape[0]) if A[i, c]]
        if not rows:
            continue
        A[[r, rows[0]]] = A[[rows[0], r]]
        for i in range(A.shape[0]):
            if i != r and A[i, c]:
                A[i] ^= A[r]
        piv.append(c)
        r += 1
    basis = []
    for f in (c for c in range(n) if c not in piv):
        x = np.zeros(n, dtype=np.uint8)
        x[f] = 1
        for i, c in enumerate(piv):
            x[c] = A[i, f]
        basis.append(x)
    return basis


def test_logicals_property_on_random_css_pairs():
    """Random CSS pairs drawn by hypothesis (H_Z random, H_X random combinations of ker H_Z, so
    H_X H_Z^T = 0, with repeated and empty rows): k = n - rank H_X - rank H_Z, every returned
    vector lies in ker H_Z, and they are independent modulo the rowspace of H_X."""
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")

    @hyp.settings(max_examples=200, deadline=None, derandomize=True)
    @hyp.given(n=st.integers(1, 24), mz=st.integers(1, 10), mx=st.integers(1, 10), seed=st.integers(0, 2 ** 32 - 1))
    def check(n, mz, mx, seed):
        rng = np.random.default_rng(seed)
        HZ = (rng.random((mz, n)) < rng.uniform(0.1, 0.6)).astype(np.uint8)
        ker = _nullspace(HZ, n)
        HX = np.zeros((mx, n), dtype=np.uint8)
        for i in range(mx):
            for b in ker:
                if rng.random() < 0.5:
                    HX[i] ^= b
        rows = lambda H: [np.nonzero(r)[0].tolist() for r in H]
        rp, ci = _csr(rows(HX), n)
        rz, cz = _csr(rows(HZ), n)
        L = _native.sagms_x_logicals(n, rp, ci, rz, cz)
        rx, rzk = _rank(list(HX)), _rank(list(HZ))
        assert L.shape[0] == n - rx - rzk
        if L.shape[0]:
            X = np.array([_bits(v, n) for v in L])
            assert not (HZ.astype(np.int64) @ X.T % 2).any()
            assert _rank(list(HX) + list(X)) == rx + L.shape[0]

    check()


def test_logicals_reject_non_css_and_bad_csr():
    rp, ci = _csr([[0, 1]], 3)
    rz, cz = _csr([[1, 2]], 3)   # overlap 1: H_X H_Z^T = 1
    with pytest.raises(_native.SagmsError, match="ERR_PARAM"):
        _native.sagms_x_logicals(3, rp, ci, rz, cz)
    bad = np.array([0, 2], dtype=np.int32)
    with pytest.raises(_native.SagmsError, match="ERR_CSR"):
        _native.sagms_x_logicals(3, bad, np.array([0, 5], dtype=np.int32), rz, cz)


def bb_code(l, m, a_terms, b_terms):
    """Bivariate-bicycle code H_X = [A | B], H_Z = [B^T | A^T] over the group Z_l x Z_m, with
    A and B sums of monomials x^p or y^p; rows list A's terms, then B's, in the given order."""
    N = l * m

    def mono(term, r, sign=1):
        i, j = divmod(r, m)
        return ((i + sign * term[1]) % l) * m + j if term[0] == "x" else i * m + (j + sign * term[1]) % m

    rows = [[mono(t, r) for t in a_terms] + [N + mono(t, r) for t in b_terms] for r in range(N)]
    rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    hz = []
    for r in range(N):
        x = 0
        for t in b_terms:
            x |= 1 << mono(t, r, -1)
        for t in a_terms:
            x |= 1 << (N + mono(t, r, -1))
        hz.append(x)
    return I.Code(m=N, n=2 * N, row_ptr=rp, col_idx=np.concatenate(rows).astype(np.int32), name=f"BB({l},{m})",
                  hz_rows=hz)


def test_bivariate_bicycle_144_has_twelve_logicals():
    """[[144,12,12]] (A = x^3 + y + y^2, B = y^3 + x + x^2 over Z_12 x Z_6): the construction
    encodes k = 12 logical qubits, so the basis has 12 X-logicals."""
    c = bb_code(12, 6, [("x", 3), ("y", 1), ("y", 2)], [("y", 3), ("x", 1), ("x", 2)])
    L = S.x_logicals(c)
    assert L.shape == (12, (144 + 31) // 32)


# ----------------------------------------------------------------------------- GPU
gpu = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@gpu
@pytest.mark.parametrize("lw,q,seed,shot0", [((63, 3), 0.05, 7, 0), ((63, 3), 0.0, 7, 0),
                                             ((255, 5), 0.3, 11, 123457), ((1023, 5), 0.01, 2**40 + 3, 2**33 + 5),
                                             ((1023, 5), 0.0005, 99, 17)])
def test_sampler_matches_input_generator(dev, lw, q, seed, shot0):
    c = I.gb_code(*lw)
    dc = S.DeviceCode.from_code(c)
    shots = 3001
    err, syn, L0 = S.mc_sample(dc, seed, q, shot0, shots, L0=None if q > 0 else 3.0)
    e_ref, s_ref = I.sample(c, q, shots, seed=seed, shot0=shot0)
    assert np.array_equal(err.cpu().numpy().view(np.uint32), e_ref)
    assert np.array_equal(syn.cpu().numpy().view(np.uint32), s_ref)
    if q > 0:
        assert np.allclose(L0.cpu().numpy(), np.float32(np.log((1 - q) / q)))


@gpu
def test_sampler_on_irregular_code(dev):
    c = I.tree_code(60, 3, max_deg=5, deg1_prob=0.3)
    dc = S.DeviceCode.from_code(c)
    err, syn, _ = S.mc_sample(dc, 5, 0.1, 0, 500)
    e_ref, s_ref = I.sample(c, 0.1, 500, seed=5)
    assert np.array_equal(err.cpu().numpy().view(np.uint32), e_ref)
    assert np.array_equal(syn.cpu().numpy().view(np.uint32), s_ref)


def _pipeline(dc, params, seed, q, shots):
    err, syn, L0 = S.mc_sample(dc, seed, q, 0, shots)
    ehat, conv, iters = S.decode(dc, syn, L0, params)
    fail, counts = S.mc_check(dc, err, ehat, conv, iters)
    return err, syn, ehat, conv, iters, fail, counts


def _steane():
    """[[7,1,3]] with H_X = H_Z = the Hamming(7,4) checks: distance 3, so weight-2 errors
    often decode to a logical error."""
    ham = [[3, 4, 5, 6], [1, 2, 5, 6], [0, 2, 4, 6]]
    rp, ci = _csr(ham, 7)
    hz = [sum(1 << j for j in r) for r in ham]
    return I.Code(m=3, n=7, row_ptr=rp, col_idx=ci, name="Steane", hz_rows=hz)


@gpu
@pytest.mark.parametrize("which,q,need_logical", [("steane", 0.12, True), ("gb63", 0.06, False)])
def test_check_matches_rank_test_and_counts(dev, which, q, need_logical):
    """Fail flags against conv and the rank test of e XOR e_hat in rowspace(H_Z) on the host."""
    c = _steane() if which == "steane" else I.gb_code(63, 3)
    dc = S.DeviceCode.from_code(c)
    dc.set_logicals(S.x_logicals(c))
    p = S.Params(mode="sagms", max_iter=50)
    err, _, ehat, conv, iters, fail, counts = _pipeline(dc, p, 21, q, 2000)
    e = err.cpu().numpy().view(np.uint32)
    eh = ehat.cpu().numpy().view(np.uint32)
    cv = conv.cpu().numpy()
    f = fail.cpu().numpy()
    r_bits = np.unpackbits((e ^ eh).view(np.uint8), axis=1, bitorder="little")[:, :c.n]
    ok = logical_ok(c.hz_rows, r_bits)
    want = np.where(cv == 0, 1, np.where(ok, 0, 2))
    assert np.array_equal(f, want)
    assert (want == 1).sum() > 0
    if need_logical:
        assert (want == 2).sum() > 0
    assert counts == {"shots": 2000, "failures": int((want != 0).sum()), "not_converged": int((want == 1).sum()),
                      "logical": int((want == 2).sum()), "iters_sum": int(iters.cpu().numpy().sum())}


@gpu
def test_pipeline_decodes_like_the_oracle(dev):
    """The engine's decoder outputs on its own frames against the FP64 oracle."""
    from tests import gpu_helpers as G
    c = I.gb_code(255, 5)
    dc = S.DeviceCode.from_code(c)
    p = S.Params(mode="sagms", max_iter=100)
    err, syn, L0 = S.mc_sample(dc, 31, 0.02, 0, 600)
    G.compare(c, dc, syn.cpu().numpy().view(np.uint32), L0.cpu().numpy(), p)


@gpu
def test_run_equals_manual_batches_and_continues(dev):
    c = I.gb_code(127, 4)
    dc = S.DeviceCode.from_code(c)
    dc.set_logicals(S.x_logicals(c))
    p = S.Params(mode="sagms", max_iter=60)
    q = 0.04
    _, _, _, _, _, _, manual = _pipeline(dc, p, 77, q, 10000)
    whole = S.mc_run(dc, p, 77, q, target_failures=10**9, max_shots=10000, batch=3333)
    assert whole == manual
    part = S.mc_run(dc, p, 77, q, target_failures=10**9, max_shots=4000, batch=1024)
    rest = S.mc_run(dc, p, 77, q, target_failures=10**9, max_shots=10000, batch=1500, counts=part)
    assert rest == manual


@gpu
def test_run_stops_between_batches_at_the_failure_target(dev):
    c = I.gb_code(63, 3)
    dc = S.DeviceCode.from_code(c)
    dc.set_logicals(np.zeros((0, c.nw), dtype=np.uint32))    # k = 0: decoder failures only
    p = S.Params(mode="ms", max_iter=20)
    r = S.mc_run(dc, p, 5, 0.08, target_failures=50, max_shots=10**6, batch=256)
    assert r["failures"] >= 50 and r["logical"] == 0
    assert r["shots"] % 256 == 0 and r["shots"] < 10**6
    prev = S.mc_run(dc, p, 5, 0.08, target_failures=10**9, max_shots=r["shots"] - 256, batch=256)
    assert prev["failures"] < 50


@gpu
def test_run_needs_logicals(dev):
    c = I.gb_code(63, 3)
    dc = S.DeviceCode.from_code(c)
    with pytest.raises(_native.SagmsError, match="logical"):
        S.mc_run(dc, S.Params(), 1, 0.01, max_shots=10)


@gpu
def test_sms_alpha_sweep_rows_are_independent_runs(dev):
    """The sweep is one Monte Carlo run per alpha on the same frames: each row equals a
    direct run, the best alpha has the lowest FER, and alpha* is Eq. 9 for the prior."""
    from paper_2605_10433_gb300.sweep import sms_alpha_sweep
    import oracle
    c = I.gb_code(63, 3)
    dc = S.DeviceCode.from_code(c)
    dc.set_logicals(S.x_logicals(c))
    alphas = [0.5, 0.7, 0.9, 1.0]
    sw = sms_alpha_sweep(dc, alphas, 0.05, seed=9, target_failures=10**9, max_shots=4000, max_iter=30, batch=1000)
    for row, a in zip(sw["rows"], alphas):
        r = S.mc_run(dc, S.Params(mode="sms", alpha=a, max_iter=30), 9, 0.05, target_failures=10**9,
                     max_shots=4000, batch=4000)
        assert (row["failures"], row["shots"], row["logical"]) == (r["failures"], r["shots"], r["logical"])
    assert sw["best_alpha"] == min(sw["rows"], key=lambda x: (x["fer"], x["alpha"]))["alpha"]
    assert sw["alpha_star"] == pytest.approx(oracle.alpha_star(np.log(0.95 / 0.05), 6), rel=1e-12)


def test_checkpointed_run_resumes_from_the_last_record(tmp_path, monkeypatch):
    """Host logic of the JSONL checkpoint (CPU, with a stand-in for the GPU run that draws
    a fixed number of failures per frame index): an interrupted run resumes at the last
    recorded frame and ends with the counts of an uninterrupted one; records of other runs
    in the same file are ignored."""
    import json
    import paper_2605_10433_gb300 as pkg
    from paper_2605_10433_gb300 import sweep

    def fake_run(code, params, seed, q, L0=None, target_failures=0, max_shots=0, batch=0, counts=None):
        c = dict(counts)
        while c["failures"] < target_failures and c["shots"] < max_shots:
            b = min(batch, max_shots - c["shots"])
            c["failures"] += sum(1 for t in range(c["shots"], c["shots"] + b) if (t * 7 + seed) % 97 == 0)
            c["shots"] += b
            c["iters_sum"] += 2 * b
        return c

    monkeypatch.setattr(pkg, "mc_run", fake_run)
    p = S.Params(mode="sagms")
    ck = str(tmp_path / "ck.jsonl")
    with open(ck, "w") as f:   # a record of another run (different seed) in the same file
        f.write(json.dumps({**sweep._key("GB(63,3)", p, 0.01, S.llr(0.01), 99), "shots": 5, "failures": 5,
                            "not_converged": 5, "logical": 0, "iters_sum": 1}) + "\n")
    part = sweep.mc_run_checkpointed(None, "GB(63,3)", p, 3, 0.01, ck, target_failures=10**9, max_shots=3000, batch=1000)
    assert part["shots"] == 3000
    full = sweep.mc_run_checkpointed(None, "GB(63,3)", p, 3, 0.01, ck, target_failures=10**9, max_shots=10000, batch=1000)
    ref = fake_run(None, p, 3, 0.01, target_failures=10**9, max_shots=10000, batch=1000,
                   counts={"shots": 0, "failures": 0, "not_converged": 0, "logical": 0, "iters_sum": 0})
    assert full == ref
    lines = [json.loads(x) for x in open(ck)]
    assert len(lines) == 1 + 10 and lines[-1]["shots"] == 10000 and lines[0]["seed"] == 99

    # a crash mid-write leaves a torn last record: the run resumes from the last complete one
    torn = str(tmp_path / "torn.jsonl")
    sweep.mc_run_checkpointed(None, "GB(63,3)", p, 3, 0.01, torn, target_failures=10**9, max_shots=4000, batch=1000)
    good = open(torn).read()
    with open(torn, "a") as f:
        f.write(good.splitlines()[-1][:37])            # half of a 5000-shot record, no newline
    again = sweep.mc_run_checkpointed(None, "GB(63,3)", p, 3, 0.01, torn, target_failures=10**9, max_shots=10000,
                                      batch=1000)
    assert again == ref
    recs = [x for x in open(torn).read().splitlines() if x]
    assert len(recs) == 4 + 1 + 6 and all(json.loads(x)["shots"] == 1000 * (k + 1)
                                          for k, x in enumerate(recs[:4] + recs[5:]))


@gpu
def test_checkpointed_run_on_the_gpu_equals_one_run(dev, tmp_path):
    from paper_2605_10433_gb300 import sweep
    c = I.gb_code(127, 4)
    dc = S.DeviceCode.from_code(c)
    dc.set_logicals(S.x_logicals(c))
    p = S.Params(mode="sagms", max_iter=40)
    ck = str(tmp_path / "ck.jsonl")
    sweep.mc_run_checkpointed(dc, "GB(127,4)", p, 5, 0.04, ck, target_failures=10**9, max_shots=4096, batch=2048)
    got = sweep.mc_run_checkpointed(dc, "GB(127,4)", p, 5, 0.04, ck, target_failures=10**9, max_shots=10240,
                                    batch=2048)
    assert got == S.mc_run(dc, p, 5, 0.04, target_failures=10**9, max_shots=10240, batch=10240)


@gpu
def test_sharded_run_on_one_gpu_equals_one_run(dev):
    """mc_run_sharded without a process group (one rank): its per-batch sample -> decode ->
    check through the Python entry points counts the same frames as the library's fused
    mc_run, failure target and frame cap included."""
    from paper_2605_10433_gb300 import sweep
    c = I.gb_code(127, 4)
    dc = S.DeviceCode.from_code(c)
    dc.set_logicals(S.x_logicals(c))
    p = S.Params(mode="sagms", max_iter=40)
    for target, cap in ((25, 10**6), (10**9, 9000)):
        got = sweep.mc_run_sharded(dc, p, 5, 0.05, target_failures=target, max_shots=cap, batch=2048)
        assert got == S.mc_run(dc, p, 5, 0.05, target_failures=target, max_shots=cap, batch=2048)
