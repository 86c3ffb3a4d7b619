"""Pins of the GF(4) oracle (oracle/gf4.c), each against something other than itself:

* BP4 on tree-structured stabilizer matrices (random Pauli entries) reaches the exact Pauli
  marginals: its posterior LLRs ln P(E_j = I | s) / P(E_j = W | s) equal a brute-force sum over
  all 4^n errors to 1e-9, and its decision is the marginal maximiser;
* a matrix of X-type checks with priors that forbid X and Y (a Z-flip channel) reduces every
  mode to the binary oracle (pinned in test_oracle_pins.py): same decisions, iteration counts,
  and Lambda(Z) equal to the binary posterior;
* the CSS stacking is symplectic-orthogonal and the depolarising sampler's syndromes are the
  trace inner products <E, H_i>;
* zero syndrome -> identity estimate in round 0; SMS(1) = MS; SAGMS(a, a, eta = 1) = SMS(a).
"""
import itertools

import numpy as np
import pytest

import oracle
from oracle import gf4 as O4
from paper_2605_10433_gb300 import inputs as I
from paper_2605_10433_gb300.inputs import gf4 as I4

PAULI_XZ = {0: (0, 0), 1: (1, 0), 2: (0, 1), 3: (1, 1)}


def _anti(a, b):
    ax, az = PAULI_XZ[a]
    bx, bz = PAULI_XZ[b]
    return (ax & bz) ^ (az & bx)


def _star_tree(n, seed):
    """A tree with checks of degree up to 3: chain of checks sharing one qubit each."""
    rng = np.random.default_rng(seed)
    rows = []
    nxt = 1
    frontier = [0]
    while nxt < n:
        u = int(rng.choice(frontier))
        k = int(min(rng.integers(1, 3), n - nxt))
        r = [u] + list(range(nxt, nxt + k))
        frontier += list(range(nxt, nxt + k))
        nxt += k
        rows.append(r)
    pauli = np.array([int(rng.integers(1, 4)) for r in rows for _ in r], dtype=np.uint8)
    row_ptr = np.cumsum([0] + [len(r) for r in rows]).astype(np.int32)
    col_idx = np.array([j for r in rows for j in r], dtype=np.int32)
    return I4.Gf4Code(m=len(rows), n=n, row_ptr=row_ptr, col_idx=col_idx, pauli=pauli, name=f"star{seed}")


def _syndrome_of(g, errs):
    s = np.zeros(g.m, dtype=np.uint8)
    for i in range(g.m):
        for e in range(g.row_ptr[i], g.row_ptr[i + 1]):
            s[i] ^= _anti(int(errs[g.col_idx[e]]), int(g.pauli[e]))
    return s


def _brute_marginals(g, s, eps):
    """log P(E_j = I | s) - log P(E_j = W | s) for W = X, Z, Y, by summing all 4^n errors."""
    n = g.n
    p = np.array([1 - eps, eps / 3, eps / 3, eps / 3])
    marg = np.zeros((n, 4))
    for errs in itertools.product(range(4), repeat=n):
        if np.array_equal(_syndrome_of(g, errs), s):
            w = np.prod(p[list(errs)])
            for j, e in enumerate(errs):
                marg[j, e] += w
    with np.errstate(divide="ignore"):
        return np.log(marg[:, [0]]) - np.log(marg[:, [1, 2, 3]])


def _pack(bits):
    return I.pack_bits(np.asarray(bits, dtype=np.uint8)[None, :])[0]


@pytest.mark.parametrize("seed", range(8))
def test_bp4_on_trees_equals_brute_force_marginals(seed):
    g = _star_tree(7, seed)
    rng = np.random.default_rng(100 + seed)
    eps = 0.15
    errs = rng.choice(4, size=g.n, p=[1 - eps, eps / 3, eps / 3, eps / 3])
    s = _syndrome_of(g, errs)
    ref = _brute_marginals(g, s, eps)
    L0 = np.array([I4.prior(eps)])
    out = O4.decode(g, _pack(s)[None, :], L0, mode=oracle.BP, max_iter=12, flags=O4.FLAG_NO_EARLY_STOP, trace=True)
    post = out["trace"][0, 12]
    assert np.allclose(post, ref, rtol=0, atol=1e-9), np.max(np.abs(post - ref))
    # decision = the marginal maximiser (argmin of the LLRs with I at 0; ties to I, X, Z, Y)
    full = np.concatenate([np.zeros((g.n, 1)), ref], axis=1)
    want = np.argmin(full, axis=1)               # 0 I, 1 X, 2 Z, 3 Y
    code_of = np.array([0, 1, 2, 3])
    ex = I.unpack_bits(out["ex"], g.n)[0]
    ez = I.unpack_bits(out["ez"], g.n)[0]
    got = ex + 2 * ez
    assert np.array_equal(got, code_of[want])


@pytest.mark.parametrize("mode", [oracle.MS, oracle.SMS, oracle.SAGMS, oracle.BP])
def test_z_channel_on_x_checks_reduces_to_the_binary_oracle(mode):
    code = I.gb_code(63, 3)
    g = I4.Gf4Code(m=code.m, n=code.n, row_ptr=code.row_ptr, col_idx=code.col_idx,
                   pauli=np.full(code.nnz, I4.X, np.uint8))
    q = 0.05
    _, syn, _, _ = I.workload(code, [q], 60, seed=77)
    L = float(I.llr_prior(q))
    pq = np.tile(np.array([np.inf, L, np.inf]), (code.n, 1))
    kw = dict(mode=mode, alpha=0.75, max_iter=40)
    a = O4.decode(g, syn, pq, flags=O4.FLAG_L0_PER_QUBIT, trace=True, **kw)
    b = oracle.decode_code(code, syn, np.full(len(syn), L), flags=oracle.FLAG_NATURAL_UNITS, trace=True, **kw)
    assert not a["ex"].any()
    same = (a["ez"] == b["err"]).all(axis=1) & (a["iters"] == b["iters"]) & (a["conv"] == b["conv"])
    assert same.mean() >= 0.95
    for s in np.nonzero(same)[0]:
        it = int(b["iters"][s])
        za = a["trace"][s, :it + 1, :, 1]
        zb = b["trace"][s, :it + 1]
        assert np.allclose(za, zb, rtol=1e-9, atol=1e-9)
        assert np.all(np.isinf(a["trace"][s, :it + 1, :, [0, 2]]))


def test_css_stack_is_symplectic_orthogonal_and_syndromes_are_trace_products():
    code = I.gb_code(63, 5)
    g = I4.css_code(code)
    assert g.m == 2 * code.m and g.n == code.n
    rows = []
    for i in range(g.m):
        v = np.zeros(g.n, dtype=np.int64)
        for e in range(g.row_ptr[i], g.row_ptr[i + 1]):
            v[g.col_idx[e]] = g.pauli[e]
        rows.append(v)
    for i in range(0, g.m, 7):
        for k in range(g.m):
            assert sum(_anti(int(a), int(b)) for a, b in zip(rows[i], rows[k]) if a and b) % 2 == 0
    ex, ez, syn = I4.depolarizing(g, 0.05, 20, seed=3)
    xb = I.unpack_bits(ex, g.n)
    zb = I.unpack_bits(ez, g.n)
    for s in range(20):
        errs = xb[s] + 2 * zb[s]
        assert np.array_equal(I.unpack_bits(syn[s:s + 1], g.m)[0], _syndrome_of(g, errs))
    # every Pauli appears at the rate eps / 3
    ex, ez, _ = I4.depolarizing(g, 0.3, 4000, seed=4)
    xb = I.unpack_bits(ex, g.n).astype(int)
    zb = I.unpack_bits(ez, g.n).astype(int)
    kinds = xb + 2 * zb
    for k in (1, 2, 3):
        assert abs((kinds == k).mean() - 0.1) < 0.005


def test_zero_syndrome_and_mode_reductions():
    g = I4.css_code(I.gb_code(63, 5))
    ex, ez, syn = I4.depolarizing(g, 0.03, 200, seed=9)
    L0 = np.full(200, I4.prior(0.03))
    z = O4.decode(g, np.zeros_like(syn), L0, mode=oracle.SAGMS, max_iter=10)
    assert not z["ex"].any() and not z["ez"].any() and (z["conv"] == 1).all() and (z["iters"] == 0).all()
    ms = O4.decode(g, syn, L0, mode=oracle.MS, max_iter=20, trace=True)
    sms1 = O4.decode(g, syn, L0, mode=oracle.SMS, alpha=1.0, max_iter=20, trace=True)
    for k in ("ex", "ez", "conv", "iters", "trace"):
        assert np.array_equal(ms[k], sms1[k])
    sms = O4.decode(g, syn, L0, mode=oracle.SMS, alpha=0.6, max_iter=20, trace=True)
    sag = O4.decode(g, syn, L0, mode=oracle.SAGMS, alpha_min=0.6, alpha_max=0.6, eta_unsat=1.0, max_iter=20,
                    trace=True)
    for k in ("ex", "ez", "conv", "iters", "trace"):
        assert np.array_equal(sms[k], sag[k])
