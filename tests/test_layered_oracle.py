"""Pins of the oracle's layered schedule (FLAG_LAYERED) against things other than itself.
CPU only.  The paper decodes with the flooding schedule; the layered one is an option of
this library, read as: first-fit layers of the checks in index order, layers visited in
increasing order, each check taking its inputs from the messages as they stand, gains from
the residual at the start of the round.

* cycle-free Tanner graphs: any schedule run to convergence gives BP's exact marginals and
  MS's min-marginals, so brute force over all error patterns pins both rules;
* a hand-worked three-check chain whose first-fit order (c0, c2, c1) differs from the index
  order and from flooding (tests/golden/hand_layered_ms_chain.json);
* codes whose checks share no qubit form a single layer, where the layered round is the
  flooding round: bitwise identical to the flooding oracle in every mode.
The CUDA library's own layering (sagms_check_layers, host side) is checked here too, against
the rule written out on the dense matrix.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2605_10433_gb300 import inputs as I
from tests import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
LAYERED = oracle.FLAG_LAYERED


def _tree_case(seed, mode):
    rng = np.random.default_rng(2000 + seed)
    c = I.tree_code(int(rng.integers(6, 13)), seed, max_deg=4)
    H = c.dense()
    L0 = rng.uniform(0.4, 3.0, size=c.n)
    e = (rng.random(c.n) < 0.3).astype(np.uint8)
    s = (H.astype(np.int64) @ e) % 2
    syn = I.pack_bits(s[None, :].astype(np.uint8))
    it = 2 * (c.n + c.m)
    r = oracle.decode_code(c, syn, L0, mode=mode, max_iter=it,
                           flags=oracle.FLAG_L0_PER_QUBIT | oracle.FLAG_NO_EARLY_STOP | LAYERED, trace=True)
    return c, H, s, L0, r["trace"][0, it], r


@pytest.mark.parametrize("seed", range(12))
def test_layered_bp_on_trees_equals_exact_marginals(seed):
    c, H, s, L0, post, _ = _tree_case(seed, oracle.BP)
    assert np.max(np.abs(post)) < oracle.BP_CLIP
    np.testing.assert_allclose(post, brute.exact_llr(H, s, L0), rtol=0, atol=1e-9)


@pytest.mark.parametrize("seed", range(12))
def test_layered_ms_on_trees_equals_min_marginals(seed):
    c, H, s, L0, post, r = _tree_case(seed, oracle.MS)
    np.testing.assert_allclose(post, brute.min_marginal_diff(H, s, L0), rtol=0, atol=1e-9)
    best, unique = brute.ml_pattern(H, s, L0)
    if unique:
        assert np.array_equal(I.unpack_bits(r["err"], c.n)[0], best)


def _chain():
    g = json.load(open(os.path.join(GOLDEN, "hand_layered_ms_chain.json")))
    H = np.zeros((len(g["rows"]), g["n"]), dtype=np.uint8)
    for i, row in enumerate(g["rows"]):
        H[i, row] = 1
    return g, I.code_from_dense(H), I.pack_bits(np.array([g["syndrome"]], dtype=np.uint8))


def test_hand_worked_layered_chain():
    g, c, syn = _chain()
    L0 = np.array(g["L0"])
    f = oracle.FLAG_L0_PER_QUBIT | LAYERED
    r = oracle.decode_code(c, syn, L0, mode=oracle.MS, max_iter=5, flags=f, trace=True)
    np.testing.assert_allclose(r["trace"][0, :2], np.array(g["trace_early_stop"]), rtol=0, atol=1e-12)
    assert list(I.unpack_bits(r["err"], c.n)[0]) == g["err_bits"]
    assert r["conv"][0] == g["conv"] and r["iters"][0] == g["iters"]
    r2 = oracle.decode_code(c, syn, L0, mode=oracle.MS, max_iter=2, flags=f | oracle.FLAG_NO_EARLY_STOP, trace=True)
    np.testing.assert_allclose(r2["trace"][0], np.array(g["trace_two_rounds"]), rtol=0, atol=1e-12)
    fl = oracle.decode_code(c, syn, L0, mode=oracle.MS, max_iter=1,
                            flags=oracle.FLAG_L0_PER_QUBIT | oracle.FLAG_NO_EARLY_STOP, trace=True)
    np.testing.assert_allclose(fl["trace"][0, 1], np.array(g["flooding_round_one"]), rtol=0, atol=1e-12)


@pytest.mark.parametrize("mode", [oracle.MS, oracle.SMS, oracle.SAGMS, oracle.BP])
def test_single_layer_codes_match_flooding_bitwise(mode):
    """Checks with pairwise disjoint supports (every qubit in at most one check)."""
    rng = np.random.default_rng(mode)
    n = 60
    perm = rng.permutation(n)
    cuts = np.sort(rng.choice(np.arange(1, n), size=11, replace=False))
    rows = [r for r in np.split(perm, cuts) if len(r)][:10]   # the last block's qubits stay unchecked
    H = np.zeros((len(rows), n), dtype=np.uint8)
    for i, row in enumerate(rows):
        H[i, row] = 1
    c = I.code_from_dense(H)
    _, syn, L0, _ = I.workload(c, [0.05, 0.2], 40, seed=3)
    kw = dict(mode=mode, alpha=0.8, max_iter=6, trace=True)
    a = oracle.decode_code(c, syn, L0, flags=oracle.FLAG_NO_EARLY_STOP, **kw)
    b = oracle.decode_code(c, syn, L0, flags=oracle.FLAG_NO_EARLY_STOP | LAYERED, **kw)
    assert np.array_equal(a["trace"], b["trace"]) and np.array_equal(a["err"], b["err"])


def test_layered_differs_from_flooding_on_a_loopy_code():
    """Sanity of the flag itself: on a GB code the layered posteriors after one round differ
    from the flooding ones (a later layer sees messages replaced earlier in the round)."""
    c = I.gb_code(63, 3)
    _, syn, L0, _ = I.workload(c, [0.05], 8, seed=4)
    kw = dict(mode=oracle.SAGMS, max_iter=1, trace=True)
    a = oracle.decode_code(c, syn, L0, flags=oracle.FLAG_NO_EARLY_STOP, **kw)["trace"][:, 1]
    b = oracle.decode_code(c, syn, L0, flags=oracle.FLAG_NO_EARLY_STOP | LAYERED, **kw)["trace"][:, 1]
    assert not np.array_equal(a, b)


def _first_fit(c):
    """The layering rule written out on the dense matrix: check i takes the smallest layer
    not used by an earlier check it shares a qubit with."""
    H = c.dense().astype(bool)
    layer = []
    for i in range(c.m):
        used = {layer[k] for k in range(i) if (H[k] & H[i]).any()}
        layer.append(next(l for l in range(c.m + 1) if l not in used))
    return np.array(layer)


@pytest.mark.parametrize("make", [lambda: I.gb_code(63, 3), lambda: I.gb_code(127, 4), lambda: I.gb_code(255, 8),
                                  lambda: I.tree_code(40, 3, max_deg=4)])
def test_library_layering_is_the_first_fit_rule(make):
    """The CUDA library's layers (host side, no GPU) follow the same rule, checked against the
    rule written out on the dense matrix; every layer's checks share no qubit."""
    from paper_2605_10433_gb300 import _native
    c = make()
    layer, L = _native.sagms_check_layers(c.m, c.n, c.row_ptr, c.col_idx)
    assert np.array_equal(layer, _first_fit(c)) and L == layer.max() + 1
    H = c.dense().astype(np.int64)
    for l in range(L):
        assert (H[layer == l].sum(axis=0) <= 1).all()


def test_hand_chain_layers():
    from paper_2605_10433_gb300 import _native
    _, c, _ = _chain()
    layer, L = _native.sagms_check_layers(c.m, c.n, c.row_ptr, c.col_idx)
    assert list(layer) == [0, 1, 0] and L == 2


def test_library_layering_property_on_small_irregular_codes():
    """The first-fit rule on small irregular codes drawn by hypothesis (empty checks, unused
    qubits, repeated neighbourhoods), against the rule written out on the dense matrix."""
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")
    from paper_2605_10433_gb300 import _native

    @hyp.settings(max_examples=300, deadline=None, derandomize=True)
    @hyp.given(m=st.integers(1, 20), n=st.integers(1, 30), seed=st.integers(0, 2 ** 32 - 1),
               dmax=st.integers(0, 8))
    def check(m, n, seed, dmax):
        rng = np.random.default_rng(seed)
        rows = [sorted(rng.choice(n, size=min(int(rng.integers(0, dmax + 1)), n), replace=False).tolist())
                for _ in range(m)]
        rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
        c = I.Code(m=m, n=n, row_ptr=rp, col_idx=np.array([x for r in rows for x in r], dtype=np.int32))
        layer, L = _native.sagms_check_layers(c.m, c.n, c.row_ptr, c.col_idx)
        assert np.array_equal(layer, _first_fit(c)) and L == layer.max() + 1

    check()


@pytest.mark.parametrize("lw", [(63, 3), (127, 4)])
def test_layered_decode_is_invariant_under_relabelling_into_layer_order(lw):
    """The oracle visits checks in first-fit layer order.  Relabel the checks so that their
    index order is that order (layer by layer, by index within a layer, from the rule written
    out on the dense matrix): first-fit then assigns every check the same layer, so the
    layered decode must not change, bit for bit, in every round.  An oracle whose layers or
    visiting order follow any other rule fails this on codes with several layers."""
    c = I.gb_code(*lw)
    layer = _first_fit(c)
    assert layer.max() >= 3
    order = np.lexsort((np.arange(c.m), layer))         # by (layer, index)
    rows = [c.col_idx[c.row_ptr[i]:c.row_ptr[i + 1]] for i in order]
    rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    c2 = I.Code(m=c.m, n=c.n, row_ptr=rp, col_idx=np.concatenate(rows).astype(np.int32))
    assert np.array_equal(_first_fit(c2), layer[order])
    _, syn, L0, _ = I.workload(c, [0.05], 40, seed=lw[0])
    bits = I.unpack_bits(syn, c.m)[:, order]
    syn2 = I.pack_bits(bits)
    kw = dict(mode=oracle.MS, max_iter=12, trace=True, flags=LAYERED | oracle.FLAG_NO_EARLY_STOP)
    a = oracle.decode_code(c, syn, L0, **kw)
    b = oracle.decode_code(c2, syn2, L0, **kw)
    assert np.array_equal(a["err"], b["err"]) and np.array_equal(a["iters"], b["iters"])
    assert np.array_equal(np.nan_to_num(a["trace"], nan=7.0), np.nan_to_num(b["trace"], nan=7.0))
