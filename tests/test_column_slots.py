"""Edge order of the column-indexed kernels (sagms_column_slots, host only): every edge gets a
slot in [0, 2D), distinct within its check, with slot mod D distinct among its qubit's edges.
The CSR order is kept when it already has the property; otherwise the slots are a proper
D-edge-colouring of the graph of qubits and check halves, which exists whenever qubit degrees
are <= D and check degrees <= 2D (Koenig's edge-colouring theorem).  The tests check the
property itself on codes that need the colouring, including tight ones where every degree
reaches its bound, and that shift structure survives a column sort of a circulant code."""
import numpy as np
import pytest

from paper_2605_10433_gb300 import _native
from paper_2605_10433_gb300 import inputs as I


def _valid(m, n, rp, ci, slots, D):
    for i in range(m):
        s = slots[rp[i]:rp[i + 1]]
        if len(set(s.tolist())) != len(s) or s.min(initial=0) < 0 or s.max(initial=0) >= 2 * D:
            return False
    seen = {}
    for i in range(m):
        for e in range(rp[i], rp[i + 1]):
            key = (int(ci[e]), int(slots[e]) % D)
            if key in seen:
                return False
            seen[key] = e
    return True


def _sorted_rows(rp, ci):
    return np.concatenate([np.sort(ci[rp[i]:rp[i + 1]]) for i in range(len(rp) - 1)]).astype(np.int32)


def _random_code(m, n, dv, dc, seed):
    """Configuration-model graph: every qubit has dv stubs, dealt to checks of at most dc edges
    (repeated pairs dropped, so degrees stay within their bounds)."""
    rng = np.random.default_rng(seed)
    stubs = rng.permutation(np.repeat(np.arange(n), dv))
    rows = [sorted(set(stubs[k:k + dc].tolist())) for k in range(0, len(stubs), dc)][:m]
    rows += [[] for _ in range(m - len(rows))]
    rows = [rng.permutation(r).tolist() for r in rows]
    rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    return rp, np.array([c for r in rows for c in r], dtype=np.int32)


@pytest.mark.parametrize("l,w", [(63, 3), (127, 4), (255, 5)])
def test_generalized_bicycle_term_order_is_kept(l, w):
    """Rows listed by polynomial term already have the property: the CSR order comes back."""
    c = I.gb_code(l, w)
    s = _native.sagms_column_slots(c.m, c.n, c.row_ptr, c.col_idx, w)
    expect = np.concatenate([np.arange(c.row_ptr[i + 1] - c.row_ptr[i]) for i in range(c.m)])
    assert np.array_equal(s, expect)


@pytest.mark.parametrize("l,w", [(63, 3), (127, 4), (255, 5), (1023, 5)])
def test_sorted_generalized_bicycle_rows_keep_the_circulant_structure(l, w):
    """With each row's columns sorted the CSR order breaks the property at the circulant wrap;
    the colouring restores one slot per (block, exponent) pair, so neighbouring checks reach
    neighbouring columns in every slot (the conflict-free shared-memory pattern of the kernel)."""
    c = I.gb_code(l, w)
    ci = _sorted_rows(c.row_ptr, c.col_idx)
    s = _native.sagms_column_slots(c.m, c.n, c.row_ptr, ci, w)
    assert _valid(c.m, c.n, c.row_ptr, ci, s, w)
    slot_of = {}
    for i in range(c.m):
        for e in range(c.row_ptr[i], c.row_ptr[i + 1]):
            key = (int(ci[e]) // l, (int(ci[e]) % l - i) % l)
            assert slot_of.setdefault(key, int(s[e])) == int(s[e])
    assert len(set(slot_of.values())) == 2 * w


def test_sorted_bivariate_bicycle_rows():
    from tests.test_mc import bb_code
    c = bb_code(12, 6, [("x", 3), ("y", 1), ("y", 2)], [("y", 3), ("x", 1), ("x", 2)])
    ci = _sorted_rows(c.row_ptr, c.col_idx)
    s = _native.sagms_column_slots(c.m, c.n, c.row_ptr, ci, 3)
    assert _valid(c.m, c.n, c.row_ptr, ci, s, 3)


@pytest.mark.parametrize("D", [2, 3, 4, 5, 8])
@pytest.mark.parametrize("seed", range(6))
def test_random_codes_at_their_degree_bounds(D, seed):
    """Random graphs with qubit degree D and check degree 2D (after dropped repeats, at most
    that): the greedy choice alone fails on them, so alternating-path swaps are exercised."""
    n = 64 * (seed + 1)
    m = n // 2
    rp, ci = _random_code(m, n, D, 2 * D, seed)
    s = _native.sagms_column_slots(m, n, rp, ci, D)
    assert _valid(m, n, rp, ci, s, D)


def test_tight_random_code_needs_more_than_the_csr_order():
    rp, ci = _random_code(512, 1024, 5, 10, 7)
    expect = np.concatenate([np.arange(rp[i + 1] - rp[i]) for i in range(512)])
    assert not _valid(512, 1024, rp, ci, expect, 5)
    assert _valid(512, 1024, rp, ci, _native.sagms_column_slots(512, 1024, rp, ci, 5), 5)


def test_errors():
    rp = np.array([0, 3], dtype=np.int32)
    with pytest.raises(_native.SagmsError) as ex:   # check degree 3 > 2D
        _native.sagms_column_slots(1, 4, rp, np.array([0, 1, 2], dtype=np.int32), 1)
    assert ex.value.code == -3   # ERR_DEGREE
    with pytest.raises(_native.SagmsError) as ex:   # repeated column
        _native.sagms_column_slots(1, 4, rp, np.array([0, 1, 1], dtype=np.int32), 2)
    assert ex.value.code == -2   # ERR_CSR
    with pytest.raises(_native.SagmsError) as ex:
        _native.sagms_column_slots(1, 4, rp, np.array([0, 1, 2], dtype=np.int32), 0)
    assert ex.value.code == -1   # ERR_ARG


def test_qubit_degree_above_the_row_count_is_refused():
    rp = np.array([0, 1, 2], dtype=np.int32)
    with pytest.raises(_native.SagmsError) as ex:   # qubit 0 in two checks, one message row
        _native.sagms_column_slots(2, 3, rp, np.array([0, 0], dtype=np.int32), 1)
    assert ex.value.code == -3   # ERR_DEGREE


def test_property_on_small_irregular_codes():
    """Any code with qubit degrees <= D and check degrees <= 2D, in any column order, with
    empty checks and unused qubits, gets valid slots (hypothesis draws the graphs)."""
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")

    @hyp.settings(max_examples=300, deadline=None, derandomize=True)
    @hyp.given(D=st.integers(1, 6), m=st.integers(1, 24), n=st.integers(1, 40), seed=st.integers(0, 2 ** 32 - 1),
               fill=st.floats(0.0, 1.0))
    def check(D, m, n, seed, fill):
        rng = np.random.default_rng(seed)
        qdeg = np.zeros(n, dtype=int)
        rows = []
        for _ in range(m):
            want = int(rng.integers(0, 2 * D + 1) * fill + 0.5)
            free = [c for c in rng.permutation(n).tolist() if qdeg[c] < D][:want]
            for c in free:
                qdeg[c] += 1
            rows.append(free)
        rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
        ci = np.array([c for r in rows for c in r], dtype=np.int32)
        s = _native.sagms_column_slots(m, n, rp, ci, D)
        assert _valid(m, n, rp, ci, s, D)

    check()
