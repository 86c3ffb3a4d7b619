"""Pins of the seeded input generators (codes, noise, syndromes).  CPU only."""
import json
import os

import numpy as np
import pytest

from paper_2605_10433_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    kat = json.load(open(os.path.join(GOLDEN, "philox4x32_10_kat.json")))
    for v in kat["vectors"]:
        ctr = [int(x, 16) for x in v["ctr"]]
        key = [int(x, 16) for x in v["key"]]
        out = [int(x, 16) for x in v["out"]]
        assert list(I.philox4x32_10(ctr, key)) == out


@pytest.mark.parametrize("l,w", [(63, 3), (127, 4), (255, 3), (255, 4), (255, 5), (255, 6), (255, 8), (511, 5), (1023, 5)])
def test_gb_code_structure(l, w):
    c = I.gb_code(l, w)
    H = c.dense()
    assert H.shape == (l, 2 * l)
    assert (H.sum(axis=1) == 2 * w).all()            # check degree 2w
    assert (H.sum(axis=0) == w).all()                # qubit degree w
    # H_X H_Z^T = A B + B A = 0 (mod 2): circulants commute (GB family, Sec. II)
    hz = np.zeros((l, 2 * l), dtype=np.int64)
    for r, x in enumerate(c.hz_rows):
        for j in range(2 * l):
            hz[r, j] = (x >> j) & 1
    assert ((H.astype(np.int64) @ hz.T) % 2 == 0).all()
    assert c.k > 0


@pytest.mark.parametrize("l,w", [(63, 3), (127, 4), (255, 8)])
def test_gb_dimension_matches_rank(l, w):
    """k from the gcd formula equals n - rank(H_X) - rank(H_Z) by elimination."""
    c = I.gb_code(l, w)
    rx = I.gf2_rank(c.row_bitsets())
    rz = I.gf2_rank(list(c.hz_rows))
    assert c.n - rx - rz == c.k


def test_syndrome_matches_dense_product():
    c = I.gb_code(63, 3)
    err, syn = I.sample(c, 0.05, 300, seed=7)
    bits = I.unpack_bits(err, c.n)
    s_dense = (c.dense().astype(np.int64) @ bits.T.astype(np.int64) % 2).T
    assert np.array_equal(I.unpack_bits(syn, c.m), s_dense.astype(np.uint8))
    assert np.array_equal(I.syndrome(c, err), syn)


def test_pack_roundtrip():
    rng = np.random.default_rng(0)
    b = rng.integers(0, 2, size=(17, 77)).astype(np.uint8)
    assert np.array_equal(I.unpack_bits(I.pack_bits(b), 77), b)


@pytest.mark.parametrize("q", [0.005, 0.02, 0.05, 0.3])
def test_sampler_flip_rate_and_independence(q):
    """Per-qubit flip frequency within 5 sigma of q; per-shot weight variance ~ n q (1-q)."""
    c = I.gb_code(255, 4)
    shots = 4000
    err, _ = I.sample(c, q, shots, seed=11)
    bits = I.unpack_bits(err, c.n).astype(np.float64)
    tot = bits.size
    rate = bits.sum() / tot
    assert abs(rate - q) < 5 * np.sqrt(q * (1 - q) / tot)
    wt = bits.sum(axis=1)
    var_expected = c.n * q * (1 - q)
    assert abs(wt.var() / var_expected - 1) < 0.15
    # first and last qubits are hit at the same rate (no positional bias of the gaps)
    for j in (0, c.n - 1):
        col = bits[:, j].mean()
        assert abs(col - q) < 6 * np.sqrt(q * (1 - q) / shots) + 1e-12


def test_sampler_deterministic_and_chunk_invariant():
    c = I.gb_code(127, 4)
    e1, s1 = I.sample(c, 0.02, 5000, seed=3)
    e2, s2 = I.sample(c, 0.02, 5000, seed=3, threads=1)
    assert np.array_equal(e1, e2) and np.array_equal(s1, s2)
    e3, s3 = I.sample(c, 0.02, 1000, seed=3, shot0=2000)
    assert np.array_equal(e3, e1[2000:3000]) and np.array_equal(s3, s1[2000:3000])


def test_zero_probability_gives_zero_error():
    c = I.gb_code(63, 3)
    err, syn = I.sample(c, 0.0, 50, seed=1)
    assert not err.any() and not syn.any()


def test_tree_code_is_a_forest():
    for seed in range(10):
        c = I.tree_code(12, seed)
        # acyclic bipartite graph: edges = nodes - components
        edges = c.nnz
        parent = list(range(c.n + c.m))

        def find(x):
            while parent[x] != x:
                parent[x] = parent[parent[x]]
                x = parent[x]
            return x
        for i in range(c.m):
            for t in range(c.row_ptr[i], c.row_ptr[i + 1]):
                a, b = find(c.n + i), find(int(c.col_idx[t]))
                assert a != b, "cycle"
                parent[a] = b
        assert edges <= c.n + c.m - 1


def _gap_sampler_by_definition(n, q, seed, shot):
    """The documented sampler, restated in plain Python for one frame: uniform u32 draws
    u_d = Philox4x32-10(counter (d // 4, shot low, shot high, 0x53414721), key (seed low,
    seed high))[d mod 4]; the gap table T[g] = floor((1 - q)^g 2^32) with the powers formed
    by repeated double multiplication, T[0] = 2^32 - 1 and T[g] = 2^32 - 1 while the product
    is at least 2^32, 0 once it drops below 1; each draw skips the largest g <= n with
    u < T[g] unflipped qubits (0 if none) and flips the next one, until the position passes n.
    A zero probability consumes one draw and flips nothing."""
    two32 = 4294967296.0
    T, pw = [], 1.0
    for g in range(n + 1):
        t = pw * two32
        T.append(0xFFFFFFFF if (g == 0 or t >= two32) else (0 if t < 1.0 else int(t)))
        pw *= (1.0 - q)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    flips, pos, d = [], 0, 0
    while True:
        u = I.philox4x32_10((d >> 2, shot & 0xFFFFFFFF, shot >> 32, 0x53414721), key)[d & 3]
        d += 1
        if q == 0.0:
            break
        pos += max([g for g in range(n + 1) if u < T[g]], default=0)
        if pos >= n:
            break
        flips.append(pos)
        pos += 1
        if pos >= n:
            break
    return flips


@pytest.mark.parametrize("q", [0.0, 0.02, 0.3, 0.9])
def test_sampler_bits_equal_its_definition(q):
    """Every flipped position of the C sampler, frame by frame, against the plain-Python
    statement of its definition (the frames the tests and the on-device sampler share)."""
    c = I.gb_code(63, 3)
    seed, shot0, shots = 0x1234_5678_9ABC, 2**33 + 5, 25
    err, _ = I.sample(c, q, shots, seed=seed, shot0=shot0)
    bits = I.unpack_bits(err, c.n)
    for k in range(shots):
        assert np.nonzero(bits[k])[0].tolist() == _gap_sampler_by_definition(c.n, q, seed, shot0 + k), k


def test_splitmix64_known_answers():
    """The code generator's exponent stream (GB polynomials from splitmix64 draws) against the
    generator's published first outputs for seed 0."""
    kat = json.load(open(os.path.join(GOLDEN, "splitmix64_kat.json")))
    g = I.splitmix64_stream(kat["seed"])
    assert [next(g) for _ in kat["outputs"]] == [int(x, 16) for x in kat["outputs"]]
