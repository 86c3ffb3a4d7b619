"""Seeded synthetic inputs for the SAGMS decoder: codes, error patterns, syndromes, priors.

This module serves both the FP64 oracle and the CUDA decoder and holds none of the
decoder's arithmetic.  It builds

* generalized-bicycle (GB) codes H_X = [A | B], H_Z = [B^T | A^T] from two weight-w
  polynomials a(x), b(x) over GF(2)[x]/(x^l - 1) (the GB family of Sec. II), with A, B
  the l x l circulants sum_t P^t (P the cyclic shift, A[r][(r + t) mod l] = 1);
* iid Z-flip error patterns e and their syndromes s = H_X e (mod 2) (the channel of
  Sec. II marginalised to one Pauli component), from the counter-based C sampler in
  ``gen.c``;
* channel priors L0 = ln((1 - q) / q) for flip probability q (the prior LLR of Sec. II
  written for a binary symbol).

Packed bit layout: bit j of a pattern is bit j % 32 of uint32 word j // 32.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libsagms_inputs.so")
_lib = None

MASK64 = (1 << 64) - 1


def build_lib(force: bool = False) -> str:
    """Compile gen.c into libsagms_inputs.so (plain C, host only)."""
    src = os.path.join(_HERE, "gen.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", src, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build_lib()
        lib = ctypes.CDLL(_LIB_PATH)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        i32p = ctypes.POINTER(ctypes.c_int32)
        lib.sagms_gen_philox4x32_10.argtypes = [u32p, u32p, u32p]
        lib.sagms_gen_philox4x32_10.restype = None
        lib.sagms_gen_sample.argtypes = [ctypes.c_int32, ctypes.c_int32, i32p, i32p, ctypes.c_uint64,
                                         ctypes.c_int64, ctypes.c_int64,
                                         ctypes.POINTER(ctypes.c_double), u32p, u32p]
        lib.sagms_gen_sample.restype = ctypes.c_int
        lib.sagms_gen_syndrome.argtypes = [ctypes.c_int32, ctypes.c_int32, i32p, i32p, ctypes.c_int64, u32p, u32p]
        lib.sagms_gen_syndrome.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype)) if a is not None else None


# --------------------------------------------------------------------------- Philox
def philox4x32_10(counter, key) -> tuple:
    """One Philox4x32-10 block (Salmon et al., SC'11) from the C generator."""
    lib = _load()
    c = np.asarray(counter, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.sagms_gen_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32), _ptr(out, ctypes.c_uint32))
    return tuple(int(x) for x in out)


# --------------------------------------------------------------------------- GF(2) helpers
def splitmix64_stream(seed: int):
    """splitmix64 (Steele, Lea, Flood 2014) as an infinite generator of 64-bit words."""
    state = seed & MASK64
    while True:
        state = (state + 0x9E3779B97F4A7C15) & MASK64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        yield z ^ (z >> 31)


def poly_from_exponents(exps) -> int:
    """GF(2) polynomial as a Python int (bit t = coefficient of x^t)."""
    p = 0
    for t in exps:
        p ^= 1 << t
    return p


def poly_mod(a: int, b: int) -> int:
    db = b.bit_length() - 1
    while a and a.bit_length() - 1 >= db:
        a ^= b << (a.bit_length() - 1 - db)
    return a


def poly_gcd(a: int, b: int) -> int:
    while b:
        a, b = b, poly_mod(a, b)
    return a


def gf2_rank(rows) -> int:
    """Rank over GF(2) of a list of row bitsets (Python ints), by elimination."""
    pivots = {}
    rank = 0
    for r in rows:
        x = r
        while x:
            top = x.bit_length() - 1
            if top in pivots:
                x ^= pivots[top]
            else:
                pivots[top] = x
                rank += 1
                break
    return rank


# --------------------------------------------------------------------------- codes
@dataclass
class Code:
    """A binary parity-check matrix H (m x n) in CSR form plus its CSC lists.

    ``col_idx`` keeps the order in which the rows were built (for GB codes: the terms of
    a(x), then those of b(x)); the decoder library keeps that order as each check's edge
    order where it suits its column-indexed layout, and picks its own otherwise."""
    m: int
    n: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    name: str = ""
    l: int = 0
    w: int = 0
    a: tuple = ()
    b: tuple = ()
    k: int = 0
    seed: int = 0
    hz_rows: list = field(default_factory=list)   # H_Z rows as bitsets (GB codes)
    col_ptr: np.ndarray = None
    row_idx: np.ndarray = None

    def __post_init__(self):
        self.row_ptr = np.ascontiguousarray(self.row_ptr, dtype=np.int32)
        self.col_idx = np.ascontiguousarray(self.col_idx, dtype=np.int32)
        if self.col_ptr is None:
            self.col_ptr, self.row_idx = csr_to_csc(self.m, self.n, self.row_ptr, self.col_idx)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def mw(self) -> int:
        return (self.m + 31) // 32

    @property
    def nw(self) -> int:
        return (self.n + 31) // 32

    def dense(self) -> np.ndarray:
        H = np.zeros((self.m, self.n), dtype=np.uint8)
        for i in range(self.m):
            for t in range(self.row_ptr[i], self.row_ptr[i + 1]):
                H[i, self.col_idx[t]] ^= 1
        return H

    def row_bitsets(self):
        rows = []
        for i in range(self.m):
            x = 0
            for t in range(self.row_ptr[i], self.row_ptr[i + 1]):
                x |= 1 << int(self.col_idx[t])
            rows.append(x)
        return rows


def csr_to_csc(m, n, row_ptr, col_idx):
    col_cnt = np.bincount(col_idx, minlength=n).astype(np.int64)
    col_ptr = np.zeros(n + 1, dtype=np.int32)
    col_ptr[1:] = np.cumsum(col_cnt)
    row_idx = np.zeros(len(col_idx), dtype=np.int32)
    fill = col_ptr[:-1].astype(np.int64).copy()
    for i in range(m):
        for t in range(row_ptr[i], row_ptr[i + 1]):
            j = col_idx[t]
            row_idx[fill[j]] = i
            fill[j] += 1
    return col_ptr, row_idx


def code_from_dense(H: np.ndarray, name: str = "") -> Code:
    H = np.asarray(H, dtype=np.uint8)
    m, n = H.shape
    row_ptr = [0]
    cols = []
    for i in range(m):
        nz = np.nonzero(H[i])[0]
        cols.extend(int(c) for c in nz)
        row_ptr.append(len(cols))
    return Code(m=m, n=n, row_ptr=np.array(row_ptr), col_idx=np.array(cols, dtype=np.int32), name=name)


def gb_exponents(l: int, w: int, seed: int, max_tries: int = 100000):
    """Draw exponent sets a, b (w distinct values in [0, l) each) from splitmix64(seed'),
    seed' = seed, seed + 1, ..., until a != b and k = 2 deg gcd(a(x), b(x), x^l - 1) > 0.

    Returns (a, b, k, seed').  The GB polynomials of the paper's codes are not printed in
    it, so the codes here are seeded stand-ins of the same family."""
    if not (1 <= w <= l):
        raise ValueError("need 1 <= w <= l")
    xl1 = (1 << l) | 1
    for tries in range(max_tries):
        s = seed + tries
        g = splitmix64_stream(s)
        a, b = [], []
        while len(a) < w:
            t = next(g) % l
            if t not in a:
                a.append(t)
        while len(b) < w:
            t = next(g) % l
            if t not in b:
                b.append(t)
        if sorted(a) == sorted(b):
            continue
        d = poly_gcd(poly_gcd(xl1, poly_from_exponents(a)), poly_from_exponents(b))
        k = 2 * (d.bit_length() - 1)
        if k > 0:
            return tuple(a), tuple(b), k, s
    raise RuntimeError("no GB code with k > 0 found")


def gb_code(l: int, w: int, seed: int | None = None) -> Code:
    """GB code with H_X = [A | B] (m = l checks, n = 2l qubits, check degree 2w, qubit
    degree w).  Row r lists columns (r + a_t) mod l for the terms of a(x) in draw order,
    then l + (r + b_t) mod l for the terms of b(x)."""
    if seed is None:
        seed = 1000 * l + w
    a, b, k, s = gb_exponents(l, w, seed)
    m, n = l, 2 * l
    row_ptr = np.arange(0, m * 2 * w + 1, 2 * w, dtype=np.int32)
    r = np.arange(l, dtype=np.int64)[:, None]
    colsA = (r + np.array(a)[None, :]) % l
    colsB = l + (r + np.array(b)[None, :]) % l
    col_idx = np.concatenate([colsA, colsB], axis=1).reshape(-1).astype(np.int32)
    # H_Z = [B^T | A^T]: row r of B^T has ones at columns (r - b_t) mod l.
    hz = []
    for rr in range(l):
        x = 0
        for t in b:
            x |= 1 << ((rr - t) % l)
        for t in a:
            x |= 1 << (l + (rr - t) % l)
        hz.append(x)
    return Code(m=m, n=n, row_ptr=row_ptr, col_idx=col_idx, name=f"GB(l={l},w={w})", l=l, w=w,
                a=a, b=b, k=k, seed=s, hz_rows=hz)


def tree_code(n_vars: int, seed: int, max_deg: int = 4, deg1_prob: float = 0.0) -> Code:
    """Random Tanner forest: every check joins 2..max_deg variables from distinct
    components (union-find), so the Tanner graph has no cycle.  Used to pin the BP
    and MS update rules to exact marginals / max-product values."""
    rng = np.random.default_rng(seed)
    parent = list(range(n_vars))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    rows = []
    for _ in range(4 * n_vars):
        comps = {}
        for v in rng.permutation(n_vars):
            comps.setdefault(find(int(v)), int(v))
        if len(comps) < 2:
            break
        d = int(rng.integers(2, max_deg + 1))
        picks = list(comps.values())
        rng.shuffle(picks)
        picks = picks[:d]
        for v in picks[1:]:
            parent[find(v)] = find(picks[0])
        rows.append(sorted(picks) if rng.random() < 0.5 else picks)
        if deg1_prob > 0 and rng.random() < deg1_prob:
            # a degree-1 check adds a leaf factor and keeps the graph a forest
            rows.append([int(rng.integers(0, n_vars))])
    row_ptr = [0]
    cols = []
    for r in rows:
        cols.extend(r)
        row_ptr.append(len(cols))
    return Code(m=len(rows), n=n_vars, row_ptr=np.array(row_ptr), col_idx=np.array(cols, dtype=np.int32),
                name=f"tree(n={n_vars},seed={seed})")


# --------------------------------------------------------------------------- noise
def llr_prior(q) -> np.ndarray:
    """Binary channel prior L0 = ln((1 - q) / q)."""
    q = np.asarray(q, dtype=np.float64)
    return np.log((1.0 - q) / q)


def depolarizing_to_z(p):
    """Marginal Z-flip probability 2p/3 of a depolarising channel with rate p (Y and Z)."""
    return 2.0 * np.asarray(p, dtype=np.float64) / 3.0


def sample(code: Code, q, shots: int, seed: int, shot0: int = 0, want_err: bool = True,
           threads: int | None = None):
    """Draw `shots` iid flip patterns (per-shot flip probability q: scalar or [shots])
    and their syndromes.  Returns (err [shots][nw] or None, syn [shots][mw]) as uint32."""
    lib = _load()
    qa = np.broadcast_to(np.asarray(q, dtype=np.float64), (shots,)).copy()
    err = np.zeros((shots, code.nw), dtype=np.uint32) if want_err else None
    syn = np.zeros((shots, code.mw), dtype=np.uint32)
    if threads is None:
        threads = min(16, os.cpu_count() or 1)
    chunk = max(1, -(-shots // max(1, threads)))
    if shots >= 4096 and threads > 1:
        starts = list(range(0, shots, chunk))
    else:
        starts = [0] if shots else []
        chunk = shots

    def run(st):
        cnt = min(chunk, shots - st)
        e = err[st:st + cnt] if err is not None else None
        rc = lib.sagms_gen_sample(code.m, code.n, _ptr(code.col_ptr, ctypes.c_int32),
                                  _ptr(code.row_idx, ctypes.c_int32), ctypes.c_uint64(seed & MASK64),
                                  shot0 + st, cnt, _ptr(qa[st:st + cnt], ctypes.c_double),
                                  _ptr(e, ctypes.c_uint32) if e is not None else None,
                                  _ptr(syn[st:st + cnt], ctypes.c_uint32))
        if rc != 0:
            raise RuntimeError("sample: bad arguments")

    if len(starts) > 1:
        with ThreadPoolExecutor(len(starts)) as ex:
            list(ex.map(run, starts))
    elif starts:
        run(0)
    return err, syn


def syndrome(code: Code, err: np.ndarray) -> np.ndarray:
    """s = H e (mod 2) for packed error patterns [shots][nw]."""
    lib = _load()
    err = np.ascontiguousarray(err, dtype=np.uint32)
    shots = err.shape[0]
    syn = np.zeros((shots, code.mw), dtype=np.uint32)
    rc = lib.sagms_gen_syndrome(code.m, code.n, _ptr(code.row_ptr, ctypes.c_int32), _ptr(code.col_idx, ctypes.c_int32),
                                shots, _ptr(err, ctypes.c_uint32), _ptr(syn, ctypes.c_uint32))
    if rc != 0:
        raise RuntimeError("syndrome: bad arguments")
    return syn


def pack_bits(bits: np.ndarray) -> np.ndarray:
    """[shots][k] 0/1 array -> [shots][ceil(k/32)] uint32 words (LSB first)."""
    bits = np.asarray(bits, dtype=np.uint8)
    shots, k = bits.shape
    kw = (k + 31) // 32
    pad = np.zeros((shots, kw * 32), dtype=np.uint8)
    pad[:, :k] = bits
    b = np.packbits(pad.reshape(shots, kw, 4, 8)[:, :, :, ::-1], axis=-1).reshape(shots, kw, 4)
    return (b[:, :, 0].astype(np.uint32) | (b[:, :, 1].astype(np.uint32) << 8)
            | (b[:, :, 2].astype(np.uint32) << 16) | (b[:, :, 3].astype(np.uint32) << 24))


def unpack_bits(words: np.ndarray, k: int) -> np.ndarray:
    """[shots][kw] uint32 -> [shots][k] uint8 bits (LSB first)."""
    words = np.ascontiguousarray(words, dtype=np.uint32)
    shots = words.shape[0]
    by = words.view(np.uint8).reshape(shots, -1)
    bits = np.unpackbits(by, axis=1, bitorder="little")
    return bits[:, :k]


def workload(code: Code, p_values, shots: int, seed: int, want_err: bool = False, shot0: int = 0):
    """Interleaved multi-p batch: shot t uses p_values[t % len(p_values)] with iid Z
    flips at q = p and prior L0 = ln((1-p)/p).  Returns (err|None, syn, L0 float32, q)."""
    pv = np.asarray(p_values, dtype=np.float64)
    q = pv[(np.arange(shots) + shot0) % len(pv)]
    err, syn = sample(code, q, shots, seed, shot0=shot0, want_err=want_err)
    L0 = llr_prior(q).astype(np.float32)
    return err, syn, L0, q
