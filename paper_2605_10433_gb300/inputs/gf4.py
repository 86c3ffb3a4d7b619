"""Seeded synthetic inputs for the quaternary (GF(4)) setting of Sec. II: a stabilizer matrix
with Pauli entries, depolarising Pauli errors and their syndromes.  Shared by the FP64 oracle
and the CUDA decoder; none of the decoder's arithmetic lives here.

* ``css_code(code)``: the overcomplete stabilizer matrix of a CSS code, its X-type rows
  (H_X, Pauli X on the support) stacked over its Z-type rows (H_Z, Pauli Z on the support):
  m = m_X + m_Z rows.  For a GB code with l, w this is the 2l x 2l matrix with check and qubit
  degree 2w, the shape of the paper's [[126, k]] experiments (l = 63, w = 5: d_c = d_v = 10).
* ``depolarizing(gcode, eps, shots, seed)``: iid Pauli errors with P(I) = 1 - eps and
  P(X) = P(Y) = P(Z) = eps / 3 (Sec. II); which qubits are hit comes from the counter-based
  sampler of the binary inputs at rate eps, and each hit's Pauli from numpy's Philox
  generator keyed by the seed; syndrome s_i = <E, H_i> (X-type rows see the z bits, Z-type
  rows the x bits).
* ``prior(eps0)``: L0 = ln((1 - eps0) / (eps0 / 3)), the per-Pauli channel LLR of Sec. II.

Pauli codes follow the symplectic map phi_s: X = (1, 0) -> 1, Z = (0, 1) -> 2, Y = (1, 1) -> 3.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import Code, sample, syndrome

X, Z, Y = 1, 2, 3


@dataclass
class Gf4Code:
    """A stabilizer matrix over GF(4) in CSR form: ``pauli[e]`` is the Pauli of edge e."""
    m: int
    n: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    pauli: np.ndarray
    name: str = ""
    k: int = 0
    hx: Code = None   # the X-type rows as a binary code (they see the z bits of an error)
    hz: Code = None   # the Z-type rows (they see the x bits)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def mw(self) -> int:
        return (self.m + 31) // 32

    @property
    def nw(self) -> int:
        return (self.n + 31) // 32


def hz_code(code: Code) -> Code:
    """H_Z of a GB code as a binary Code (rows from its bitsets, columns ascending)."""
    rows = [[j for j in range(code.n) if (r >> j) & 1] for r in code.hz_rows]
    row_ptr = np.cumsum([0] + [len(r) for r in rows])
    return Code(m=len(rows), n=code.n, row_ptr=row_ptr, col_idx=np.array([j for r in rows for j in r], dtype=np.int32),
                name=code.name + " H_Z")


def css_code(code: Code, hz: Code | None = None) -> Gf4Code:
    """X-type rows of ``code`` (H_X) over the Z-type rows of ``hz`` (default: the GB code's
    H_Z)."""
    hz = hz if hz is not None else hz_code(code)
    if hz.n != code.n:
        raise ValueError("H_X and H_Z must act on the same qubits")
    row_ptr = np.concatenate([code.row_ptr, code.row_ptr[-1] + hz.row_ptr[1:]]).astype(np.int32)
    col_idx = np.concatenate([code.col_idx, hz.col_idx]).astype(np.int32)
    pauli = np.concatenate([np.full(code.nnz, X, np.uint8), np.full(hz.nnz, Z, np.uint8)])
    return Gf4Code(m=code.m + hz.m, n=code.n, row_ptr=row_ptr, col_idx=col_idx, pauli=pauli,
                   name=f"CSS[{code.name}]", k=code.k, hx=code, hz=hz)


def depolarizing(gcode: Gf4Code, eps, shots: int, seed: int):
    """Returns (ex, ez, syn): packed x bits and z bits of the errors [shots][nw] and the
    syndromes [shots][mw] (the X-type rows' bits first)."""
    if gcode.hx is None or gcode.hz is None:
        raise ValueError("depolarizing() needs a CSS stabilizer matrix (css_code)")
    hit, _ = sample(gcode.hx, eps, shots, seed=seed)
    bits = np.unpackbits(hit.view(np.uint8), axis=1, bitorder="little")[:, :gcode.n]
    rng = np.random.Generator(np.random.Philox(key=seed & ((1 << 64) - 1)))
    kind = np.zeros_like(bits)
    pos = np.nonzero(bits)
    kind[pos] = rng.integers(1, 4, size=len(pos[0]))   # 1 X, 2 Z, 3 Y, equally likely
    from . import pack_bits
    ex = pack_bits((kind & 1).astype(np.uint8))
    ez = pack_bits((kind >> 1).astype(np.uint8))
    sx = syndrome(gcode.hx, ez)   # X-type rows anticommute with the z part
    sz = syndrome(gcode.hz, ex)   # Z-type rows with the x part
    mx = gcode.hx.m
    sbits = np.concatenate([np.unpackbits(sx.view(np.uint8), axis=1, bitorder="little")[:, :mx],
                            np.unpackbits(sz.view(np.uint8), axis=1, bitorder="little")[:, :gcode.hz.m]], axis=1)
    return ex, ez, pack_bits(sbits)


def prior(eps0) -> np.ndarray:
    """L0 = ln((1 - eps0) / (eps0 / 3))."""
    e = np.asarray(eps0, dtype=np.float64)
    return np.log((1.0 - e) / (e / 3.0))
