"""FP64 CPU oracle of the quaternary (GF(4)) decoders, BP4 and the Min-Sum family on a
stabilizer matrix with Pauli entries (test infrastructure; ``gf4.c``).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` import
this module.  Parity status: pinned by ``tests/test_gf4_oracle.py`` -- BP4 on tree-structured
stabilizer matrices equals brute-force Pauli marginals over all 4^n errors, a matrix of
X-type checks with priors that forbid X and Y reduces it exactly to the binary oracle (itself
pinned), and the mode reductions and zero-syndrome case hold bit for bit.  ``shadow`` (the
acceptance replay of GPU traces, not the method) is pinned in ``tests/test_gf4_shadow.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import CFLAGS, MS, SMS, SAGMS, BP   # noqa: F401  (mode numbers shared with the binary oracle)

FLAG_L0_PER_QUBIT = 1
FLAG_NO_EARLY_STOP = 2

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libgf4.so")
_lib = None


def build_lib(force: bool = False) -> str:
    """Compile gf4.c.  With ORACLE_GF4_LIB_OVERRIDE set (the test that plants mistakes in a copy
    of gf4.c and checks that the pins fail), that prebuilt library is used instead."""
    override = os.environ.get("ORACLE_GF4_LIB_OVERRIDE")
    if override:
        return override
    src = os.path.join(_HERE, "gf4.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, src, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_lib())
        P = ctypes.POINTER
        lib.oracle_gf4_decode.argtypes = [ctypes.c_int, ctypes.c_int, P(ctypes.c_int32), P(ctypes.c_int32),
                                          P(ctypes.c_uint8), ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_uint,
                                          ctypes.c_int64, P(ctypes.c_uint32), P(ctypes.c_double),
                                          P(ctypes.c_uint32), P(ctypes.c_uint8), P(ctypes.c_int32),
                                          P(ctypes.c_double)]
        lib.oracle_gf4_decode.restype = ctypes.c_int
        lib.oracle_gf4_shadow.argtypes = [ctypes.c_int, ctypes.c_int, P(ctypes.c_int32), P(ctypes.c_int32),
                                          P(ctypes.c_uint8), ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_uint, P(ctypes.c_uint32),
                                          P(ctypes.c_double), ctypes.c_int, P(ctypes.c_float), P(ctypes.c_double),
                                          P(ctypes.c_double), P(ctypes.c_int32)]
        lib.oracle_gf4_shadow.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct)) if a is not None else None


def decode(gcode, syn, L0, mode=SAGMS, alpha=0.75, alpha_min=0.30, alpha_max=0.50, eta_unsat=1.10, max_iter=100,
           flags=0, trace=False, threads=1):
    """Decode packed syndromes ``syn`` [shots][ceil(m/32)] on the GF(4) matrix ``gcode``
    (row_ptr, col_idx, pauli).  ``L0``: [shots] per-shot prior LLR (the same for X, Z, Y), or
    [n][3] LLRs ln P(I)/P(W) for W = X, Z, Y with FLAG_L0_PER_QUBIT.  Returns ``ex``, ``ez``
    [shots][ceil(n/32)] (x and z bits of e_hat), ``conv``, ``iters`` and with ``trace=True``
    ``trace`` [shots][max_iter+1][n][3] posterior LLRs (X, Z, Y) at each check."""
    lib = _load()
    m, n = gcode.m, gcode.n
    row_ptr = np.ascontiguousarray(gcode.row_ptr, dtype=np.int32)
    col_idx = np.ascontiguousarray(gcode.col_idx, dtype=np.int32)
    pauli = np.ascontiguousarray(gcode.pauli, dtype=np.uint8)
    syn = np.ascontiguousarray(syn, dtype=np.uint32).reshape(-1, (m + 31) // 32)
    shots = syn.shape[0]
    per_qubit = bool(flags & FLAG_L0_PER_QUBIT)
    L0 = np.ascontiguousarray(L0, dtype=np.float64)
    if per_qubit and L0.shape != (n, 3):
        raise ValueError("per-qubit L0 must be [n][3]")
    if not per_qubit:
        L0 = L0.reshape(-1)
        if L0.shape[0] != shots:
            raise ValueError("per-shot L0 must have one entry per shot")
    nw = (n + 31) // 32
    err = np.zeros((shots, 2, nw), dtype=np.uint32)
    conv = np.zeros(shots, dtype=np.uint8)
    iters = np.zeros(shots, dtype=np.int32)
    tr = np.zeros((shots, max_iter + 1, n, 3), dtype=np.float64) if trace else None

    def run(lo, hi):
        if hi <= lo:
            return
        Ls = L0 if per_qubit else np.ascontiguousarray(L0[lo:hi])
        rc = lib.oracle_gf4_decode(m, n, _p(row_ptr, ctypes.c_int32), _p(col_idx, ctypes.c_int32),
                                   _p(pauli, ctypes.c_uint8), mode, alpha, alpha_min, alpha_max, eta_unsat,
                                   max_iter, flags, hi - lo, _p(syn[lo:hi], ctypes.c_uint32), _p(Ls, ctypes.c_double),
                                   _p(err[lo:hi], ctypes.c_uint32), _p(conv[lo:hi], ctypes.c_uint8),
                                   _p(iters[lo:hi], ctypes.c_int32),
                                   _p(tr[lo:hi] if tr is not None else None, ctypes.c_double))
        if rc != 0:
            raise RuntimeError("oracle_gf4_decode: bad arguments")

    threads = max(1, int(threads))
    if threads == 1 or shots < 2 * threads:
        run(0, shots)
    else:
        bounds = np.linspace(0, shots, threads + 1).astype(int)
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(lambda k: run(bounds[k], bounds[k + 1]), range(threads)))
    out = {"ex": err[:, 0], "ez": err[:, 1], "conv": conv, "iters": iters}
    if tr is not None:
        out["trace"] = tr
    return out


def shadow(gcode, syn_row, L0, G, rounds, mode=SAGMS, alpha=0.75, alpha_min=0.30, alpha_max=0.50, eta_unsat=1.10,
           flags=0):
    """Replay one shot's rounds from another implementation's binary32 per-Pauli posterior trace
    ``G`` [>= rounds+1][n][3] and bound its rounding (``oracle_gf4_shadow``; test acceptance
    only).  Returns (dev, bnd, flips) with dev, bnd [rounds+1][n][3]."""
    lib = _load()
    n = gcode.n
    row_ptr = np.ascontiguousarray(gcode.row_ptr, dtype=np.int32)
    col_idx = np.ascontiguousarray(gcode.col_idx, dtype=np.int32)
    pauli = np.ascontiguousarray(gcode.pauli, dtype=np.uint8)
    syn_row = np.ascontiguousarray(syn_row, dtype=np.uint32).reshape(-1)
    L0 = np.ascontiguousarray(L0, dtype=np.float64).reshape(-1)
    G = np.ascontiguousarray(np.asarray(G, dtype=np.float32)[:rounds + 1]).reshape(rounds + 1, n, 3)
    dev = np.zeros((rounds + 1, n, 3))
    bnd = np.zeros((rounds + 1, n, 3))
    flips = np.zeros(rounds + 1, dtype=np.int32)
    rc = lib.oracle_gf4_shadow(gcode.m, n, _p(row_ptr, ctypes.c_int32), _p(col_idx, ctypes.c_int32),
                               _p(pauli, ctypes.c_uint8), mode, alpha, alpha_min, alpha_max, eta_unsat, flags,
                               _p(syn_row, ctypes.c_uint32), _p(L0, ctypes.c_double), rounds, _p(G, ctypes.c_float),
                               _p(dev, ctypes.c_double), _p(bnd, ctypes.c_double), _p(flips, ctypes.c_int32))
    if rc != 0:
        raise RuntimeError("oracle_gf4_shadow: bad arguments")
    return dev, bnd, flips
