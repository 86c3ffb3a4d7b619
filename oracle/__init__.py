"""FP64 CPU oracle of the SAGMS / SMS / MS / BP decoder (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
import this package.  It shares no code with the CUDA library: the arithmetic lives in
``oracle.c`` (plain C, double precision, explicit per-edge message arrays and direct
leave-one-out loops, following Algorithm 1 with Eqs. 1-8 of the paper), which this module
compiles with gcc and calls through ctypes.

Parity status per function:
* ``decode`` (MS, SMS, SAGMS, BP): pinned by the tests in ``tests/test_oracle_pins.py``
  (tree-code brute force, closed forms at the first iteration, reductions between modes,
  the single-check ratio of Eq. 9, the zero-syndrome case).
* ``decode`` with FLAG_LAYERED (the layered schedule, not used by the paper): pinned by
  ``tests/test_layered_oracle.py`` (tree-code brute force, a hand-worked example, the
  first-fit layering on a hand-drawn graph, single-layer codes, information speed on
  a chain).
* ``alpha_star`` / ``alpha_star_approx``: pinned to the values the paper prints (Sec. V).
* ``shadow`` (acceptance machinery, not the method): pinned by ``tests/test_shadow.py`` -- the
  oracle's own trajectories replay with zero deviation, a plain binary32 decoder written in
  the test passes its bound, and planted mistakes in that decoder (Eqs. 1-8) exceed it.
* The pins themselves are checked by ``tests/test_oracle_mutants.py``: mistakes planted in a
  copy of ``oracle.c`` (one per case, across Eqs. 1-8, Algorithm 1, the readings, the
  automatic ceiling and the layered schedule) must each make a pin fail.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

MS, SMS, SAGMS, BP = 0, 1, 2, 3
FLAG_L0_PER_QUBIT = 1
FLAG_NO_EARLY_STOP = 2
FLAG_NATURAL_UNITS = 8
FLAG_AUTO_CEILING = 16
FLAG_LAYERED = 32
FLAG_PERTURB = 64        # test acceptance only: FP32 rounding model (oracle.c)
FLAG_PERTURB_NEG = 128   # its mirror image

MSFAM_CLIP = 1.0e6
BP_CLIP = 23.718998

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


# Compiler flags of the checker (portable: the same source builds on x86 and Arm hosts).
CFLAGS = ["-O2", "-std=c99", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off"]


def build_lib(force: bool = False) -> str:
    """Compile oracle.c.  With ORACLE_LIB_OVERRIDE set (tests that plant mistakes in a copy
    of oracle.c and check that the pins fail), that prebuilt library is used instead."""
    override = os.environ.get("ORACLE_LIB_OVERRIDE")
    if override:
        return override
    src = os.path.join(_HERE, "oracle.c")
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
        lib.oracle_decode.argtypes = [ctypes.c_int, ctypes.c_int, P(ctypes.c_int32), P(ctypes.c_int32),
                                      ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_int, ctypes.c_uint, ctypes.c_int64,
                                      P(ctypes.c_uint32), P(ctypes.c_double), P(ctypes.c_uint32),
                                      P(ctypes.c_uint8), P(ctypes.c_int32), P(ctypes.c_double),
                                      P(ctypes.c_double), P(ctypes.c_int64)]
        lib.oracle_decode.restype = ctypes.c_int
        lib.oracle_shadow.argtypes = [ctypes.c_int, ctypes.c_int, P(ctypes.c_int32), P(ctypes.c_int32), ctypes.c_int,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_uint, P(ctypes.c_uint32), P(ctypes.c_double), ctypes.c_int,
                                      P(ctypes.c_float), P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_int32)]
        lib.oracle_shadow.restype = ctypes.c_int
        lib.oracle_alpha_star.argtypes = [ctypes.c_double, ctypes.c_int]
        lib.oracle_alpha_star.restype = ctypes.c_double
        lib.oracle_alpha_star_approx.argtypes = [ctypes.c_double, ctypes.c_int]
        lib.oracle_alpha_star_approx.restype = ctypes.c_double
        _lib = lib
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct)) if a is not None else None


def decode(m, n, row_ptr, col_idx, syn, L0, mode=SAGMS, alpha=0.75, alpha_min=0.30, alpha_max=0.50,
           eta_unsat=1.10, max_iter=100, flags=0, trace=False, threads=1):
    """Decode packed syndromes ``syn`` [shots][ceil(m/32)].

    ``L0``: [shots] per-shot prior, or [n] with FLAG_L0_PER_QUBIT.  Returns a dict with
    ``err`` [shots][ceil(n/32)] uint32, ``conv`` [shots] uint8, ``iters`` [shots] int32,
    ``clips`` [shots] int64 (check-node outputs the clip bound) and,
    with ``trace=True``, ``trace`` [shots][max_iter+1][n] float64 posteriors (units the
    decoder runs in: L0-normalised for the MS family with a per-shot prior) and ``scale``
    (same shape): |L0_j| + sum of |messages| into qubit j, the size of P_j's terms."""
    lib = _load()
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
    syn = np.ascontiguousarray(syn, dtype=np.uint32).reshape(-1, (m + 31) // 32)
    shots = syn.shape[0]
    L0 = np.ascontiguousarray(L0, dtype=np.float64).reshape(-1)
    per_qubit = bool(flags & FLAG_L0_PER_QUBIT)
    if per_qubit and L0.shape[0] != n:
        raise ValueError("per-qubit L0 must have n entries")
    if not per_qubit and L0.shape[0] != shots:
        raise ValueError("per-shot L0 must have one entry per shot")
    nw = (n + 31) // 32
    err = np.zeros((shots, nw), dtype=np.uint32)
    conv = np.zeros(shots, dtype=np.uint8)
    iters = np.zeros(shots, dtype=np.int32)
    clips = np.zeros(shots, dtype=np.int64)
    tr = np.zeros((shots, max_iter + 1, n), dtype=np.float64) if trace else None
    sc = np.zeros((shots, max_iter + 1, n), dtype=np.float64) if trace else None

    def run(lo, hi):
        if hi <= lo:
            return
        Ls = L0 if per_qubit else L0[lo:hi]
        rc = lib.oracle_decode(m, n, _p(row_ptr, ctypes.c_int32), _p(col_idx, ctypes.c_int32), mode,
                               alpha, alpha_min, alpha_max, eta_unsat, max_iter, flags, hi - lo,
                               _p(syn[lo:hi], ctypes.c_uint32), _p(np.ascontiguousarray(Ls), ctypes.c_double),
                               _p(err[lo:hi], ctypes.c_uint32), _p(conv[lo:hi], ctypes.c_uint8),
                               _p(iters[lo:hi], ctypes.c_int32), _p(tr[lo:hi] if tr is not None else None, ctypes.c_double),
                               _p(sc[lo:hi] if sc is not None else None, ctypes.c_double),
                               _p(clips[lo:hi], ctypes.c_int64))
        if rc != 0:
            raise RuntimeError("oracle_decode: bad arguments")

    threads = max(1, int(threads))
    if threads == 1 or shots < 2 * threads:
        run(0, shots)
    else:
        bounds = np.linspace(0, shots, threads + 1).astype(int)
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(lambda k: run(bounds[k], bounds[k + 1]), range(threads)))
    out = {"err": err, "conv": conv, "iters": iters, "clips": clips}
    if tr is not None:
        out["trace"] = tr
        out["scale"] = sc
    return out


def decode_code(code, syn, L0, **kw):
    return decode(code.m, code.n, code.row_ptr, code.col_idx, syn, L0, **kw)


def shadow(m, n, row_ptr, col_idx, syn, L0, G, rounds, mode=SAGMS, alpha=0.75, alpha_min=0.30, alpha_max=0.50,
           eta_unsat=1.10, flags=0):
    """Replay one shot's flooding rounds from another implementation's binary32 posterior
    trace ``G`` [>= rounds+1][n] (rows 0..rounds) and bound its rounding (oracle.c,
    ``oracle_shadow``; test acceptance only).  ``syn``: one packed row; ``L0``: the shot's prior
    (one value) or [n] with FLAG_L0_PER_QUBIT.  Returns (dev, bnd, flips): dev[l][j] =
    G_l(j) minus the FP64 step applied to G_{l-1}, bnd the binary32 rounding bound on |dev|,
    flips[l] the qubits whose G_l sign differs from that step's sign."""
    lib = _load()
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
    syn = np.ascontiguousarray(syn, dtype=np.uint32).reshape(-1)
    L0 = np.ascontiguousarray(L0, dtype=np.float64).reshape(-1)
    G = np.ascontiguousarray(np.asarray(G, dtype=np.float32)[:rounds + 1]).reshape(rounds + 1, n)
    dev = np.zeros((rounds + 1, n), dtype=np.float64)
    bnd = np.zeros((rounds + 1, n), dtype=np.float64)
    flips = np.zeros(rounds + 1, dtype=np.int32)
    rc = lib.oracle_shadow(m, n, _p(row_ptr, ctypes.c_int32), _p(col_idx, ctypes.c_int32), mode, alpha, alpha_min,
                           alpha_max, eta_unsat, flags, _p(syn, ctypes.c_uint32), _p(L0, ctypes.c_double), rounds,
                           _p(G, ctypes.c_float), _p(dev, ctypes.c_double), _p(bnd, ctypes.c_double),
                           _p(flips, ctypes.c_int32))
    if rc != 0:
        raise RuntimeError("oracle_shadow: bad arguments")
    return dev, bnd, flips


def shadow_code(code, syn, L0, G, rounds, **kw):
    return shadow(code.m, code.n, code.row_ptr, code.col_idx, syn, L0, G, rounds, **kw)


def alpha_star(L0: float, dc: int) -> float:
    """Eq. 9, exact form."""
    return _load().oracle_alpha_star(float(L0), int(dc))


def alpha_star_approx(L0: float, dc: int) -> float:
    """Eq. 9, first-order form 1 - ln(dc - 1)/L0."""
    return _load().oracle_alpha_star_approx(float(L0), int(dc))
