"""Build libsagms.so (CUDA, sm_103a) in-tree with nvcc.

The library is compiled for sm_103a only (``-gencode arch=compute_103a,code=sm_103a``),
without fast-math, so the BP rule's log1pf / expm1f are the accurate library functions.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libsagms.so")
SOURCES = [os.path.join(HERE, "csrc", f)
           for f in ("kernels_qc_large.cu", "kernels_qc_small.cu", "kernels_qc_bp.cu", "kernels_slots.cu", "kernels_generic.cu",
                     "kernels_layered.cu", "sagms.cu",
                     "server.cu", "mc.cu", "gf4.cu")]
DEPS = SOURCES + [os.path.join(HERE, "csrc", f) for f in os.listdir(os.path.join(HERE, "csrc"))] + \
    [os.path.join(ROOT, "include", "sagms.h")]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsagms.so")
    return cand


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in DEPS if os.path.exists(p))


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    """Compile every translation unit to an object in parallel, then link the library."""
    if not force and not stale():
        return LIB
    from concurrent.futures import ThreadPoolExecutor
    tag = f".tmp{os.getpid()}"
    flags = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
             *extra]
    if verbose:
        flags.insert(0, "-Xptxas=-v")
    objs = [os.path.join(HERE, "csrc", os.path.basename(src) + tag + ".o") for src in SOURCES]

    def compile_one(args):
        src, obj = args
        cmd = [nvcc(), *flags, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        return subprocess.run(cmd, capture_output=True, text=True)

    try:
        with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
            results = list(ex.map(compile_one, zip(SOURCES, objs)))
        for r in results:
            sys.stderr.write(r.stdout + r.stderr)
        failed = [src for src, r in zip(SOURCES, results) if r.returncode != 0]
        if failed:
            raise RuntimeError(f"nvcc failed for {', '.join(os.path.basename(f) for f in failed)}")
        tmp = LIB + tag
        subprocess.check_call([nvcc(), *ARCH, "-shared", *objs, "-o", tmp])
        os.replace(tmp, LIB)
    finally:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose="-v" in sys.argv)
