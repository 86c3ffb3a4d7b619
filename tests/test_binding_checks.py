"""The Python binding refuses buffers whose dtype, shape, layout or memory space does not
match the code before any pointer reaches the library (a wrong shape would let a kernel or
a copy run past a buffer's end).  Host logic only: a stand-in code object, CPU tensors and
numpy arrays."""
from types import SimpleNamespace

import numpy as np
import pytest
import torch

import paper_2605_10433_gb300 as S

CODE = SimpleNamespace(m=63, n=126, mw=2, nw=4, device=0)


def host_bufs(shots=5, per_qubit=False, lib="numpy"):
    syn = np.zeros((shots, CODE.mw), np.uint32)
    L0 = np.ones(CODE.n if per_qubit else shots, np.float32)
    err = np.zeros((shots, CODE.nw), np.int32)
    conv = np.zeros(shots, np.uint8)
    iters = np.zeros(shots, np.int32)
    bufs = [syn, L0, err, conv, iters]
    return [torch.from_numpy(b) for b in bufs] if lib == "torch" else bufs


def check(bufs, flags=0, host=True):
    return S._check_buffers(CODE, S.Params(flags=flags), tuple(bufs), host=host)


@pytest.mark.parametrize("lib", ["numpy", "torch"])
def test_matching_host_buffers_pass(lib):
    assert check(host_bufs(lib=lib)) == 5
    assert check(host_bufs(per_qubit=True, lib=lib), flags=S.FLAG_L0_PER_QUBIT) == 5
    assert check(host_bufs(shots=0, lib=lib)) == 0


def test_outputs_may_be_longer_than_the_batch():
    b = host_bufs(shots=5)
    b[0], b[1] = b[0][:3], b[1][:3]          # three shots into five-row outputs
    assert check(b) == 3
    b = host_bufs(shots=5)
    b[0], b[1] = b[0][:0], b[1][:0]          # zero shots: left to the library to refuse
    assert check(b) == 0


@pytest.mark.parametrize("k,bad,exc", [
    (0, np.zeros((5, 3), np.uint32), ValueError),            # syndrome row width != ceil(m/32)
    (0, np.zeros(10, np.uint32), ValueError),                # flat syndromes
    (0, np.zeros((5, 2), np.uint64), TypeError),             # 8-byte words
    (1, np.ones(4, np.float32), ValueError),                 # fewer priors than shots
    (1, np.ones(5, np.float64), TypeError),                  # FP64 priors
    (1, np.ones(CODE.n, np.float32), ValueError),            # per-qubit length without the flag
    (2, np.zeros((5, 3), np.int32), ValueError),             # err row width != ceil(n/32)
    (2, np.zeros((4, 4), np.int32), ValueError),             # err shorter than the batch
    (2, np.zeros((5, 4), np.float32), TypeError),            # float err
    (3, np.zeros(4, np.uint8), ValueError),                  # conv shorter than the batch
    (3, np.zeros(5, np.int32), TypeError),                   # 4-byte conv
    (4, np.zeros(5, np.int64), TypeError),                   # 8-byte iters
    (4, np.zeros(5, np.uint32), TypeError),                  # unsigned iters
    (4, np.zeros((5, 2), np.int32)[:, 0], ValueError),       # strided view
])
def test_mismatched_buffers_are_refused(k, bad, exc):
    b = host_bufs()
    b[k] = bad
    with pytest.raises(exc):
        check(b)


def test_per_qubit_flag_wants_one_prior_per_qubit():
    b = host_bufs(shots=CODE.n - 1)
    with pytest.raises(ValueError):
        check(b, flags=S.FLAG_L0_PER_QUBIT)     # shots priors, but the flag wants n


def test_memory_space_is_checked():
    with pytest.raises(ValueError):
        check(host_bufs(lib="torch"), host=False)      # CPU tensors on the device path
    with pytest.raises(TypeError):
        b = host_bufs(lib="torch")
        b[1] = b[1].to(torch.bfloat16)
        check(b)
