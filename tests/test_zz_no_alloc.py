"""sagms_decode_noalloc: decoding for callers that cannot allocate device memory.

Serving threads with latency budgets, processes confined to a device-memory budget fixed
at start-up, and frameworks that own every allocation cannot let the decoder call
cudaMalloc (or grow a cudaMallocAsync pool) per batch.  The no-allocation entry point
takes its only scratch -- the shot counters the two-slot kernel claims shots from -- from
a fixed array in the library's device memory.  These tests call it through the C ABI and
check that it returns exactly what sagms_decode returns, on two calls in a row (the
array keeps the previous call's counters, so the second call checks that each call
resets what it uses).

A launch limit (sagms_set_launch_limit) splits a call into several launches, so the
fixed counters beyond the first are exercised as well.

This file is collected last so that a run stopping at the first failure has already run
every other test."""
import ctypes

import numpy as np
import pytest
import torch

import paper_2605_10433_gb300 as S
from paper_2605_10433_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _noalloc(native, dcode, params, d_syn, d_L0, shots, stream):
    err = torch.full((shots, dcode.nw), -1, dtype=torch.int32, device="cuda")
    conv = torch.full((shots,), 7, dtype=torch.uint8, device="cuda")
    iters = torch.full((shots,), -5, dtype=torch.int32, device="cuda")
    rc = native.lib().sagms_decode_noalloc(dcode.handle, ctypes.byref(params), shots, d_syn.data_ptr(),
                                           d_L0.data_ptr(), err.data_ptr(), conv.data_ptr(), iters.data_ptr(),
                                           ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0, native.sagms_last_error_string()
    return err, conv, iters


@pytest.mark.parametrize("lw,mode", [((1023, 5), "sagms"), ((63, 3), "sms"), ((255, 8), "ms"), ((127, 4), "bp")])
def test_noalloc_matches_decode_on_two_calls(lw, mode):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_10433_gb300 import _native
    code = I.gb_code(*lw)
    dcode = S.DeviceCode.from_code(code)
    shots = 20011
    _, syn, L0, _ = I.workload(code, [0.01, 0.02, 0.05], shots, seed=4242 + lw[0])
    d_syn = torch.from_numpy(syn.view(np.int32)).cuda()
    d_L0 = torch.from_numpy(L0).cuda()
    params = S.Params(mode=mode, max_iter=100)
    stream = torch.cuda.current_stream()
    ref = S.decode(dcode, d_syn, d_L0, params, stream=stream)
    torch.cuda.synchronize()
    for _ in range(2):
        out = _noalloc(_native, dcode, params.to_c(), d_syn, d_L0, shots, stream)
        torch.cuda.synchronize()
        # same kernel, same arithmetic: identical results (the tests' tolerance for the MS
        # family's two kernels is bitwise identity, and BP runs the same kernel either way)
        for a, b in zip(out, ref):
            assert torch.equal(a, b)


@pytest.mark.parametrize("lw,mode", [((1023, 5), "sagms"), ((255, 5), "sms")])
def test_noalloc_split_over_several_counters(lw, mode):
    """A launch limit below the batch splits each call into several launches, so the call
    uses fixed counters 0..k (one per launch), each reset before its launch: the results
    must still equal sagms_decode's single launch, on two calls in a row."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_10433_gb300 import _native
    code = I.gb_code(*lw)
    dcode = S.DeviceCode.from_code(code)
    shots = 20011
    _, syn, L0, _ = I.workload(code, [0.01, 0.02], shots, seed=777 + lw[0])
    d_syn = torch.from_numpy(syn.view(np.int32)).cuda()
    d_L0 = torch.from_numpy(L0).cuda()
    params = S.Params(mode=mode, max_iter=100)
    stream = torch.cuda.current_stream()
    ref = S.decode(dcode, d_syn, d_L0, params, stream=stream)   # one launch
    torch.cuda.synchronize()
    try:
        _native.sagms_set_launch_limit(dcode.handle, 5003)          # four launches: counters 0..3
        for _ in range(2):
            out = _noalloc(_native, dcode, params.to_c(), d_syn, d_L0, shots, stream)
            torch.cuda.synchronize()
            for a, b in zip(out, ref):
                assert torch.equal(a, b)
    finally:
        _native.sagms_set_launch_limit(dcode.handle, 0)


def test_noalloc_rejects_batches_beyond_the_fixed_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_10433_gb300 import _native
    code = I.gb_code(63, 3)
    dcode = S.DeviceCode.from_code(code)
    params = S.Params(mode="sagms").to_c()
    too_many = 64 * (2 ** 31 - 1) + 1
    dummy = torch.zeros(16, dtype=torch.int32, device="cuda")
    # d_err is deliberately misaligned: should the size check ever stop refusing first, the
    # launcher's host-side alignment check still refuses the call before any launch.
    rc = _native.lib().sagms_decode_noalloc(dcode.handle, ctypes.byref(params), too_many, dummy.data_ptr(),
                                            dummy.data_ptr(), dummy.data_ptr() + 2, dummy.data_ptr(),
                                            dummy.data_ptr(), None)
    assert rc == -9 and "fixed scratch" in _native.sagms_last_error_string()
