"""One code handle shared by several host threads, each decoding on its own CUDA stream
(the handle's launch plan is immutable apart from the atomic sagms_set_plan): every
thread's results must equal the serial decode of the same batch, bit for bit, while
another thread keeps switching the plan among the kernels (results do not depend on it)."""
import threading

import numpy as np
import pytest
import torch

import paper_2605_10433_gb300 as S
from paper_2605_10433_gb300 import _native
from paper_2605_10433_gb300 import inputs as I
from tests import gpu_helpers as G

pytestmark = pytest.mark.gpu

PARAMS = [
    S.Params(mode="sagms", alpha_min=0.30, alpha_max=0.50, eta_unsat=1.10, max_iter=60),
    S.Params(mode="ms", max_iter=60),
    S.Params(mode="sms", alpha=0.75, max_iter=60),
    S.Params(mode="sagms", alpha_min=0.30, alpha_max=0.50, eta_unsat=1.10, max_iter=60, flags=S.FLAG_LAYERED),
    S.Params(mode="bp", max_iter=40),
    S.Params(mode="sagms", alpha_min=0.30, alpha_max=0.50, eta_unsat=1.10, max_iter=60, flags=S.FLAG_AUTO_CEILING),
]


@pytest.fixture(scope="module", autouse=True)
def dev_check():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("lw", [(255, 5), (1023, 5)])
def test_threads_and_streams_share_a_code_handle(lw):
    c = I.gb_code(*lw)
    dc = S.DeviceCode.from_code(c)
    jobs = []
    for k, p in enumerate(PARAMS):
        _, syn, L0, _ = I.workload(c, [0.005, 0.02, 0.05], 6000 + 37 * k, seed=900 + k)
        jobs.append((p, syn, L0, G.gpu_decode(dc, syn, L0, p)))
    errors = []
    stop = threading.Event()

    def worker(k):
        try:
            torch.cuda.set_device(0)
            p, syn, L0, ref = jobs[k]
            st = torch.cuda.Stream()
            d_syn = torch.from_numpy(np.ascontiguousarray(syn).view(np.int32)).cuda()
            d_L0 = torch.from_numpy(np.ascontiguousarray(L0, dtype=np.float32)).cuda()
            torch.cuda.synchronize()
            for _ in range(4):
                err, conv, iters = S.decode(dc, d_syn, d_L0, p, stream=st)[:3]
                st.synchronize()
                assert np.array_equal(err.cpu().numpy().view(np.uint32), ref["err"]), k
                assert np.array_equal(conv.cpu().numpy(), ref["conv"]), k
                assert np.array_equal(iters.cpu().numpy(), ref["iters"]), k
        except Exception as e:   # reported by the main thread
            errors.append(e)

    def planner():
        kernels = (0, 4, 3, 2, 1)
        k = 0
        while not stop.is_set():
            _native.sagms_set_plan(dc.handle, kernels[k % len(kernels)])
            k += 1
            stop.wait(0.002)

    threads = [threading.Thread(target=worker, args=(k,)) for k in range(len(jobs))]
    pt = threading.Thread(target=planner)
    pt.start()
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    stop.set()
    pt.join(timeout=30)
    assert not any(t.is_alive() for t in threads)
    if errors:
        raise errors[0]
