"""Serving loop (continuous batching) on the GPU: every request's result is the same alone
and in the mix, admission is gated by the memory budget, and host-side failures (cancelled
and malformed requests, timeouts) leave the server serving."""
import numpy as np
import pytest
import torch

import paper_2605_10433_gb300 as S
from paper_2605_10433_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def codes():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out = []
    for l, w in [(63, 3), (255, 4), (511, 5), (1023, 5)]:
        c = I.gb_code(l, w)
        out.append((c, S.DeviceCode.from_code(c)))
    return out


def make_requests(codes, n, seed, max_shots=2048):
    rng = np.random.default_rng(seed)
    reqs = []
    for k in range(n):
        ci = int(rng.integers(0, len(codes)))
        c, dc = codes[ci]
        shots = int(np.floor(np.exp(rng.uniform(0, np.log(max_shots)))))
        p = float(rng.uniform(0.005, 0.03))
        _, syn, L0, _ = I.workload(c, [p], shots, seed=10_000 * seed + k)
        hs = torch.from_numpy(syn.view(np.int32)).pin_memory()
        hl = torch.from_numpy(L0).pin_memory()
        out = (torch.empty((shots, dc.nw), dtype=torch.int32).pin_memory(), torch.empty(shots, dtype=torch.uint8).pin_memory(),
               torch.empty(shots, dtype=torch.int32).pin_memory())
        reqs.append((ci, hs, hl, out))
    return reqs


def alone(codes, ci, hs, hl, params):
    dc = codes[ci][1]
    out = S.decode(dc, hs.cuda(), hl.cuda(), params)
    torch.cuda.synchronize()
    return [t.cpu() for t in out]


@pytest.mark.parametrize("mode", ["continuous", "plain"])
def test_each_result_is_the_same_alone_and_in_the_mix(codes, mode):
    params = S.Params(mode="sagms", max_iter=100)
    srv = S.Server(mem_budget=64 << 20, max_inflight=8, mode=mode, shots_per_cta=16)
    ids = [srv.add_code(dc, params) for _, dc in codes]
    reqs = make_requests(codes, 60, seed=1)
    tickets = [srv.submit(ids[ci], hs, hl, *out) for ci, hs, hl, out in reqs]
    for t in tickets:
        srv.wait(t, 120)
    for (ci, hs, hl, out), t in zip(reqs, tickets):
        ref = alone(codes, ci, hs, hl, params)
        for a, b in zip(out, ref):
            assert torch.equal(a, b)
        s_ns, d_ns = srv.times(t)
        assert d_ns >= s_ns > 0
        assert srv.release(t) == 0
    srv.close()


def test_admission_waits_for_memory_and_rejects_oversized_requests(codes):
    params = S.Params(mode="sagms")
    c, dc = codes[3]
    # budget for about one 2000-shot request of the n=2046 code at a time
    srv = S.Server(mem_budget=1 << 20, max_inflight=8, mode="continuous")
    cid = srv.add_code(dc, params)
    reqs = []
    for k in range(6):
        _, syn, L0, _ = I.workload(c, [0.01], 2000, seed=500 + k)
        reqs.append((torch.from_numpy(syn.view(np.int32)).pin_memory(), torch.from_numpy(L0).pin_memory(),
                     torch.empty((2000, dc.nw), dtype=torch.int32).pin_memory(),
                     torch.empty(2000, dtype=torch.uint8).pin_memory(), torch.empty(2000, dtype=torch.int32).pin_memory()))
    tickets = [srv.submit(cid, *r) for r in reqs]
    # the last request cannot be admitted before the ones ahead of it free the arena
    assert srv.poll(tickets[-1], 0) in (-7, 0)
    for t in tickets:
        srv.wait(t, 60)
    for r in reqs:
        ref = alone(codes, 3, r[0], r[1], params)
        assert all(torch.equal(a, b) for a, b in zip(r[2:], ref))
    big = 200000
    _, syn, L0, _ = I.workload(c, [0.01], big, seed=9)
    with pytest.raises(S._native.SagmsError) as ei:
        srv.submit(cid, syn.view(np.int32), L0, np.empty((big, dc.nw), np.int32), np.empty(big, np.uint8),
                   np.empty(big, np.int32))
    assert ei.value.code == -9
    srv.close()


def test_cancel_malformed_requests_and_timeouts_leave_the_server_serving(codes):
    params = S.Params(mode="sagms")
    c, dc = codes[3]
    srv = S.Server(mem_budget=4 << 20, max_inflight=1, mode="continuous")
    cid = srv.add_code(dc, params)

    def req(shots, seed):
        _, syn, L0, _ = I.workload(c, [0.02], shots, seed=seed)
        return (torch.from_numpy(syn.view(np.int32)).pin_memory(), torch.from_numpy(L0).pin_memory(),
                torch.empty((shots, dc.nw), dtype=torch.int32).pin_memory(),
                torch.empty(shots, dtype=torch.uint8).pin_memory(), torch.empty(shots, dtype=torch.int32).pin_memory())

    first = req(10000, 1)
    queued = [req(500, 2 + k) for k in range(3)]
    t_first = srv.submit(cid, *first)
    t_q = [srv.submit(cid, *r) for r in queued]
    # one request on the GPU at a time: the queued ones cannot have finished yet
    assert srv.poll(t_q[-1], 0) == -7
    assert srv.cancel(t_q[1]) == 0
    assert srv.poll(t_q[1], 1000) == -10            # cancelled
    assert srv.release(t_q[1]) == 0                 # released while its turn is still ahead
    # malformed requests mid-stream are refused on the host and change nothing
    bad = req(10, 99)
    with pytest.raises(S._native.SagmsError):
        srv.submit(cid + 7, *bad)                     # unknown code
    with pytest.raises(S._native.SagmsError):
        srv.submit(cid, bad[0][:0], bad[1][:0], *bad[2:])   # zero shots
    for t in [t_first, t_q[0], t_q[2]]:
        srv.wait(t, 60)
    for r in [first, queued[0], queued[2]]:
        ref = alone(codes, 3, r[0], r[1], params)
        assert all(torch.equal(a, b) for a, b in zip(r[2:], ref))
    srv.close()
