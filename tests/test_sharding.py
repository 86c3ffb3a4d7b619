"""Shot sharding across ranks (the multi-GPU path: independent shots, no data-path
collective), exercised as world-size-2 gloo process groups on CPU.

Each rank generates its own shard with the bench's per-rank shot offset and decodes it
with the FP64 oracle; the shards must be disjoint slices of the single-process batch, and
the failure / iteration counters summed with one all-reduce must equal the single-process
counters."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SHOTS_PER_RANK = 600


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import oracle
    from paper_2605_10433_gb300 import inputs as I
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    code = I.gb_code(127, 4)
    _, syn, L0, _ = I.workload(code, [0.01, 0.02, 0.04], SHOTS_PER_RANK, seed=31337, shot0=rank * SHOTS_PER_RANK)
    r = oracle.decode_code(code, syn, L0.astype(np.float64), mode=oracle.SAGMS, max_iter=100)
    np.save(os.path.join(outdir, f"syn{rank}.npy"), syn)
    counters = torch.tensor([SHOTS_PER_RANK, int((r["conv"] == 0).sum()), int(r["iters"].sum())], dtype=torch.int64)
    dist.all_reduce(counters)
    if rank == 0:
        np.save(os.path.join(outdir, "counters.npy"), counters.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shards_match_single_process(tmp_path):
    import oracle
    from paper_2605_10433_gb300 import inputs as I
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    code = I.gb_code(127, 4)
    _, syn_all, L0_all, _ = I.workload(code, [0.01, 0.02, 0.04], world * SHOTS_PER_RANK, seed=31337)
    for rank in range(world):
        shard = np.load(os.path.join(tmp_path, f"syn{rank}.npy"))
        assert np.array_equal(shard, syn_all[rank * SHOTS_PER_RANK:(rank + 1) * SHOTS_PER_RANK])
    r = oracle.decode_code(code, syn_all, L0_all.astype(np.float64), mode=oracle.SAGMS, max_iter=100)
    got = np.load(os.path.join(tmp_path, "counters.npy"))
    assert list(got) == [world * SHOTS_PER_RANK, int((r["conv"] == 0).sum()), int(r["iters"].sum())]


def _fake_frames(code, params, seed, q, shot0, shots, L0):
    """Stand-in for the GPU batch runner: counts of frames shot0 .. shot0 + shots - 1 as a
    fixed function of the frame index (a failure every 97 frames, half of them logical)."""
    t = np.arange(shot0, shot0 + max(shots, 0), dtype=np.int64)
    fail = ((t * 7 + seed) % 97) == 0
    logical = fail & (t % 2 == 0)
    return {"shots": int(t.size), "failures": int(fail.sum()), "not_converged": int((fail & ~logical).sum()),
            "logical": int(logical.sum()), "iters_sum": int((1 + t % 3).sum())}


def _mc_rank_main(rank, world, port, outdir, target, max_shots, batch):
    import sys
    sys.path.insert(0, ROOT)
    import json
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2605_10433_gb300 import sweep
    seen = []

    def frames(code, params, seed, q, shot0, shots, L0):
        seen.append([shot0, shots])
        return _fake_frames(code, params, seed, q, shot0, shots, L0)

    total = sweep.mc_run_sharded(None, None, 5, 0.01, target_failures=target, max_shots=max_shots, batch=batch,
                                 frames=frames)
    with open(os.path.join(outdir, f"mc{rank}.json"), "w") as f:
        json.dump({"total": total, "seen": seen}, f)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("target,max_shots", [(40, 10**7), (10**9, 23_000)])
def test_two_rank_monte_carlo_matches_single_process(tmp_path, target, max_shots):
    """The sharded Monte Carlo protocol on two gloo ranks: the ranks decode disjoint frame
    ranges that together are [0, K W B), stop in the same round (failure target or frame cap,
    clipped at the cap), and both end with the counts of one process running the protocol with
    batch W B."""
    import json
    from paper_2605_10433_gb300 import sweep
    world, batch = 2, 1000
    mp.start_processes(_mc_rank_main, args=(world, _free_port(), str(tmp_path), target, max_shots, batch),
                       nprocs=world, join=True, start_method="spawn")
    out = [json.load(open(os.path.join(tmp_path, f"mc{r}.json"))) for r in range(world)]
    ref = dict.fromkeys(sweep.COUNT_KEYS, 0)
    while ref["failures"] < target and ref["shots"] < max_shots:
        c = _fake_frames(None, None, 5, 0.01, ref["shots"], min(world * batch, max_shots - ref["shots"]), 0.0)
        for k in sweep.COUNT_KEYS:
            ref[k] += c[k]
    assert out[0]["total"] == ref and out[1]["total"] == ref
    ranges = sorted((s0, s0 + n) for o in out for s0, n in o["seen"] if n > 0)
    assert ranges[0][0] == 0 and all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
    assert ranges[-1][1] == ref["shots"]


def _mc_failing_rank_main(rank, world, port, outdir, batch):
    """Rank 1's batch runner fails in round 2 and the process dies at once (as after a crash);
    rank 0 records how its own run ended."""
    import sys
    sys.path.insert(0, ROOT)
    import datetime
    import json
    import time
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=20))
    from paper_2605_10433_gb300 import sweep
    calls = []

    def frames(code, params, seed, q, shot0, shots, L0):
        calls.append(shot0)
        if rank == 1 and len(calls) == 2:
            raise RuntimeError("injected batch failure")
        return _fake_frames(code, params, seed, q, shot0, shots, L0)

    t0 = time.monotonic()
    try:
        total = sweep.mc_run_sharded(None, None, 5, 0.01, target_failures=10**9, max_shots=10**6, batch=batch,
                                     frames=frames)
        outcome = {"returned": total}
    except Exception as e:   # recorded for the test, then this rank leaves without further collectives
        outcome = {"error": type(e).__name__, "message": str(e)[:200]}
    outcome["seconds"] = time.monotonic() - t0
    outcome["rounds"] = len(calls)
    with open(os.path.join(outdir, f"fail{rank}.json"), "w") as f:
        json.dump(outcome, f)
    os._exit(3 if rank == 1 else 0)


def test_a_failing_rank_ends_the_sharded_run_on_every_rank(tmp_path):
    """Failure detection without a GPU: when one rank's batch fails and its process dies, the
    other rank learns of it in its next all-reduce and leaves the run with an error in bounded
    time instead of waiting forever or returning partial totals."""
    import json
    world = 2
    ctx = mp.start_processes(_mc_failing_rank_main, args=(world, _free_port(), str(tmp_path), 1000),
                             nprocs=world, join=False, start_method="spawn")
    for p in ctx.processes:
        p.join(120)
    alive = [p.pid for p in ctx.processes if p.is_alive()]
    for p in ctx.processes:
        if p.is_alive():
            p.kill()
    assert not alive, "a rank did not finish"
    assert [p.exitcode for p in ctx.processes] == [0, 3]
    r0 = json.load(open(os.path.join(tmp_path, "fail0.json")))
    r1 = json.load(open(os.path.join(tmp_path, "fail1.json")))
    assert r1["error"] == "RuntimeError" and "injected" in r1["message"] and r1["rounds"] == 2
    assert "error" in r0 and "returned" not in r0 and r0["seconds"] < 60


def test_bench_rank_shards_tile_the_single_process_batch():
    """bench.py's per-rank inputs: the shards of ranks 0 .. W-1 are disjoint, consecutive
    slices of the one-process batch of W times the shots, with the same noise levels."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    from paper_2605_10433_gb300 import inputs as I
    code = I.gb_code(63, 3)
    shots, world = 301, 3
    _, syn_all, L0_all, q_all = I.workload(code, bench.P_VALUES, shots * world, seed=bench.NOISE_SEED)
    for r in range(world):
        _, syn, L0, q = bench.rank_inputs(code, shots, r)
        sl = slice(r * shots, (r + 1) * shots)
        assert np.array_equal(syn, syn_all[sl]) and np.array_equal(L0, L0_all[sl]) and np.array_equal(q, q_all[sl])


def _slowest_rank_main(rank, world, port, outdir):
    import sys
    sys.path.insert(0, ROOT)
    import json
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    got = bench.slowest(100.0 + 37.5 * rank, dist, "cpu")   # each rank's own timed region
    with open(os.path.join(outdir, f"slow{rank}.json"), "w") as f:
        json.dump(got, f)
    dist.barrier()
    dist.destroy_process_group()


def test_bench_reports_the_slowest_rank():
    """bench.py's timing rule on two gloo ranks: every rank ends with the largest of the ranks'
    times (the job's time), and one process keeps its own."""
    import json
    import sys
    import tempfile
    sys.path.insert(0, ROOT)
    import bench
    assert bench.slowest(12.5, None, "cpu") == 12.5
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_slowest_rank_main, args=(2, _free_port(), d), nprocs=2, join=True, start_method="spawn")
        assert [json.load(open(os.path.join(d, f"slow{r}.json"))) for r in range(2)] == [137.5, 137.5]
