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
