"""Offline gain sweeps on the fused Monte Carlo engine.

``sms_alpha_sweep`` is the experiment behind the optimised-SMS points of Fig. 3: for each
candidate scale alpha, the frame-error rate of SMS(alpha) at one noise level, estimated
with the protocol of Sec. V (setup) -- frames until a failure target or a frame cap -- and
the alpha with the lowest FER.  Every alpha decodes the same frame sequence (same key),
so the comparison is paired.  ``alpha_star`` (Eq. 9, in the C library) is returned beside
it for reference: Corollary 1 places the ceiling of SAGMS there.
"""
from __future__ import annotations

import math


def sms_alpha_sweep(code, alphas, q, seed=1, target_failures=500, max_shots=20_000_000, max_iter=100, L0=None,
                    batch=1 << 22, dc=None):
    """code: a DeviceCode with logical operators attached.  Returns a dict with one row per
    alpha (alpha, fer, failures, shots, not_converged, logical, mean_iters), the best alpha
    and alpha* of Eq. 9 for the channel prior and the code's largest check degree."""
    from . import Params, _native, llr, mc_run
    prior = llr(q) if L0 is None else float(L0)
    rows = []
    for a in alphas:
        r = mc_run(code, Params(mode="sms", alpha=float(a), max_iter=max_iter), seed, q, L0=prior,
                   target_failures=target_failures, max_shots=max_shots, batch=batch)
        rows.append({"alpha": float(a), "fer": r["failures"] / r["shots"] if r["shots"] else math.nan,
                     "failures": r["failures"], "shots": r["shots"], "not_converged": r["not_converged"],
                     "logical": r["logical"], "mean_iters": r["iters_sum"] / r["shots"] if r["shots"] else math.nan})
    best = min(rows, key=lambda x: (x["fer"], x["alpha"]))
    d = code.dc_max if dc is None else dc
    return {"q": q, "L0": prior, "rows": rows, "best_alpha": best["alpha"],
            "alpha_star": _native.sagms_alpha_star(abs(prior), d)}


def _key(code_name, params, q, L0, seed):
    return {"code": code_name, "mode": params.mode, "alpha": params.alpha, "alpha_min": params.alpha_min,
            "alpha_max": params.alpha_max, "eta_unsat": params.eta_unsat, "max_iter": params.max_iter,
            "flags": params.flags, "q": float(q), "L0": float(L0), "seed": int(seed)}


def mc_run_checkpointed(code, code_name, params, seed, q, checkpoint, L0=None, target_failures=500,
                        max_shots=20_000_000, batch=1 << 22):
    """The Monte Carlo protocol of one noise level with an append-only JSONL checkpoint: after
    every batch one line records the run's identity (code name, parameters, q, L0, seed) and
    its cumulative counts.  Calling again with the same identity resumes from the last line:
    frames are indexed by a counter-based generator, so the continued run is the same frame
    sequence an uninterrupted one would draw.  A record torn by a crash mid-write (a line
    that does not parse) is skipped, so the run resumes from the last complete record; each
    record is flushed to stable storage before the next batch starts.  Returns the counts."""
    import json
    import os
    from . import llr, mc_run
    prior = llr(q) if L0 is None else float(L0)
    key = _key(code_name, params, q, prior, seed)
    counts = None
    if os.path.exists(checkpoint):
        with open(checkpoint) as f:
            for line in f:
                line = line.strip()
                if not line:
                    continue
                try:
                    rec = json.loads(line)
                except json.JSONDecodeError:   # torn by an interrupted write
                    continue
                if all(rec.get(k) == v for k, v in key.items()):
                    counts = {k: rec[k] for k in ("shots", "failures", "not_converged", "logical", "iters_sum")}
    counts = counts or {"shots": 0, "failures": 0, "not_converged": 0, "logical": 0, "iters_sum": 0}
    if os.path.exists(checkpoint) and os.path.getsize(checkpoint) > 0:
        with open(checkpoint, "rb") as f:
            f.seek(-1, os.SEEK_END)
            torn = f.read(1) != b"\n"
        if torn:   # end the torn line, so the next record starts a line of its own
            with open(checkpoint, "a") as f:
                f.write("\n")
    while counts["failures"] < target_failures and counts["shots"] < max_shots:
        counts = mc_run(code, params, seed, q, L0=prior, target_failures=target_failures,
                        max_shots=min(counts["shots"] + batch, max_shots), batch=batch, counts=counts)
        with open(checkpoint, "a") as f:
            f.write(json.dumps({**key, **counts}) + "\n")
            f.flush()
            os.fsync(f.fileno())
    return counts


COUNT_KEYS = ("shots", "failures", "not_converged", "logical", "iters_sum")


def mc_frames(code, params, seed, q, shot0, shots, L0):
    """Counts of frames shot0 .. shot0 + shots - 1 of the on-device generator: sample, decode
    and logical check on the GPU (logicals attached to ``code``)."""
    from . import decode, mc_check, mc_sample
    if shots <= 0:
        return dict.fromkeys(COUNT_KEYS, 0)
    err, syn, l0 = mc_sample(code, seed, q, shot0, shots, L0=L0)
    e_hat, conv, iters = decode(code, syn, l0, params)
    _, counts = mc_check(code, err, e_hat, conv, iters)
    return counts


def mc_run_sharded(code, params, seed, q, L0=None, target_failures=500, max_shots=20_000_000, batch=1 << 22,
                   group=None, frames=None):
    """The Monte Carlo protocol of Sec. V (setup) split across the ranks of a process group
    (one GPU per rank).  In round k rank r decodes frames [(kW + r)B, (kW + r + 1)B) of the
    counter-based generator (W ranks, batch B, clipped at ``max_shots``); one all-reduce then
    sums the five counters, and every rank applies the stopping rule to the sums, so the ranks
    stop together.  The frames decoded are those of a single-process ``mc_run`` with batch W*B
    and the totals equal its counts.  Without an initialised process group this is that run on
    one GPU.  ``frames`` replaces the per-rank batch runner (``mc_frames``)."""
    import torch
    import torch.distributed as dist
    from . import llr
    frames = frames or mc_frames
    on = dist.is_available() and dist.is_initialized()
    world = dist.get_world_size(group) if on else 1
    rank = dist.get_rank(group) if on else 0
    dev = "cuda" if on and dist.get_backend(group) == "nccl" else "cpu"
    prior = llr(q) if L0 is None else float(L0)
    total = dict.fromkeys(COUNT_KEYS, 0)
    k = 0
    while total["failures"] < target_failures and total["shots"] < max_shots:
        s0 = (k * world + rank) * batch
        c = frames(code, params, seed, q, s0, max(0, min(batch, max_shots - s0)), prior)
        t = torch.tensor([int(c[key]) for key in COUNT_KEYS], dtype=torch.int64, device=dev)
        if world > 1:
            dist.all_reduce(t, group=group)
        for key, v in zip(COUNT_KEYS, t.tolist()):
            total[key] += v
        k += 1
    return total
