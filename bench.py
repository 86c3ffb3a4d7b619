#!/usr/bin/env python3
"""Benchmark: batched SAGMS decoding of the n = 2046 generalized-bicycle code on GB300.

One step = one pass of the whole decode path (gain, check-node, variable-node, decision,
residual syndrome and early stop for every shot, up to 100 iterations) over one batch of
1e7 seeded synthetic shots, already resident in HBM: GB l=1023, w=5 (n=2046, m=1023,
d_c=10, d_v=5, 10230 edges), iid Z flips with p interleaved over {0.005, 0.01, 0.02},
L0 = ln((1-p)/p), SAGMS alpha_min=0.30, alpha_max=0.50, eta=1.10, max_iter=100.

Prints one JSON line (rank 0).  Under torchrun each rank decodes its own 1e7-shot shard on
its own GPU (weak scaling, no data-path collective); the timed region is bracketed by a
barrier and a device synchronize, and the slowest rank's time is reported.

--impl reference times the FP64 CPU oracle (the reference arm of the comparison) on the host
cores, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SAGMS shots/s (n=2046 GB, 100 it) & serving p99 us vs plain launch, FER=oracle"
UNIT = "shots/s"
L, W = 1023, 5
P_VALUES = [0.005, 0.01, 0.02]
SAGMS_KW = dict(alpha_min=0.30, alpha_max=0.50, eta_unsat=1.10)
SMS_ALPHA = 0.75
MAX_ITER = 100
NOISE_SEED = 20260513
PROFILE = os.path.join(ROOT, "profiles", "qc_kernel_gb1023_sagms.md")
KERNEL_SRC = [os.path.join(ROOT, "paper_2605_10433_gb300", "csrc", f)
              for f in ("decode_qc.cuh", "decode_groups.cuh", "decode_slots.cuh", "decode_kernel.cuh", "tmem.cuh")]
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def workload_name(shots):
    return (f"GB l={L} w={W} (n={2 * L}, m={L}, d_c={2 * W}, d_v={W}, {2 * W * L} edges), {shots:.0e} shots/GPU, "
            f"iid Z flips p in {{0.005,0.01,0.02}} interleaved, L0=ln((1-p)/p), SAGMS a_min=0.30 a_max=0.50 "
            f"eta=1.10, max_iter={MAX_ITER}")


def rank_inputs(code, shots, rank):
    """One rank's shard of the workload: shots [rank * shots, (rank + 1) * shots) of the
    seeded batch (weak scaling: every rank decodes its own, disjoint shots).  Returns the
    generator's (err, syn, L0, q) tuple."""
    from paper_2605_10433_gb300 import inputs as I
    return I.workload(code, P_VALUES, shots, seed=NOISE_SEED, shot0=rank * shots)


def slowest(value, dist, device):
    """The largest of the ranks' values (the job ends with its slowest rank): an all-reduce
    MAX over the process group (``dist`` is torch.distributed, or None for one process, which
    returns ``value``).  NCCL groups reduce on ``device`` "cuda", gloo groups on "cpu"."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples every 200 ms during the timed region."""

    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={CLOCK_FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons, power = [], [], set(), []
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, val in zip(names[1:], parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "power_w_max": max(power) if power else None}


def kernel_code(text):
    """Source text without comments and blank lines: what decides the compiled kernel."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = (re.sub(r"//.*$", "", ln).rstrip() for ln in text.splitlines())
    return "\n".join(ln for ln in lines if ln.strip())


def kernel_sha():
    h = hashlib.sha256()
    for f in KERNEL_SRC:
        h.update(kernel_code(open(f).read()).encode())
    return h.hexdigest()[:16]


def profile_traffic(shots_per_launch):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current
    kernel source (else None)."""
    try:
        txt = open(PROFILE).read()
        sha = kernel_sha()
        m_sha = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
        m_b = re.search(r"dram_bytes_per_shot:\s*([0-9.eE+-]+)", txt)
        if not m_sha or not m_b or m_sha.group(1) != sha:
            return None
        return float(m_b.group(1)) * shots_per_launch
    except Exception:
        return None


def bench_mixed_degree(S, I, steps, shots_per_code=1_000_000):
    """Mixed-degree batching: GB l=255 (n=510) with w in {3,4,5,6,8} (check degree 6..16),
    p=0.02, SAGMS max_iter=100, 1e6 shots per code in one CUDA-graph launch of a multi-code
    decode; each code's launch plan autotuned on a 1e5-shot sample first."""
    import torch
    from paper_2605_10433_gb300 import roofline
    p = S.Params(mode="sagms", max_iter=MAX_ITER, **SAGMS_KW)
    jobs, plans, ops = [], {}, []
    for w in (3, 4, 5, 6, 8):
        c = I.gb_code(255, w)
        ops.append(roofline.ops_per_iteration("sagms", c.row_ptr, c.col_idx, c.n))
        _, syn, L0, _ = I.workload(c, [0.02], shots_per_code, seed=NOISE_SEED + w)
        dc = S.DeviceCode.from_code(c)
        d_syn = torch.from_numpy(syn.view(np.int32)).cuda()
        d_L0 = torch.from_numpy(L0).cuda()
        plan, rate = S.autotune(dc, d_syn[:100000], d_L0[:100000], p)
        plans[f"w={w}"] = {**S.decode_plan(plan), "sample_shots_per_s": rate}
        jobs.append(S.Job(dc, d_syn, d_L0, p))
    g = S.Graph(jobs)
    stream = torch.cuda.current_stream()
    for _ in range(2):
        g.launch(stream)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        g.launch(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    total = shots_per_code * len(jobs) * steps
    fer = {f"w={w}": float((j.conv == 0).float().mean().item()) for w, j in zip((3, 4, 5, 6, 8), jobs)}
    iters = {f"w={w}": float(j.iters.float().mean().item()) for w, j in zip((3, 4, 5, 6, 8), jobs)}
    # issue roofline of the whole graph launch: every code's iterations x its ops per iteration
    work = sum(float(j.iters.clamp(min=0).to(torch.int64).sum()) * o for j, o in zip(jobs, ops)) * steps
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    peak = roofline.alu_peak_ops(props.multi_processor_count, float(measured_peaks().get("sm_max_mhz") or 2070.0))
    g.close()
    return {"workload": "GB l=255 (n=510) w in {3,4,5,6,8}, 1e6 shots per code, p=0.02, SAGMS max_iter=100, "
                        "one CUDA-graph launch of sagms_decode_multi per step",
            "shots_per_s": total / (ms / 1e3), "ms_per_launch": ms / steps, "launches": steps,
            "roofline_frac": work / (ms / 1e3) / peak, "plans": plans, "fer_syn": fer, "mean_iters": iters}


def bench_mc(S, I, frames=10_000_000, q=0.01, seed=NOISE_SEED + 1):
    """The fused Monte Carlo engine (sample -> decode -> logical check on the GPU, counters
    back to the host) on the headline code: frames/s of the whole protocol and its FER."""
    from paper_2605_10433_gb300.stats import wilson_interval
    code = I.gb_code(L, W)
    dc = S.DeviceCode.from_code(code)
    logicals = S.x_logicals(code)
    dc.set_logicals(logicals)
    p = S.Params(mode="sagms", max_iter=MAX_ITER, **SAGMS_KW)
    S.mc_run(dc, p, seed, q, target_failures=10**15, max_shots=1 << 20, batch=1 << 20)   # warm-up
    t0 = time.perf_counter()
    r = S.mc_run(dc, p, seed, q, target_failures=10**15, max_shots=frames, batch=1 << 22)
    dt = time.perf_counter() - t0
    lo, hi = wilson_interval(r["failures"], r["shots"])
    return {"workload": f"GB l={L} w={W}, iid Z flips q={q}, L0=ln((1-q)/q), SAGMS max_iter={MAX_ITER}, "
                        f"{frames:.0e} frames in batches of 2^22 (sagms_mc_run)",
            "frames_per_s": r["shots"] / dt, "fer": r["failures"] / r["shots"], "wilson95": [lo, hi],
            "not_converged": r["not_converged"], "logical": r["logical"], "mean_iters": r["iters_sum"] / r["shots"],
            "k_logicals": int(logicals.shape[0])}


def bench_serving(S, I, nreq=3000, load=0.6, seed=5):
    """Serving loop: Poisson-arriving requests from GB codes n in {126, 510, 1022, 2046}
    (w = 3/4/5/5), batch size floor(exp U[ln 1, ln 4096]), p ~ U[0.005, 0.03], SAGMS
    max_iter=100.  Plain per-request launches (one stream, one request at a time) give the
    capacity; the same arrival schedule at `load` x that capacity is then replayed through the
    continuous-batching server and through plain launches.  A sweep replays it at 30, 60, 80 and
    95% of the continuous mode's own capacity (all requests at once) in both modes.  Latency = completion - submit,
    measured by the server's clock, host copies included."""
    import torch
    rng = np.random.default_rng(seed)
    params = S.Params(mode="sagms", max_iter=MAX_ITER, **SAGMS_KW)
    codes = [I.gb_code(l, w) for l, w in ((63, 3), (255, 4), (511, 5), (1023, 5))]
    dcodes = [S.DeviceCode.from_code(c) for c in codes]
    cid = rng.integers(0, len(codes), size=nreq)
    shots = np.floor(np.exp(rng.uniform(0, np.log(4096), size=nreq))).astype(np.int64)
    pv = rng.uniform(0.005, 0.03, size=nreq)
    reqs = []
    for k in range(len(codes)):
        sel = np.nonzero(cid == k)[0]
        tot = int(shots[sel].sum())
        q = np.repeat(pv[sel], shots[sel])
        _, syn = I.sample(codes[k], q, tot, seed=seed * 1000 + k)
        L0 = I.llr_prior(q).astype(np.float32)
        hs = torch.from_numpy(syn.view(np.int32)).pin_memory()
        hl = torch.from_numpy(L0).pin_memory()
        he = torch.empty((tot, dcodes[k].nw), dtype=torch.int32).pin_memory()
        hc = torch.empty(tot, dtype=torch.uint8).pin_memory()
        hi = torch.empty(tot, dtype=torch.int32).pin_memory()
        off = 0
        for i in sel:
            n = int(shots[i])
            reqs.append((int(i), k, (hs[off:off + n], hl[off:off + n], he[off:off + n], hc[off:off + n], hi[off:off + n])))
            off += n
    reqs.sort()
    total = int(shots.sum())

    def run(mode, arrival_ns):
        srv = S.Server(mem_budget=512 << 20, max_inflight=16, mode=mode, shots_per_cta=16)
        ids = [srv.add_code(dc, params) for dc in dcodes]
        tickets = srv.replay([ids[k] for _, k, _ in reqs], [r for _, _, r in reqs], arrival_ns)
        for t in tickets:
            srv.wait(t, 300)
        times = np.array([srv.times(t) for t in tickets], dtype=np.int64)
        srv.close()
        lat_us = (times[:, 1] - times[:, 0]) / 1e3
        span = (times[:, 1].max() - times[:, 0].min()) / 1e9
        return {"p50_us": float(np.percentile(lat_us, 50)), "p99_us": float(np.percentile(lat_us, 99)),
                "mean_us": float(lat_us.mean()), "shots_per_s": total / span}

    burst = np.zeros(nreq, dtype=np.int64)
    run("plain", burst)   # warm-up
    cap = run("plain", burst)["shots_per_s"]
    run("continuous", burst)   # warm-up
    cap_cont = run("continuous", burst)["shots_per_s"]
    gaps = rng.exponential(1.0, size=nreq)   # one Poisson schedule, rescaled to each offered rate

    def schedule(rate_shots):
        rate_req = rate_shots / shots.mean()
        arrival = np.cumsum(gaps / rate_req) * 1e9
        return (arrival - arrival[0]).astype(np.int64)

    arrival = schedule(load * cap)
    cont = run("continuous", arrival)
    plain = run("plain", arrival)
    # the same schedule at fractions of the continuous mode's own capacity, both modes
    sweep = []
    for f in (0.3, 0.6, 0.8, 0.95):
        arr = schedule(f * cap_cont)
        c, pl = run("continuous", arr), run("plain", arr)
        sweep.append({"load_of_continuous_capacity": f, "offered_shots_per_s": f * cap_cont,
                      "continuous": c, "plain": pl, "p99_speedup_vs_plain": pl["p99_us"] / c["p99_us"]})
    return {"workload": f"{nreq} Poisson requests, GB n in {{126,510,1022,2046}}, batch floor(exp U[ln1,ln4096]) "
                        f"(mean {shots.mean():.0f} shots), p~U[0.005,0.03], SAGMS max_iter=100, "
                        f"offered load {load:.0%} of plain-launch capacity",
            "plain_capacity_shots_per_s": cap, "continuous_capacity_shots_per_s": cap_cont,
            "offered_shots_per_s": load * cap,
            "continuous": cont, "plain": plain,
            "p99_speedup_vs_plain": plain["p99_us"] / cont["p99_us"], "sweep": sweep}


def bench_gf4(S, I, steps, shots=1_000_000):
    """The paper's own decoding setting (Sec. II, Sec. V): GF(4) decoding of the overcomplete CSS
    matrix of a GB code with l = 63, w = 5 (m = 126 rows, check and qubit degree 10) under
    depolarising noise at eps = 0.01; SAGMS (0.30, 0.50, 1.10), SMS(0.5) and BP4 with the matched
    prior (eps0 = eps) and SAGMS / BP4 with the mismatched one (eps0 = 0.1): shots/s and FER."""
    import torch
    from paper_2605_10433_gb300 import roofline
    from paper_2605_10433_gb300.inputs import gf4 as I4
    g = I4.css_code(I.gb_code(63, 5))
    dc = S.Gf4DeviceCode(g)
    eps = 0.01
    _, _, syn = I4.depolarizing(g, eps, shots, seed=NOISE_SEED + 4)
    d_syn = torch.from_numpy(syn.view(np.int32)).cuda()
    out = {"workload": f"CSS stack of GB l=63 w=5 ([[126,{g.k}]], m=126, d_c=d_v=10), depolarising eps={eps}, "
                       f"{shots:.0e} shots, max_iter={MAX_ITER}, GF(4) scalar messages",
           "kernel": "gf4_css_kernel<10,5> (column-indexed)" if dc.css_layout else "gf4_kernel<10,10>"}
    runs = [("sagms", S.Params(mode="sagms", max_iter=MAX_ITER, **SAGMS_KW), eps),
            ("sms", S.Params(mode="sms", alpha=0.5, max_iter=MAX_ITER), eps),
            ("bp4", S.Params(mode="bp", max_iter=MAX_ITER), eps),
            ("sagms_mismatch", S.Params(mode="sagms", max_iter=MAX_ITER, **SAGMS_KW), 0.1),
            ("bp4_mismatch", S.Params(mode="bp", max_iter=MAX_ITER), 0.1),
            # the same SAGMS decode on the generic (index-list) kernel, for comparison
            ("sagms_generic_kernel", S.Params(mode="sagms", max_iter=MAX_ITER, flags=S.FLAG_GENERIC_KERNEL, **SAGMS_KW),
             eps)]
    stream = torch.cuda.current_stream()
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    peak = roofline.alu_peak_ops(props.multi_processor_count, float(measured_peaks().get("sm_max_mhz") or 2070.0))
    for name, p, eps0 in runs:
        d_L0 = torch.full((shots,), float(I4.prior(eps0)), dtype=torch.float32, device="cuda")
        S.gf4_decode(dc, d_syn, d_L0, p, stream=stream)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            _, conv, iters = S.gf4_decode(dc, d_syn, d_L0, p, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        ops = roofline.gf4_ops_per_iteration(p.mode, g.row_ptr, g.col_idx, g.n)
        it_sum = float(iters.clamp(min=0).to(torch.int64).sum())
        out[name] = {"eps0": eps0, "shots_per_s": shots / (ms / 1e3), "fer_syn": float((conv == 0).float().mean()),
                     "mean_iters": float(iters.float().mean()), "ops_per_iteration": ops,
                     "roofline_frac": it_sum * ops / (ms / 1e3) / peak}
    dc.close()
    return out


def bench_small_configs(S, I, steps, shots=1_000_000, cpu_shots=20000):
    """Configs 1 and 2: SAGMS (and the other modes on config 2) on GB l=63 w=3 at iid Z flips
    p = 0.05, and on GB l=127 w=4 at depolarising p in {0.01, 0.02, 0.04} marginalised to 2p/3;
    GPU shots/s and FER, and the FP64 oracle's rate on the host cores on a bounded sample."""
    import torch
    import oracle
    threads = os.cpu_count() or 1
    out = {}
    cases = [("config1 GB l=63 w=3 p=0.05", (63, 3), [0.05], 50, ["sagms", "sms", "ms", "bp"]),
             ("config2 GB l=127 w=4 p_dep=0.01,0.02,0.04 (q=2p/3)", (127, 4), [0.01 * 2 / 3, 0.02 * 2 / 3, 0.04 * 2 / 3],
              MAX_ITER, ["sagms", "sms", "ms", "bp"])]
    from paper_2605_10433_gb300 import roofline
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    peak = roofline.alu_peak_ops(props.multi_processor_count, float(measured_peaks().get("sm_max_mhz") or 2070.0))
    stream = torch.cuda.current_stream()
    for name, lw, qs, max_iter, modes in cases:
        code = I.gb_code(*lw)
        dc = S.DeviceCode.from_code(code)
        _, syn, L0, _ = I.workload(code, qs, shots, seed=NOISE_SEED + lw[0])
        d_syn = torch.from_numpy(syn.view(np.int32)).cuda()
        d_L0 = torch.from_numpy(L0).cuda()
        entry = {}
        for mode in modes:
            p = S.Params(mode=mode, alpha=SMS_ALPHA, max_iter=max_iter, **SAGMS_KW)
            err, conv, iters = S.decode(dc, d_syn, d_L0, p, stream=stream)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                S.decode(dc, d_syn, d_L0, p, out=(err, conv, iters), stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            om = {"ms": oracle.MS, "sms": oracle.SMS, "sagms": oracle.SAGMS, "bp": oracle.BP}[mode]
            t0 = time.perf_counter()
            oracle.decode_code(code, syn[:cpu_shots], L0[:cpu_shots].astype(np.float64), mode=om, alpha=SMS_ALPHA,
                               max_iter=max_iter, threads=threads, **SAGMS_KW)
            cpu = cpu_shots / (time.perf_counter() - t0)
            ops = roofline.ops_per_iteration(mode, code.row_ptr, code.col_idx, code.n)
            it_sum = float(iters.clamp(min=0).to(torch.int64).sum())
            entry[mode] = {"shots_per_s": shots / (ms / 1e3), "fer_syn": float((conv == 0).float().mean()),
                           "mean_iters": float(iters.float().mean()), "ops_per_iteration": ops,
                           "roofline_frac": it_sum * ops / (ms / 1e3) / peak, "oracle_shots_per_s": cpu,
                           "oracle_cores": threads, "oracle_sample": cpu_shots}
        out[name] = entry
        dc.close()
    return out


def classify_mismatches(S, code, dcode, syn, L0, params, g_err, g_conv, g_it, o):
    """Per-shot decision parity of the GPU batch against the FP64 oracle on the same shots,
    with the acceptance of the parity tests: every mismatching shot is re-decoded on the GPU
    with its posterior trace and replayed by the oracle's shadow check (each round re-done in
    FP64 from the GPU's own previous posteriors must land within the binary32 rounding bound);
    it is a near-tie when the first differing decision has an oracle posterior |LLR| < 1e-4,
    else amplified.  Returns the counts."""
    import oracle
    import torch
    mode = {"ms": oracle.MS, "sms": oracle.SMS, "sagms": oracle.SAGMS, "bp": oracle.BP}[params.mode]
    kw = dict(mode=mode, alpha=params.alpha, alpha_min=params.alpha_min, alpha_max=params.alpha_max,
              eta_unsat=params.eta_unsat, flags=params.flags)
    same = (g_err == o["err"]).all(axis=1) & (g_conv == o["conv"]) & (g_it == o["iters"])
    bad = np.nonzero(~same)[0]
    near, amp, shadow_fail, worst = 0, 0, 0, 0.0
    n = code.n
    for c0 in range(0, len(bad), 64):
        idx = bad[c0:c0 + 64]
        d_syn = torch.from_numpy(np.ascontiguousarray(syn[idx]).view(np.int32)).cuda()
        d_L0 = torch.from_numpy(np.ascontiguousarray(L0[idx])).cuda()
        _, _, it_t, tr = S.decode(dcode, d_syn, d_L0, params, trace=True)
        torch.cuda.synchronize()
        it_t, tr = it_t.cpu().numpy(), tr.cpu().numpy()
        ot = oracle.decode_code(code, syn[idx], L0[idx].astype(np.float64), max_iter=params.max_iter, trace=True,
                                threads=os.cpu_count() or 1, **{k: v for k, v in kw.items()})
        for k, s in enumerate(idx):
            rounds = int(it_t[k])
            dev, bnd, _ = oracle.shadow_code(code, syn[s], L0[s:s + 1], tr[k], rounds, **kw)
            with np.errstate(divide="ignore", invalid="ignore"):
                ratio = float(np.max(np.where(dev == 0.0, 0.0, np.abs(dev) / bnd)))
            worst = max(worst, ratio)
            if ratio > 1.0 or rounds != int(g_it[s]):
                shadow_fail += 1
                continue
            last = min(rounds, int(ot["iters"][k]))
            for l in range(last + 1):
                diff = np.signbit(tr[k, l, :n]) != (ot["trace"][k, l, :n] < 0)
                if diff.any():
                    scale = abs(float(L0[s])) if params.mode != "bp" else 1.0
                    if float(np.abs(ot["trace"][k, l, :n][diff]).max()) * scale < 1e-4:
                        near += 1
                    else:
                        amp += 1
                    break
    shots = len(same)
    return {"shots": shots, "identical": int(same.sum()), "identical_frac": float(same.mean()),
            "near_tie": near, "near_tie_frac": near / shots, "amplified": amp, "amplified_frac": amp / shots,
            "shadow_failures": shadow_fail, "shadow_worst": worst}


def cpu_oracle_sample(code, syn, L0, shots, threads):
    import oracle
    t0 = time.perf_counter()
    r = oracle.decode_code(code, syn[:shots], L0[:shots].astype(np.float64), mode=oracle.SAGMS,
                           max_iter=MAX_ITER, threads=threads, **SAGMS_KW)
    dt = time.perf_counter() - t0
    return r, dt


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores, on bounded samples of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2605_10433_gb300 import inputs as I
    import oracle
    oracle.build_lib()
    code = I.gb_code(L, W)
    threads = os.cpu_count() or 1
    sample = args.ref_sample
    _, syn, L0, _ = I.workload(code, P_VALUES, sample * (args.steps + args.warmup), seed=NOISE_SEED)
    times = []
    for k in range(args.warmup + args.steps):
        sl = slice(k * sample, (k + 1) * sample)
        _, dt = cpu_oracle_sample(code, syn[sl], L0[sl], sample, threads)
        if k >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = sample * args.steps / total
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(sample) + f" (bounded sample of {sample} shots per step)",
                       "code_seed": code.seed, "a": list(code.a), "b": list(code.b), "k": code.k,
                       "l2": "CPU run"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{sample} shots per step x {args.steps} steps of the same workload"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--shots", type=int, default=10_000_000)
    ap.add_argument("--ref-sample", type=int, default=40000)
    ap.add_argument("--cpu-sample", type=int, default=100000)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--mode-steps", type=int, default=3)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the SMS / MS / BP / layered lines, the other configs and the CPU baseline")
    ap.add_argument("--layered", action="store_true",
                    help="time the layered schedule (SAGMS_FLAG_LAYERED) instead of Algorithm 1's flooding one")
    ap.add_argument("--mode", default="sagms", choices=["sagms", "sms", "ms", "bp"],
                    help="decoder timed (default SAGMS, the headline; the others for profiling)")
    ap.add_argument("--only", default=None, choices=["gf4", "mc", "serving", "mixed", "small"],
                    help="run one secondary workload alone and print its JSON (profiling)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        return run_reference(args)
    if args.only:
        import torch
        import paper_2605_10433_gb300 as S
        from paper_2605_10433_gb300 import inputs as I
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        fn = {"gf4": lambda: bench_gf4(S, I, args.mode_steps, shots=min(args.shots, 1_000_000)),
              "mc": lambda: bench_mc(S, I), "serving": lambda: bench_serving(S, I),
              "mixed": lambda: bench_mixed_degree(S, I, args.mode_steps),
              "small": lambda: bench_small_configs(S, I, args.mode_steps)}[args.only]
        print(json.dumps(fn()))
        return 0

    import torch
    import paper_2605_10433_gb300 as S
    from paper_2605_10433_gb300 import inputs as I
    from paper_2605_10433_gb300 import roofline
    from paper_2605_10433_gb300.stats import wilson_interval

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    code = I.gb_code(L, W)
    shots = args.shots
    t0 = time.perf_counter()
    _, syn, L0, qv = rank_inputs(code, shots, rank)
    gen_s = time.perf_counter() - t0
    dcode = S.DeviceCode.from_code(code)
    d_syn = torch.from_numpy(syn.view(np.int32)).cuda()
    d_L0 = torch.from_numpy(L0).cuda()
    err = torch.empty((shots, code.nw), dtype=torch.int32, device="cuda")
    conv = torch.empty((shots,), dtype=torch.uint8, device="cuda")
    iters = torch.empty((shots,), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    sagms = S.Params(mode=args.mode, alpha=SMS_ALPHA, max_iter=MAX_ITER, flags=S.FLAG_LAYERED if args.layered else 0,
                     **SAGMS_KW)

    def step(p):
        S.decode(dcode, d_syn, d_L0, p, out=(err, conv, iters), stream=stream)

    def timed(p, warm, steps, clocks=False):
        for _ in range(warm):
            step(p)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler() if clocks else None
        if sampler:
            sampler.start()
            time.sleep(0.5)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            step(p)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        clk = sampler.stop() if sampler else None
        barrier()
        return slowest(ms, dist, "cuda"), clk

    ms, clk = timed(sagms, args.warmup, args.steps, clocks=True)
    it_host = iters.cpu().numpy()
    conv_host = conv.cpu().numpy()
    value = shots * world * args.steps / (ms / 1e3)
    ms_step = ms / args.steps

    # roofline: algorithmic ops of this launch over the launch's average duration
    props = torch.cuda.get_device_properties(local)
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz") or (clk or {}).get("sm_max_mhz") or 2070.0)
    ops_it = roofline.ops_per_iteration(args.mode, code.row_ptr, code.col_idx, code.n)
    ops_launch = float(it_host.astype(np.int64).sum()) * ops_it
    achieved = ops_launch / (ms_step / 1e3)
    peak = roofline.alu_peak_ops(props.multi_processor_count, sm_max)
    traffic = None if (args.layered or args.mode != "sagms") else profile_traffic(shots)
    roof = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "Tops/s",
            "frac": achieved / peak, "traffic": traffic,
            "kernel": ("sagms::layered_kernel<10,64>" if args.layered else
                       "sagms::qc_kernel<10,5,2,512,2048,BP>" if args.mode == "bp" else "sagms::qc_kernel<10,5,4>"),
            "note": (f"ops = sum over shots of iters x {ops_it} per iteration (Eq. 15 / Table I CN cost + VN sum, "
                     f"decision, residual XOR, popcount); peak = {props.multi_processor_count} SMs x 128 lanes x "
                     f"{sm_max:.0f} MHz (derived from unit counts and clock); HBM bound "
                     f"{roofline.hbm_bytes_per_shot(code.m, code.n)} B/shot at "
                     + (f"{peaks['hbm_gbs']} GB/s (of measured)" if "hbm_gbs" in peaks else "6800 GB/s (of fallback)")
                     + f" is {(peaks.get('hbm_gbs', 6800.0) * 1e9 / roofline.hbm_bytes_per_shot(code.m, code.n)):.3g} "
                     "shots/s")}
    tmem = "qc_tmem=1" in S._native.sagms_version() and args.mode != "bp" and not args.layered
    smem_b = roofline.smem_bytes(it_host, code.nnz, code.n, old_in_smem=not tmem)
    smem_peak = roofline.smem_peak_bytes(props.multi_processor_count, sm_max)
    roof_smem = {"bound": "smem", "achieved": smem_b / (ms_step / 1e3) / 1e9, "peak": smem_peak / 1e9, "unit": "GB/s",
                 "frac": smem_b / (ms_step / 1e3) / smem_peak,
                 "note": ("diagnostic roof: shared-memory bytes of the flooding schedule per shot of r iterations "
                          + ("(12E r + 4n r: old messages in tensor memory)" if tmem else "(16E r - 4E + 4n r)")
                          + " over SMs x 128 B x clock (derived)")}

    fer = {}
    for k, p in enumerate(P_VALUES):
        sel = np.arange(shots) % len(P_VALUES) == k
        f = int((conv_host[sel] == 0).sum())
        lo, hi = wilson_interval(f, int(sel.sum()))
        fer[str(p)] = {"fer_syn": f / sel.sum(), "wilson95": [lo, hi], "mean_iters": float(it_host[sel].mean())}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": workload_name(shots) + (", layered schedule" if args.layered else "")
                      + ("" if args.mode == "sagms" else f", decoder {args.mode} instead of SAGMS"),
                      "global_batch": shots * world, "code_seed": code.seed,
                      "a": list(code.a), "b": list(code.b), "k": code.k,
                      "l2": f"inputs larger than L2: {syn.nbytes / 1e9:.2f} GB syndromes per GPU",
                      "parallelism": f"shot-sharded x{world}"},
           "gpu_launches": args.steps, "mean_iters": float(it_host.mean()), "fer": fer, "roofline": roof,
           "roofline_smem": None if args.layered else roof_smem,
           "clocks": clk, "input_gen_s": gen_s}

    # e2e: the C-ABI host entry point, host<->device copies inside the timed region
    h_syn = torch.from_numpy(syn.view(np.int32)).pin_memory()
    h_L0 = torch.from_numpy(L0).pin_memory()
    h_err = torch.empty((shots, code.nw), dtype=torch.int32).pin_memory()
    h_conv = torch.empty((shots,), dtype=torch.uint8).pin_memory()
    h_it = torch.empty((shots,), dtype=torch.int32).pin_memory()
    S.decode_host(dcode, h_syn, h_L0, sagms, out=(h_err, h_conv, h_it))
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        S.decode_host(dcode, h_syn, h_L0, sagms, out=(h_err, h_conv, h_it))
    e2e_s = slowest(time.perf_counter() - t0, dist, "cuda")
    assert np.array_equal(h_it.numpy(), it_host), "host path disagrees with the device path"
    out["e2e"] = {"value": shots * world * args.e2e_steps / e2e_s, "unit": UNIT,
                  "h2d_bytes_per_step": int(syn.nbytes + L0.nbytes),
                  "d2h_bytes_per_step": int(shots * code.nw * 4 + shots + shots * 4),
                  "api": "sagms_decode_host (pinned host buffers, chunked copy/compute overlap)"}

    if not args.no_extras:
        modes = {}
        for name, p in (("sms", S.Params(mode="sms", alpha=SMS_ALPHA, max_iter=MAX_ITER)),
                        ("ms", S.Params(mode="ms", max_iter=MAX_ITER)),
                        ("bp", S.Params(mode="bp", max_iter=MAX_ITER)),
                        ("sagms_layered", S.Params(mode="sagms", alpha_min=SAGMS_KW["alpha_min"],
                                                   alpha_max=SAGMS_KW["alpha_max"], eta_unsat=SAGMS_KW["eta_unsat"],
                                                   max_iter=MAX_ITER, flags=S.FLAG_LAYERED))):
            m_ms, _ = timed(p, 1, args.mode_steps)
            cv = conv.cpu().numpy()
            it_m = iters.cpu().numpy()
            ops_m = roofline.ops_per_iteration(p.mode, code.row_ptr, code.col_idx, code.n)
            t_m = m_ms / 1e3 / args.mode_steps
            modes[name] = {"shots_per_s": shots * world * args.mode_steps / (m_ms / 1e3),
                           "mean_iters": float(it_m.mean()), "fer_syn": float((cv == 0).mean()),
                           "roofline_frac": float(it_m.astype(np.int64).sum()) * ops_m / t_m / peak,
                           "ops_per_iteration": ops_m}
        out["modes"] = modes
        step(sagms)
        torch.cuda.synchronize()
        if world == 1:
            # one batch per noise level (same size as the headline batch): shots/s, mean
            # iterations and the issue-roofline fraction of each p on its own
            per_p = {}
            for k, q in enumerate(P_VALUES):
                _, syn_q, L0_q, _ = I.workload(code, [q], shots, seed=NOISE_SEED + 1 + k)
                ds_q = torch.from_numpy(syn_q.view(np.int32)).cuda()
                dl_q = torch.from_numpy(L0_q).cuda()
                for _ in range(args.warmup):
                    S.decode(dcode, ds_q, dl_q, sagms, out=(err, conv, iters), stream=stream)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(args.mode_steps):
                    S.decode(dcode, ds_q, dl_q, sagms, out=(err, conv, iters), stream=stream)
                e1.record(stream)
                torch.cuda.synchronize()
                t_q = e0.elapsed_time(e1) / 1e3 / args.mode_steps
                it_q = iters.cpu().numpy()
                per_p[str(q)] = {"shots_per_s": shots / t_q, "mean_iters": float(it_q.mean()),
                                 "fer_syn": float((conv.cpu().numpy() == 0).mean()),
                                 "roofline_frac": float(it_q.astype(np.int64).sum()) * ops_it / t_q / peak}
                del ds_q, dl_q
            out["per_p"] = per_p
            step(sagms)
            torch.cuda.synchronize()
            out["config3_mixed_degree"] = bench_mixed_degree(S, I, args.mode_steps)
            out["serving"] = bench_serving(S, I)
            out["monte_carlo"] = bench_mc(S, I)
            out["gf4"] = bench_gf4(S, I, args.mode_steps)

    if rank == 0 and world == 1 and not args.no_extras:
        threads = os.cpu_count() or 1
        r, dt = cpu_oracle_sample(code, syn, L0, args.cpu_sample, threads)
        cs = args.cpu_sample
        parity = classify_mismatches(S, code, dcode, syn[:cs], L0[:cs], sagms, err.cpu().numpy().view(np.uint32)[:cs],
                                     conv_host[:cs], it_host[:cs], r)
        out["cpu_baseline"] = {"value": cs / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
                               "sample": f"first {cs} shots of the same batch (FP64 C oracle, {threads} threads)",
                               "oracle_fer_syn": float((r["conv"] == 0).mean()),
                               "gpu_oracle_identical": parity["identical_frac"], "decision_parity": parity}
        one = max(1, args.cpu_sample // 16)
        _, dt1 = cpu_oracle_sample(code, syn, L0, one, 1)
        out["cpu_baseline"]["single_thread"] = {"value": one / dt1, "unit": UNIT, "cores": 1,
                                                "sample": f"first {one} shots, one thread"}
    if rank == 0:
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
