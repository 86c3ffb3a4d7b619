"""Shared helpers of the GPU parity tests: run the CUDA path and the FP64 oracle on the
same seeded shots and compare them element by element.

Acceptance (the tolerances of the decoder's specification, with the readings below):
* Per-shot outputs (e_hat, conv, iters) identical to the oracle's.  Every shot whose outputs
  differ is re-decoded on the GPU with its posterior trace, and:
  - the traced run must reproduce the batch run's outputs, and the outputs must be the ones
    the trace implies (e_hat = the sign bits of the last posteriors, conv = a zero residual,
    iters = the first round with a zero residual under early stop);
  - the shadow replay (``oracle.shadow``) must accept the trace: every round of it, re-done in
    FP64 from the GPU's own previous posteriors, lands within the first-order binary32
    rounding bound of the GPU's posteriors.  The replay is a perturbed FP64 run of the method
    (perturbed by at most that bound per round) whose outcome is the GPU's outcome;
  - the shot is then classified at its first divergent check from the free-running FP64 run:
    a near-tie when every differing bit has an oracle posterior |LLR| < 1e-4 (counted against
    the 0.01% of ``min_frac``), else amplified (rounding differences of earlier rounds grown
    through the loopy graph until a decision differs).  Amplified shots are capped per
    workload by ``max_amplified`` (a fraction of the shots), the measured values recorded in
    the design notes.
* Posteriors: normwise relative error max_j |g_j - o_j| / max(max_j |o_j|, 1) <= 1e-5 at
  every check up to the shot's conditioning horizon (the last check at which an FP32-level
  perturbation of priors and gains moves the FP64 posteriors by <= 1e-6 normwise) and before
  any hard-decision divergence; past the horizon every traced shot must pass the shadow
  replay.  Normwise, because a posterior is a sum of d_v + 1 messages and the rounding error
  of a sum scales with the size of its terms, not with a result that may cancel to near zero.
MS in L0-normalised units is integer-valued: it must match exactly, with no exemption.
"""
import os

import numpy as np
import torch

import oracle
import paper_2605_10433_gb300 as S
from paper_2605_10433_gb300 import inputs as I

ORACLE_MODE = {"ms": oracle.MS, "sms": oracle.SMS, "sagms": oracle.SAGMS, "bp": oracle.BP}
THREADS = max(1, min(32, os.cpu_count() or 1))
MSG_RTOL = 1e-5
TIE_ABS = 1e-4
TIE_U = 64.0 * 2.0 ** -24   # FP32 resolution of a posterior, relative to the size of its terms
PERTURB = 2.0 ** -23
HORIZON_RTOL = 1e-6


def oracle_decode(code, syn, L0, p: S.Params, trace=False):
    return oracle.decode_code(code, syn, np.asarray(L0, dtype=np.float64), mode=ORACLE_MODE[p.mode],
                              alpha=p.alpha, alpha_min=p.alpha_min, alpha_max=p.alpha_max,
                              eta_unsat=p.eta_unsat, max_iter=p.max_iter, flags=p.flags, trace=trace,
                              threads=THREADS)


def gpu_decode(dcode, syn, L0, p: S.Params, trace=False):
    d_syn = torch.from_numpy(np.ascontiguousarray(syn).view(np.int32)).cuda()
    d_L0 = torch.from_numpy(np.ascontiguousarray(L0, dtype=np.float32)).cuda()
    out = S.decode(dcode, d_syn, d_L0, p, trace=trace)
    torch.cuda.synchronize()
    res = {"err": out[0].cpu().numpy().view(np.uint32), "conv": out[1].cpu().numpy(),
           "iters": out[2].cpu().numpy()}
    if trace:
        res["trace"] = out[3].cpu().numpy()
    return res


def first_divergence(gt, ot, iters_g, iters_o, n):
    """First check index where the sign-bit hard decisions of the two traces differ."""
    last = min(iters_g, iters_o)
    for l in range(last + 1):
        gd = np.signbit(gt[l, :n])
        od = ot[l, :n] < 0
        if (gd != od).any():
            return l, np.nonzero(gd != od)[0]
    return None, None


def perturbed(p: S.Params, L0, sign, n):
    """FP32-level perturbation used to measure how well a shot's FP64 trajectory is
    determined: every prior scaled by (1 + sign sigma_j 2^-23) with a fixed pseudo-random
    sign sigma_j per qubit (a uniform scaling would be invisible to the positively
    homogeneous MS family), and the SMS / SAGMS gains by (1 + sign 2^-23).  The perturbed run
    uses per-qubit priors in the units the original run decodes in.  Returns (params, priors)
    or (None, None) for MS in L0-normalised units, which is integer-valued and exact."""
    per_qubit = bool(p.flags & 1)
    L0 = np.asarray(L0, dtype=np.float64)
    if p.mode == "ms" and not per_qubit:
        return None, None
    sigma = np.where(np.random.default_rng(20260513).random(n) < 0.5, -1.0, 1.0)
    if per_qubit:
        base = L0
    elif p.mode == "bp":
        base = np.full(n, L0[0])
    else:
        base = np.full(n, np.sign(L0[0]))
    LL = base * (1.0 + sign * sigma * PERTURB)
    f = 1.0 + sign * PERTURB
    kw = {**p.__dict__, "flags": p.flags | 1}
    if p.mode == "sms":
        kw["alpha"] = p.alpha * f
    elif p.mode == "sagms":
        kw["alpha_min"] = p.alpha_min * f
        kw["alpha_max"] = p.alpha_max * f
    return S.Params(**kw), LL


def _normwise(a, b):
    return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), 1.0)) if a.size else 0.0


def conditioning(code, syn1, L01, p: S.Params):
    """FP64 trajectory of one shot and its FP32-level perturbations: priors and gains scaled by
    1 +- 2^-23, and the oracle's FP32 rounding model (every posterior and every VN->CN input
    moved by +-2^-23 times the size of its terms, both sign patterns).  Returns (trace,
    outcome stable?, horizon), horizon = last check whose normwise posterior change stays
    <= 1e-6 under all of them."""
    o = oracle_decode(code, syn1, L01, p, trace=True)
    n = code.n
    last = int(o["iters"][0])
    horizon = last
    stable = True
    for sign in (+1, -1):
        pp, LL = perturbed(p, L01, sign, n)
        if pp is None:
            continue
        q = oracle_decode(code, syn1, LL, pp, trace=True)
        if not (np.array_equal(q["err"], o["err"]) and q["iters"][0] == o["iters"][0] and q["conv"][0] == o["conv"][0]):
            stable = False
        for l in range(min(last, int(q["iters"][0])) + 1):
            if _normwise(q["trace"][0, l, :n], o["trace"][0, l, :n]) > HORIZON_RTOL:
                horizon = min(horizon, l - 1)
                break
    if not (p.mode == "ms" and not (p.flags & 1)):   # L0-normalised MS is integer-exact
        for extra in (oracle.FLAG_PERTURB, oracle.FLAG_PERTURB | oracle.FLAG_PERTURB_NEG):
            q = oracle_decode(code, syn1, L01, S.Params(**{**p.__dict__, "flags": p.flags | extra}), trace=True)
            if not (np.array_equal(q["err"], o["err"]) and q["iters"][0] == o["iters"][0] and q["conv"][0] == o["conv"][0]):
                stable = False
            for l in range(min(last, int(q["iters"][0])) + 1):
                if _normwise(q["trace"][0, l, :n], o["trace"][0, l, :n]) > HORIZON_RTOL:
                    horizon = min(horizon, l - 1)
                    break
    return o, stable, horizon


def shadow_kw(p: S.Params):
    return dict(mode=ORACLE_MODE[p.mode], alpha=p.alpha, alpha_min=p.alpha_min, alpha_max=p.alpha_max,
                eta_unsat=p.eta_unsat, flags=p.flags)


def _shadow_ratio(dev, bnd):
    a = np.abs(dev)
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(a == 0.0, 0.0, a / bnd)
    return float(np.max(r)) if r.size else 0.0


def trace_outcome_ok(code, syn1, G, rounds, err1, conv1, p: S.Params):
    """The outputs a trace implies: e_hat = sign bits of the last posteriors, conv = zero
    residual, and under early stop no earlier round with a zero residual."""
    n = code.n
    dec = np.signbit(G[:rounds + 1, :n])
    res = [(I.syndrome(code, I.pack_bits(dec[l][None, :])) != syn1[None, :]).any() for l in range(rounds + 1)]
    if not np.array_equal(I.pack_bits(dec[rounds][None, :])[0], err1):
        return "e_hat differs from the sign bits of the last traced posteriors"
    if bool(conv1) != (not res[rounds]):
        return "conv differs from the residual of the last traced posteriors"
    early = not (p.flags & S.FLAG_NO_EARLY_STOP)
    if early and any(not x for x in res[:rounds]):
        return "a zero residual before the reported round"
    if early and rounds < p.max_iter and res[rounds]:
        return "stopped before max_iter without a zero residual"
    return None


def amplified_cap(max_amplified, shots, oracle_failures):
    """Largest accepted number of amplified mismatches: ``max_amplified`` x shots for the
    workloads whose caps are set from measurements, else (targeted tests of adversarial codes)
    ten times the oracle's non-converged shots plus 2e-4 of the shots plus 2 -- amplification
    needs trajectories that wander, and those are the non-converging and slowly converging
    shots."""
    if max_amplified is not None:
        return int(np.ceil(max_amplified * shots - 1e-9))
    return 10 * int(oracle_failures) + int(np.ceil(2e-4 * shots)) + 2


def compare(code, dcode, syn, L0, p: S.Params, min_frac=0.9999, ref=None, max_amplified=None, gpu=None):
    """Decode on both sides and enforce the acceptance above.  Returns a summary dict.
    ``gpu``: outputs of these shots taken from an earlier GPU launch (for instance a sample of
    a full-size batch), used instead of decoding them here.  ``min_frac``: the near-tie budget
    is (1 - min_frac) of the shots; ``max_amplified``: see amplified_cap."""
    g = gpu if gpu is not None else gpu_decode(dcode, syn, L0, p)
    o = ref if ref is not None else oracle_decode(code, syn, L0, p)
    same = (g["err"] == o["err"]).all(axis=1) & (g["conv"] == o["conv"]) & (g["iters"] == o["iters"])
    shots = len(same)
    bad = np.nonzero(~same)[0]
    per_qubit = bool(p.flags & 1)
    normalised = p.mode != "bp" and not per_qubit
    n = code.n
    counted, amplified = [], []
    worst_shadow = 0.0
    kw = shadow_kw(p)
    for c0 in range(0, len(bad), 64):
        idx = bad[c0:c0 + 64]
        Lc = L0 if per_qubit else L0[idx]
        gt = gpu_decode(dcode, syn[idx], Lc, p, trace=True)
        ot = oracle_decode(code, syn[idx], Lc, p, trace=True)
        for k, s in enumerate(idx):
            for key in ("err", "conv", "iters"):
                assert np.array_equal(gt[key][k], g[key][s]), f"shot {s}: traced run differs from the batch run ({key})"
            rounds = int(gt["iters"][k])
            assert rounds >= 0, f"shot {s}: valid on one side only"
            L1 = L0 if per_qubit else L0[s:s + 1]
            G = gt["trace"][k]
            why = trace_outcome_ok(code, syn[s], G, rounds, g["err"][s], g["conv"][s], p)
            assert why is None, f"shot {s} ({p.mode}): {why}"
            dev, bnd, _ = oracle.shadow_code(code, syn[s], L1, G, rounds, **kw)
            ratio = _shadow_ratio(dev, bnd)
            worst_shadow = max(worst_shadow, ratio)
            assert ratio <= 1.0, (f"shot {s} ({p.mode}): GPU posteriors at {ratio:.3g} of the binary32 rounding "
                                  f"bound of the FP64 step from its own previous state")
            l, bits = first_divergence(G, ot["trace"][k], rounds, int(ot["iters"][k]), n)
            assert l is not None, f"shot {s}: outputs differ but no posterior sign differs"
            p_llr = np.abs(ot["trace"][k, l, bits]) * (abs(float(L0[s])) if normalised else 1.0)
            (counted if float(p_llr.max()) < TIE_ABS else amplified).append(int(s))
    allowed = int(np.floor((1 - min_frac) * shots + 1e-6))
    assert len(counted) <= allowed, f"{len(counted)} near-tie mismatches / {shots} shots ({p.mode}), allowed {allowed}"
    cap = amplified_cap(max_amplified, shots, int((o["conv"] == 0).sum()))
    assert len(amplified) <= cap, f"{len(amplified)} amplified mismatches / {shots} shots ({p.mode}), cap {cap}"
    fer_g = float(1 - g["conv"].mean()) if shots else 0.0
    fer_o = float(1 - o["conv"].mean()) if shots else 0.0
    return {"shots": shots, "mismatch": len(bad), "near_tie": len(counted), "amplified": len(amplified),
            "shadow_worst": worst_shadow,
            "fer_gpu": fer_g, "fer_oracle": fer_o, "gpu": g, "oracle": o}


def mcnemar_p(gpu_conv, oracle_conv):
    """Exact two-sided McNemar p-value of the paired convergence flags (the same shots decoded
    by both sides): under equal FER the discordant shots split evenly."""
    from math import comb
    g = np.asarray(gpu_conv) == 0
    o = np.asarray(oracle_conv) == 0
    b, c = int((g & ~o).sum()), int((o & ~g).sum())
    k, n = min(b, c), b + c
    if n == 0:
        return 1.0
    tail = sum(comb(n, i) for i in range(k + 1)) / 2.0 ** n
    return min(1.0, 2.0 * tail)


def fer_check(r, shots, alpha=0.01):
    """FER parity: the GPU FER lies in the oracle's 95% Wilson interval, or -- the two FERs come
    from the same shots, so their difference is the discordant shots' -- the exact McNemar test
    of the paired convergence flags does not reject equality at level ``alpha``.  Returns
    (oracle interval, McNemar p)."""
    from paper_2605_10433_gb300.stats import wilson_interval
    fails_o = int((r["oracle"]["conv"] == 0).sum())
    lo, hi = wilson_interval(fails_o, shots)
    pm = mcnemar_p(r["gpu"]["conv"], r["oracle"]["conv"])
    inside = lo - 1e-12 <= r["fer_gpu"] <= hi + 1e-12
    assert inside or pm >= alpha, (f"FER gpu {r['fer_gpu']:.3e} outside the oracle's interval [{lo:.3e}, {hi:.3e}] "
                                   f"and McNemar p = {pm:.3g}")
    return (lo, hi), pm


def compare_traces(code, dcode, syn, L0, p: S.Params):
    """Posterior traces within the normwise tolerance up to each shot's conditioning horizon.
    Returns (largest normwise error inside the horizons, largest anywhere, mean horizon)."""
    g = gpu_decode(dcode, syn, L0, p, trace=True)
    n = code.n
    per_qubit = bool(p.flags & 1)
    worst_in, worst_all, hz = 0.0, 0.0, []
    for s in range(syn.shape[0]):
        L1 = L0 if per_qubit else L0[s:s + 1]
        o, _, horizon = conditioning(code, syn[s:s + 1], L1, p)
        ot = o["trace"][0]
        gi, oi = int(g["iters"][s]), int(o["iters"][0])
        l_div, _ = first_divergence(g["trace"][s], ot, gi, oi, n)
        last = min(gi, oi) if l_div is None else l_div - 1
        hz.append(horizon)
        if gi >= 0:
            dev, bnd, _ = oracle.shadow_code(code, syn[s], L1, g["trace"][s], gi, **shadow_kw(p))
            ratio = _shadow_ratio(dev, bnd)
            assert ratio <= 1.0, f"shot {s}: traced posteriors at {ratio:.3g} of the binary32 rounding bound"
        for l in range(last + 1):
            e = _normwise(g["trace"][s, l, :n].astype(np.float64), ot[l, :n])
            worst_all = max(worst_all, e)
            if l <= horizon:
                worst_in = max(worst_in, e)
                assert e <= MSG_RTOL, f"shot {s} check {l} (horizon {horizon}): normwise posterior error {e:.3g}"
    return worst_in, worst_all, float(np.mean(hz)) if hz else 0.0


def residual_ok(code, syn, err):
    """conv must equal [s XOR H e_hat == 0] (a property that holds at any size)."""
    s_hat = I.syndrome(code, err)
    return (s_hat == syn).all(axis=1)
