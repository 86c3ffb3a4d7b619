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
