"""Reporting helpers for decoder runs: frame-error statistics and the logical check.

These post-process decoder outputs for reports; neither the decoder nor its FP64 checker
calls them."""
from __future__ import annotations

import math

import numpy as np


def wilson_interval(failures: int, trials: int, z: float = 1.959963984540054):
    """95% Wilson score interval of a binomial proportion, the confidence interval the
    Monte Carlo protocol of Sec. V (setup) reports per FER point."""
    if trials <= 0:
        return (0.0, 1.0)
    ph = failures / trials
    den = 1 + z * z / trials
    c = (ph + z * z / (2 * trials)) / den
    h = z * math.sqrt(ph * (1 - ph) / trials + z * z / (4 * trials * trials)) / den
    return (max(0.0, c - h), min(1.0, c + h))


def log_ratio_interval(f1: int, n1: int, f2: int, n2: int, z: float = 1.959963984540054):
    """Two-sample CI of the ratio of two failure rates (log-ratio normal approximation),
    the statistic quoted for the SAGMS/SMS FER ratio in Sec. V (results)."""
    if min(f1, f2) == 0:
        return (0.0, math.inf)
    r = (f1 / n1) / (f2 / n2)
    se = math.sqrt(1 / f1 - 1 / n1 + 1 / f2 - 1 / n2)
    return (r * math.exp(-z * se), r * math.exp(z * se))


def _gf2_rank(rows) -> int:
    pivots = {}
    rank = 0
    for r in rows:
        x = r
        while x:
            top = x.bit_length() - 1
            if top in pivots:
                x ^= pivots[top]
            else:
                pivots[top] = x
                rank += 1
                break
    return rank


def logical_ok(hz_rows, residual_bits: np.ndarray) -> np.ndarray:
    """Per shot: whether the residual e XOR e_hat lies in the row space of H_Z, i.e. is a
    stabilizer and leaves no logical error.  residual_bits: [shots][n] 0/1."""
    base = _gf2_rank(hz_rows)
    out = np.zeros(residual_bits.shape[0], dtype=bool)
    for s in range(residual_bits.shape[0]):
        r = residual_bits[s]
        if not r.any():
            out[s] = True
            continue
        x = 0
        for j in np.nonzero(r)[0]:
            x |= 1 << int(j)
        out[s] = _gf2_rank(list(hz_rows) + [x]) == base
    return out
