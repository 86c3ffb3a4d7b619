"""Brute-force references over all 2^n error patterns (tiny codes only).

These are independent of the oracle's message passing: they enumerate every error
pattern e, keep those with H e = s, and read off
* exact posterior LLRs log P(e_j = 0 | s) / P(e_j = 1 | s) under the prior
  P(e) ~ exp(-sum_j L0_j e_j)  (what BP computes exactly on a cycle-free Tanner graph);
* min-marginal cost differences min_{e_j=1} cost(e) - min_{e_j=0} cost(e) with
  cost(e) = sum_j L0_j e_j  (what Min-Sum computes exactly on a cycle-free graph);
* the maximum-likelihood (minimum-cost) pattern.
"""
import numpy as np


def all_patterns(n):
    idx = np.arange(1 << n, dtype=np.int64)
    return ((idx[:, None] >> np.arange(n)[None, :]) & 1).astype(np.uint8)


def consistent(H, s):
    E = all_patterns(H.shape[1])
    S = (E.astype(np.int64) @ H.T.astype(np.int64)) % 2
    ok = (S == np.asarray(s)[None, :]).all(axis=1)
    return E[ok]


def exact_llr(H, s, L0):
    E = consistent(H, s)
    cost = E.astype(np.float64) @ np.asarray(L0, dtype=np.float64)
    out = np.zeros(H.shape[1])
    for j in range(H.shape[1]):
        c0 = -cost[E[:, j] == 0]
        c1 = -cost[E[:, j] == 1]
        l0 = np.logaddexp.reduce(c0) if c0.size else -np.inf
        l1 = np.logaddexp.reduce(c1) if c1.size else -np.inf
        out[j] = l0 - l1
    return out


def min_marginal_diff(H, s, L0):
    E = consistent(H, s)
    cost = E.astype(np.float64) @ np.asarray(L0, dtype=np.float64)
    out = np.zeros(H.shape[1])
    for j in range(H.shape[1]):
        c0 = cost[E[:, j] == 0]
        c1 = cost[E[:, j] == 1]
        out[j] = (c1.min() if c1.size else np.inf) - (c0.min() if c0.size else np.inf)
    return out


def ml_pattern(H, s, L0):
    """Minimum-cost pattern and whether it is unique."""
    E = consistent(H, s)
    cost = E.astype(np.float64) @ np.asarray(L0, dtype=np.float64)
    order = np.argsort(cost, kind="stable")
    best = E[order[0]]
    unique = len(cost) == 1 or cost[order[1]] > cost[order[0]] + 1e-12
    return best, unique
