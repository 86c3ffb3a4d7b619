"""A plain binary32 GF(4) decoder in numpy, written only to pin the oracle's GF(4) shadow replay.

Rounds of Algorithm 1 on a Pauli matrix, every operation rounded to binary32: per-Pauli
posteriors summed from the messages of the edges whose entry anticommutes with the Pauli, the
Pauli decision, the residual and gains, the scalar inputs lambda_T(posteriors) minus the edge's
own message, and the binary CN rules.  Its reported posteriors are its state.  ``MUTANTS`` lists
the planted mistakes the replay must reject.  Slow (Python loops): small matrices only.
"""
import numpy as np

import oracle

F = np.float32
MSFAM_CLIP = F(1.0e6)
BP_CLIP = F(23.718998)
PAULIS = (1, 2, 3)   # X, Z, Y

MUTANTS = (
    "vn_every_pauli",    # Eq. 2 per Pauli: a message added to every Pauli, commuting or not
    "commute_swapped",   # the scalar message: commuting and anticommuting Paulis swapped
    "not_extrinsic",     # the scalar message without the edge's own message removed
    "eta_input",         # Eq. 7: eta on the input syndrome bit
    "no_syn_sign",       # Eqs. 3, 4, 8: the syndrome sign dropped
)


def _anti(a, b):
    return ((a & (b >> 1)) ^ ((a >> 1) & b)) & 1


def _softplus_neg(a):
    return F(max(-a, F(0)) + np.log1p(np.exp(F(-abs(a)))))


def _lse_neg(b, c):
    lo, hi = min(b, c), max(b, c)
    if lo == np.inf:
        return F(-np.inf)
    return F(-lo + np.log1p(np.exp(F(lo - hi))))


def _lam(L, T, mutant):
    t = {1: 0, 2: 1, 3: 2}[T]
    u, v = (t + 1) % 3, (t + 2) % 3
    if mutant == "commute_swapped":
        t, u = u, t
    return F(_softplus_neg(L[t]) - _lse_neg(L[u], L[v]))


def _phi(x):
    with np.errstate(divide="ignore", over="ignore"):
        return np.log1p(F(2.0) / np.expm1(F(x)))


def decode(g, syn_row, L0, mode=oracle.SAGMS, alpha=0.75, alpha_min=0.30, alpha_max=0.50, eta_unsat=1.10,
           max_iter=30, mutant=None):
    """One shot, per-shot prior L0.  Returns (trace [rounds+1][n][3] float32, rounds)."""
    m, n = g.m, g.n
    rp, ci, pa = np.asarray(g.row_ptr), np.asarray(g.col_idx), np.asarray(g.pauli).astype(int)
    E = len(ci)
    s = ((np.asarray(syn_row, dtype=np.uint32)[np.arange(m) >> 5] >> (np.arange(m) & 31)) & 1).astype(int)
    l0 = F(np.asarray(L0).reshape(-1)[0])
    vn = [[] for _ in range(n)]
    for e in range(E):
        vn[ci[e]].append(e)
    r = np.zeros(E, dtype=F)
    Lam = np.full((n, 3), l0, dtype=F)
    trace, l = [], 0
    while True:
        trace.append(Lam.copy())
        dec = np.zeros(n, dtype=int)
        for j in range(n):
            best = F(0)
            for w in range(3):
                if Lam[j, w] < best:
                    best, dec[j] = Lam[j, w], PAULIS[w]
        res = s.copy()
        for i in range(m):
            for e in range(rp[i], rp[i + 1]):
                res[i] ^= _anti(dec[ci[e]], pa[e])
        cnt = int(res.sum())
        if cnt == 0 or l == max_iter:
            break
        if mode == oracle.SAGMS:
            base = F(alpha_max) - (F(alpha_max) - F(alpha_min)) * (F(cnt) * F(1.0 / m))
            bit = s if mutant == "eta_input" else res
            gain = np.where(bit == 1, base * F(eta_unsat), base).astype(F)
        elif mode == oracle.SMS:
            gain = np.full(m, F(alpha), dtype=F)
        else:
            gain = np.ones(m, dtype=F)
        q = np.zeros(E, dtype=F)
        for e in range(E):
            lam = _lam(Lam[ci[e]], pa[e], mutant)
            q[e] = lam if mutant == "not_extrinsic" else F(lam - r[e])
        rn = np.zeros(E, dtype=F)
        for i in range(m):
            for e in range(rp[i], rp[i + 1]):
                others = [f for f in range(rp[i], rp[i + 1]) if f != e]
                neg = 0 if mutant == "no_syn_sign" else int(s[i])
                for f in others:
                    neg ^= int(np.signbit(q[f]))
                if mode != oracle.BP:
                    mn = min((abs(q[f]) for f in others), default=F(np.inf))
                    mag = min(F(gain[i] * F(mn)), MSFAM_CLIP)
                else:
                    S_ = F(0.0)
                    for f in others:
                        S_ = F(S_ + _phi(abs(q[f])))
                    mag = min(F(_phi(S_)), BP_CLIP)
                rn[e] = -mag if neg else mag
        r = rn
        Lam = np.empty((n, 3), dtype=F)
        for j in range(n):
            for w in range(3):
                acc = l0
                for e in vn[j]:
                    if mutant == "vn_every_pauli" or _anti(PAULIS[w], pa[e]):
                        acc = F(acc + r[e])
                Lam[j, w] = acc
        l += 1
    return np.array(trace, dtype=F), l
