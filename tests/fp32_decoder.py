"""A plain binary32 decoder in numpy (flooding, or the layered schedule), written only to pin the oracle's shadow replay.

It states Algorithm 1 with Eqs. 1-8 the way a binary32 implementation evaluates them: the
check-node inputs are formed as posterior minus the edge's own message (Eq. 2's extrinsic
sum), every operation rounds to binary32, and its reported posteriors are its state.  The
shadow replay (``oracle.shadow``) must accept its traces and must reject the traces of the
planted mistakes ``MUTANTS`` lists.  Slow (Python loops over checks): small codes only.
"""
import numpy as np

import oracle

F = np.float32
MSFAM_CLIP = F(1.0e6)
BP_CLIP = F(23.718998)

MUTANTS = (
    "eta_input",      # Eq. 7: eta on the input syndrome bit instead of the residual bit
    "gamma_over_n",   # Eq. 6: unsatisfied fraction over n instead of m
    "nonextrinsic",   # Eqs. 4, 8: the minimum includes the edge's own input
    "no_syn_sign",    # Eqs. 3, 4, 8: (-1)^{s_i} dropped
    "drop_message",   # Eq. 2: a qubit's first message left out of its posterior
    "stale_input",    # Eq. 2 / Algorithm 1: inputs from the previous round's posterior
    "bp_half",        # Eq. 3: phi(2x), i.e. tanh(|q|) instead of tanh(|q|/2)
    "layer_stale",    # layered schedule: inputs from the round-start posterior, not the current one
)


def _phi(x):
    with np.errstate(divide="ignore", over="ignore"):
        return np.log1p(F(2.0) / np.expm1(F(x)))


def first_fit_order(code):
    """Checks by (first-fit layer, index): check i takes the smallest layer that no earlier
    check sharing a qubit with it uses."""
    rp, ci = np.asarray(code.row_ptr), np.asarray(code.col_idx)
    cols = [set(ci[rp[i]:rp[i + 1]].tolist()) for i in range(code.m)]
    layer = []
    for i in range(code.m):
        used = {layer[k] for k in range(i) if cols[k] & cols[i]}
        lay = 0
        while lay in used:
            lay += 1
        layer.append(lay)
    return sorted(range(code.m), key=lambda i: (layer[i], i))


def decode(code, syn_row, L0, mode=oracle.SAGMS, alpha=0.75, alpha_min=0.30, alpha_max=0.50, eta_unsat=1.10,
           max_iter=50, flags=0, mutant=None, rebuild_above=None):
    """One shot.  Returns (trace [rounds+1][n] float32, rounds, conv).  With
    oracle.FLAG_LAYERED, the layered schedule with in-place posterior updates
    P = (P - r_old) + r_new; ``rebuild_above``: after a round in which some |P| exceeds it,
    P is recomputed as L0 + sum r."""
    m, n = code.m, code.n
    rp = np.asarray(code.row_ptr, dtype=np.int64)
    ci = np.asarray(code.col_idx, dtype=np.int64)
    E = len(ci)
    s = ((np.asarray(syn_row, dtype=np.uint32)[np.arange(m) >> 5] >> (np.arange(m) & 31)) & 1).astype(np.int64)
    per_qubit = bool(flags & oracle.FLAG_L0_PER_QUBIT)
    msfam = mode != oracle.BP
    if per_qubit:
        prior = np.asarray(L0, dtype=F).copy()
    elif msfam:
        prior = np.full(n, F(np.sign(float(np.asarray(L0).reshape(-1)[0]))), dtype=F)
    else:
        prior = np.full(n, F(np.asarray(L0).reshape(-1)[0]), dtype=F)
    early = not (flags & oracle.FLAG_NO_EARLY_STOP)
    vn = [[] for _ in range(n)]
    for e in range(E):
        vn[ci[e]].append(e)
    r = np.zeros(E, dtype=F)
    P = prior.copy()
    Pprev = prior.copy()
    trace = []
    conv = 0
    l = 0
    while True:
        trace.append(P.copy())
        dec = np.signbit(P).astype(np.int64)
        res = s.copy()
        for i in range(m):
            res[i] ^= int(np.bitwise_xor.reduce(dec[ci[rp[i]:rp[i + 1]]])) if rp[i + 1] > rp[i] else 0
        cnt = int(res.sum())
        if cnt == 0 and early:
            conv = 1
            break
        if l == max_iter:
            conv = int(cnt == 0)
            break
        if mode == oracle.SAGMS:
            denom = n if mutant == "gamma_over_n" else m
            base = F(alpha_max) - (F(alpha_max) - F(alpha_min)) * (F(cnt) * F(1.0 / denom))
            bit = s if mutant == "eta_input" else res
            gain = np.where(bit == 1, base * F(eta_unsat), base).astype(F)
        elif mode == oracle.SMS:
            gain = np.full(m, F(alpha), dtype=F)
        else:
            gain = np.ones(m, dtype=F)
        layered = bool(flags & oracle.FLAG_LAYERED)
        src = Pprev if (mutant == "stale_input" and l > 0) else P
        q = (src[ci] - r).astype(F)
        rn = np.zeros(E, dtype=F)
        Pl = P.copy()
        for i in (first_fit_order(code) if layered else range(m)):
            lo, hi = rp[i], rp[i + 1]
            if layered:
                base = P if mutant == "layer_stale" else Pl
                q[lo:hi] = (base[ci[lo:hi]] - r[lo:hi]).astype(F)
            for e in range(lo, hi):
                others = [f for f in range(lo, hi) if f != e or mutant == "nonextrinsic"]
                neg = 0 if mutant == "no_syn_sign" else int(s[i])
                for f in others:
                    neg ^= int(np.signbit(q[f]))
                if msfam:
                    mn = min((abs(q[f]) for f in others), default=F(np.inf))
                    mag = min(F(gain[i] * F(mn)), MSFAM_CLIP)
                else:
                    S = F(0.0)
                    for f in others:
                        x = abs(q[f]) * (F(2.0) if mutant == "bp_half" else F(1.0))
                        S = F(S + _phi(x))
                    mag = min(F(_phi(S)), BP_CLIP)
                rn[e] = -mag if neg else mag
            if layered:
                r[lo:hi] = rn[lo:hi]
                Pl[ci[lo:hi]] = (q[lo:hi] + rn[lo:hi]).astype(F)
        r = rn if not layered else r
        Pprev = P
        if layered:
            P = Pl
            l += 1
            if rebuild_above is None or not (np.abs(P) > rebuild_above).any():
                continue
        P = np.empty(n, dtype=F)
        for j in range(n):
            acc = prior[j]
            for k, e in enumerate(vn[j]):
                if mutant == "drop_message" and k == 0:
                    continue
                acc = F(acc + r[e])
            P[j] = acc
        if not layered:
            l += 1
    return np.array(trace, dtype=F), l, conv
