"""Algorithmic work model of one decoder iteration and the ALU-issue roofline.

The per-check-node cost follows the weighted operation count of Eq. 15 / Table I
(additions, multiplications, comparisons weight 1, transcendentals weight 10):
    MS    2 d_c - 3   (Table I: d_c - 1 multiplications, d_c - 2 comparisons)
    SMS   2 d_c - 2   (Eq. 15: MS plus the alpha multiplication)
    SAGMS 2 d_c + 3   (Eq. 15 / Table I: 3 additions, d_c + 1 multiplications, d_c - 1 comparisons)
    BP    22 d_c - 13 (Eq. 15 / Table I: d_c - 2 additions, d_c - 1 multiplications, 2 d_c - 1 transcendentals)
To that one iteration adds, per qubit j of degree d_v, the posterior sum, the d_v extrinsic
subtractions and the hard decision (2 d_v + 1), one XOR per edge for the residual syndrome
(Eq. 1), and one popcount step per check (Eq. 6).  Retired shots do no work, so the work of a
batch is sum over shots of iters x ops_per_iteration.
"""
from __future__ import annotations

import numpy as np

CN_OPS = {
    "ms": lambda dc: 2 * dc - 3,
    "sms": lambda dc: 2 * dc - 2,
    "sagms": lambda dc: 2 * dc + 3,
    "bp": lambda dc: 22 * dc - 13,
}

THREAD_OPS_PER_SM_CLK = 128   # 4 schedulers x 32 lanes issue one instruction each per clock


def ops_per_iteration(mode: str, row_ptr, col_idx, n: int) -> int:
    row_ptr = np.asarray(row_ptr)
    dc = np.diff(row_ptr)
    dv = np.bincount(np.asarray(col_idx), minlength=n)
    cn = int(sum(CN_OPS[mode](int(d)) for d in dc))
    vn = int((2 * dv + 1).sum())
    edges = int(row_ptr[-1])
    return cn + vn + edges + len(dc)


# Quaternary variable node (Sec. II, scalar messages): per qubit of degree d_v, the three Pauli
# totals Lambda(X), Lambda(Z), Lambda(Y) take two additions per edge (an edge's message enters
# the two Paulis that anticommute with its entry), the decision argmin(0, Lambda(X), Lambda(Z),
# Lambda(Y)) three comparisons, and each of the three commute LLRs
# lambda_T = ln(1 + e^{-Lambda(T)}) - ln(e^{-Lambda(T')} + e^{-Lambda(T'')}) two exponentials
# and two logarithms (weight 10 each, as Eq. 15 weighs transcendentals) plus four simple
# operations; every edge then takes one subtraction for its extrinsic message.
GF4_LAMBDA_OPS = 4 * 10 + 4


def gf4_ops_per_iteration(mode: str, row_ptr, col_idx, n: int) -> int:
    """One iteration of the GF(4) decoder on a stabilizer matrix with Pauli entries: the check
    rule of Eq. 15 / Table I per row (BP4 for mode "bp"), the quaternary variable node above
    (3 d_v + 3 + 3 x 44 per qubit), one anticommutation test per edge for the residual
    syndrome (Eq. 1 with the trace inner product) and one popcount step per check."""
    row_ptr = np.asarray(row_ptr)
    dc = np.diff(row_ptr)
    dv = np.bincount(np.asarray(col_idx), minlength=n)
    cn = int(sum(CN_OPS[mode](int(d)) for d in dc))
    vn = int((3 * dv + 3 + 3 * GF4_LAMBDA_OPS).sum())
    edges = int(row_ptr[-1])
    return cn + vn + edges + len(dc)


def alu_peak_ops(sms: int, sm_mhz: float) -> float:
    """Thread-instruction issue rate of the whole GPU: SMs x 128 lanes x clock."""
    return sms * THREAD_OPS_PER_SM_CLK * sm_mhz * 1e6


SMEM_BYTES_PER_SM_CLK = 128  # shared-memory pipe: one 128-byte wavefront per clock per SM


def smem_bytes(iters, edges: int, n: int, old_in_smem: bool = True) -> float:
    """Shared-memory bytes of the flooding schedule, summed over shots.  A shot with r >= 1
    iterations reads P_j for each of its r residual checks (4E per check; rounds 2..r take
    their check-node inputs from the same read), writes L_new (4E) and reads it back in the
    variable-node sum (4E) in every round, and writes P (4n) in every round.  With the check
    threads' old messages in shared memory it also reads L_old (4E) in rounds 2..r (round 1
    starts from zero messages): 16E r - 4E + 4n r bytes; with them in tensor memory (the
    headline kernel shape) that read leaves shared memory: 12E r + 4n r.  A shot stopped at its
    first check (r = 0) moves none."""
    r = np.asarray(iters, dtype=np.int64)
    r = r[r > 0]
    if not old_in_smem:
        return float((12 * edges + 4 * n) * r.sum())
    return float((16 * edges + 4 * n) * r.sum() - 4 * edges * r.size)


def smem_peak_bytes(sms: int, sm_mhz: float) -> float:
    """Shared-memory bandwidth of the whole GPU: SMs x 128 B x clock."""
    return sms * SMEM_BYTES_PER_SM_CLK * sm_mhz * 1e6


def hbm_bytes_per_shot(m: int, n: int) -> int:
    """Syndrome in, prior in, packed estimate + flag + count out."""
    return ((m + 31) // 32) * 4 + 4 + ((n + 31) // 32) * 4 + 1 + 4
