// Two-group decoder kernel with column-indexed message storage, for the MS family.  Every
// edge has a check slot j (distinct within its check) such that the j mod DV are distinct
// among each qubit's edges; the edge's message lives at row j mod DV of its qubit's column.
// Generalized-bicycle codes H = [A | B] with rows listed in polynomial-term order have such
// slots as listed (slot j < w is term j of a(x), slot w + k term k of b(x); DC = 2w, DV = w);
// for any other code with qubit degrees <= DV and check degrees <= DC the host assigns them
// by edge colouring (sagms_column_slots).
//
// A 512-thread CTA holds NG = 512 / T independent groups of T threads; each group decodes one
// shot at a time and refills as shots finish (as in decode_groups.cuh), synchronised by its
// own named barrier (a warp barrier when T = 32), so one group's arithmetic-bound check-node
// phase overlaps another's shared-memory-bound phases.  Thread tg of a group owns the K checks
// tg + kT and the qubit pairs (2tg + 2hT, 2tg + 2hT + 1), h < NP / 2T.  The byte offsets of
// its checks' columns stay in registers for the whole launch, biased by its group's
// shared-memory base, so every access of the loop is a register plus an immediate and one
// code body serves all groups (K * DC offsets: with K = 4 a thread has 128 registers).
//
// Shared memory per group g:
//   P_g[NP + 4]            posteriors; P_g[NP] = +inf is the column padded check slots read
//   C_g[q][NP + 4]         negated message D = -L_{i->c} of qubit c's q-th edge at [q][c];
//                          column NP is scratch for padded check slots
// then the groups' bookkeeping and the first-check flip words.  A check thread reaches
// P_g[col] and C_g[j mod DV][col] from the same offset register, and a qubit thread reads its
// messages at fixed offsets: no index loads at all.  A freshly loaded shot's first round has
// every check send the same message on all of its edges (all inputs are the prior), so that
// round stores one closed-form value per check instead of running the check-node minimum
// search.
//
// The arithmetic of every check and qubit is that of decode_kernel.cuh, operation for
// operation, except the MS-family check-node output of shapes up to DC = 10, which takes an
// exactly equivalent form (see there): results are bitwise identical to the other kernels.
#pragma once

#include "decode_groups.cuh"
#include "tmem.cuh"

#ifndef SAGMS_QC_TMEM
#define SAGMS_QC_TMEM 1
#endif

namespace sagms {

constexpr int kQcMisc = 320;     // per-group bookkeeping bytes
constexpr int kQcThreads = 512;  // threads per CTA

// One kernel shape: DC x DV slot degrees, K checks per thread, T threads per group, NP qubit
// columns.  Byte layout of the CTA's shared memory (see the file comment).
template <int DC_, int DV_, int K_, int T_, int NP_>
struct QcShape {
    static constexpr int DC = DC_, DV = DV_, K = K_, T = T_, NP = NP_;
    static constexpr int NG = kQcThreads / T;               // groups per CTA
    static constexpr int MC = K * T;                        // checks a group covers
    static constexpr size_t ROW = (size_t)(NP + 4) * 4;     // one qubit-indexed row + padding
    static constexpr uint32_t PAD = (uint32_t)NP * 4;       // byte offset of the padding column
    static constexpr size_t GROUP = (size_t)(1 + DV) * ROW;
    static constexpr size_t MISC = (size_t)NG * GROUP;
    static constexpr size_t SMEM = MISC + (size_t)NG * kQcMisc + 32 * 4;
    // per-qubit priors (shared by the groups) and their negativity bits, after the rest
    static constexpr size_t PQS = SMEM;
    static constexpr size_t NEGW = PQS + (size_t)(NP + 4) * 4;
    static constexpr size_t SMEM_PQ = NEGW + (size_t)(NP / 32) * 4;
    // Check threads keep their outgoing messages in tensor memory too (tmem.cuh): the shapes
    // with four checks of ten slots per thread in 256-thread groups, one CTA per SM (40 of the
    // 64 columns a warp's lane row gets; 4 warps per lane quadrant, 256 columns per CTA).
    static constexpr bool TM = SAGMS_QC_TMEM != 0 && DC == 10 && K == 4 && T == 256;
    static constexpr uint32_t TM_COLS = 256, TM_WARP_COLS = 64;
    static_assert(DC == 2 * DV && (K == 2 || K == 4) && NG * T == kQcThreads, "shape");
    static_assert(NP % (2 * T) == 0 && MC <= 1024 && (T == 32 || NG <= 15), "layout");
};

// Group barrier: a warp barrier for warp-sized groups, else named barrier 1 + g (an
// immediate when the group index is known at compile time, GC >= 0).
template <int T, int GC>
__device__ __forceinline__ void qc_sync(int g) {
    if constexpr (T == 32) __syncwarp();
    else if constexpr (GC >= 0) asm volatile("bar.sync %0, %1;" ::"n"(1 + GC), "n"(T) : "memory");
    else asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "n"(T) : "memory");
}

// Bits of a per-check field for check k of a thread (K <= 4 checks, 8 bits each).
__device__ __forceinline__ uint32_t qc_byte(uint32_t x, int k) { return (x >> (8 * k)) & 0xffu; }

// GC: the group index when it is fixed at compile time (one copy of the loop per group, every
// group address an immediate), or -1 (one copy for all groups, g at run time).  PQ: one prior
// per qubit shared by all shots (SAGMS_FLAG_L0_PER_QUBIT; LLR units), pq_ok = all finite.
// BPK: the BP rule of Eq. 3 (per-shot priors in LLR units) instead of the MS family.
// tm: the thread's tensor-memory address (its lane, its warp's columns) when S::TM and !BPK: the
// check thread's outgoing messages are kept there as well as in C_g, and the next round reads its
// old messages from there.  Checks 2p and 2p + 1 share columns 2p DC .. 2p DC + 2 DC - 1, slot j
// of check 2p + h at column 2p DC + 2j + h, so each loaded pair lands in adjacent registers as
// the FP32x2 operand of the input sums.  The closed-form first round sends one value per check
// on all its edges: it stores slot 0 of the pair only (2 columns), and the round after it
// (flag `uni`) reads those two columns and adds them to every slot.
template <class S, bool AUTO, bool PQ, int GC, bool BPK>
__device__ __forceinline__ void qc_group(const DecodeArgs& a, unsigned char* smem, const int tg, const int g_rt,
                                         const uint32_t (&off)[S::K][S::DC], const uint32_t degs, const bool pq_ok,
                                         const uint32_t tm) {
    constexpr int DC = S::DC, DV = S::DV, K = S::K, T = S::T, NP = S::NP;
    constexpr bool TM = S::TM && !BPK;
    const int g = GC >= 0 ? GC : g_rt;
    const size_t PO = (size_t)g * S::GROUP;
    const bool early = (a.flags & kFlagNoEarlyStop) == 0;
    const int lane = tg & 31;
    const int n = a.n, m = a.m;
    const int mw = (m + 31) >> 5, nw = (n + 31) >> 5;
    const float inf = __uint_as_float(0x7f800000u);
    float* P = reinterpret_cast<float*>(smem + PO);
    unsigned char* misc = smem + S::MISC;
    int* cnt = reinterpret_cast<int*>(misc + g * kQcMisc);   // [2 parity]
    int* claim = cnt + 2;
    int* pfidx = cnt + 4;
    int* shotsm = cnt + 6;
    float* pfl0 = reinterpret_cast<float*>(cnt + 8);
    float* amaxsh = reinterpret_cast<float*>(cnt + 10);   // alpha_max of the group's shot (Eq. 7)
    uint32_t* pfsyn = reinterpret_cast<uint32_t*>(cnt + 16);
    const uint32_t* flipw = reinterpret_cast<const uint32_t*>(misc + S::NG * kQcMisc);
    // o: the column's byte offset biased by the group's base
    auto Pat = [&](uint32_t o) -> float& { return *reinterpret_cast<float*>(smem + o); };
    // per-qubit prior of a column, from the same biased offset
    auto PQat = [&](uint32_t o) -> float { return *reinterpret_cast<const float*>(smem + S::PQS + o - PO); };
    const float* PQs = reinterpret_cast<const float*>(smem + S::PQS);
    const uint32_t* negw = reinterpret_cast<const uint32_t*>(smem + S::NEGW);
    auto Cat = [&](int j, uint32_t o) -> float& {
        return *reinterpret_cast<float*>(smem + o + (size_t)(1 + j % DV) * S::ROW);
    };

    const int nshots = (int)a.shots;
    const int clg = a.chunk_lg;
    const int cmask = (1 << clg) - 1;
    const bool dynamic = a.work != nullptr;
    const int gid = S::NG * (int)blockIdx.x + g;
    const int gstride = S::NG * (int)gridDim.x;
    if (tg == 0) {
        claim[0] = dynamic ? atomicAdd(a.work, 1) : gid;
        claim[1] = dynamic ? atomicAdd(a.work, 1) : gid + gstride;
    }
    qc_sync<T, GC>(g);
    // Shots: chunks of 2^chunk_lg consecutive shots, claimed dynamically through the work
    // counter (one atomic per chunk, a chunk ahead of its use, via the two-entry ring
    // `claim`), or statically: group b = NG * CTA + g takes chunks b, b + NG * grid, ...
    int seqp = 0;
    auto assign = [&]() -> int {
        const int p = seqp++;
        const int c = p >> clg;
        const long long idx = ((long long)claim[c & 1] << clg) + (p & cmask);
        if ((p & cmask) == 0 && c > 0 && tg == 0)
            claim[(c + 1) & 1] = dynamic ? atomicAdd(a.work, 1) : gid + (c + 1) * gstride;
        return idx < (long long)nshots ? (int)idx : nshots;
    };
    // The next shot's syndrome row and prior are copied into shared memory by warp 0 with
    // cp.async one refill ahead (double-buffered).
    auto prefetch = [&](int b, int s) {
        if (tg < 32 && s < nshots) {
            if (lane < mw) cp_async4(pfsyn + b * 32 + lane, a.syn + s * mw + lane);
            if (lane == 0 && !PQ) cp_async4(pfl0 + b, a.L0 + s);
            cp_async_commit();
        }
    };
    {
        const int first = assign();
        if (tg == 0) pfidx[0] = first;
        prefetch(0, first);
    }

    enum { kActive = 0, kPending = 1, kDone = 2 };
    int state = kPending;
    int itk = 0;
    float prior = 0.0f;
    uint32_t sbits = 0;   // bit k: syndrome bit of check tg + kT
    int pbuf = 0;
    int ph = 0;
    const bool tracing = a.trace != nullptr;
    bool uni = false;   // the last round was the closed form (tensor memory holds slot 0 of each check)

    while (true) {
        // A5: gather the checks' posteriors, residual bits, unsatisfied count
        float2 v[K / 2][DC];
        uint32_t xb = 0;   // bit k: residual bit of check k
#pragma unroll
        for (int p = 0; p < K / 2; ++p) {
#pragma unroll
            for (int j = 0; j < DC; ++j) v[p][j] = make_float2(Pat(off[2 * p][j]), Pat(off[2 * p + 1][j]));
            uint32_t x0 = ((sbits >> (2 * p)) & 1u) << 31, x1 = ((sbits >> (2 * p + 1)) & 1u) << 31;
#pragma unroll
            for (int j = 0; j < DC; j += 2) {
                x0 ^= __float_as_uint(v[p][j].x) ^ __float_as_uint(v[p][j + 1].x);
                x1 ^= __float_as_uint(v[p][j].y) ^ __float_as_uint(v[p][j + 1].y);
            }
            xb |= ((x0 >> 31) << (2 * p)) | ((x1 >> 31) << (2 * p + 1));
        }
        const int part = __reduce_add_sync(0xffffffffu, __popc(xb));
        if (lane == 0) atomicAdd(&cnt[ph], part);
        if (tg < 32) cp_async_wait_all();
        qc_sync<T, GC>(g);
        int gcnt = cnt[ph];
        uint32_t stb = xb;   // bit k: residual bit of check k this round
        if (tg == 0) cnt[ph ^ 1] = 0;
        if (tracing && state == kActive) {
            float* tr = a.trace + ((size_t)shotsm[pbuf ^ 1] * (size_t)(a.max_iter + 1) + (size_t)itk) * (size_t)n;
            for (int c = tg; c < n; c += T) tr[c] = P[c];
        }

        // A6: finish, refill, or count the round about to run.
        bool idle = false, fresh = false;
        int consumed = -1;
        const bool fin = state == kActive && ((gcnt == 0 && early) || itk == a.max_iter);
        if (state == kActive && !fin) {
            itk++;
        } else {
            if (fin) {
                const int s = shotsm[pbuf ^ 1];
#pragma unroll
                for (int vv = 0; vv < NP / T; ++vv) {
                    const int c = vv * T + tg;
                    const uint32_t word = __ballot_sync(0xffffffffu, (c < n) && (__float_as_uint(P[c]) >> 31));
                    if (lane == 0 && c < n) a.err[s * nw + (c >> 5)] = word;
                }
                if (tg == 0) { a.conv[s] = (gcnt == 0) ? 1 : 0; a.iters[s] = itk; }
                state = kPending;
            }
            idle = true;
            const int b = pbuf;
            const int s = pfidx[b];
            if (s >= nshots) {
                state = kDone;
            } else {
                if (tg == 0) shotsm[b] = s;
                pbuf ^= 1;
                consumed = b;
                const uint32_t* row = pfsyn + b * 32;
                const float l0 = PQ ? 0.0f : pfl0[b];
                const uint32_t word = (lane < mw) ? row[lane] : 0u;
                if (!(PQ ? pq_ok : isfinite(l0))) {
                    for (int w = tg; w < nw; w += T) a.err[s * nw + w] = 0u;
                    if (tg == 0) { a.conv[s] = 0; a.iters[s] = -1; }
                } else {
                    const float pi = PQ ? 0.0f
                                        : (BPK ? l0 + 0.0f : ((l0 > 0.0f) ? 1.0f : ((l0 < 0.0f) ? -1.0f : 0.0f)));
                    const bool flipped = PQ || pi < 0.0f;
                    // First check (l = 0), Eqs. 1 and 6: popcount of s XOR flip.
                    const uint32_t flip_lane = (flipped && lane < mw) ? flipw[lane] : 0u;
                    const int c0 = __reduce_add_sync(0xffffffffu, (int)__popc(word ^ flip_lane));
                    if (tracing) {
                        float* tr = a.trace + (size_t)s * (size_t)(a.max_iter + 1) * (size_t)n;
                        for (int c = tg; c < n; c += T) tr[c] = PQ ? PQs[c] : pi;
                    }
                    if ((c0 == 0 && early) || a.max_iter == 0) {
                        for (int w = tg; w < nw; w += T)
                            a.err[s * nw + w] =
                                PQ ? negw[w]
                                   : ((pi < 0.0f) ? ((w == nw - 1 && (n & 31)) ? ((1u << (n & 31)) - 1u) : 0xffffffffu) : 0u);
                        if (tg == 0) { a.conv[s] = (c0 == 0) ? 1 : 0; a.iters[s] = 0; }
                    } else {
                        // Round 1 runs now on the priors themselves (Eq. 2 at l = 1).
                        state = kActive;
                        itk = 1;
                        idle = false;
                        fresh = true;
                        prior = pi;
                        // alpha_max of the new shot.  Every thread of the group stores the
                        // same value, so each thread's own read-back is that value.
                        if (AUTO) *amaxsh = shot_alpha_max(a, l0);
                        gcnt = c0;
                        sbits = 0;
                        stb = 0;
#pragma unroll
                        for (int k = 0; k < K; ++k) {
                            const int i = tg + k * T;
                            const uint32_t bit = (i < m) ? ((row[i >> 5] >> (i & 31)) & 1u) : 0u;
                            sbits |= bit << k;
                            const uint32_t flip = PQ ? ((flipw[i >> 5] >> (i & 31)) & 1u) : (qc_byte(degs, k) & 1u);
                            stb |= (bit ^ (flipped ? flip : 0u)) << k;
                        }
                    }
                }
            }
        }
        if (state == kDone) break;

        if (!idle) {
            // A2 gains (Eq. 7)
            float g[K];
            if (a.mode == kModeSAGMS) {
                const float amax = AUTO ? *amaxsh : a.amax;
            const float base = amax - (amax - a.amin) * ((float)gcnt * a.inv_m);
#pragma unroll
                for (int k = 0; k < K; ++k) g[k] = base * (((stb >> k) & 1u) ? a.eta : 1.0f);
            } else {
#pragma unroll
                for (int k = 0; k < K; ++k) g[k] = (a.mode == kModeSMS) ? a.alpha : 1.0f;
            }
            if (fresh && !PQ && BPK) {
                // A3 (Eq. 3) on round-1 inputs, as decode_kernel.cuh: each real edge's sum over
                // the other edges is (deg - 1) phi(|s|); the parity is the syndrome bit XOR the
                // sign of s once per edge.  Stored negated (D = -L), the same on every slot.
                const uint32_t sgn = __float_as_uint(prior) & kSign;
                const float ph0 = phi_fn(fabsf(prior));
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const uint32_t deg = qc_byte(degs, k);
                    const uint32_t par = (((sbits >> k) & 1u) << 31) ^ ((deg & 1u) ? sgn : 0u);
                    const float S1 = (deg >= 2) ? (float)(int)(deg - 1) * ph0 : 0.0f;
                    const float mag = fminf(phi_fn(S1), kBpClip);
                    const float d = __uint_as_float(__float_as_uint(mag) | (~(par ^ sgn) & kSign));
#pragma unroll
                    for (int j = 0; j < DC; ++j) Cat(j, off[k][j]) = d;
                }
            } else if (fresh && !PQ) {
                // A3 on round-1 inputs: every real edge carries the prior s, padded slots +inf.
                // The minimum and second minimum of |v| are |s| (a check with one edge has no
                // second: +inf), the parity is the syndrome bit XOR the sign of s once per
                // edge, and every real edge gets the second-minimum output (|v_j| = m1).
                const uint32_t sgn = __float_as_uint(prior) & kSign;
                const float ms = fabsf(prior);
                uint32_t dk[K];
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const uint32_t deg = qc_byte(degs, k);
                    const uint32_t par = (((sbits >> k) & 1u) << 31) ^ ((deg & 1u) ? sgn : 0u);
                    const float m2 = (deg >= 2) ? ms : inf;
                    const float o2 = __uint_as_float(__float_as_uint(fminf(g[k] * m2, kMsFamClip)) | par);
                    const float d = __uint_as_float(__float_as_uint(o2) ^ (~__float_as_uint(prior) & kSign));
#pragma unroll
                    for (int j = 0; j < DC; ++j) Cat(j, off[k][j]) = d;
                    if constexpr (TM) {
                        // every edge of the check carries d: slot 0 of the pair stands for all
                        dk[k] = __float_as_uint(d);
                        if (k & 1) tmem_st2(tm + (uint32_t)((k - 1) * DC), dk[k - 1], dk[k]);
                    }
                }
            } else {
                if (PQ && fresh) {
                    // round-1 inputs are the qubits' own priors (+inf on padded slots)
#pragma unroll
                    for (int p = 0; p < K / 2; ++p)
#pragma unroll
                        for (int j = 0; j < DC; ++j) v[p][j] = make_float2(PQat(off[2 * p][j]), PQat(off[2 * p + 1][j]));
                }
#pragma unroll
                for (int p = 0; p < K / 2; ++p) {
                    // A3 check-node update for checks 2p and 2p + 1 (C holds negated
                    // messages: P - L = P + D; a fresh shot has no old messages)
                    if (!(PQ && fresh)) {
                        if constexpr (TM) {
                            __syncwarp();
                            if (uni) {
                                // the previous round was the closed form: one message per check
                                uint32_t d0, d1;
                                tmem_ld2(tm + (uint32_t)(2 * p * DC), d0, d1);
                                const float2 d = make_float2(__uint_as_float(d0), __uint_as_float(d1));
#pragma unroll
                                for (int j = 0; j < DC; ++j) v[p][j] = add2(v[p][j], d);
                            } else {
                                uint32_t o[2 * DC];
                                tmem_ld20(tm + (uint32_t)(2 * p * DC), o);
#pragma unroll
                                for (int j = 0; j < DC; ++j)
                                    v[p][j] = add2(v[p][j], make_float2(__uint_as_float(o[2 * j]), __uint_as_float(o[2 * j + 1])));
                            }
                        } else {
#pragma unroll
                            for (int j = 0; j < DC; ++j)
                                v[p][j] = add2(v[p][j], make_float2(Cat(j, off[2 * p][j]), Cat(j, off[2 * p + 1][j])));
                        }
                    }
                    uint32_t par0 = ((sbits >> (2 * p)) & 1u) << 31, par1 = ((sbits >> (2 * p + 1)) & 1u) << 31;
#pragma unroll
                    for (int j = 0; j < DC; j += 2) {
                        par0 ^= __float_as_uint(v[p][j].x) ^ __float_as_uint(v[p][j + 1].x);
                        par1 ^= __float_as_uint(v[p][j].y) ^ __float_as_uint(v[p][j + 1].y);
                    }
                    par0 &= kSign;
                    par1 &= kSign;
                    if constexpr (BPK) {
                        // A3, BP rule (Eq. 3): phi sums over the other edges by prefix and suffix
                        // sums, in the slot order and arithmetic of decode_kernel.cuh (padded slots
                        // add phi(+inf) = 0); stored negated, D = -L.
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const uint32_t par = h ? par1 : par0;
                            float ph[DC];
#pragma unroll
                            for (int j = 0; j < DC; ++j) ph[j] = phi_fn(fabsf(h ? v[p][j].y : v[p][j].x));
                            float suf[DC + 1];
                            suf[DC] = 0.0f;
#pragma unroll
                            for (int j = DC - 1; j >= 0; --j) suf[j] = suf[j + 1] + ph[j];
                            float pre = 0.0f;
#pragma unroll
                            for (int j = 0; j < DC; ++j) {
                                const float Sj = pre + suf[j + 1];
                                pre += ph[j];
                                const float mag = fminf(phi_fn(Sj), kBpClip);
                                const uint32_t vb = __float_as_uint(h ? v[p][j].y : v[p][j].x);
                                Cat(j, off[2 * p + h][j]) = __uint_as_float(__float_as_uint(mag) | (~(par ^ vb) & kSign));
                            }
                        }
                    } else if constexpr (DC <= 10 && !(PQ && T == 128)) {
                        // Eqs. 4 and 8: edge j receives min(g * min_{i != j} |v_i|, clip) with
                        // the parity of the other edges.  The gain is positive (host-checked),
                        // so fl(g x) is monotone in x and the minimum may be taken after the
                        // scaling: min_{i != j} fl(g |v_i|).  The parity bit rides on the gain,
                        // making every scaled value of the check the same sign, and floats of
                        // one sign order like their bit patterns as unsigned integers.  So
                        // each edge's output is an unsigned minimum over the others: over its
                        // slot pair's partner, the pairs before it (running prefix) and the
                        // pairs after it (suffix, seeded with the clip).  These are the same
                        // bits as the smallest / second-smallest selection below, with no
                        // compare and select per edge and a short dependency chain.  (Shapes
                        // where the values do not fit the register budget keep the selection.)
                        constexpr int NPR = DC / 2;
                        uint32_t wvp[2][DC];   // both checks' outputs, for the interleaved store
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const uint32_t par = h ? par1 : par0;
                            const float gs = __uint_as_float(__float_as_uint(g[2 * p + h]) | par);
                            uint32_t x[DC], pm[NPR], sp[NPR];
#pragma unroll
                            for (int j = 0; j < DC; ++j) x[j] = __float_as_uint(gs * fabsf(h ? v[p][j].y : v[p][j].x));
#pragma unroll
                            for (int i = 0; i < NPR; ++i) pm[i] = min(x[2 * i], x[2 * i + 1]);
                            sp[NPR - 1] = __float_as_uint(kMsFamClip) | par;
#pragma unroll
                            for (int i = NPR - 2; i >= 0; --i) sp[i] = min(sp[i + 1], pm[i + 1]);
                            uint32_t pre = 0u;
                            uint32_t wv[DC];
#pragma unroll
                            for (int i = 0; i < NPR; ++i) {
                                const uint32_t o0 = i ? __vimin3_u32(x[2 * i + 1], pre, sp[i]) : min(x[1], sp[0]);
                                const uint32_t o1 = i ? __vimin3_u32(x[2 * i], pre, sp[i]) : min(x[0], sp[0]);
                                pre = i ? min(pre, pm[i]) : pm[0];
                                const uint32_t b0 = __float_as_uint(h ? v[p][2 * i].y : v[p][2 * i].x);
                                const uint32_t b1 = __float_as_uint(h ? v[p][2 * i + 1].y : v[p][2 * i + 1].x);
                                wv[2 * i] = o0 ^ (~b0 & kSign);
                                wv[2 * i + 1] = o1 ^ (~b1 & kSign);
                                Cat(2 * i, off[2 * p + h][2 * i]) = __uint_as_float(wv[2 * i]);
                                Cat(2 * i + 1, off[2 * p + h][2 * i + 1]) = __uint_as_float(wv[2 * i + 1]);
                            }
#pragma unroll
                            for (int j = 0; j < DC; ++j) wvp[h][j] = wv[j];
                        }
                        if constexpr (TM) {
                            uint32_t il[2 * DC];
#pragma unroll
                            for (int j = 0; j < DC; ++j) { il[2 * j] = wvp[0][j]; il[2 * j + 1] = wvp[1][j]; }
                            tmem_st20(tm + (uint32_t)(2 * p * DC), il);
                        }
                    } else {
                        // Smallest and second smallest |v|, two edges at a time:
                        // m2 = min(m2, hi, max(m1, lo)), m1 = min(m1, lo).
                        float m1a = inf, m2a = inf, m1b = inf, m2b = inf;
#pragma unroll
                        for (int j = 0; j < DC; j += 2) {
                            const float a0 = fabsf(v[p][j].x), a1 = fabsf(v[p][j + 1].x);
                            const float c0 = fabsf(v[p][j].y), c1 = fabsf(v[p][j + 1].y);
                            const float loa = fminf(a0, a1), hia = fmaxf(a0, a1);
                            const float lob = fminf(c0, c1), hib = fmaxf(c0, c1);
                            m2a = fminf(fminf(m2a, hia), fmaxf(m1a, loa));
                            m1a = fminf(m1a, loa);
                            m2b = fminf(fminf(m2b, hib), fmaxf(m1b, lob));
                            m1b = fminf(m1b, lob);
                        }
                        const float o1a = __uint_as_float(__float_as_uint(fminf(g[2 * p] * m1a, kMsFamClip)) | par0);
                        const float o2a = __uint_as_float(__float_as_uint(fminf(g[2 * p] * m2a, kMsFamClip)) | par0);
                        const float o1b = __uint_as_float(__float_as_uint(fminf(g[2 * p + 1] * m1b, kMsFamClip)) | par1);
                        const float o2b = __uint_as_float(__float_as_uint(fminf(g[2 * p + 1] * m2b, kMsFamClip)) | par1);
#pragma unroll
                        for (int j = 0; j < DC; ++j) {
                            const float ma = (fabsf(v[p][j].x) == m1a) ? o2a : o1a;
                            const float mb = (fabsf(v[p][j].y) == m1b) ? o2b : o1b;
                            Cat(j, off[2 * p][j]) = __uint_as_float(__float_as_uint(ma) ^ (~__float_as_uint(v[p][j].x) & kSign));
                            Cat(j, off[2 * p + 1][j]) = __uint_as_float(__float_as_uint(mb) ^ (~__float_as_uint(v[p][j].y) & kSign));
                        }
                    }
                }
            }
            if constexpr (TM) tmem_wait_st();   // this round's stores land before the next reads
            uni = fresh && !PQ && !BPK;
        }
        qc_sync<T, GC>(g);

        // Claim and prefetch the group's next shot (warp 0 of the group).
        if (consumed >= 0 && tg < 32) {
            const int nx = assign();
            if (tg == 0) pfidx[consumed ^ 1] = nx;
            prefetch(consumed ^ 1, nx);
        }

        if (!idle) {
            // A4 variable-node update: qubit pairs (2tg + 2hT, 2tg + 2hT + 1)
            const float2 npr = make_float2(-prior, -prior);
            unsigned char* vbase = smem + PO + (size_t)tg * 8;
#pragma unroll
            for (int h = 0; h < NP / (2 * T); ++h) {
                float2 acc = npr;
                if (PQ) {
                    const float2 pq = *reinterpret_cast<const float2*>(smem + S::PQS + (size_t)tg * 8 + (size_t)h * 8 * T);
                    acc = make_float2(-pq.x, -pq.y);
                }
#pragma unroll
                for (int q = 0; q < DV; ++q)
                    acc = add2(acc, *reinterpret_cast<const float2*>(vbase + (size_t)(1 + q) * S::ROW + (size_t)h * 8 * T));
                *reinterpret_cast<float2*>(vbase + (size_t)h * 8 * T) =
                    __ffma2_rn(acc, make_float2(-1.0f, -1.0f), make_float2(0.0f, 0.0f));
            }
        }
        qc_sync<T, GC>(g);
        ph ^= 1;
    }
}

// colQ: [K][DC][T] u32, byte offset 4 * col of check tg + kT in slot j (S::PAD for a padded
// slot or a check past m).  AUTO: the gain ceiling of each shot comes from its prior
// (SAGMS_FLAG_AUTO_CEILING), a separate instantiation so the default one carries no trace of it.
// Two CTAs per SM (64 registers) for the small shapes and for BP with two checks per thread,
// where BP's transcendental chains need the warps more than the registers (a few bytes spill
// at DC = 10; still 1.15-1.5x faster).  The MS family keeps four checks per thread at 128
// registers: at 64 it measured 10-21% slower.
template <class S, bool AUTO, bool PQ, bool BPK = false>
__global__ void __launch_bounds__(kQcThreads, (S::K * S::DC <= 12 || (BPK && S::K == 2 && S::DC <= 10)) ? 2 : 1)
qc_kernel(const DecodeArgs a, const uint32_t* __restrict__ colQ) {
    constexpr int DC = S::DC, K = S::K, T = S::T;
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr bool TMK = S::TM && !BPK;
    __shared__ uint32_t tm_slot;
    const int t = threadIdx.x;
    const int g = t / T;
    const int tg = t % T;
    // Tensor memory for the check threads' messages: warp 0 allocates the CTA's columns; the
    // barrier after the zeroing below publishes the base (fenced on both sides).
    if constexpr (TMK) {
        if (t < 32) tmem_alloc(&tm_slot, S::TM_COLS);
        tmem_fence_before();
    }
    const float inf = __uint_as_float(0x7f800000u);
    uint32_t off[K][DC];
    uint32_t degs = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        uint32_t d = 0;
#pragma unroll
        for (int j = 0; j < DC; ++j) {
            const uint32_t o = __ldg(colQ + (k * DC + j) * T + tg);
            d += (o != S::PAD) ? 1u : 0u;
            off[k][j] = o + (uint32_t)(g * S::GROUP);   // into this group's arrays
        }
        degs |= d << (8 * k);
    }
    // Posteriors, messages and bookkeeping of every group start at zero; the padding columns
    // of the posteriors hold +inf.
    {
        float* z = reinterpret_cast<float*>(smem);
        for (int k = t; k < (int)(S::MISC / 4); k += kQcThreads) z[k] = 0.0f;
        int* misc = reinterpret_cast<int*>(smem + S::MISC);
        for (int k = t; k < S::NG * kQcMisc / 4; k += kQcThreads) misc[k] = 0;
    }
    int pq_ok = 1;
    if constexpr (PQ) {
        // per-qubit priors (LLR units), +inf past n; all finite or every shot is invalid
        float* pqs = reinterpret_cast<float*>(smem + S::PQS);
        for (int c = t; c < S::NP + 4; c += kQcThreads) {
            const float v = (c < a.n) ? __ldg(a.L0 + c) + 0.0f : inf;   // -0 -> +0: sign bits are decisions
            pqs[c] = v;
            if (c < a.n) pq_ok &= isfinite(v) ? 1 : 0;
        }
    }
    __syncthreads();
    if (t < S::NG) *reinterpret_cast<float*>(smem + (size_t)t * S::GROUP + S::PAD) = inf;
    // First residual bits under the priors' signs: a check's degree parity under a negative
    // per-shot prior, the parity of its negative priors with per-qubit priors.
    uint32_t* flipw = reinterpret_cast<uint32_t*>(smem + S::MISC + S::NG * kQcMisc);
    if (t < T) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            uint32_t f = qc_byte(degs, k) & 1u;
            if constexpr (PQ) {
                f = 0u;
#pragma unroll
                for (int j = 0; j < DC; ++j)   // group 0: offsets are the plain column offsets
                    f ^= __float_as_uint(*reinterpret_cast<const float*>(smem + S::PQS + off[k][j])) >> 31;
            }
            const uint32_t w = __ballot_sync(0xffffffffu, f);
            if ((t & 31) == 0) flipw[(t + k * T) >> 5] = w;
        }
    }
    if constexpr (PQ) {
        // [L0_c < 0]: the decision of a shot stopped at its first check
        uint32_t* negw = reinterpret_cast<uint32_t*>(smem + S::NEGW);
        const float* pqs = reinterpret_cast<const float*>(smem + S::PQS);
        for (int c = t; c < S::NP; c += kQcThreads) {
            const uint32_t w = __ballot_sync(0xffffffffu, (c < a.n) && (__float_as_uint(pqs[c]) >> 31));
            if ((t & 31) == 0) negw[c >> 5] = w;
        }
    }
    pq_ok = __syncthreads_and(pq_ok);
    uint32_t tm = 0;
    if constexpr (TMK) {
        tmem_fence_after();
        const int w = t >> 5;
        tm = tm_slot + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(w >> 2) * S::TM_WARP_COLS;
    }
    if constexpr (S::NG == 2) {
        if (g == 0) qc_group<S, AUTO, PQ, 0, BPK>(a, smem, tg, g, off, degs, pq_ok != 0, tm);
        else qc_group<S, AUTO, PQ, 1, BPK>(a, smem, tg, g, off, degs, pq_ok != 0, tm);
    } else {
        qc_group<S, AUTO, PQ, -1, BPK>(a, smem, tg, g, off, degs, pq_ok != 0, tm);
    }
    if constexpr (TMK) {
        // every tensor-memory access of the CTA has completed (each load and each round's
        // stores were waited for); warp 0 releases the columns
        tmem_fence_before();
        __syncthreads();
        tmem_fence_after();
        if (t < 32) tmem_dealloc(tm_slot, S::TM_COLS);
    }
}

}  // namespace sagms
