// Two-group decoder kernel with column-indexed message storage, for the MS family on codes
// whose edges line up slot by slot: every edge in check slot j is, at its qubit, the edge
// numbered q = j mod DV, and a qubit's edges in increasing check slot have increasing q.
// Generalized-bicycle codes H = [A | B] with rows listed in polynomial-term order have this
// structure (slot j < w is term j of a(x) and qubit c < l meets it as its j-th edge; slot
// w + k is term k of b(x)), with DC = 2w and DV = w.
//
// Groups and shots are those of decode_groups.cuh: a 1024-thread CTA holds two independent
// 512-thread groups, each decoding one shot at a time with its own named barriers.  Thread
// tg of a group owns checks tg and tg + 512 and the qubit pairs (2tg, 2tg + 1) and
// (1024 + 2tg, 1024 + 2tg + 1).
//
// Shared memory per group g (byte offsets are compile-time for each group):
//   P_g[2048 + 4]          posteriors; P_g[2048] = +inf is the column padded check slots read
//   C_g[q][2048 + 4]       negated message D = -L_{i->c} of qubit c's q-th edge at [q][c];
//                          column 2048 is scratch for padded check slots
// and, shared by both groups,
//   colQ[DC][512]          u32: byte offsets 4 * col of checks tg (low half) and tg + 512
//                          (high half) in slot j (2048 for a padded slot)
// A check thread reaches P_g[col] and C_g[j mod DV][col] from the same offset register, and a
// qubit thread reads its messages at fixed offsets: no index loads in the variable-node
// update.  A freshly loaded shot's first round has every check send the same message on all
// of its edges (all inputs are the prior), so that round stores one closed-form value per
// check instead of running the check-node minimum search.
//
// The arithmetic of every check and qubit is, operation for operation, that of
// decode_kernel.cuh: results are bitwise identical to the other kernels.
#pragma once

#include "decode_groups.cuh"

namespace sagms {

constexpr int kQcRowBytes = (kGrpQubits + 4) * 4;    // one qubit-indexed row plus padding column
constexpr uint32_t kQcPadOff = (uint32_t)kGrpQubits * 4;

__host__ __device__ constexpr size_t qc_group_bytes(int DV) { return (size_t)(1 + DV) * kQcRowBytes; }
__host__ __device__ constexpr size_t qc_P_off(int DV, int g) { return (size_t)g * qc_group_bytes(DV); }
__host__ __device__ constexpr size_t qc_C_off(int DV, int g, int q) {
    return qc_P_off(DV, g) + (size_t)(1 + q) * kQcRowBytes;
}
__host__ __device__ constexpr size_t qc_col_off(int DV) { return 2 * qc_group_bytes(DV); }
__host__ __device__ constexpr size_t qc_misc_off(int DC, int DV) {
    return qc_col_off(DV) + (size_t)DC * kGrpThreads * 4;
}
__host__ __device__ constexpr size_t qc_smem_bytes(int DC, int DV) {
    return qc_misc_off(DC, DV) + 2 * kGrpMiscPerGroup + 32 * 4;
}

template <int DC, int DV, int G>
__device__ __forceinline__ void qc_group(const DecodeArgs& a, unsigned char* smem, const int tg,
                                         const uint32_t degs) {
    constexpr int NP = kGrpQubits;
    constexpr size_t PO = qc_P_off(DV, G);
    const bool early = (a.flags & kFlagNoEarlyStop) == 0;
    const int lane = tg & 31;
    const int n = a.n, m = a.m;
    const int mw = (m + 31) >> 5, nw = (n + 31) >> 5;
    const float inf = __uint_as_float(0x7f800000u);
    float* P = reinterpret_cast<float*>(smem + PO);
    const uint32_t* colQ = reinterpret_cast<const uint32_t*>(smem + qc_col_off(DV));
    unsigned char* misc = smem + qc_misc_off(DC, DV);
    int* cnt = reinterpret_cast<int*>(misc + G * kGrpMiscPerGroup);   // [2 parity]
    int* claim = cnt + 2;
    int* pfidx = cnt + 4;
    int* shotsm = cnt + 6;
    float* pfl0 = reinterpret_cast<float*>(cnt + 8);
    uint32_t* pfsyn = reinterpret_cast<uint32_t*>(cnt + 16);
    const uint32_t* flipw = reinterpret_cast<const uint32_t*>(misc + 2 * kGrpMiscPerGroup);
    auto Pat = [&](uint32_t o) -> float& { return *reinterpret_cast<float*>(smem + PO + o); };
    auto Cat = [&](int j, uint32_t o) -> float& {
        return *reinterpret_cast<float*>(smem + qc_C_off(DV, G, j % DV) + o);
    };

    const int nshots = (int)a.shots;
    const int clg = a.chunk_lg;
    const int cmask = (1 << clg) - 1;
    const bool dynamic = a.work != nullptr;
    const int gid = 2 * (int)blockIdx.x + G;
    const int gstride = 2 * (int)gridDim.x;
    if (tg == 0) {
        claim[0] = dynamic ? atomicAdd(a.work, 1) : gid;
        claim[1] = dynamic ? atomicAdd(a.work, 1) : gid + gstride;
    }
    group_barrier(G);
    int seqp = 0;
    auto assign = [&]() -> int {
        const int p = seqp++;
        const int c = p >> clg;
        const long long idx = ((long long)claim[c & 1] << clg) + (p & cmask);
        if ((p & cmask) == 0 && c > 0 && tg == 0)
            claim[(c + 1) & 1] = dynamic ? atomicAdd(a.work, 1) : gid + (c + 1) * gstride;
        return idx < (long long)nshots ? (int)idx : nshots;
    };
    auto prefetch = [&](int b, int s) {
        if (tg < 32 && s < nshots) {
            if (lane < mw) cp_async4(pfsyn + b * 32 + lane, a.syn + s * mw + lane);
            if (lane == 0) cp_async4(pfl0 + b, a.L0 + s);
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
    uint32_t sbits = 0;   // bit 0: syndrome bit of check tg, bit 1: of check tg + 512
    int pbuf = 0;
    int ph = 0;
    // degs: degree of check tg in bits 0-7, of check tg + 512 in bits 8-15; a negative
    // prior flips a check's first residual bit when its degree is odd.

    while (true) {
        // A5: gather the two checks' posteriors, residual bits, unsatisfied count
        uint32_t wq[DC];
        float2 v[DC];
#pragma unroll
        for (int j = 0; j < DC; ++j) {
            wq[j] = colQ[j * kGrpThreads + tg];
            v[j] = make_float2(Pat(wq[j] & 0xffffu), Pat(wq[j] >> 16));
        }
        uint32_t x0 = (sbits & 1u) << 31, x1 = (sbits >> 1) << 31;
#pragma unroll
        for (int j = 0; j < DC; j += 2) {
            x0 ^= __float_as_uint(v[j].x) ^ __float_as_uint(v[j + 1].x);
            x1 ^= __float_as_uint(v[j].y) ^ __float_as_uint(v[j + 1].y);
        }
        const uint32_t b0 = __ballot_sync(0xffffffffu, x0 >> 31);
        const uint32_t b1 = __ballot_sync(0xffffffffu, x1 >> 31);
        if (lane == 0) atomicAdd(&cnt[ph], __popc(b0) + __popc(b1));
        if (tg < 32) cp_async_wait_all();
        group_barrier(G);
        int gcnt = cnt[ph];
        uint32_t st0 = x0 >> 31, st1 = x1 >> 31;
        if (tg == 0) cnt[ph ^ 1] = 0;
        if (a.trace && state == kActive) {
            float* tr = a.trace + ((size_t)shotsm[pbuf ^ 1] * (size_t)(a.max_iter + 1) + (size_t)itk) * (size_t)n;
            for (int c = tg; c < n; c += kGrpThreads) tr[c] = P[c];
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
                for (int vv = 0; vv < 4; ++vv) {
                    const int c = vv * kGrpThreads + tg;
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
                const float l0 = pfl0[b];
                const uint32_t bit0 = (tg < m) ? ((row[tg >> 5] >> (tg & 31)) & 1u) : 0u;
                const uint32_t bit1 = (tg + 512 < m) ? ((row[(tg + 512) >> 5] >> ((tg + 512) & 31)) & 1u) : 0u;
                const uint32_t word = (lane < mw) ? row[lane] : 0u;
                if (!isfinite(l0)) {
                    for (int w = tg; w < nw; w += kGrpThreads) a.err[s * nw + w] = 0u;
                    if (tg == 0) { a.conv[s] = 0; a.iters[s] = -1; }
                } else {
                    const float pi = (l0 > 0.0f) ? 1.0f : ((l0 < 0.0f) ? -1.0f : 0.0f);
                    const bool flipped = pi < 0.0f;
                    // First check (l = 0), Eqs. 1 and 6: popcount of s XOR flip.
                    const uint32_t flip_lane = (flipped && lane < mw) ? flipw[lane] : 0u;
                    const int c0 = __reduce_add_sync(0xffffffffu, (int)__popc(word ^ flip_lane));
                    if (a.trace) {
                        float* tr = a.trace + (size_t)s * (size_t)(a.max_iter + 1) * (size_t)n;
                        for (int c = tg; c < n; c += kGrpThreads) tr[c] = pi;
                    }
                    if ((c0 == 0 && early) || a.max_iter == 0) {
                        for (int w = tg; w < nw; w += kGrpThreads)
                            a.err[s * nw + w] =
                                (pi < 0.0f) ? ((w == nw - 1 && (n & 31)) ? ((1u << (n & 31)) - 1u) : 0xffffffffu) : 0u;
                        if (tg == 0) { a.conv[s] = (c0 == 0) ? 1 : 0; a.iters[s] = 0; }
                    } else {
                        // Round 1 runs now on the priors themselves (Eq. 2 at l = 1).
                        state = kActive;
                        itk = 1;
                        idle = false;
                        fresh = true;
                        prior = pi;
                        sbits = bit0 | (bit1 << 1);
                        gcnt = c0;
                        st0 = bit0 ^ (flipped ? (degs & 1u) : 0u);
                        st1 = bit1 ^ (flipped ? ((degs >> 8) & 1u) : 0u);
                    }
                }
            }
        }
        if (state == kDone) break;

        if (!idle) {
            // A2 gains of the two checks (Eq. 7)
            float g0 = 1.0f, g1 = 1.0f;
            if (a.mode == kModeSAGMS) {
                const float base = a.amax - (a.amax - a.amin) * ((float)gcnt * a.inv_m);
                g0 = base * (st0 ? a.eta : 1.0f);
                g1 = base * (st1 ? a.eta : 1.0f);
            } else if (a.mode == kModeSMS) {
                g0 = a.alpha;
                g1 = a.alpha;
            }
            if (fresh) {
                // A3 on round-1 inputs: every real edge carries the prior s, padded slots +inf.
                // The minimum and second minimum of |v| are |s| (a check with one edge has no
                // second: +inf), the parity is the syndrome bit XOR the sign of s once per
                // edge, and every real edge gets the second-minimum output (|v_j| = m1).
                const uint32_t sgn = __float_as_uint(prior) & kSign;
                const float ms = fabsf(prior);
                const uint32_t deg0 = degs & 0xffu, deg1 = degs >> 8;
                const uint32_t par0 = ((sbits & 1u) << 31) ^ ((deg0 & 1u) ? sgn : 0u);
                const uint32_t par1 = ((sbits >> 1) << 31) ^ ((deg1 & 1u) ? sgn : 0u);
                const float m2a = (deg0 >= 2) ? ms : inf;
                const float m2b = (deg1 >= 2) ? ms : inf;
                const float o2a = __uint_as_float(__float_as_uint(fminf(g0 * m2a, kMsFamClip)) | par0);
                const float o2b = __uint_as_float(__float_as_uint(fminf(g1 * m2b, kMsFamClip)) | par1);
                const float d0 = __uint_as_float(__float_as_uint(o2a) ^ (~__float_as_uint(prior) & kSign));
                const float d1 = __uint_as_float(__float_as_uint(o2b) ^ (~__float_as_uint(prior) & kSign));
#pragma unroll
                for (int j = 0; j < DC; ++j) {
                    Cat(j, wq[j] & 0xffffu) = d0;
                    Cat(j, wq[j] >> 16) = d1;
                }
            } else {
                // A3 check-node update (C holds negated messages: P - L = P + D)
#pragma unroll
                for (int j = 0; j < DC; ++j)
                    v[j] = add2(v[j], make_float2(Cat(j, wq[j] & 0xffffu), Cat(j, wq[j] >> 16)));
                uint32_t par0 = (sbits & 1u) << 31, par1 = (sbits >> 1) << 31;
#pragma unroll
                for (int j = 0; j < DC; j += 2) {
                    par0 ^= __float_as_uint(v[j].x) ^ __float_as_uint(v[j + 1].x);
                    par1 ^= __float_as_uint(v[j].y) ^ __float_as_uint(v[j + 1].y);
                }
                par0 &= kSign;
                par1 &= kSign;
                float m1a = inf, m2a = inf, m1b = inf, m2b = inf;
#pragma unroll
                for (int j = 0; j < DC; j += 2) {
                    const float a0 = fabsf(v[j].x), a1 = fabsf(v[j + 1].x);
                    const float c0 = fabsf(v[j].y), c1 = fabsf(v[j + 1].y);
                    const float loa = fminf(a0, a1), hia = fmaxf(a0, a1);
                    const float lob = fminf(c0, c1), hib = fmaxf(c0, c1);
                    m2a = fminf(fminf(m2a, hia), fmaxf(m1a, loa));
                    m1a = fminf(m1a, loa);
                    m2b = fminf(fminf(m2b, hib), fmaxf(m1b, lob));
                    m1b = fminf(m1b, lob);
                }
                const float o1a = __uint_as_float(__float_as_uint(fminf(g0 * m1a, kMsFamClip)) | par0);
                const float o2a = __uint_as_float(__float_as_uint(fminf(g0 * m2a, kMsFamClip)) | par0);
                const float o1b = __uint_as_float(__float_as_uint(fminf(g1 * m1b, kMsFamClip)) | par1);
                const float o2b = __uint_as_float(__float_as_uint(fminf(g1 * m2b, kMsFamClip)) | par1);
#pragma unroll
                for (int j = 0; j < DC; ++j) {
                    const float ma = (fabsf(v[j].x) == m1a) ? o2a : o1a;
                    const float mb = (fabsf(v[j].y) == m1b) ? o2b : o1b;
                    Cat(j, wq[j] & 0xffffu) = __uint_as_float(__float_as_uint(ma) ^ (~__float_as_uint(v[j].x) & kSign));
                    Cat(j, wq[j] >> 16) = __uint_as_float(__float_as_uint(mb) ^ (~__float_as_uint(v[j].y) & kSign));
                }
            }
        }
        group_barrier(G);

        // Claim and prefetch the group's next shot (warp 0 of the group).
        if (consumed >= 0 && tg < 32) {
            const int nx = assign();
            if (tg == 0) pfidx[consumed ^ 1] = nx;
            prefetch(consumed ^ 1, nx);
        }

        if (!idle) {
            // A4 variable-node update: qubit pairs (2tg, 2tg + 1) and (1024 + 2tg, 1025 + 2tg)
            const float2 npr = make_float2(-prior, -prior);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int c = h * (NP / 2) + 2 * tg;
                float2 acc = npr;
#pragma unroll
                for (int q = 0; q < DV; ++q)
                    acc = add2(acc, *reinterpret_cast<const float2*>(smem + qc_C_off(DV, G, q) + (size_t)c * 4));
                *reinterpret_cast<float2*>(smem + PO + (size_t)c * 4) =
                    __ffma2_rn(acc, make_float2(-1.0f, -1.0f), make_float2(0.0f, 0.0f));
            }
        }
        group_barrier(G);
        ph ^= 1;
    }
}

template <int DC, int DV>
__global__ void __launch_bounds__(1024, 1) qc_kernel(const DecodeArgs a, const uint32_t* __restrict__ colQ) {
    static_assert(DC == 2 * DV && DC % 2 == 0, "slot j meets its qubit as edge j mod DV");
    extern __shared__ __align__(16) unsigned char smem[];
    const int t = threadIdx.x;
    const int tg = t % kGrpThreads;
    const float inf = __uint_as_float(0x7f800000u);
    {
        const int4* s = reinterpret_cast<const int4*>(colQ);
        int4* d = reinterpret_cast<int4*>(smem + qc_col_off(DV));
        for (int k = t; k < DC * kGrpThreads * 4 / 16; k += 1024) d[k] = __ldg(s + k);
    }
    // Posteriors (sentinel +inf), messages and bookkeeping of both groups start at zero.
    {
        float* z = reinterpret_cast<float*>(smem);
        for (int k = t; k < (int)(2 * qc_group_bytes(DV) / 4); k += 1024) z[k] = 0.0f;
        int* misc = reinterpret_cast<int*>(smem + qc_misc_off(DC, DV));
        if (t < 2 * kGrpMiscPerGroup / 4) misc[t] = 0;
    }
    __syncthreads();
    if (t < 2) *reinterpret_cast<float*>(smem + qc_P_off(DV, t) + kQcPadOff) = inf;
    // Check degrees (first-check flips for a negative prior: degree parity; the closed-form
    // first round needs the degree itself).
    const uint32_t* cq = reinterpret_cast<const uint32_t*>(smem + qc_col_off(DV));
    uint32_t deg0 = 0, deg1 = 0;
#pragma unroll
    for (int j = 0; j < DC; ++j) {
        const uint32_t w = cq[j * kGrpThreads + tg];
        deg0 += ((w & 0xffffu) != kQcPadOff) ? 1u : 0u;
        deg1 += ((w >> 16) != kQcPadOff) ? 1u : 0u;
    }
    uint32_t* flipw = reinterpret_cast<uint32_t*>(smem + qc_misc_off(DC, DV) + 2 * kGrpMiscPerGroup);
    if (t < kGrpThreads) {
        const uint32_t w0 = __ballot_sync(0xffffffffu, deg0 & 1u);
        const uint32_t w1 = __ballot_sync(0xffffffffu, deg1 & 1u);
        if ((t & 31) == 0) { flipw[t >> 5] = w0; flipw[(t + kGrpThreads) >> 5] = w1; }
    }
    __syncthreads();
    if (t < kGrpThreads)
        qc_group<DC, DV, 0>(a, smem, tg, deg0 | (deg1 << 8));
    else
        qc_group<DC, DV, 1>(a, smem, tg, deg0 | (deg1 << 8));
}

}  // namespace sagms
