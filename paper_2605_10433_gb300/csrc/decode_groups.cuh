// Two-group decoder kernel for the MS family on codes of up to 1024 checks and 2048 qubits
// (per-shot priors).
//
// A 1024-thread CTA holds two independent groups of 512 threads.  Each group decodes one
// shot at a time and refills as shots finish, exactly like one slot of decode_slots.cuh;
// a thread owns two checks of its group's shot (checks t and t + 512, paired in FP32x2
// registers) and four qubits.  The groups synchronise with their own named barriers, so
// they drift out of phase: while one group runs its arithmetic-bound check-node phase the
// other runs its shared-memory-bound gather and variable-node phases, which a single
// one-CTA-per-SM kernel of this size cannot overlap.
//
// Shared memory (byte offsets from grp_* below; host and device use the same arithmetic):
//   P_g[2048 + 4]         posteriors of group g's shot; P_g[2048] = +inf is the sentinel
//                         padding slots read
//   C_g[DC * 1024 + 4]    negated CN->VN messages D = -L_{i->j} at [j * 1024 + i];
//                         C_g[DC * 1024] = 0 is the target of padded qubit slots
//   colB[2][DC][1024]     u16: byte offset of P_g[col(i, j)] from the shared base
//   vneB[2][DV][2048]     u32: byte offset of the q-th edge message of qubit c in C_g
//   per-group bookkeeping (counts, claims, prefetch buffers) and the first-check flip words
// Every per-check access is then a register plus an immediate.  The arithmetic of each
// check and qubit is, operation for operation, the one of decode_kernel.cuh (bitwise
// identical results).
#pragma once

#include "decode_slots.cuh"

namespace sagms {

constexpr int kGrpThreads = 512;
constexpr int kGrpChecks = 1024;
constexpr int kGrpQubits = 2048;
constexpr int kGrpMiscPerGroup = 320;   // cnt[2] claim[2] pfidx[2] shotsm[2] pfl0[2] pad, pfsyn[2][32]

__host__ __device__ inline size_t grp_P_off(int g) { return (size_t)g * (kGrpQubits + 4) * 4; }
__host__ __device__ inline size_t grp_C_off(int DC, int g) {
    return grp_P_off(2) + (size_t)g * ((size_t)DC * kGrpChecks + 4) * 4;
}
__host__ __device__ inline size_t grp_colB_off(int DC) { return grp_C_off(DC, 2); }
__host__ __device__ inline size_t grp_vneB_off(int DC) { return grp_colB_off(DC) + (size_t)2 * DC * kGrpChecks * 2; }
__host__ __device__ inline size_t grp_misc_off(int DC, int DV) {
    return grp_vneB_off(DC) + (size_t)2 * DV * kGrpQubits * 4;
}
__host__ __device__ inline size_t grp_smem_bytes(int DC, int DV) {
    return grp_misc_off(DC, DV) + 2 * kGrpMiscPerGroup + 32 * 4;
}

struct GroupLayout {
    const uint16_t* colB;  // [2][DC][1024]
    const uint32_t* vneB;  // [2][DV][2048]
};

__device__ __forceinline__ void group_barrier(int g) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(kGrpThreads) : "memory");
}

template <int DC, int DV>
__global__ void __launch_bounds__(1024, 1) group_kernel(const DecodeArgs a, const GroupLayout lay) {
    static_assert(DC % 2 == 0, "edge pairs");
    constexpr int G = kGrpThreads, MC = kGrpChecks, NP = kGrpQubits, VPT = NP / G;
    extern __shared__ __align__(16) unsigned char smem[];
    const bool early = (a.flags & kFlagNoEarlyStop) == 0;
    const int t = threadIdx.x;
    const int g = t / G;
    const int tg = t % G;
    const int lane = t & 31;
    const int n = a.n, m = a.m;
    const int mw = (m + 31) >> 5, nw = (n + 31) >> 5;
    const float inf = __uint_as_float(0x7f800000u);

    float* P = reinterpret_cast<float*>(smem + grp_P_off(g));
    float* C = reinterpret_cast<float*>(smem + grp_C_off(DC, g));
    const uint16_t* colB = reinterpret_cast<const uint16_t*>(smem + grp_colB_off(DC)) + g * DC * MC;
    const uint32_t* vneB = reinterpret_cast<const uint32_t*>(smem + grp_vneB_off(DC)) + g * DV * NP;
    unsigned char* misc = smem + grp_misc_off(DC, DV);
    int* cnt = reinterpret_cast<int*>(misc + g * kGrpMiscPerGroup);   // [2 parity]
    int* claim = cnt + 2;                                              // [2]
    int* pfidx = cnt + 4;                                              // [2 buffers]
    int* shotsm = cnt + 6;                                             // [2 buffers]
    float* pfl0 = reinterpret_cast<float*>(cnt + 8);                   // [2 buffers]
    float* amaxsh = reinterpret_cast<float*>(cnt + 10);                // alpha_max of the group's shot
    uint32_t* pfsyn = reinterpret_cast<uint32_t*>(cnt + 16);           // [2 buffers][32]
    uint32_t* flipw = reinterpret_cast<uint32_t*>(misc + 2 * kGrpMiscPerGroup);   // [32]
    const uint16_t pad = (uint16_t)(grp_P_off(g) + (size_t)NP * 4);

    // Stage the code graph and initialise both groups' state (whole CTA).
    {
        const int4* s1 = reinterpret_cast<const int4*>(lay.colB);
        int4* d1 = reinterpret_cast<int4*>(smem + grp_colB_off(DC));
        for (int k = t; k < 2 * DC * MC * 2 / 16; k += 1024) d1[k] = __ldg(s1 + k);
        const int4* s2 = reinterpret_cast<const int4*>(lay.vneB);
        int4* d2 = reinterpret_cast<int4*>(smem + grp_vneB_off(DC));
        for (int k = t; k < 2 * DV * NP * 4 / 16; k += 1024) d2[k] = __ldg(s2 + k);
    }
    for (int c = tg; c < NP + 4; c += G) P[c] = (c < n) ? 0.0f : inf;
    for (int k = tg; k < DC * MC + 4; k += G) C[k] = 0.0f;
    if (tg < 16) cnt[tg] = 0;
    __syncthreads();
    // First check of a shot with a negative prior: every hard decision is 1, so a check's
    // residual bit (Eq. 1) is s_i XOR its degree parity.
    int haspad_local = 0;
    {
        int d = 0;
#pragma unroll
        for (int j = 0; j < DC; ++j) d += (colB[j * MC + tg] != pad) ? 1 : 0;
        int d2 = 0;
#pragma unroll
        for (int j = 0; j < DC; ++j) d2 += (colB[j * MC + tg + G] != pad) ? 1 : 0;
        if ((tg < m && d < DC) || (tg + G < m && d2 < DC)) haspad_local = 1;
        if (g == 0) {
            const uint32_t w0 = __ballot_sync(0xffffffffu, (tg < m) && (d & 1));
            const uint32_t w1 = __ballot_sync(0xffffffffu, (tg + G < m) && (d2 & 1));
            if (lane == 0) { flipw[tg >> 5] = w0; flipw[(tg + G) >> 5] = w1; }
        }
    }
    // Shots: each group takes chunks of 2^chunk_lg consecutive shots (see decode_slots.cuh);
    // with a work counter the chunks are claimed dynamically, else group b = 2 * CTA + g
    // takes chunks b, b + 2G, ...
    const int nshots = (int)a.shots;
    const int clg = a.chunk_lg;
    const int cmask = (1 << clg) - 1;
    const bool dynamic = a.work != nullptr;
    const int gid = 2 * (int)blockIdx.x + g;
    const int gstride = 2 * (int)gridDim.x;
    if (tg == 0) {
        claim[0] = dynamic ? atomicAdd(a.work, 1) : gid;
        claim[1] = dynamic ? atomicAdd(a.work, 1) : gid + gstride;
    }
    const bool haspad = __syncthreads_or(haspad_local) != 0;
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
    int pbuf = 0;         // prefetch buffer the next refill reads
    int ph = 0;
    const uint32_t fl0 = (flipw[tg >> 5] >> (tg & 31)) & 1u;
    const uint32_t fl1 = (flipw[(tg + G) >> 5] >> ((tg + G) & 31)) & 1u;

    while (state != kDone) {
        // A5: gather the two checks' posteriors, residual bits, unsatisfied count
        float2 v[DC];
#pragma unroll
        for (int j = 0; j < DC; ++j)
            v[j] = make_float2(*reinterpret_cast<const float*>(smem + colB[j * MC + tg]),
                               *reinterpret_cast<const float*>(smem + colB[j * MC + tg + G]));
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
        group_barrier(g);
        int gcnt = cnt[ph];
        uint32_t st0 = x0 >> 31, st1 = x1 >> 31;
        if (tg == 0) cnt[ph ^ 1] = 0;
        if (a.trace && state == kActive) {
            float* tr = a.trace + ((size_t)shotsm[pbuf ^ 1] * (size_t)(a.max_iter + 1) + (size_t)itk) * (size_t)n;
            for (int c = tg; c < n; c += G) tr[c] = P[c];
        }

        // A6: finish, refill, or count the round about to run.
        bool zero = false, fresh = false;
        int consumed = -1;   // prefetch buffer taken this round
        const bool fin = state == kActive && ((gcnt == 0 && early) || itk == a.max_iter);
        if (state == kActive && !fin) {
            itk++;
        } else {
            if (fin) {
                const int s = shotsm[pbuf ^ 1];
#pragma unroll
                for (int vv = 0; vv < VPT; ++vv) {
                    const int c = vv * G + tg;
                    const uint32_t word = __ballot_sync(0xffffffffu, (c < n) && (__float_as_uint(P[c]) >> 31));
                    if (lane == 0 && c < n) a.err[s * nw + (c >> 5)] = word;
                }
                if (tg == 0) { a.conv[s] = (gcnt == 0) ? 1 : 0; a.iters[s] = itk; }
                state = kPending;
            }
            zero = true;
            if (state == kPending) {
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
                    const uint32_t bit1 = (tg + G < m) ? ((row[(tg + G) >> 5] >> ((tg + G) & 31)) & 1u) : 0u;
                    const uint32_t word = (lane < mw) ? row[lane] : 0u;
                    if (!isfinite(l0)) {
                        for (int w = tg; w < nw; w += G) a.err[s * nw + w] = 0u;
                        if (tg == 0) { a.conv[s] = 0; a.iters[s] = -1; }
                    } else {
                        const float pi = (l0 > 0.0f) ? 1.0f : ((l0 < 0.0f) ? -1.0f : 0.0f);
                        prior = pi;
                        // alpha_max of the new shot.  Every thread of the group stores the
                        // same value, so each thread's own read-back is that value.
                        if (a.flags & kFlagAutoCeiling) *amaxsh = shot_alpha_max(a, l0);
                        sbits = bit0 | (bit1 << 1);
                        const bool flipped = pi < 0.0f;
                        // First check (l = 0), Eqs. 1 and 6: popcount of s XOR flip.
                        const uint32_t flip_lane = (flipped && lane < mw) ? flipw[lane] : 0u;
                        const int c0 = __reduce_add_sync(0xffffffffu, (int)__popc(word ^ flip_lane));
                        if (a.trace) {
                            float* tr = a.trace + (size_t)s * (size_t)(a.max_iter + 1) * (size_t)n;
                            for (int c = tg; c < n; c += G) tr[c] = pi;
                        }
                        if ((c0 == 0 && early) || a.max_iter == 0) {
                            for (int w = tg; w < nw; w += G)
                                a.err[s * nw + w] =
                                    (pi < 0.0f) ? ((w == nw - 1 && (n & 31)) ? ((1u << (n & 31)) - 1u) : 0xffffffffu) : 0u;
                            if (tg == 0) { a.conv[s] = (c0 == 0) ? 1 : 0; a.iters[s] = 0; }
                        } else {
                            // Round 1 runs now on the priors themselves (Eq. 2 at l = 1).
                            state = kActive;
                            itk = 1;
                            zero = false;
                            fresh = true;
                            gcnt = c0;
                            st0 = bit0 ^ (flipped ? fl0 : 0u);
                            st1 = bit1 ^ (flipped ? fl1 : 0u);
                        }
                    }
                }
            }
        }
        if (state == kDone) break;

        // A2 gains of the two checks (Eq. 7)
        float g0 = 1.0f, g1 = 1.0f;
        if (a.mode == kModeSAGMS) {
            const float amax = (a.flags & kFlagAutoCeiling) ? *amaxsh : a.amax;
            const float base = amax - (amax - a.amin) * ((float)gcnt * a.inv_m);
            g0 = base * (st0 ? a.eta : 1.0f);
            g1 = base * (st1 ? a.eta : 1.0f);
        } else if (a.mode == kModeSMS) {
            g0 = a.alpha;
            g1 = a.alpha;
        }
        // A3 check-node update for both checks (C holds negated messages: P - L = P + D)
#pragma unroll
        for (int j = 0; j < DC; ++j) v[j] = add2(v[j], make_float2(C[j * MC + tg], C[j * MC + tg + G]));
        if (fresh) {
            if (haspad) {
#pragma unroll
                for (int j = 0; j < DC; ++j)
                    v[j] = make_float2((colB[j * MC + tg] == pad) ? inf : prior,
                                       (colB[j * MC + tg + G] == pad) ? inf : prior);
            } else {
#pragma unroll
                for (int j = 0; j < DC; ++j) v[j] = make_float2(prior, prior);
            }
        }
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
        const float o1a = zero ? 0.0f : __uint_as_float(__float_as_uint(fminf(g0 * m1a, kMsFamClip)) | par0);
        const float o2a = zero ? 0.0f : __uint_as_float(__float_as_uint(fminf(g0 * m2a, kMsFamClip)) | par0);
        const float o1b = zero ? 0.0f : __uint_as_float(__float_as_uint(fminf(g1 * m1b, kMsFamClip)) | par1);
        const float o2b = zero ? 0.0f : __uint_as_float(__float_as_uint(fminf(g1 * m2b, kMsFamClip)) | par1);
#pragma unroll
        for (int j = 0; j < DC; ++j) {
            const float ma = (fabsf(v[j].x) == m1a) ? o2a : o1a;
            const float mb = (fabsf(v[j].y) == m1b) ? o2b : o1b;
            C[j * MC + tg] = __uint_as_float(__float_as_uint(ma) ^ (~__float_as_uint(v[j].x) & kSign));
            C[j * MC + tg + G] = __uint_as_float(__float_as_uint(mb) ^ (~__float_as_uint(v[j].y) & kSign));
        }
        group_barrier(g);

        // Claim and prefetch the group's next shot (warp 0 of the group).
        if (consumed >= 0 && tg < 32) {
            const int nx = assign();
            if (tg == 0) pfidx[consumed ^ 1] = nx;
            prefetch(consumed ^ 1, nx);
        }

        // A4 variable-node update: qubits (tg, tg + 512) and (tg + 1024, tg + 1536) in pairs
        const float2 npr = make_float2(-prior, -prior);
#pragma unroll
        for (int vv = 0; vv < VPT; vv += 2) {
            const int c0 = vv * G + tg, c1 = c0 + G;
            float2 acc = npr;
#pragma unroll
            for (int q = 0; q < DV; ++q)
                acc = add2(acc, make_float2(*reinterpret_cast<const float*>(smem + vneB[q * NP + c0]),
                                            *reinterpret_cast<const float*>(smem + vneB[q * NP + c1])));
            const float2 pp = __ffma2_rn(acc, make_float2(-1.0f, -1.0f), make_float2(0.0f, 0.0f));
            P[c0] = pp.x;
            P[c1] = pp.y;
        }
        group_barrier(g);
        ph ^= 1;
    }
}

}  // namespace sagms
