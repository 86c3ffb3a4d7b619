// Two-slot continuous-batching decoder kernel for the MS family (MS / SMS / SAGMS).
//
// A CTA owns two shot slots that advance independently through Algorithm 1.  When a slot's
// residual syndrome reaches zero (or its iteration budget runs out) the CTA writes that
// shot's result and loads the next shot into the slot in the same iteration: the slot's
// check-node outputs are forced to zero for one round, so the variable-node update leaves
// P = L0 of the new shot, and its first check happens at the next iteration.  No slot waits
// for the other, and the code graph, the barriers and the index loads are shared by two
// shots.
//
// Layout (shared memory, sizes fixed at compile time for the thread count MP = padded check
// count and NP = padded qubit count, so every per-thread address is a register plus an
// immediate):
//   P2[NP]         float2: posterior of qubit c for slot 0 (.x) and slot 1 (.y); +inf past n
//   C2[DC*MP + 2]  float2: CN->VN message of edge (i, j) at [j*MP + i]; C2[DC*MP] = 0
//   colB[DC*MP]    u16: byte offset of P2[col(i, j)]
//   vneB[DV*NP]    u32: byte offset (from C2) of the q-th edge of qubit c; padding -> zero slot
// Packed FP32 pairs (add/sub.rn.f32x2) update both slots' edges in one instruction; min /
// compare work stays per slot.  The arithmetic of each slot is, operation for operation and
// in the same order, the one of decode_kernel.cuh, so both kernels give bitwise identical
// results.
#pragma once

#include "decode_kernel.cuh"

namespace sagms {

// Paired FP32 add (round to nearest).
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

struct SlotLayout {
    const uint16_t* colB;  // [DC][MP]
    const uint32_t* vneB;  // [DV][NP]
};

// Shared memory of one CTA (bytes), in the order the kernel carves it up.
__host__ __device__ inline size_t slot_smem_bytes(int DC, int DV, int MP, int NP, bool per_qubit) {
    return (size_t)(NP + 2) * 8                      // P2 (+ sentinel)
           + ((size_t)DC * MP + 2) * 8               // C2 (+ zero slot)
           + (per_qubit ? (size_t)(NP + 4) * 4 : 0)  // PQ
           + (size_t)DC * MP * 2                     // colB
           + (size_t)DV * NP * 4                     // vneB
           + 16 + 32 * 4 + 64 * 4 + 16 + 16 + 16     // cnt, flipw, negw, claim, pfidx, shotsm
           + 16                                      // amaxsh
           + 2 * 2 * 32 * 4 + 2 * 2 * 4;             // prefetch buffers (syndrome rows, priors)
}

// Resident CTAs per SM the register allocation must allow: 1024 threads per SM, except the
// widest checks at 256 threads, which trade a fourth CTA for spill-free registers.
template <int DC, int MP>
struct SlotBounds {
    static constexpr int kMinBlocks = (DC >= 12 && MP == 256) ? 3 : ((1024 / MP) > 0 ? (1024 / MP) : 1);
};

__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <int DC, int DV, int MP, int NP>
__global__ void __launch_bounds__(MP, SlotBounds<DC, MP>::kMinBlocks)
slot_kernel(const DecodeArgs a, const SlotLayout lay) {
    static_assert(NP % MP == 0, "qubit padding must be a multiple of the thread count");
    static_assert(MP <= 1024, "one thread per check");
    constexpr int VPT = NP / MP;
    extern __shared__ __align__(16) unsigned char smem[];
    const bool per_qubit = (a.flags & kFlagPerQubit) != 0;
    const bool early = (a.flags & kFlagNoEarlyStop) == 0;
    float2* P2 = reinterpret_cast<float2*>(smem);
    float2* C2 = P2 + NP + 2;
    float* PQ = reinterpret_cast<float*>(C2 + DC * MP + 2);
    uint16_t* colB = reinterpret_cast<uint16_t*>(PQ + (per_qubit ? NP + 4 : 0));
    uint32_t* vneB = reinterpret_cast<uint32_t*>(colB + DC * MP);
    int* cnt = reinterpret_cast<int*>(vneB + DV * NP);       // [2 parity][2 slots]
    uint32_t* flipw = reinterpret_cast<uint32_t*>(cnt + 4);  // [32] first-check flip bit per check
    uint32_t* negw = flipw + 32;                              // [64] per-qubit [L0_j < 0] bits
    int* claim = reinterpret_cast<int*>(negw + 64);           // [2 slots][2] claimed shot indices
    uint32_t* pfsyn = reinterpret_cast<uint32_t*>(claim + 4); // [2 slots][2 buffers][32] syndrome rows
    float* pfl0 = reinterpret_cast<float*>(pfsyn + 128);      // [2 slots][2 buffers] priors
    int* pfidx = reinterpret_cast<int*>(pfl0 + 4);            // [2 slots][2 buffers] shot in each buffer
    int* shotsm = pfidx + 4;                                  // [2 slots][2] shot being decoded
    float* amaxsh = reinterpret_cast<float*>(shotsm + 4);     // [2 slots] alpha_max of the slot's shot
    const unsigned char* c2base = reinterpret_cast<const unsigned char*>(C2);

    const int t = threadIdx.x;
    const int lane = t & 31;
    const int n = a.n, m = a.m;
    const int mw = (m + 31) >> 5, nw = (n + 31) >> 5;
    const float inf = __uint_as_float(0x7f800000u);
    const uint16_t pad = (uint16_t)(NP * 8);   // padding slots read the sentinel P2[NP] = +inf
    // C2 holds NEGATED messages D = -L_{i->j}: the check node then forms P_j - L_{i->j} as the
    // plain sum P_j + D, and the variable node sums Q = -L0 + sum D and stores P = -Q + 0.
    // Round-to-nearest is symmetric under negation, so every value is bitwise the one of
    // the unnegated formulation (decode_kernel.cuh), including +0 for an exact cancellation.

    {
        const int4* s1 = reinterpret_cast<const int4*>(lay.colB);
        int4* d1 = reinterpret_cast<int4*>(colB);
        for (int k = t; k < DC * MP * 2 / 16; k += MP) d1[k] = __ldg(s1 + k);
        const int4* s2 = reinterpret_cast<const int4*>(lay.vneB);
        int4* d2 = reinterpret_cast<int4*>(vneB);
        for (int k = t; k < DV * NP * 4 / 16; k += MP) d2[k] = __ldg(s2 + k);
    }
    for (int c = t; c < NP + 2; c += MP) P2[c] = (c < n) ? make_float2(0.0f, 0.0f) : make_float2(inf, inf);
    if (per_qubit)
        for (int c = t; c < NP + 4; c += MP) PQ[c] = (c < n) ? __ldg(a.L0 + c) + 0.0f : inf;   // -0 -> +0
    if (t < 2) C2[DC * MP + t] = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int j = 0; j < DC; ++j) C2[j * MP + t] = make_float2(0.0f, 0.0f);
    if (t < 4) cnt[t] = 0;
    __syncthreads();
    // First check of a shot: every hard decision is [prior_j < 0], so the residual bit of a
    // check (Eq. 1) is s_i XOR flip_i with flip_i = parity of its negative priors:
    // per-qubit priors -> from PQ; a negative per-shot prior -> the check's degree parity.
    int pq_ok = 1;
    int haspad_local = 0;
    {
        uint32_t f = 0u;
        int d = DC;
        if (t < m) {
            d = 0;
#pragma unroll
            for (int j = 0; j < DC; ++j) {
                const uint16_t off = colB[j * MP + t];
                if (off != pad) {
                    ++d;
                    if (per_qubit) f ^= __float_as_uint(PQ[off >> 3]) >> 31;
                }
            }
            if (!per_qubit) f = (uint32_t)d & 1u;
        }
        const uint32_t w = __ballot_sync(0xffffffffu, f);
        if (lane == 0) flipw[t >> 5] = w;
        if (t < m && d < DC) haspad_local = 1;
        if (per_qubit) {
            for (int c = t; c < n; c += MP) pq_ok &= isfinite(PQ[c]) ? 1 : 0;
#pragma unroll
            for (int vv = 0; vv < VPT; ++vv) {
                const int c = vv * MP + t;
                const uint32_t nb = __ballot_sync(0xffffffffu, (c < n) && (__float_as_uint(PQ[c]) >> 31));
                if (lane == 0 && c < n) negw[c >> 5] = nb;
            }
        }
    }

    // Shot indices fit in 32 bits: the host splits larger batches into several launches.
    // A CTA takes its shots as chunks of 2^chunk_lg consecutive shots, assigned to its two
    // slots in order.  With a work counter the chunks are claimed dynamically (thread 0,
    // one atomic per chunk, a chunk ahead of its use, through the two-entry ring `claim`);
    // without one, CTA b takes chunks b, b + G, b + 2G, ...
    const int nshots = (int)a.shots;
    const int clg = a.chunk_lg;
    const int cmask = (1 << clg) - 1;
    const bool dynamic = a.work != nullptr;
    if (t == 0) {
        claim[0] = dynamic ? atomicAdd(a.work, 1) : (int)blockIdx.x;
        claim[1] = dynamic ? atomicAdd(a.work, 1) : (int)blockIdx.x + (int)gridDim.x;
    }
    int seqp = 0;   // shots this CTA has assigned to its slots so far
    pq_ok = __syncthreads_and(pq_ok);
    const bool haspad = __syncthreads_or(haspad_local) != 0;   // some check has fewer than DC edges
    // Next shot of this CTA's sequence.  Entering chunk c (c > 0) claims chunk c + 1 into the
    // ring entry that held chunk c - 1, which is fully assigned; the claim has a whole chunk
    // of refills to land before it is read.
    auto assign = [&]() -> int {
        const int p = seqp++;
        const int c = p >> clg;
        const long long idx = ((long long)claim[c & 1] << clg) + (p & cmask);
        if ((p & cmask) == 0 && c > 0 && t == 0)
            claim[(c + 1) & 1] = dynamic ? atomicAdd(a.work, 1) : (int)blockIdx.x + (c + 1) * (int)gridDim.x;
        return idx < (long long)nshots ? (int)idx : nshots;
    };
    const int first0 = assign();
    const int first1 = assign();
    if (t == 0) { pfidx[0] = first0; pfidx[2] = first1; }
    // Inputs of the shot a slot starts next (its syndrome row and prior) are copied into
    // shared memory by warp 0 with cp.async one refill ahead, double-buffered per slot;
    // warp 0 waits for its copies before each CTA barrier that precedes their use.
    auto prefetch = [&](int k, int b, int s) {
        if (t < 32 && s < nshots) {
            if (lane < mw) cp_async4(pfsyn + (k * 2 + b) * 32 + lane, a.syn + s * mw + lane);
            if (lane == 0 && !per_qubit) cp_async4(pfl0 + k * 2 + b, a.L0 + s);
            cp_async_commit();
        }
    };
    prefetch(0, 0, first0);
    prefetch(1, 0, first1);

    // Slot states: decoding, waiting for its next shot, no shots left.
    enum { kActive = 0, kPending = 1, kDone = 2 };
    int state[2] = {kPending, kPending};
    int itk[2] = {0, 0};
    float prior[2] = {0.0f, 0.0f};
    uint32_t sbits = 0;  // bit k: this thread's check syndrome bit of slot k
    uint32_t pbits = 0;  // bit k: prefetch buffer slot k reads at its next refill

    int ph = 0;
    while (state[0] != kDone || state[1] != kDone) {
        // A5: gather, residual bits, unsatisfied counts of both slots
        float2 v[DC];
        uint32_t x0 = (sbits & 1u) << 31, x1 = (sbits >> 1) << 31;
#pragma unroll
        for (int j = 0; j < DC; ++j) v[j] = *reinterpret_cast<const float2*>(smem + colB[j * MP + t]);
#pragma unroll
        for (int j = 0; j < DC; j += 2) {
            x0 ^= __float_as_uint(v[j].x) ^ __float_as_uint(v[j + 1].x);
            x1 ^= __float_as_uint(v[j].y) ^ __float_as_uint(v[j + 1].y);
        }
        const uint32_t b0 = __ballot_sync(0xffffffffu, x0 >> 31);
        const uint32_t b1 = __ballot_sync(0xffffffffu, x1 >> 31);
        if (lane == 0) {
            atomicAdd(&cnt[ph * 2 + 0], __popc(b0));
            atomicAdd(&cnt[ph * 2 + 1], __popc(b1));
        }
        if (t < 32) cp_async_wait_all();
        __syncthreads();
        int gcnt[2] = {cnt[ph * 2 + 0], cnt[ph * 2 + 1]};
        uint32_t gst[2] = {x0 >> 31, x1 >> 31};
        if (t == 0) { cnt[(ph ^ 1) * 2 + 0] = 0; cnt[(ph ^ 1) * 2 + 1] = 0; }
        if (a.trace) {
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                if (state[k] != kActive) continue;
                const int sk = shotsm[2 * k + (((pbits >> k) & 1) ^ 1)];
                float* tr = a.trace + ((size_t)sk * (size_t)(a.max_iter + 1) + (size_t)itk[k]) * (size_t)n;
                for (int c = t; c < n; c += MP) tr[c] = k ? P2[c].y : P2[c].x;
            }
        }

        // A6 per slot: the common case (both slots decoding, neither finished) is one test.
        bool zero[2] = {false, false};
        uint32_t fresh = 0u;    // bit k: slot k runs the first round of a newly loaded shot
        uint32_t consumed = 0u; // bit 2k: slot k took its prefetched shot; bit 2k+1: from buffer 1
        const bool fin0 = state[0] == kActive && ((gcnt[0] == 0 && early) || itk[0] == a.max_iter);
        const bool fin1 = state[1] == kActive && ((gcnt[1] == 0 && early) || itk[1] == a.max_iter);
        if (!(fin0 || fin1 || state[0] != kActive || state[1] != kActive)) {
            itk[0]++;
            itk[1]++;
        } else {
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const bool fin = k ? fin1 : fin0;
                if (fin) {
                    const int s = shotsm[2 * k + (((pbits >> k) & 1) ^ 1)];
#pragma unroll
                    for (int vv = 0; vv < VPT; ++vv) {
                        const int c = vv * MP + t;
                        const float pc = k ? P2[c].y : P2[c].x;
                        const uint32_t word = __ballot_sync(0xffffffffu, (c < n) && (__float_as_uint(pc) >> 31));
                        if (lane == 0 && c < n) a.err[s * nw + (c >> 5)] = word;
                    }
                    if (t == 0) { a.conv[s] = (gcnt[k] == 0) ? 1 : 0; a.iters[s] = itk[k]; }
                    state[k] = kPending;
                } else if (state[k] == kActive) {
                    itk[k]++;
                    continue;
                }
                zero[k] = true;
                if (state[k] != kPending) continue;
                // Start the prefetched shot (at most one per round: a shot finished at its
                // first check leaves the slot pending for the next round).
                const int b = (pbits >> k) & 1;
                const int s = pfidx[2 * k + b];
                if (s >= nshots) { state[k] = kDone; continue; }
                if (t == 0) shotsm[2 * k + b] = s;
                pbits ^= 1u << k;
                consumed |= (1u | ((uint32_t)b << 1)) << (2 * k);   // warp 0 claims and prefetches later
                const uint32_t* row = pfsyn + (k * 2 + b) * 32;
                const float l0 = per_qubit ? 0.0f : pfl0[k * 2 + b];
                const uint32_t bit = (t < m) ? ((row[t >> 5] >> (t & 31)) & 1u) : 0u;
                const uint32_t word = (lane < mw) ? row[lane] : 0u;
                if (!(per_qubit ? (pq_ok != 0) : isfinite(l0))) {
                    for (int w = t; w < nw; w += MP) a.err[s * nw + w] = 0u;
                    if (t == 0) { a.conv[s] = 0; a.iters[s] = -1; }
                    continue;
                }
                const float pi = per_qubit ? 0.0f : ((l0 > 0.0f) ? 1.0f : ((l0 < 0.0f) ? -1.0f : 0.0f));
                prior[k] = pi;
                // alpha_max of the new shot.  Every thread stores the same value, so each
                // thread's own read-back below is that value without a barrier.
                if (a.flags & kFlagAutoCeiling) amaxsh[k] = shot_alpha_max(a, l0);
                sbits = (sbits & ~(1u << k)) | (bit << k);
                const bool flipped = per_qubit || pi < 0.0f;
                // First check (l = 0) of the new shot, Eqs. 1 and 6: popcount of s XOR flip.
                const uint32_t flip_lane = (flipped && lane < mw) ? flipw[lane] : 0u;
                const int c0 = __reduce_add_sync(0xffffffffu, (int)__popc(word ^ flip_lane));
                if (a.trace) {
                    float* tr = a.trace + (size_t)s * (size_t)(a.max_iter + 1) * (size_t)n;
                    for (int c = t; c < n; c += MP) tr[c] = per_qubit ? PQ[c] : pi;
                }
                if ((c0 == 0 && early) || a.max_iter == 0) {
                    for (int w = t; w < nw; w += MP) {
                        uint32_t e0;
                        if (per_qubit) e0 = negw[w];
                        else e0 = (pi < 0.0f) ? ((w == nw - 1 && (n & 31)) ? ((1u << (n & 31)) - 1u) : 0xffffffffu) : 0u;
                        a.err[s * nw + w] = e0;
                    }
                    if (t == 0) { a.conv[s] = (c0 == 0) ? 1 : 0; a.iters[s] = 0; }
                    continue;
                }
                // Round 1 runs now: its inputs are the priors themselves (C = 0), Eq. 2 at l = 1;
                // the check-node phase substitutes them for this slot.
                state[k] = kActive;
                itk[k] = 1;
                zero[k] = false;
                fresh |= 1u << k;
                gcnt[k] = c0;
                gst[k] = bit ^ ((flipped && t < m) ? ((flipw[t >> 5] >> (t & 31)) & 1u) : 0u);
            }
            if (state[0] == kDone && state[1] == kDone) break;
        }

        // A2 gains (Eq. 7 with this round's count and residual bit)
        float g0 = 1.0f, g1 = 1.0f;
        if (a.mode == kModeSAGMS) {
            const bool autoc = (a.flags & kFlagAutoCeiling) != 0;
            const float am0 = autoc ? amaxsh[0] : a.amax;
            const float am1 = autoc ? amaxsh[1] : a.amax;
            g0 = (am0 - (am0 - a.amin) * ((float)gcnt[0] * a.inv_m)) * (gst[0] ? a.eta : 1.0f);
            g1 = (am1 - (am1 - a.amin) * ((float)gcnt[1] * a.inv_m)) * (gst[1] ? a.eta : 1.0f);
        } else if (a.mode == kModeSMS) {
            g0 = a.alpha;
            g1 = a.alpha;
        }
        // A3 check-node update for both slots
#pragma unroll
        for (int j = 0; j < DC; ++j) v[j] = add2(v[j], C2[j * MP + t]);   // P - L_old (C2 is negated)
        if (fresh) {
            // A freshly loaded slot's round-1 inputs are its priors (+inf on padding slots).
            if (per_qubit || haspad) {
#pragma unroll
                for (int j = 0; j < DC; ++j) {
                    const uint16_t off = colB[j * MP + t];
                    const float pq = per_qubit ? PQ[off >> 3] : 0.0f;
                    const float p0 = (off == pad) ? inf : (per_qubit ? pq : prior[0]);
                    const float p1 = (off == pad) ? inf : (per_qubit ? pq : prior[1]);
                    if (fresh & 1u) v[j].x = p0;
                    if (fresh & 2u) v[j].y = p1;
                }
            } else if (fresh == 1u) {
#pragma unroll
                for (int j = 0; j < DC; ++j) v[j].x = prior[0];
            } else if (fresh == 2u) {
#pragma unroll
                for (int j = 0; j < DC; ++j) v[j].y = prior[1];
            } else {
#pragma unroll
                for (int j = 0; j < DC; ++j) v[j] = make_float2(prior[0], prior[1]);
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
        // Smallest and second smallest |v| per slot, two edges at a time:
        // lo/hi of the pair, then m2 = min(m2, hi, max(m1, lo)), m1 = min(m1, lo).
        float m1a = inf, m2a = inf, m1b = inf, m2b = inf;
#pragma unroll
        for (int j = 0; j < DC; j += 2) {
            const float a0 = fabsf(v[j].x), a1 = fabsf(v[j + 1].x);
            const float b0 = fabsf(v[j].y), b1 = fabsf(v[j + 1].y);
            const float loa = fminf(a0, a1), hia = fmaxf(a0, a1);
            const float lob = fminf(b0, b1), hib = fmaxf(b0, b1);
            m2a = fminf(fminf(m2a, hia), fmaxf(m1a, loa));
            m1a = fminf(m1a, loa);
            m2b = fminf(fminf(m2b, hib), fmaxf(m1b, lob));
            m1b = fminf(m1b, lob);
        }
        const float o1a = zero[0] ? 0.0f : __uint_as_float(__float_as_uint(fminf(g0 * m1a, kMsFamClip)) | par0);
        const float o2a = zero[0] ? 0.0f : __uint_as_float(__float_as_uint(fminf(g0 * m2a, kMsFamClip)) | par0);
        const float o1b = zero[1] ? 0.0f : __uint_as_float(__float_as_uint(fminf(g1 * m1b, kMsFamClip)) | par1);
        const float o2b = zero[1] ? 0.0f : __uint_as_float(__float_as_uint(fminf(g1 * m2b, kMsFamClip)) | par1);
#pragma unroll
        for (int j = 0; j < DC; ++j) {
            const float ma = (fabsf(v[j].x) == m1a) ? o2a : o1a;
            const float mb = (fabsf(v[j].y) == m1b) ? o2b : o1b;
            // store D = -L_{i->j}: the sign of the output flipped once more
            C2[j * MP + t] = make_float2(__uint_as_float(__float_as_uint(ma) ^ (~__float_as_uint(v[j].x) & kSign)),
                                         __uint_as_float(__float_as_uint(mb) ^ (~__float_as_uint(v[j].y) & kSign)));
        }
        __syncthreads();

        // Claims and prefetches for the slots that took a shot this round (warp 0 only; the
        // next refill of a slot reads them after the next barrier).
        if (consumed && t < 32) {
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                if (!((consumed >> (2 * k)) & 1u)) continue;
                const int b = (consumed >> (2 * k + 1)) & 1u;
                const int nx = assign();
                if (t == 0) pfidx[2 * k + (b ^ 1)] = nx;
                prefetch(k, b ^ 1, nx);
            }
        }

        // A4 variable-node update for both slots (qubits past n compute on the zero slot and
        // are never read: no bounds test in the loop)
        const float2 npr = make_float2(-prior[0], -prior[1]);
#pragma unroll
        for (int vv = 0; vv < VPT; ++vv) {
            const int c = vv * MP + t;
            float2 acc = npr;
            if (per_qubit) {
                const float p = -PQ[c];
                acc = make_float2(p, p);
            }
#pragma unroll
            for (int q = 0; q < DV; ++q)
                acc = add2(acc, *reinterpret_cast<const float2*>(c2base + vneB[q * NP + c]));
            // P = -Q exactly, with either zero mapped to +0 (a posterior of -0.0 would read as a
            // negative sign bit): -Q + 0 by one fused multiply-add per pair.
            P2[c] = __ffma2_rn(acc, make_float2(-1.0f, -1.0f), make_float2(0.0f, 0.0f));
        }
        __syncthreads();
        ph ^= 1;
    }
}

}  // namespace sagms
