// Batched flooding-schedule decoder kernel (MS / SMS / SAGMS and the phi-domain BP rule).
//
// One CTA decodes one shot at a time and loops over shots (persistent).  One thread owns
// one check node i (its DC padded edge slots), and threads stride over the variable nodes.
// All per-shot state lives in shared memory for the whole decode:
//   P[Np]        posterior of every qubit (Alg. 1, hard-decision input), +inf past n
//   C[DC*Mp + 4] CN->VN message of every edge, slot-major: C[j*Mp + i]; C[DC*Mp] = 0 is the
//                target of padded qubit slots
//   colT[DC*Mp]  column of edge (i, j) (u16), padded slots point at the +inf qubit n
//   vneT[DV*Np]  edge position j*Mp + i of the q-th edge of qubit c (u16), padded -> zero slot
// Nothing goes back to global memory between iterations; global traffic per shot is the
// syndrome in, the prior, and the packed estimate / flag / count out.
//
// Per iteration l (Algorithm 1):
//   A5  gather P over the check's edges; residual bit s~_i = s_i XOR (XOR of sign bits)
//       (Eq. 1); warp ballot + popcount -> shared counter -> |s~|_0 (Eq. 6 numerator)
//   A6  stop if |s~|_0 == 0 (early termination) or l == max_iter
//   A2  gain g_i: 1 (MS), alpha (SMS), [a_max - (a_max - a_min) |s~|_0/m] * (eta if s~_i)
//       (SAGMS, Eq. 7)
//   A3  VN->CN inputs v_j = P_j - C_old(i,j) (= L0 + sum over the other checks, Eq. 2),
//       one pass for min1 / min2 / sign parity, then the extrinsic output per edge:
//       MS family (Eqs. 4, 8): (-1)^{s_i + parity + sgn v_j} * min(g * (|v_j| == min1 ? min2 : min1), clip)
//       BP (Eq. 3): (-1)^{...} * min(phi(sum_{k != j} phi(|v_k|)), clip), with prefix/suffix sums
//       (in round 1 with one prior per shot every real input is the prior: the sum is
//       (deg - 1) phi(|L0|) on every real edge)
//   A4  P_c = L0_c + sum over the qubit's edges of C (Eq. 2's full sum)
// Sign bits are read straight from the IEEE representation: no -0.0 ever arises (every
// value is a sum whose first term is the prior, or a difference of two finite values, and
// per-qubit priors are loaded as L0 + 0, which turns a -0.0 prior into +0.0).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace sagms {

constexpr float kMsFamClip = 1.0e6f;     // |CN output| cap, MS family (normalised units)
constexpr float kBpClip = 23.718998f;    // |CN output| cap, BP: ln(2e10)
constexpr uint32_t kSign = 0x80000000u;

struct DecodeArgs {
    const uint16_t* colT;   // [DC][Mp]
    const uint16_t* vneT;   // [DV][Np]
    int m, n, Mp, Np;
    int mode;
    float alpha, amin, amax, eta, inv_m;
    int dcmax;     // largest check degree (the auto gain ceiling's d_c)
    int max_iter;
    unsigned flags;
    long long shots;
    const uint32_t* syn;
    const float* L0;
    uint32_t* err;
    uint8_t* conv;
    int32_t* iters;
    float* trace;
    int* work;     // continuous-batching kernels: zero-initialised chunk counter, or null (static)
    int chunk_lg;  // continuous-batching kernels: log2 of the shots per claimed chunk
};

enum { kModeMS = 0, kModeSMS = 1, kModeSAGMS = 2, kModeBP = 3 };
enum { kFlagPerQubit = 1u, kFlagNoEarlyStop = 2u, kFlagAutoCeiling = 16u };

// alpha_max of a shot under the automatic ceiling (Corollary 1): alpha*(|L0|, d_c) of Eq. 9,
// clamped to [alpha_min, 1/eta].  alpha* = 2 atanh(t) / x with t = tanh(x/2)^(d_c - 1) is
// evaluated as (ln(2 - w) - ln w) / x with w = 1 - t = -expm1((d_c - 1) log1p(-u)) and
// u = 1 - tanh(x/2) = 2 / (e^x + 1), which keeps its accuracy when t rounds to 1 in FP32
// (|L0| above about 18).  x = 0 gives alpha_min.
__device__ __forceinline__ float auto_alpha_max(float l0, int dc, float amin, float eta) {
    const float x = fabsf(l0);
    float a = 0.0f;
    if (x > 0.0f) {
        const float u = 2.0f / (expf(x) + 1.0f);
        const float w = -expm1f((float)(dc - 1) * log1pf(-u));
        a = (logf(2.0f - w) - logf(w)) / x;
    }
    return fminf(fmaxf(a, amin), 1.0f / eta);
}

// alpha_max of a shot: the parameter, or the automatic ceiling of its prior.
__device__ __forceinline__ float shot_alpha_max(const DecodeArgs& a, float l0) {
    return (a.flags & kFlagAutoCeiling) ? auto_alpha_max(l0, a.dcmax, a.amin, a.eta) : a.amax;
}

__host__ __device__ inline size_t smem_bytes(int DC, int DV, int Mp, int Np, bool per_qubit) {
    size_t floats = (size_t)Np + (size_t)DC * Mp + 4 + (per_qubit ? (size_t)Np : 0);
    size_t halves = (size_t)DC * Mp + (size_t)DV * Np;
    return floats * 4 + halves * 2 + 16;
}

// phi(x) = -ln tanh(x/2) = 2 atanh(e^-x), x >= 0; phi(0) = +inf, phi(+inf) = 0.  Evaluated
// from two polynomial forms with one CUDA logf or expf each, instead of log1pf(2 / expm1f(x)):
//   x < 1:  phi = -ln y + t P(t), y = x/2, t = y^2, where t P(t) approximates -ln(tanh(y) / y)
//           (= t/3 - 7t^2/90 + ...) on t in [0, 1/4);
//   x >= 1: phi = 2u S(t), u = e^-x <= 1/e, t = u^2, where S(t) approximates
//           atanh(u)/u = sum_k t^k / (2k + 1) on t in (0, e^-2].
// P (degree 4) and S (degree 5) are near-minimax fits in relative error computed for this
// library (iteratively reweighted least squares on a dense grid, FP64): P within 3.7e-9 of
// -ln(tanh(y)/y)/t, S within 3.9e-10 of atanh(u)/u, both far below FP32 resolution; the
// coefficients are those fits rounded to FP32.  A GPU test bounds the result against the
// library composition log1pf(2 / expm1f(x)) and an FP64 reference.
__device__ __forceinline__ float phi_fn(float x) {
    if (x < 1.0f) {
        const float yv = 0.5f * x, t = yv * yv;
        float s = 1.7822636291e-3f;
        s = fmaf(s, t, -6.6359406337e-3f);
        s = fmaf(s, t, 2.1862298250e-2f);
        s = fmaf(s, t, -7.7777564526e-2f);
        s = fmaf(s, t, 3.3333334327e-1f);
        return fmaf(s, t, -logf(yv));
    }
    const float u = expf(-x), t = u * u;
    float s = 1.3069644570e-1f;
    s = fmaf(s, t, 1.0458538681e-1f);
    s = fmaf(s, t, 1.4332985878e-1f);
    s = fmaf(s, t, 1.9998490810e-1f);
    s = fmaf(s, t, 3.3333349228e-1f);
    s = fmaf(s, t, 1.0f);
    return 2.0f * u * s;
}

// The composition the decoder used before phi_fn, kept as the reference of the phi test.
__device__ __forceinline__ float phi_ref(float x) { return log1pf(2.0f / expm1f(x)); }

template <int DC, int DV, bool BP>
__global__ void __launch_bounds__(1024, 1) decode_kernel(const DecodeArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const bool per_qubit = (a.flags & kFlagPerQubit) != 0;
    const bool early = (a.flags & kFlagNoEarlyStop) == 0;
    float* P = reinterpret_cast<float*>(smem);
    float* C = P + a.Np;
    float* PQ = C + DC * a.Mp + 4;
    uint16_t* colT = reinterpret_cast<uint16_t*>(PQ + (per_qubit ? a.Np : 0));
    uint16_t* vneT = colT + DC * a.Mp;
    int* cnt_sh = reinterpret_cast<int*>(vneT + DV * a.Np);

    const int t = threadIdx.x;
    const int T = blockDim.x;   // == Mp
    const int lane = t & 31;
    const int Mp = a.Mp, Np = a.Np, n = a.n, m = a.m;
    const int mw = (m + 31) >> 5, nw = (n + 31) >> 5;

    // Stage the code graph once per CTA (16-byte vector copies; both arrays are multiples of 16 B).
    {
        const int4* src = reinterpret_cast<const int4*>(a.colT);
        int4* dst = reinterpret_cast<int4*>(colT);
        const int cnt16 = (DC * Mp * 2) / 16;
        for (int k = t; k < cnt16; k += T) dst[k] = __ldg(src + k);
        const int4* src2 = reinterpret_cast<const int4*>(a.vneT);
        int4* dst2 = reinterpret_cast<int4*>(vneT);
        const int cnt16b = (DV * Np * 2) / 16;
        for (int k = t; k < cnt16b; k += T) dst2[k] = __ldg(src2 + k);
    }
    for (int c = n + t; c < Np; c += T) P[c] = __uint_as_float(0x7f800000u);  // +inf
    if (t < 4) C[DC * Mp + t] = 0.0f;
    int pq_ok = 1;
    if (per_qubit) {
        for (int c = t; c < n; c += T) {
            const float v = __ldg(a.L0 + c) + 0.0f;   // -0 -> +0: sign bits are decisions
            PQ[c] = v;
            pq_ok &= isfinite(v) ? 1 : 0;
        }
    }
    pq_ok = __syncthreads_and(pq_ok);
    const float clip = BP ? kBpClip : kMsFamClip;
    int deg = 0;   // real edges of this thread's check
#pragma unroll
    for (int j = 0; j < DC; ++j) deg += (colT[j * Mp + t] != (uint16_t)n) ? 1 : 0;

    // CN->VN messages start at zero once per launch: every slot is rewritten by its check in
    // each round, and a shot's first round reads no old message, so no shot has to clear them.
#pragma unroll
    for (int j = 0; j < DC; ++j) C[j * Mp + t] = 0.0f;
    // The next shot's prior and syndrome word are loaded one shot ahead, so their latency
    // overlaps the current shot's rounds.
    float l0_next = 0.0f;
    uint32_t sw_next = 0u;
    if (blockIdx.x < a.shots) {
        if (!per_qubit) l0_next = __ldg(a.L0 + blockIdx.x);
        sw_next = (t < m) ? __ldg(a.syn + (long long)blockIdx.x * mw + (t >> 5)) : 0u;
    }
    for (long long shot = blockIdx.x; shot < a.shots; shot += gridDim.x) {
        const float l0_cur = l0_next;
        const uint32_t sw = sw_next;
        if (shot + gridDim.x < a.shots) {
            if (!per_qubit) l0_next = __ldg(a.L0 + shot + gridDim.x);
            sw_next = (t < m) ? __ldg(a.syn + (shot + gridDim.x) * mw + (t >> 5)) : 0u;
        }
        float prior = 0.0f;
        float amax = a.amax;
        bool valid;
        if (per_qubit) {
            valid = pq_ok != 0;
        } else {
            const float l0 = l0_cur;
            valid = isfinite(l0);
            if (BP) prior = l0 + 0.0f;
            else prior = (l0 > 0.0f) ? 1.0f : ((l0 < 0.0f) ? -1.0f : 0.0f);
            if (valid) amax = shot_alpha_max(a, l0);
        }
        if (!valid) {
            for (int w = t; w < nw; w += T) a.err[shot * nw + w] = 0u;
            if (t == 0) { a.conv[shot] = 0; a.iters[shot] = -1; }
            continue;
        }
        // A0: P = L0 (no CN message yet: round 1 reads none), s_i
        for (int c = t; c < n; c += T) P[c] = per_qubit ? PQ[c] : prior;
        const uint32_t s_bit = (t < m) ? ((sw >> (t & 31)) & 1u) : 0u;
        if (t == 0) { cnt_sh[0] = 0; cnt_sh[1] = 0; }
        __syncthreads();

        int it = 0;
        int cnt = 0;
        for (;; ++it) {
            // A5: gather posteriors of this check's qubits, residual bit, unsatisfied count
            float v[DC];
            uint32_t x = s_bit << 31;
#pragma unroll
            for (int j = 0; j < DC; ++j) {
                v[j] = P[colT[j * Mp + t]];
                x ^= __float_as_uint(v[j]);
            }
            const uint32_t st = x >> 31;
            const uint32_t bal = __ballot_sync(0xffffffffu, st);
            if (lane == 0 && bal) atomicAdd(&cnt_sh[it & 1], __popc(bal));
            __syncthreads();
            cnt = cnt_sh[it & 1];
            if (a.trace) {
                float* tr = a.trace + ((size_t)shot * (size_t)(a.max_iter + 1) + (size_t)it) * (size_t)n;
                for (int c = t; c < n; c += T) tr[c] = P[c];
            }
            // A6
            if ((cnt == 0 && early) || it == a.max_iter) break;
            if (t == 0) cnt_sh[(it + 1) & 1] = 0;

            // A2: gain
            float g;
            if (a.mode == kModeSAGMS)
                g = (amax - (amax - a.amin) * ((float)cnt * a.inv_m)) * (st ? a.eta : 1.0f);
            else if (a.mode == kModeSMS)
                g = a.alpha;
            else
                g = 1.0f;

            // A3: check-node update
            uint32_t par = s_bit << 31;
            if (it > 0) {   // round 1 has no old message (v - 0 = v exactly)
#pragma unroll
                for (int j = 0; j < DC; ++j) v[j] = v[j] - C[j * Mp + t];
            }
#pragma unroll
            for (int j = 0; j < DC; ++j) par ^= __float_as_uint(v[j]);
            par &= kSign;
            if (!BP) {
                float m1 = __uint_as_float(0x7f800000u), m2 = m1;
#pragma unroll
                for (int j = 0; j < DC; ++j) {
                    const float av = fabsf(v[j]);
                    m2 = fminf(m2, fmaxf(m1, av));
                    m1 = fminf(m1, av);
                }
                const float o1 = __uint_as_float(__float_as_uint(fminf(g * m1, clip)) | par);
                const float o2 = __uint_as_float(__float_as_uint(fminf(g * m2, clip)) | par);
#pragma unroll
                for (int j = 0; j < DC; ++j) {
                    const float mag = (fabsf(v[j]) == m1) ? o2 : o1;
                    C[j * Mp + t] = __uint_as_float(__float_as_uint(mag) ^ (__float_as_uint(v[j]) & kSign));
                }
            } else if (it == 0 && !per_qubit) {
                // Round 1: every real input is the shot's prior, so each real edge's sum over
                // the other edges is (deg - 1) phi(|L0|) (none for a degree-1 check)
                const float ph0 = phi_fn(fabsf(prior));
                const float S1 = (deg >= 2) ? (float)(deg - 1) * ph0 : 0.0f;
                const float mag = fminf(phi_fn(S1), clip);
#pragma unroll
                for (int j = 0; j < DC; ++j)
                    C[j * Mp + t] = __uint_as_float(__float_as_uint(mag) | (par ^ (__float_as_uint(v[j]) & kSign)));
            } else {
                float ph[DC];
#pragma unroll
                for (int j = 0; j < DC; ++j) ph[j] = phi_fn(fabsf(v[j]));
                float suf[DC + 1];
                suf[DC] = 0.0f;
#pragma unroll
                for (int j = DC - 1; j >= 0; --j) suf[j] = suf[j + 1] + ph[j];
                float pre = 0.0f;
#pragma unroll
                for (int j = 0; j < DC; ++j) {
                    const float S = pre + suf[j + 1];
                    pre += ph[j];
                    const float mag = fminf(phi_fn(S), clip);
                    C[j * Mp + t] = __uint_as_float(__float_as_uint(mag) | (par ^ (__float_as_uint(v[j]) & kSign)));
                }
            }
            __syncthreads();

            // A4: variable-node update (posterior), Eq. 2 summed over all of N(c)
            for (int c = t; c < n; c += T) {
                float acc = per_qubit ? PQ[c] : prior;
#pragma unroll
                for (int q = 0; q < DV; ++q) acc += C[vneT[q * Np + c]];
                P[c] = acc;
            }
            __syncthreads();
        }

        // A7: write-out (packed hard decision, flag, count)
        for (int base = 0; base < n; base += T) {
            const int c = base + t;
            const bool b = (c < n) && (__float_as_uint(P[c]) >> 31);
            const uint32_t word = __ballot_sync(0xffffffffu, b);
            if (lane == 0 && c < n) a.err[shot * nw + (c >> 5)] = word;
        }
        if (t == 0) {
            a.conv[shot] = (cnt == 0) ? 1 : 0;
            a.iters[shot] = it;
        }
        __syncthreads();
    }
}

}  // namespace sagms
