// Quaternary decoder kernel for CSS stabilizer matrices (every row all X or all Z), the paper's
// setting of Sec. II (the X-type rows of a GB code over its Z-type rows), with the
// column-indexed layout of the binary decoders.  Same rounds and arithmetic per check and
// qubit as gf4_kernel.cuh (Algorithm 1 read per Pauli, scalar messages); only the storage and
// the order of each qubit's message sums differ.
//
// Every edge has a slot j < DC within its check such that, among each qubit's edges of one
// row type, the j mod DH are distinct (the CSR order or a load-time edge colouring of each
// type's rows).  Shared memory holds two halves, X and Z, each of (2 + DH) rows of Np + 4
// 32-bit cells:
//   row 0       lambda_T of every qubit (T = X in the X half, Z in the Z half): the scalar input
//               that a row of type T reads, before its own old message is removed
//   row 1       the decision bit a row of type T sees, in the sign position: the z bit of the
//               qubit's Pauli decision in the X half (an X row anticommutes with Z and Y), the x
//               bit in the Z half
//   rows 2 + r  the CN->VN message of the qubit's edge of that type in slot r (mod DH)
// Column n is the padding column: lambda = +inf, bit 0, message cells scratch for padded slots.
// A check thread keeps the byte offsets of its DC columns in registers, biased by its half, so
// each of its accesses is a register plus an immediate; a qubit thread reads its messages at
// fixed rows.  No index loads and no per-edge Pauli tests.
//
// Per round, as gf4_kernel.cuh:
//   A5  residual bit of each check: s_i XOR the decision bits of its qubits (Eq. 1 with the
//       trace inner product); unsatisfied count by ballot and shared counter; stop test
//   A2  gain (Eq. 7)
//   A3  inputs lambda_T(Lambda) - (own old message), which is the extrinsic lambda because the
//       own message enters the two Paulis anticommuting with T alike; MS-family min1/min2 or BP
//       phi sums (Eqs. 3, 4, 8)
//   A4  per qubit: Lambda(Z) = L0 + its X-type messages, Lambda(X) = L0 + its Z-type messages,
//       Lambda(Y) = L0 + all of them (Eq. 2 per Pauli); decision argmin(0, Lambda(X),
//       Lambda(Z), Lambda(Y)) (ties to I, X, Z, Y); lambda_X and lambda_Z
// The trace row of a checked round is written by the variable-node update that produced it.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gf4_kernel.cuh"

namespace sagms {

// Bytes of one half (2 + DH rows of Np + 4 cells) and of the CTA's shared memory.
__host__ __device__ inline size_t gf4_css_half_bytes(int DH, int Np) { return (size_t)(2 + DH) * (size_t)(Np + 4) * 4; }
__host__ __device__ inline size_t gf4_css_smem_bytes(int DH, int Np) { return 2 * gf4_css_half_bytes(DH, Np) + 64; }

// colS: [DC][Mp] u32, byte offset of slot j's column of check i within the shared block,
// 4 * column plus the half of the check's type (padded slots and checks past m: column n).
// Two 512-thread CTAs' register budget (64), eight 128-thread CTAs per SM for the m = 126
// stack, for the shapes up to DC = 10 that fit it without spilling (all but BP at DC = 8).
template <int DC, int DH, bool BP>
__global__ void __launch_bounds__(512, (DC <= 10 && !(BP && DC == 8)) ? 2 : 1) gf4_css_kernel(const DecodeArgs a, const uint32_t* __restrict__ colS) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int t = threadIdx.x;
    const int T = blockDim.x;   // == Mp
    const int lane = t & 31;
    const int Np = a.Np, n = a.n, m = a.m;
    const int mw = (m + 31) >> 5, nw = (n + 31) >> 5;
    const bool early = (a.flags & kFlagNoEarlyStop) == 0;
    const size_t ROW = (size_t)(Np + 4) * 4;
    const size_t HALF = (size_t)(2 + DH) * ROW;
    float* LXh = reinterpret_cast<float*>(smem);                 // X half, row 0
    float* LZh = reinterpret_cast<float*>(smem + HALF);          // Z half, row 0
    uint32_t* BXh = reinterpret_cast<uint32_t*>(smem + ROW);     // X half, row 1
    uint32_t* BZh = reinterpret_cast<uint32_t*>(smem + HALF + ROW);
    int* cnt_sh = reinterpret_cast<int*>(smem + 2 * HALF);
    const float inf = __uint_as_float(0x7f800000u);
    auto cell = [&](uint32_t o, int row) -> float& { return *reinterpret_cast<float*>(smem + o + (size_t)row * ROW); };
    // message row r of qubit c in half h
    auto msg = [&](int h, int r, int c) -> float {
        return *reinterpret_cast<const float*>(smem + (size_t)h * HALF + (size_t)(2 + r) * ROW + (size_t)c * 4);
    };

    uint32_t off[DC];
#pragma unroll
    for (int j = 0; j < DC; ++j) off[j] = __ldg(colS + j * T + t);
    // the padding column: no sign, no minimum, phi = 0
    if (t < 2) {
        *reinterpret_cast<float*>(smem + (size_t)t * HALF + (size_t)n * 4) = inf;
        *reinterpret_cast<uint32_t*>(smem + (size_t)t * HALF + ROW + (size_t)n * 4) = 0u;
    }
    const float clip = BP ? kBpClip : kMsFamClip;
    // Message cells start at zero once per launch.  A cell that no edge maps to (a qubit with
    // fewer than DH edges of a type) stays zero; every other one is rewritten by its check in
    // each round, and a shot's first round reads no old message, so no shot has to clear them.
    for (int k = t; k < DH * (Np + 4); k += T) {
        reinterpret_cast<float*>(smem + 2 * ROW)[k] = 0.0f;
        reinterpret_cast<float*>(smem + HALF + 2 * ROW)[k] = 0.0f;
    }

    // The next shot's prior and syndrome word are loaded one shot ahead, so their latency
    // overlaps the current shot's rounds.
    float l0_next = 0.0f;
    uint32_t sw_next = 0u;
    if (blockIdx.x < a.shots) {
        l0_next = __ldg(a.L0 + blockIdx.x);
        sw_next = (t < m) ? __ldg(a.syn + (long long)blockIdx.x * mw + (t >> 5)) : 0u;
    }
    // lambda_T(L0) of the last prior seen (the first-round input; the prior's bits as the key,
    // and no finite prior has the bits of a NaN)
    uint32_t prior_last = 0x7fffffffu;
    float lam0 = 0.0f;
    for (long long shot = blockIdx.x; shot < a.shots; shot += gridDim.x) {
        const float l0 = l0_next;
        const uint32_t sw = sw_next;
        if (shot + gridDim.x < a.shots) {
            l0_next = __ldg(a.L0 + shot + gridDim.x);
            sw_next = (t < m) ? __ldg(a.syn + (shot + gridDim.x) * mw + (t >> 5)) : 0u;
        }
        if (!isfinite(l0)) {
            for (int w = t; w < 2 * nw; w += T) a.err[shot * 2 * nw + w] = 0u;
            if (t == 0) { a.conv[shot] = 0; a.iters[shot] = -1; }
            continue;
        }
        const float prior = l0 + 0.0f;
        // A0: no CN message yet; posteriors are the prior, scalar inputs lambda_T(prior), the
        // decision X when L0 < 0 (argmin(0, L0, L0, L0), ties to I): x bit set, z bit clear
        if (__float_as_uint(prior) != prior_last) {   // a batch-wide prior: once per CTA
            lam0 = gf4_softplus_neg(prior) - gf4_lse_neg(prior, prior);
            prior_last = __float_as_uint(prior);
        }
        const uint32_t xb0 = (prior < 0.0f) ? kSign : 0u;
        for (int c = t; c < n; c += T) {
            LXh[c] = lam0;
            LZh[c] = lam0;
            BXh[c] = 0u;
            BZh[c] = xb0;
        }
        if (a.trace) {
            float* tr = a.trace + (size_t)shot * (size_t)(a.max_iter + 1) * (size_t)n * 3;
            for (int c = t; c < n; c += T) { tr[3 * c] = prior; tr[3 * c + 1] = prior; tr[3 * c + 2] = prior; }
        }
        const uint32_t s_bit = (t < m) ? ((sw >> (t & 31)) & 1u) : 0u;
        if (t == 0) { cnt_sh[0] = 0; cnt_sh[1] = 0; }
        __syncthreads();

        int it = 0;
        int cnt = 0;
        for (;; ++it) {
            // A5: residual bit of this check from its qubits' decision bits (Eq. 1)
            uint32_t par = s_bit << 31;
#pragma unroll
            for (int j = 0; j < DC; j += 2)
                par ^= __float_as_uint(cell(off[j], 1)) ^ __float_as_uint(cell(off[j + 1], 1));
            const uint32_t st = par >> 31;
            const uint32_t bal = __ballot_sync(0xffffffffu, st);
            if (lane == 0 && bal) atomicAdd(&cnt_sh[it & 1], __popc(bal));
            __syncthreads();
            cnt = cnt_sh[it & 1];
            // A6
            if ((cnt == 0 && early) || it == a.max_iter) break;
            if (t == 0) cnt_sh[(it + 1) & 1] = 0;

            // A2: gain (Eq. 7)
            float g;
            if (a.mode == kModeSAGMS)
                g = (a.amax - (a.amax - a.amin) * ((float)cnt * a.inv_m)) * (st ? a.eta : 1.0f);
            else if (a.mode == kModeSMS)
                g = a.alpha;
            else
                g = 1.0f;

            // A3: check-node update on the extrinsic scalar inputs (Eqs. 3, 4, 8)
            float v[DC];
            uint32_t sp = s_bit << 31;
            if (it == 0) {
                // no CN message yet: the input is lambda_T itself (lambda - 0 exactly)
#pragma unroll
                for (int j = 0; j < DC; ++j) v[j] = cell(off[j], 0);
            } else {
#pragma unroll
                for (int j = 0; j < DC; ++j) v[j] = cell(off[j], 0) - cell(off[j], 2 + j % DH);
            }
#pragma unroll
            for (int j = 0; j < DC; ++j) sp ^= __float_as_uint(v[j]);
            sp &= kSign;
            if (!BP) {
                float m1 = inf, m2 = inf;
#pragma unroll
                for (int j = 0; j < DC; ++j) {
                    const float av = fabsf(v[j]);
                    m2 = fminf(m2, fmaxf(m1, av));
                    m1 = fminf(m1, av);
                }
                const float o1 = __uint_as_float(__float_as_uint(fminf(g * m1, clip)) | sp);
                const float o2 = __uint_as_float(__float_as_uint(fminf(g * m2, clip)) | sp);
#pragma unroll
                for (int j = 0; j < DC; ++j) {
                    const float mag = (fabsf(v[j]) == m1) ? o2 : o1;
                    cell(off[j], 2 + j % DH) = __uint_as_float(__float_as_uint(mag) ^ (__float_as_uint(v[j]) & kSign));
                }
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
                    cell(off[j], 2 + j % DH) = __uint_as_float(__float_as_uint(mag) | (sp ^ (__float_as_uint(v[j]) & kSign)));
                }
            }
            __syncthreads();

            // A4: per-Pauli posteriors (Eq. 2 per Pauli), decision, lambda_X and lambda_Z
            for (int c = t; c < n; c += T) {
                float lz = prior, lx = prior, ly = prior;
#pragma unroll
                for (int r = 0; r < DH; ++r) {
                    const float rx = msg(0, r, c);
                    lz += rx;
                    ly += rx;
                }
#pragma unroll
                for (int r = 0; r < DH; ++r) {
                    const float rz = msg(1, r, c);
                    lx += rz;
                    ly += rz;
                }
                uint32_t d = 0;
                float best = 0.0f;
                if (lx < best) { best = lx; d = 1; }
                if (lz < best) { best = lz; d = 2; }
                if (ly < best) { best = ly; d = 3; }
                LXh[c] = gf4_softplus_neg(lx) - gf4_lse_neg(lz, ly);
                LZh[c] = gf4_softplus_neg(lz) - gf4_lse_neg(lx, ly);
                BXh[c] = (d >> 1) << 31;   // z bit
                BZh[c] = (d & 1u) << 31;   // x bit
                if (a.trace) {
                    float* tr = a.trace + ((size_t)shot * (size_t)(a.max_iter + 1) + (size_t)(it + 1)) * (size_t)n * 3;
                    tr[3 * c] = lx;
                    tr[3 * c + 1] = lz;
                    tr[3 * c + 2] = ly;
                }
            }
            __syncthreads();
        }

        // A7: write-out (x bits, z bits of the Pauli decisions), flag, count
        for (int base = 0; base < n; base += T) {
            const int c = base + t;
            const uint32_t wx = __ballot_sync(0xffffffffu, (c < n) && (BZh[c] >> 31));
            const uint32_t wz = __ballot_sync(0xffffffffu, (c < n) && (BXh[c] >> 31));
            if (lane == 0 && c < n) {
                a.err[shot * 2 * nw + (c >> 5)] = wx;
                a.err[shot * 2 * nw + nw + (c >> 5)] = wz;
            }
        }
        if (t == 0) {
            a.conv[shot] = (cnt == 0) ? 1 : 0;
            a.iters[shot] = it;
        }
        __syncthreads();
    }
}

}  // namespace sagms
