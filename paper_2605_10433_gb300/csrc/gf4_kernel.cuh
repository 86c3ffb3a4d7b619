// Quaternary (GF(4)) flooding decoder kernel: BP4 and its Min-Sum family (MS / SMS / SAGMS) on a
// stabilizer matrix with Pauli entries (Sec. II), scalar messages.
//
// One CTA decodes one shot at a time and loops over shots (persistent); one thread owns one
// check (its DC padded edge slots; at most 512 checks) and threads stride over the qubits.  Per-shot state in
// shared memory:
//   LX, LZ, LY [Np]   posterior LLRs ln P(I)/P(W) of every qubit for W = X, Z, Y
//   D [Np]            the qubit's Pauli decision (0 I, 1 X, 2 Z, 3 Y)
//   C [DC*Mp + 4]     CN->VN message of every edge, slot-major C[j*Mp + i]; C[DC*Mp] = 0 is the
//                     target of padded qubit slots
//   Lam [DC*Mp + 4]   VN->CN scalar message of every edge, same index; +inf on padded check slots
//   colT [DC*Mp]      column of edge (i, j) | Pauli << 14 (u16); padded slots: column n, Pauli 0
//   vneT [DV*Np]      edge position j*Mp + i of the q-th edge of qubit c | Pauli << 16 (u32);
//                     padded: the zero slot, Pauli 0
//
// Round l (Algorithm 1 with the paper's equations read per Pauli):
//   A5  residual bit s~_i = s_i XOR (XOR over the check's qubits of <D_c, H_ic>) (Eq. 1),
//       count of unsatisfied checks by warp ballot + shared counter; stop test
//   A2  gain (Eq. 7), as the binary kernels
//   A3  CN update on the scalar inputs Lam (Eqs. 3, 4, 8): sign parity with s_i, then the
//       extrinsic min1/min2 selection (MS family) or phi prefix/suffix sums (BP), clipped
//   A4  per qubit: Lambda(W) = L0 + sum of C over the edges whose Pauli anticommutes with W
//       (Eq. 2 per Pauli), decision D = argmin(0, Lambda(X), Lambda(Z), Lambda(Y)) (ties to
//       I, X, Z, Y), and for every edge of Pauli T the extrinsic scalar message
//       lambda_T = ln(1 + e^{-Lambda'(T)}) - ln(e^{-Lambda'(T')} + e^{-Lambda'(T'')}), Lambda' =
//       Lambda minus the edge's own message on the Paulis it anticommutes with.  Since that
//       message enters T' and T'' alike, lambda_T(Lambda') = lambda_T(Lambda) - message: one
//       lambda per Pauli and qubit, then one subtraction per edge (as q = P - r in the
//       binary kernels).
// LLR units throughout (lambda_T is not homogeneous).  Outputs: e_hat as x bits then z bits
// ([shots][2][nw]), conv, iters; the trace holds Lambda(X, Z, Y) of every checked round.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "decode_kernel.cuh"

namespace sagms {

// Pauli codes 1 X, 2 Z, 3 Y (symplectic bits x | z << 1); anticommutation is the symplectic
// product.
__device__ __forceinline__ uint32_t gf4_anti(uint32_t a, uint32_t b) { return ((a & (b >> 1)) ^ ((a >> 1) & b)) & 1u; }

// ln(1 + e^{-a}) and ln(e^{-b} + e^{-c}) in FP32, overflow-safe; the latter is -inf when both
// are +inf.
__device__ __forceinline__ float gf4_softplus_neg(float a) { return fmaxf(-a, 0.0f) + log1pf(expf(-fabsf(a))); }
__device__ __forceinline__ float gf4_lse_neg(float b, float c) {
    const float lo = fminf(b, c), hi = fmaxf(b, c);
    if (lo == __uint_as_float(0x7f800000u)) return __uint_as_float(0xff800000u);
    return -lo + log1pf(expf(lo - hi));
}

// DecodeArgs::flags bits kGf4PauliShift + P, P = 1 (X), 2 (Z), 3 (Y): the matrix has an entry
// of Pauli P.  Internal to the GF(4) launch, above every public flag bit.
constexpr int kGf4PauliShift = 8;

__host__ __device__ inline size_t gf4_smem_bytes(int DC, int DV, int Mp, int Np) {
    const size_t floats = 3 * (size_t)Np + 2 * ((size_t)DC * Mp + 4);
    return floats * 4 + (size_t)Np + (size_t)DC * Mp * 2 + (size_t)DV * Np * 4 + 64;
}

struct Gf4Layout {
    const uint16_t* colT;   // [DC][Mp]
    const uint32_t* vneT;   // [DV][Np]
};

// Up to d_c = 10 the kernel fits 64 registers without spilling, so two 512-thread CTAs (eight
// of the 128 threads an m <= 128 code launches) share an SM; larger slot counts keep the
// register budget of one 512-thread CTA.
template <int DC, int DV, bool BP>
__global__ void __launch_bounds__(512, DC <= 10 ? 2 : 1) gf4_kernel(const DecodeArgs a, const Gf4Layout lay) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int t = threadIdx.x;
    const int T = blockDim.x;   // == Mp
    const int lane = t & 31;
    const int Mp = a.Mp, Np = a.Np, n = a.n, m = a.m;
    const int mw = (m + 31) >> 5, nw = (n + 31) >> 5;
    const bool early = (a.flags & kFlagNoEarlyStop) == 0;
    // bit P (1 X, 2 Z, 3 Y): the matrix has an entry of Pauli P (set by the host)
    const uint32_t pauli_set = (a.flags >> kGf4PauliShift) & 0xeu;
    float* LX = reinterpret_cast<float*>(smem);
    float* LZ = LX + Np;
    float* LY = LZ + Np;
    float* C = LY + Np;
    float* Lam = C + DC * Mp + 4;
    uint32_t* vneT = reinterpret_cast<uint32_t*>(Lam + DC * Mp + 4);
    uint16_t* colT = reinterpret_cast<uint16_t*>(vneT + DV * Np);
    uint8_t* D = reinterpret_cast<uint8_t*>(colT + DC * Mp);
    int* cnt_sh = reinterpret_cast<int*>(D + ((Np + 15) & ~15));
    const float inf = __uint_as_float(0x7f800000u);

    for (int k = t; k < DC * Mp; k += T) colT[k] = __ldg(lay.colT + k);
    for (int k = t; k < DV * Np; k += T) vneT[k] = __ldg(lay.vneT + k);
    __syncthreads();
    // padded check slots: +inf input (no sign, no minimum, phi = 0); the zero slot
#pragma unroll
    for (int j = 0; j < DC; ++j)
        if ((colT[j * Mp + t] & 0x3fffu) == (uint16_t)n) Lam[j * Mp + t] = inf;
    if (t < 4) C[DC * Mp + t] = 0.0f;
    const float clip = BP ? kBpClip : kMsFamClip;

    // The next shot's prior and syndrome word are loaded one shot ahead, so their latency
    // overlaps the current shot's rounds.
    float l0_next = 0.0f;
    uint32_t sw_next = 0u;
    if (blockIdx.x < a.shots) {
        l0_next = __ldg(a.L0 + blockIdx.x);
        sw_next = (t < m) ? __ldg(a.syn + (long long)blockIdx.x * mw + (t >> 5)) : 0u;
    }
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
        // A0: no CN message yet; posteriors are the prior, scalar inputs lambda_T(prior)
        const float lam0 = gf4_softplus_neg(prior) - gf4_lse_neg(prior, prior);
        for (int c = t; c < n; c += T) {
            LX[c] = prior;
            LZ[c] = prior;
            LY[c] = prior;
            D[c] = (prior < 0.0f) ? 1 : 0;   // argmin(0, L0, L0, L0): X when L0 < 0 (ties to I)
        }
#pragma unroll
        for (int j = 0; j < DC; ++j) {
            C[j * Mp + t] = 0.0f;
            if ((colT[j * Mp + t] & 0x3fffu) != (uint16_t)n) Lam[j * Mp + t] = lam0;
        }
        const uint32_t s_bit = (t < m) ? ((sw >> (t & 31)) & 1u) : 0u;
        if (t == 0) { cnt_sh[0] = 0; cnt_sh[1] = 0; }
        __syncthreads();

        int it = 0;
        int cnt = 0;
        for (;; ++it) {
            // A5: residual bit of this check from the qubits' Pauli decisions (Eq. 1)
            uint32_t st = s_bit;
#pragma unroll
            for (int j = 0; j < DC; ++j) {
                const uint32_t ct = colT[j * Mp + t];
                const uint32_t c = ct & 0x3fffu;
                if (c != (uint32_t)n) st ^= gf4_anti(D[c], ct >> 14);
            }
            const uint32_t bal = __ballot_sync(0xffffffffu, st);
            if (lane == 0 && bal) atomicAdd(&cnt_sh[it & 1], __popc(bal));
            __syncthreads();
            cnt = cnt_sh[it & 1];
            if (a.trace) {
                float* tr = a.trace + ((size_t)shot * (size_t)(a.max_iter + 1) + (size_t)it) * (size_t)n * 3;
                for (int c = t; c < n; c += T) {
                    tr[3 * c] = LX[c];
                    tr[3 * c + 1] = LZ[c];
                    tr[3 * c + 2] = LY[c];
                }
            }
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

            // A3: check-node update on the scalar inputs (Eqs. 3, 4, 8)
            float v[DC];
            uint32_t par = s_bit << 31;
#pragma unroll
            for (int j = 0; j < DC; ++j) {
                v[j] = Lam[j * Mp + t];
                par ^= __float_as_uint(v[j]);
            }
            par &= kSign;
            if (!BP) {
                float m1 = inf, m2 = inf;
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

            // A4: per-Pauli posteriors (Eq. 2 per Pauli), decision, extrinsic scalar messages
            for (int c = t; c < n; c += T) {
                float lx = prior, lz = prior, ly = prior;
                float r[DV];
                uint32_t pt[DV];
#pragma unroll
                for (int q = 0; q < DV; ++q) {
                    const uint32_t e = vneT[q * Np + c];
                    r[q] = C[e & 0xffffu];
                    pt[q] = e >> 16;
                    // an X entry's message counts toward Z and Y, a Z entry's toward X and Y,
                    // a Y entry's toward X and Z (Pauli 0: the padded zero slot, toward none)
                    if (gf4_anti(1u, pt[q])) lx += r[q];
                    if (gf4_anti(2u, pt[q])) lz += r[q];
                    if (gf4_anti(3u, pt[q])) ly += r[q];
                }
                LX[c] = lx;
                LZ[c] = lz;
                LY[c] = ly;
                uint8_t d = 0;
                float best = 0.0f;
                if (lx < best) { best = lx; d = 1; }
                if (lz < best) { best = lz; d = 2; }
                if (ly < best) { best = ly; d = 3; }
                D[c] = d;
                // lambda_T of the totals, once per Pauli: an edge's own message r enters exactly
                // the two Paulis anticommuting with its entry T, so removing it multiplies
                // e^{-Lambda(T')} + e^{-Lambda(T'')} by e^{r} and leaves Lambda(T): the
                // extrinsic message is lambda_T(Lambda) - r.
                // Only the Paulis the matrix has entries of need their lambda (a CSS stack has
                // no Y entry, so lambda_Y is skipped there); the others are never selected.
                const float lamX = (pauli_set & 2u) ? gf4_softplus_neg(lx) - gf4_lse_neg(lz, ly) : 0.0f;
                const float lamZ = (pauli_set & 4u) ? gf4_softplus_neg(lz) - gf4_lse_neg(lx, ly) : 0.0f;
                const float lamY = (pauli_set & 8u) ? gf4_softplus_neg(ly) - gf4_lse_neg(lx, lz) : 0.0f;
#pragma unroll
                for (int q = 0; q < DV; ++q) {
                    if (pt[q] == 0u) continue;
                    const float lam = (pt[q] == 1u) ? lamX : ((pt[q] == 2u) ? lamZ : lamY);
                    Lam[vneT[q * Np + c] & 0xffffu] = lam - r[q];
                }
            }
            __syncthreads();
        }

        // A7: write-out (x bits, z bits of the Pauli decisions), flag, count
        for (int base = 0; base < n; base += T) {
            const int c = base + t;
            const uint32_t d = (c < n) ? D[c] : 0u;
            const uint32_t wx = __ballot_sync(0xffffffffu, d & 1u);
            const uint32_t wz = __ballot_sync(0xffffffffu, (d >> 1) & 1u);
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
