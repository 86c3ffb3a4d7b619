// Layered (serial-check) schedule for the MS family (SAGMS_FLAG_LAYERED).
//
// The checks are split into layers whose checks share no qubit: check i joins the smallest
// layer used by no earlier check sharing a qubit with it (first-fit in index order, computed
// at load time).  A round visits the layers in order; every check of a layer takes its
// inputs from the posteriors as they stand, so a later layer already sees the messages an
// earlier one replaced in the same round.  With P_j = L0_j + sum of the current CN->VN
// messages of qubit j, the check update of Eqs. 2, 4 and 8 becomes, per edge:
//   v_j = P_j - c_old(i, j)        (Eq. 2's extrinsic input)
//   c_new(i, j) from the v of the check, as in the flooding kernels
//   P_j = v_j + c_new(i, j)
// Checks of one layer touch disjoint qubits, so one thread per check updates P in place.
// The gains of a round come from the residual syndrome at its start (Eqs. 1, 6, 7).
//
// One CTA of T threads (32, 64 or 128) decodes one shot at a time (static stride over
// shots).  Shared memory holds, per shot:
//   P[Np]          posteriors (column n and up: +inf, the target of padded check slots)
//   PQ[Np]         per-qubit priors (SAGMS_FLAG_L0_PER_QUBIT only)
//   O1[Mp], O2[Mp] magnitudes min(g*min1, clip), min(g*min2, clip) of each check's last output
//   meta[Mp]       bit j: sign of the output on slot j; bits 24..28: slot of the first minimum
//   sbits, rbits   input syndrome (check order) and residual bits (layer order)
// A check's outputs take two magnitudes only, so (O1, O2, meta) reproduces every old message
// exactly: slot j carries O2 if it holds the first minimum, else O1 (two slots tying at the
// minimum have O1 == O2).  P sits at the start of shared memory, so a record's byte offsets
// address it directly.  A shot's first round reads no old message (all are zero), so it runs
// a copy of the loop without that step, and with one prior per shot the residual before it
// has a closed form.  After a later round in which a posterior exceeded 64 (normalised
// units; every round with per-qubit priors) the posteriors are summed afresh from the
// messages, through qubit-to-edge lists: in-place updates alone would keep the rounding error
// of every large value a posterior ever held.  The check records (columns, check index and
// degree, layer order) and the qubit-to-edge lists stay in global memory, read through the
// read-only cache.
#pragma once

#include <type_traits>

#include "decode_kernel.cuh"

namespace sagms {

// Record of one check in layer order, as u32 words padded to whole 16-byte vectors: the byte
// offsets 4 * col of its DC columns in P (4 * n for padding), then index | degree << 16.
template <int DC>
struct LayeredRec {
    static constexpr int R = (DC + 1 + 3) / 4 * 4;
};

struct LayeredLayout {
    const uint32_t* rec;  // [m][R]
    const int* lay_ptr;   // [L + 1] first position of each layer
    int L;
    const uint16_t* qe;   // [n][QE] edges of each qubit: layer position << 5 | record slot, 0xFFFF pads
    int QE;
};

__host__ __device__ inline size_t layered_smem_bytes(int Mp, int Np, bool per_qubit) {
    return (size_t)Np * 4 * (per_qubit ? 2 : 1) + (size_t)Mp * 12 + (size_t)(Mp / 32) * 8 + 16;
}

// Posteriors are rebuilt after a round in which one reached this magnitude (L0-normalised
// units; always with per-qubit priors): below it, an in-place update's rounding error is at
// most 2^-24 * 128 = 8e-6.
constexpr float kLayeredRebuild = 64.0f;

template <int DC, int T>
__global__ void __launch_bounds__(T, T == 32 ? 32 : (T == 64 ? 12 : 6)) layered_kernel(const DecodeArgs a, const LayeredLayout lay) {
    constexpr int R = LayeredRec<DC>::R;
    static_assert(DC <= 24 && T % 32 == 0, "layout");
    extern __shared__ __align__(16) unsigned char smem[];
    const bool per_qubit = (a.flags & kFlagPerQubit) != 0;
    const bool early = (a.flags & kFlagNoEarlyStop) == 0;
    const int t = threadIdx.x;
    const int lane = t & 31;
    const int n = a.n, m = a.m, Np = a.Np, Mp = a.Mp;
    const int mw = (m + 31) >> 5, nw = (n + 31) >> 5;
    float* P = reinterpret_cast<float*>(smem);
    float* PQ = P + Np;
    float* O1 = PQ + (per_qubit ? Np : 0);
    float* O2 = O1 + Mp;
    uint32_t* meta = reinterpret_cast<uint32_t*>(O2 + Mp);
    uint32_t* sbits = meta + Mp;
    uint32_t* rbits = sbits + Mp / 32;
    int* cnt_sh = reinterpret_cast<int*>(rbits + Mp / 32);
    const uint4* rec = reinterpret_cast<const uint4*>(lay.rec);
    const float inf = __uint_as_float(0x7f800000u);
    const bool sagms_mode = a.mode == kModeSAGMS;
    const float eta = a.eta;
    auto Pat = [&](uint32_t o) -> float& { return *reinterpret_cast<float*>(smem + o); };

    auto sync = [] {
        if constexpr (T == 32) __syncwarp();
        else __syncthreads();
    };
    // column byte offsets and check index of the check at layer position p
    auto load_rec = [&](int p, uint32_t (&off)[DC]) {
        uint32_t w[R];
#pragma unroll
        for (int k = 0; k < R / 4; ++k) {
            const uint4 u = __ldg(rec + (size_t)p * (R / 4) + k);
            w[4 * k] = u.x; w[4 * k + 1] = u.y; w[4 * k + 2] = u.z; w[4 * k + 3] = u.w;
        }
#pragma unroll
        for (int j = 0; j < DC; ++j) off[j] = w[j];
        return (int)(w[DC] & 0xffffu);
    };
    // check index and degree of the check at layer position p
    auto load_head = [&](int p, int& deg) {
        const uint32_t h = __ldg(lay.rec + (size_t)p * R + DC);
        deg = (int)(h >> 16);
        return (int)(h & 0xffffu);
    };
    // One round over the layers (A3 + A4); returns the largest |posterior| it wrote.  FRESH:
    // the shot's first round, where every old message is zero (v = P) and the check state is
    // written without being read.
    auto sweep = [&](auto fresh, float g0) {
        constexpr bool FRESH = decltype(fresh)::value;
        float pmax = 0.0f;   // largest |posterior| written this round
        for (int l = 0; l < lay.L; ++l) {
            const int p1 = __ldg(lay.lay_ptr + l + 1);
            for (int p = __ldg(lay.lay_ptr + l) + t; p < p1; p += T) {
                uint32_t off[DC];
                const int i = load_rec(p, off);
                const uint32_t s_i = (sbits[i >> 5] >> (i & 31)) & 1u;
                const float g = (sagms_mode && ((rbits[p >> 5] >> (p & 31)) & 1u)) ? g0 * eta : g0;
                float v[DC];
                uint32_t par = s_i << 31;
                if constexpr (FRESH) {
#pragma unroll
                    for (int j = 0; j < DC; ++j) {
                        v[j] = Pat(off[j]);
                        par ^= __float_as_uint(v[j]);
                    }
                } else {
                    const uint32_t mt = meta[p];
                    const float q1 = O1[p], q2 = O2[p];
                    const int am = (int)(mt >> 24);
#pragma unroll
                    for (int j = 0; j < DC; ++j) {
                        const float mag = (j == am) ? q2 : q1;
                        const float c_old = __uint_as_float(__float_as_uint(mag) | ((mt << (31 - j)) & kSign));
                        v[j] = Pat(off[j]) - c_old;
                        par ^= __float_as_uint(v[j]);
                    }
                }
                par &= kSign;
                float m1 = inf, m2 = inf;
#pragma unroll
                for (int j = 0; j < DC; ++j) {
                    const float av = fabsf(v[j]);
                    m2 = fminf(m2, fmaxf(m1, av));
                    m1 = fminf(m1, av);
                }
                const float o1 = fminf(g * m1, kMsFamClip), o2 = fminf(g * m2, kMsFamClip);
                uint32_t nm = 0u, eqm = 0u;   // output signs; slots at the minimum
#pragma unroll
                for (int j = 0; j < DC; ++j) {
                    const uint32_t sg = (par ^ __float_as_uint(v[j])) & kSign;
                    const bool eq = fabsf(v[j]) == m1;
                    const float pn = v[j] + __uint_as_float(__float_as_uint(eq ? o2 : o1) | sg);
                    Pat(off[j]) = pn;
                    pmax = fmaxf(pmax, fabsf(pn));
                    nm |= sg >> (31 - j);
                    eqm |= (uint32_t)eq << j;
                }
                O1[p] = o1;
                O2[p] = o2;
                meta[p] = nm | ((uint32_t)(__ffs(eqm) - 1) << 24);   // first slot at the minimum
            }
            sync();
        }
        return pmax;
    };

    // Posteriors rebuilt from the current messages, P_c = L0_c + sum over the qubit's edges in
    // a fixed order (Eq. 2), after a round (not the first, which starts from zero messages) in
    // which a posterior grew large: a posterior's rounding error then depends on the messages
    // of that round only, not on every large value it took while updated in place.
    auto rebuild = [&](float prior_c) {
        for (int c = t; c < n; c += T) {
            float acc = per_qubit ? PQ[c] : prior_c;
            const uint16_t* q = lay.qe + (size_t)c * lay.QE;
            for (int k = 0; k < lay.QE; ++k) {
                const uint32_t e = __ldg(q + k);
                if (e == 0xffffu) break;
                const int p = (int)(e >> 5), j = (int)(e & 31u);
                const uint32_t mt = meta[p];
                const float mag = (j == (int)(mt >> 24)) ? O2[p] : O1[p];
                acc += __uint_as_float(__float_as_uint(mag) | ((mt << (31 - j)) & kSign));
            }
            P[c] = acc;
        }
    };

    for (int c = n + t; c < Np; c += T) P[c] = inf;
    int pq_ok = 1;
    if (per_qubit) {
        for (int c = t; c < n; c += T) {
            const float v = __ldg(a.L0 + c) + 0.0f;   // -0 -> +0: the sign bit is the decision
            PQ[c] = v;
            pq_ok &= isfinite(v) ? 1 : 0;
        }
    }
    if constexpr (T == 32) pq_ok = __all_sync(0xffffffffu, pq_ok);
    else pq_ok = __syncthreads_and(pq_ok);

    for (long long shot = blockIdx.x; shot < a.shots; shot += gridDim.x) {
        float prior = 0.0f;
        float amax = a.amax;
        bool valid;
        if (per_qubit) {
            valid = pq_ok != 0;
        } else {
            const float l0 = __ldg(a.L0 + shot);
            valid = isfinite(l0);
            prior = (l0 > 0.0f) ? 1.0f : ((l0 < 0.0f) ? -1.0f : 0.0f);
            if (valid) amax = shot_alpha_max(a, l0);
        }
        if (!valid) {
            for (int w = t; w < nw; w += T) a.err[shot * nw + w] = 0u;
            if (t == 0) { a.conv[shot] = 0; a.iters[shot] = -1; }
            continue;
        }
        // A0: P = L0, load s (every message is zero: the first round reads no check state)
        for (int c = t; c < n; c += T) P[c] = per_qubit ? PQ[c] : prior;
        for (int w = t; w < mw; w += T) sbits[w] = __ldg(a.syn + shot * mw + w);
        if (t == 0) { cnt_sh[0] = 0; cnt_sh[1] = 0; }
        sync();

        int it = 0, cnt = 0;
        for (;; ++it) {
            // A5: hard decision and residual bit of every check (Eq. 1), count (Eq. 6).  Before
            // the first round with one prior per shot every decision is [L0 < 0], so a check's
            // residual is its syndrome bit XOR, under a negative prior, its degree's parity.
            const bool closed = it == 0 && !per_qubit;
            for (int base = 0; base < Mp; base += T) {
                const int p = base + t;
                uint32_t x = 0u;
                if (p < m && closed) {
                    int deg;
                    const int i = load_head(p, deg);
                    x = ((sbits[i >> 5] >> (i & 31)) ^ (prior < 0.0f ? (uint32_t)deg : 0u)) & 1u;
                } else if (p < m) {
                    uint32_t off[DC];
                    const int i = load_rec(p, off);
                    x = (sbits[i >> 5] >> (i & 31)) & 1u;
#pragma unroll
                    for (int j = 0; j < DC; ++j) x ^= __float_as_uint(Pat(off[j])) >> 31;
                }
                const uint32_t b = __ballot_sync(0xffffffffu, x);
                if (lane == 0 && p < Mp) {
                    rbits[p >> 5] = b;
                    if (b) atomicAdd(&cnt_sh[it & 1], __popc(b));
                }
            }
            sync();
            cnt = cnt_sh[it & 1];
            if (a.trace) {
                float* tr = a.trace + ((size_t)shot * (size_t)(a.max_iter + 1) + (size_t)it) * (size_t)n;
                for (int c = t; c < n; c += T) tr[c] = P[c];
            }
            // A6
            if ((cnt == 0 && early) || it == a.max_iter) break;
            if (t == 0) cnt_sh[(it + 1) & 1] = 0;
            // A2: the round's gain (Eq. 7), boosted on unsatisfied checks
            const float g0 = (a.mode == kModeSAGMS) ? amax - (amax - a.amin) * ((float)cnt * a.inv_m)
                                                    : ((a.mode == kModeSMS) ? a.alpha : 1.0f);
            // A3 + A4, layer by layer; then the rebuild when the round had a large posterior
            if (it == 0) {
                sweep(std::true_type{}, g0);
            } else {
                const float pmax = sweep(std::false_type{}, g0);
                bool big = per_qubit || pmax > kLayeredRebuild;
                if constexpr (T == 32) big = __any_sync(0xffffffffu, big);
                else big = __syncthreads_or(big);
                if (big) {
                    rebuild(prior);
                    sync();
                }
            }
        }

        // A7: write-out
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
        sync();
    }
}

}  // namespace sagms
