// The library's compiled decoder kernels and their shapes.  Each table is defined, with the
// kernel instantiations it names, in a translation unit of its own (kernels_*.cu), so the
// kernels compile in parallel; sagms.cu selects and launches them through these tables.
#pragma once

#include <cstddef>
#include <cstdint>

#include "decode_layered.cuh"
#include "decode_qc.cuh"

namespace sagms_kernels {

using sagms::DecodeArgs;

// One shot per CTA (decode_kernel.cuh), for every mode: (padded check degree, padded qubit
// degree), the first variant that covers a code's largest degrees.
struct Variant { int dc, dv; };
extern const Variant kVariants[];
extern const int kNumVariants;
using KernelFn = void (*)(const DecodeArgs);
KernelFn generic_kernel(int variant, bool bp);

// Two shot slots per CTA (decode_slots.cuh), MS family: (DC, DV, MP threads, NP qubit slots).
using SlotFn = void (*)(const DecodeArgs, const sagms::SlotLayout);
struct SlotVariant { int dc, dv, mp, np; SlotFn fn; };
extern const SlotVariant kSlotVariants[];
extern const int kNumSlotVariants;

// Two 512-thread groups per CTA (decode_groups.cuh), MS family: one compiled shape, for codes
// with more than 512 and at most 1024 checks, at most 2048 qubits and degrees up to (10, 5).
constexpr int kGroupDC = 10, kGroupDV = 5;
using GroupFn = void (*)(const DecodeArgs, const sagms::GroupLayout);
GroupFn group_kernel_fn();

// Column-indexed groups (decode_qc.cuh): one entry per compiled shape, listed by increasing
// size; a code takes the first whose slot degrees cover it (DC = 2 DV), whose checks and
// qubits it fills at least halfway, and whose slot structure it has.
using QcFn = void (*)(const DecodeArgs, const uint32_t*);
struct QcVariant {
    int dc, dv, k, t, np;
    QcFn fn[4];      // per-shot priors, per-shot priors with the automatic ceiling, per-qubit priors,
                     // BP with per-shot priors
    size_t smem[4];  // shared memory of each
};
// Two tables (kernels_qc_small.cu: n <= 512; kernels_qc_large.cu: n > 512), compiled in
// parallel and read as one list, smallest shapes first.
extern const QcVariant kQcVariantsSmall[];
extern const int kNumQcSmall;
extern const QcVariant kQcVariantsLarge[];
extern const int kNumQcLarge;
inline int num_qc_variants() { return kNumQcSmall + kNumQcLarge; }
inline const QcVariant& qc_variant(int v) {
    return v < kNumQcSmall ? kQcVariantsSmall[v] : kQcVariantsLarge[v - kNumQcSmall];
}
// Column-indexed shapes for BP alone (kernels_qc_bp.cu): two checks per thread at 64
// registers, two 512-thread CTAs per SM, for 129 to 512 and 1025 to 2048 qubits; only fn[3]
// and smem[3] are set.  A code takes the first whose message rows equal its column-indexed shape's (the same
// slots) and whose checks and qubits it fills at least halfway.
extern const QcVariant kQcBpVariants[];
extern const int kNumQcBp;

// Layered schedule (decode_layered.cuh), MS family: (padded check degree, threads per CTA).
// A code takes the first check degree that covers it, with 32 threads when no layer holds
// more than 64 checks, 64 when none holds more than 128, and 128 otherwise.
using LayeredFn = void (*)(const DecodeArgs, const sagms::LayeredLayout);
struct LayeredVariant { int dc, t; LayeredFn fn; };
extern const LayeredVariant kLayeredVariants[];
extern const int kNumLayeredVariants;

}  // namespace sagms_kernels
