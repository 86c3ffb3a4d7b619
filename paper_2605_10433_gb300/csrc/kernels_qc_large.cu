// Instantiations of the column-indexed group kernels (decode_qc.cuh), four per shape: per-shot
// priors, per-shot priors with the automatic gain ceiling, per-qubit priors, and the BP rule
// with per-shot priors.  Shapes for slot degrees (6, 3), (8, 4) and (10, 5) -- GB codes of
// weight w = 3, 4, 5 and any other code whose degrees fit -- at every size class, four checks
// per thread where the offsets and inputs fit in 128 registers (two checks per thread in
// 1024-thread CTAs measured 5-15% slower at n = 2046).
#include "kernels.h"

namespace sagms_kernels {

#define SAGMS_QC(DC, DV, K, T, NP)                                                                     \
    QcVariant {                                                                                         \
        DC, DV, K, T, NP,                                                                               \
            {sagms::qc_kernel<sagms::QcShape<DC, DV, K, T, NP>, false, false>,                          \
             sagms::qc_kernel<sagms::QcShape<DC, DV, K, T, NP>, true, false>,                           \
             sagms::qc_kernel<sagms::QcShape<DC, DV, K, T, NP>, false, true>,                           \
             sagms::qc_kernel<sagms::QcShape<DC, DV, K, T, NP>, false, false, true>},                   \
            {sagms::QcShape<DC, DV, K, T, NP>::SMEM, sagms::QcShape<DC, DV, K, T, NP>::SMEM,            \
             sagms::QcShape<DC, DV, K, T, NP>::SMEM_PQ, sagms::QcShape<DC, DV, K, T, NP>::SMEM}         \
    }
const QcVariant kQcVariantsLarge[] = {
    // n <= 1024: 128-thread groups (up to 512 checks)
    SAGMS_QC(6, 3, 4, 128, 1024), SAGMS_QC(8, 4, 4, 128, 1024), SAGMS_QC(10, 5, 4, 128, 1024),
    // n <= 2048: 256-thread groups (up to 1024 checks)
    SAGMS_QC(6, 3, 4, 256, 2048), SAGMS_QC(8, 4, 4, 256, 2048), SAGMS_QC(10, 5, 4, 256, 2048),
};
#undef SAGMS_QC
const int kNumQcLarge = sizeof(kQcVariantsLarge) / sizeof(kQcVariantsLarge[0]);

}  // namespace sagms_kernels
