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
const QcVariant kQcVariantsSmall[] = {
    // n <= 128: warp-sized groups, two checks per thread (up to 64 checks)
    SAGMS_QC(6, 3, 2, 32, 128), SAGMS_QC(8, 4, 2, 32, 128), SAGMS_QC(10, 5, 2, 32, 128),
    // n <= 256: warp-sized groups, four checks per thread (up to 128 checks)
    SAGMS_QC(6, 3, 4, 32, 256), SAGMS_QC(8, 4, 4, 32, 256), SAGMS_QC(10, 5, 4, 32, 256),
    // n <= 512: 64-thread groups (up to 256 checks); (16, 8) with two checks per thread
    SAGMS_QC(6, 3, 4, 64, 512), SAGMS_QC(8, 4, 4, 64, 512), SAGMS_QC(10, 5, 4, 64, 512),
    SAGMS_QC(12, 6, 4, 64, 512), SAGMS_QC(16, 8, 2, 128, 512),
};
#undef SAGMS_QC
const int kNumQcSmall = sizeof(kQcVariantsSmall) / sizeof(kQcVariantsSmall[0]);

}  // namespace sagms_kernels
