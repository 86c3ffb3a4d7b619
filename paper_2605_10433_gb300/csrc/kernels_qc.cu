// Instantiations of the column-indexed group kernels (decode_qc.cuh), three per shape: per-shot
// priors, per-shot priors with the automatic gain ceiling, and per-qubit priors.  Four checks per thread where the offsets and inputs
// fit in 128 registers (two checks per thread in 1024-thread CTAs measured 5-15% slower at
// n = 2046).
#include "kernels.h"

namespace sagms_kernels {

#define SAGMS_QC(DC, DV, K, T, NP)                                                                     \
    QcVariant {                                                                                         \
        DC, DV, K, T, NP,                                                                               \
            {sagms::qc_kernel<sagms::QcShape<DC, DV, K, T, NP>, false, false>,                          \
             sagms::qc_kernel<sagms::QcShape<DC, DV, K, T, NP>, true, false>,                           \
             sagms::qc_kernel<sagms::QcShape<DC, DV, K, T, NP>, false, true>},                          \
            {sagms::QcShape<DC, DV, K, T, NP>::SMEM, sagms::QcShape<DC, DV, K, T, NP>::SMEM,            \
             sagms::QcShape<DC, DV, K, T, NP>::SMEM_PQ}                                                 \
    }
const QcVariant kQcVariants[] = {
    SAGMS_QC(6, 3, 2, 32, 128),                                                       // n <= 128
    SAGMS_QC(8, 4, 4, 32, 256),                                                       // n <= 256
    SAGMS_QC(6, 3, 4, 64, 512),  SAGMS_QC(8, 4, 4, 64, 512),  SAGMS_QC(10, 5, 4, 64, 512),
    SAGMS_QC(12, 6, 4, 64, 512), SAGMS_QC(16, 8, 2, 128, 512),                        // n <= 512
    SAGMS_QC(8, 4, 4, 128, 1024), SAGMS_QC(10, 5, 4, 128, 1024),                      // n <= 1024
    SAGMS_QC(6, 3, 4, 256, 2048), SAGMS_QC(8, 4, 4, 256, 2048), SAGMS_QC(10, 5, 4, 256, 2048),
};
#undef SAGMS_QC
const int kNumQc = sizeof(kQcVariants) / sizeof(kQcVariants[0]);

}  // namespace sagms_kernels
