// Column-indexed group kernels for BP alone (decode_qc.cuh, the BP instantiation): two checks
// per thread, 64 registers, two 512-thread CTAs per SM.  Shapes for slot degrees (6, 3), (8, 4)
// and (10, 5) at 256, 512 and 2048 qubits (groups of 64, 128 and 512 threads).  At these sizes
// BP on the four-checks-per-thread shapes (128 registers, one CTA per SM) hides its
// transcendental chains worse than the one-shot-per-CTA kernel; these shapes keep 32 warps per
// SM and the column-indexed layout.  Measured against the one-shot-per-CTA kernel (BP, 1e6
// shots at p = 0.005, 0.01, 0.02): GB(127, 4) 1.44x, GB(255, 5) 1.23x, GB(1023, 5) 1.51x,
// GB(1023, 3) 1.49x; the 1024-qubit class lost (0.82x at GB(511, 5)) and has no shape here.
#include "kernels.h"

namespace sagms_kernels {

#define SAGMS_QC_BP(DC, DV, T, NP)                                                                     \
    QcVariant {                                                                                         \
        DC, DV, 2, T, NP, {nullptr, nullptr, nullptr, sagms::qc_kernel<sagms::QcShape<DC, DV, 2, T, NP>, false, false, true>}, \
            {0, 0, 0, sagms::QcShape<DC, DV, 2, T, NP>::SMEM}                                           \
    }
const QcVariant kQcBpVariants[] = {
    SAGMS_QC_BP(6, 3, 64, 256),   SAGMS_QC_BP(8, 4, 64, 256),   SAGMS_QC_BP(10, 5, 64, 256),
    SAGMS_QC_BP(6, 3, 128, 512),  SAGMS_QC_BP(8, 4, 128, 512),  SAGMS_QC_BP(10, 5, 128, 512),
    SAGMS_QC_BP(6, 3, 512, 2048), SAGMS_QC_BP(8, 4, 512, 2048), SAGMS_QC_BP(10, 5, 512, 2048),
};
#undef SAGMS_QC_BP
const int kNumQcBp = sizeof(kQcBpVariants) / sizeof(kQcBpVariants[0]);

}  // namespace sagms_kernels
