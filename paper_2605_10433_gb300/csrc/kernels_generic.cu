// Instantiations of the one-shot-per-CTA kernel (decode_kernel.cuh) for every variant.
#include "kernels.h"

namespace sagms_kernels {

const Variant kVariants[] = {{4, 2}, {6, 3}, {8, 4}, {10, 5}, {12, 6}, {16, 8}, {32, 16}};
const int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);

namespace {
template <int DC, int DV>
KernelFn pick(bool bp) { return bp ? sagms::decode_kernel<DC, DV, true> : sagms::decode_kernel<DC, DV, false>; }
}  // namespace

KernelFn generic_kernel(int variant, bool bp) {
    switch (variant) {
        case 0: return pick<4, 2>(bp);
        case 1: return pick<6, 3>(bp);
        case 2: return pick<8, 4>(bp);
        case 3: return pick<10, 5>(bp);
        case 4: return pick<12, 6>(bp);
        case 5: return pick<16, 8>(bp);
        default: return pick<32, 16>(bp);
    }
}

}  // namespace sagms_kernels
