// Instantiations of the two-slot kernels (decode_slots.cuh) and of the two-group kernel
// (decode_groups.cuh).
#include "kernels.h"

namespace sagms_kernels {

using sagms::slot_kernel;

const SlotVariant kSlotVariants[] = {
    {6, 3, 64, 128, slot_kernel<6, 3, 64, 128>},        {8, 4, 128, 256, slot_kernel<8, 4, 128, 256>},
    {6, 3, 256, 512, slot_kernel<6, 3, 256, 512>},      {8, 4, 256, 512, slot_kernel<8, 4, 256, 512>},
    {10, 5, 256, 512, slot_kernel<10, 5, 256, 512>},    {12, 6, 256, 512, slot_kernel<12, 6, 256, 512>},
    {16, 8, 256, 512, slot_kernel<16, 8, 256, 512>},    {10, 5, 512, 1024, slot_kernel<10, 5, 512, 1024>},
    {10, 5, 1024, 2048, slot_kernel<10, 5, 1024, 2048>}};
const int kNumSlotVariants = sizeof(kSlotVariants) / sizeof(kSlotVariants[0]);

GroupFn group_kernel_fn() { return sagms::group_kernel<kGroupDC, kGroupDV>; }

}  // namespace sagms_kernels
