// Instantiations of the layered-schedule kernel (decode_layered.cuh).
#include "kernels.h"

namespace sagms_kernels {

using sagms::layered_kernel;

const LayeredVariant kLayeredVariants[] = {
    {6, 32, layered_kernel<6, 32>},     {6, 64, layered_kernel<6, 64>},     {6, 128, layered_kernel<6, 128>},
    {8, 32, layered_kernel<8, 32>},     {8, 64, layered_kernel<8, 64>},     {8, 128, layered_kernel<8, 128>},
    {10, 32, layered_kernel<10, 32>},   {10, 64, layered_kernel<10, 64>},   {10, 128, layered_kernel<10, 128>},
    {12, 32, layered_kernel<12, 32>},   {12, 64, layered_kernel<12, 64>},   {12, 128, layered_kernel<12, 128>},
    {16, 32, layered_kernel<16, 32>},   {16, 64, layered_kernel<16, 64>},   {16, 128, layered_kernel<16, 128>},
    {24, 32, layered_kernel<24, 32>},   {24, 64, layered_kernel<24, 64>},   {24, 128, layered_kernel<24, 128>}};
const int kNumLayeredVariants = sizeof(kLayeredVariants) / sizeof(kLayeredVariants[0]);

}  // namespace sagms_kernels
