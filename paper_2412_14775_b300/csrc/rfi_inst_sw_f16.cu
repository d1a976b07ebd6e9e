// rfi_inst_sw_f16.cu -- overlapping-window kernels for binary16 input (two samples
// per 32-byte unit for even hops, one per 16-byte unit for odd hops).
#include "rfi_sliding.cuh"
#include "rfi_kernels.h"

namespace rfi {

static const SwInstance k_table[] = {
    RFI_SW_CH(DT_F16, 2, 1, 2), RFI_SW_CH(DT_F16, 2, 2, 2), RFI_SW_CH(DT_F16, 2, 4, 2),
    RFI_SW_CH(DT_F16, 1, 1, 2),
};

SwTable sw_instances_f16() { return {k_table, (int)(sizeof(k_table) / sizeof(k_table[0]))}; }

}  // namespace rfi
