// rfi_inst_sw_f32.cu -- overlapping-window kernels for complex64 input (L = 2 windows
// per sample), compiled apart from the other instances so that all build in
// parallel.
#include "rfi_sliding.cuh"
#include "rfi_kernels.h"

namespace rfi {

static const SwInstance k_table[] = {
    RFI_SW_CH(DT_F32, 1, 1, 2), RFI_SW_CH(DT_F32, 1, 2, 2), RFI_SW_CH(DT_F32, 1, 4, 2),
};

SwTable sw_instances_f32() { return {k_table, (int)(sizeof(k_table) / sizeof(k_table[0]))}; }

}  // namespace rfi
