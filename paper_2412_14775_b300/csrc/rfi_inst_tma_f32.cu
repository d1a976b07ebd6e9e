// rfi_inst_tma_f32.cu -- shared-memory (TMA) loader instances for complex64 input.
#include "rfi_device.cuh"
#include "rfi_kernels.h"

namespace rfi {

static const TmaInstance k_table[] = {
    RFI_TMA_PB(DT_F32, 1, 1),
    RFI_TMA_PB(DT_F32, 1, 2),
    RFI_TMA_PB(DT_F32, 1, 4),
    RFI_TMA_PB(DT_F32, 1, 8),
};

TmaTable tma_instances_f32() { return {k_table, (int)(sizeof(k_table) / sizeof(k_table[0]))}; }

}  // namespace rfi
