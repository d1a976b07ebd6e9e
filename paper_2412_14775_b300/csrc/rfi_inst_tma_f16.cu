// rfi_inst_tma_f16.cu -- shared-memory (TMA) loader instances for binary16 input (two
// samples per 32-byte unit for even M, one per 16-byte unit and one lane per row for
// odd M).
#include "rfi_device.cuh"
#include "rfi_kernels.h"

namespace rfi {

static const TmaInstance k_table[] = {
    RFI_TMA_PB(DT_F16, 2, 1),
    RFI_TMA_PB(DT_F16, 2, 2),
    RFI_TMA_PB(DT_F16, 2, 4),
    RFI_TMA_PB(DT_F16, 2, 8),
    RFI_TMA_PB(DT_F16, 1, 1),
};

TmaTable tma_instances_f16() { return {k_table, (int)(sizeof(k_table) / sizeof(k_table[0]))}; }

}  // namespace rfi
