// rfi_inst_f32.cu -- kernel instances for complex64 input (32 bytes per sample).
#include "rfi_device.cuh"
#include "rfi_kernels.h"

namespace rfi {

static const Instance k_table[] = {
    RFI_INSTM_CH(DT_F32, 1),
    RFI_INST0_P(DT_F32, 1, 0),
    RFI_INST0_P(DT_F32, 1, 1),
    RFI_INSTB_P(DT_F32, 1, 1),
    RFI_INSTB_P(DT_F32, 1, 2),
    RFI_INSTV_P(DT_F32, 1),
    RFI_INST3_P(DT_F32, 1),
};

InstanceTable instances_f32() { return {k_table, (int)(sizeof(k_table) / sizeof(k_table[0]))}; }

}  // namespace rfi
