// rfi_inst_f16.cu -- kernel instances for binary16 input (16 bytes per sample): two
// samples per 32-byte load unit when M is even, one per 16-byte unit when M is odd.
#include "rfi_device.cuh"
#include "rfi_kernels.h"

namespace rfi {

static const Instance k_table[] = {
    RFI_INSTM_CH(DT_F16, 2),
    RFI_INSTM_CH(DT_F16, 1),
    RFI_INST0_P(DT_F16, 2, 0),
    RFI_INST0_P(DT_F16, 2, 1),
    RFI_INSTB_P(DT_F16, 2, 1),
    RFI_INSTB_P(DT_F16, 2, 2),
    RFI_INST0_CH(DT_F16, 1, 1, 0),
    RFI_INST0_CH(DT_F16, 1, 1, 1),
    RFI_INSTB_CH(DT_F16, 1, 1, 1),
    RFI_INSTB_CH(DT_F16, 1, 1, 2),
    RFI_INSTV_P(DT_F16, 2),
    RFI_INST3_P(DT_F16, 2),
    RFI_INST3(DT_F16, 1, 1, 1),
    RFI_INST3(DT_F16, 1, 1, 2),
};

InstanceTable instances_f16() { return {k_table, (int)(sizeof(k_table) / sizeof(k_table[0]))}; }

}  // namespace rfi
