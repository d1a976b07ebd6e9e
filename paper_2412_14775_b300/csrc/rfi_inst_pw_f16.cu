// rfi_inst_pw_f16.cu -- kernel instances for binary16 input with partial windows
// (blocks of any length; even lengths when two samples share a load unit).
#include "rfi_device.cuh"
#include "rfi_kernels.h"

namespace rfi {

static const Instance k_table[] = {
    RFI_INSTP_P(DT_F16, 2, 0),
    RFI_INSTP_P(DT_F16, 2, 1),
    RFI_INSTP_CH(DT_F16, 1, 1, 0),
    RFI_INSTP_CH(DT_F16, 1, 1, 1),
};

InstanceTable instances_f16_pw() {
    return {k_table, (int)(sizeof(k_table) / sizeof(k_table[0]))};
}

}  // namespace rfi
