// rfi_inst_pw_f32.cu -- kernel instances for complex64 input with partial windows
// (blocks of any length); compiled apart from rfi_inst_f32.cu so that both build in
// parallel.
#include "rfi_device.cuh"
#include "rfi_kernels.h"

namespace rfi {

static const Instance k_table[] = {
    RFI_INSTP_P(DT_F32, 1, 0),
    RFI_INSTP_P(DT_F32, 1, 1),
};

InstanceTable instances_f32_pw() {
    return {k_table, (int)(sizeof(k_table) / sizeof(k_table[0]))};
}

}  // namespace rfi
