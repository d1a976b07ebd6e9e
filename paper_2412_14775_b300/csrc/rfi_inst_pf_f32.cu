// rfi_inst_pf_f32.cu -- the plain 128-register kernels for complex64 input with
// the L2 prefetch code compiled in.
#include "rfi_device.cuh"
#include "rfi_kernels.h"

namespace rfi {

static const Instance k_table[] = {
    RFI_INSTF_P(DT_F32, 1, 0),
    RFI_INSTF_P(DT_F32, 1, 1),
};

InstanceTable instances_f32_pf() {
    return {k_table, (int)(sizeof(k_table) / sizeof(k_table[0]))};
}

}  // namespace rfi
