// rfi_inst_ad_f32.cu -- kernel instances with online per-stream SK thresholds for
// complex64 input.
#include "rfi_device.cuh"
#include "rfi_kernels.h"

namespace rfi {

static const Instance k_table[] = {
    RFI_INSTA_P(DT_F32, 1, 0),
    RFI_INSTA_P(DT_F32, 1, 1),
};

InstanceTable instances_f32_ad() {
    return {k_table, (int)(sizeof(k_table) / sizeof(k_table[0]))};
}

}  // namespace rfi
