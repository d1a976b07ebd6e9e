// rfi_inst_ad_f16.cu -- kernel instances with online per-stream SK thresholds for
// binary16 input.
#include "rfi_device.cuh"
#include "rfi_kernels.h"

namespace rfi {

static const Instance k_table[] = {
    RFI_INSTA_P(DT_F16, 2, 0),
    RFI_INSTA_P(DT_F16, 2, 1),
    RFI_INSTA_CH(DT_F16, 1, 1, 0),
    RFI_INSTA_CH(DT_F16, 1, 1, 1),
};

InstanceTable instances_f16_ad() {
    return {k_table, (int)(sizeof(k_table) / sizeof(k_table[0]))};
}

}  // namespace rfi
