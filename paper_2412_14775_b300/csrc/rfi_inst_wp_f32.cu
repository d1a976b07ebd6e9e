// rfi_inst_wp_f32.cu -- window-parallel kernels for complex64 input (the lanes of a
// row take whole windows in turn), compiled apart so that all instances build in
// parallel.
#include "rfi_wpar.cuh"
#include "rfi_kernels.h"

namespace rfi {

static const WpInstance k_table[] = {
    RFI_WP_CH(DT_F32, 1, 2), RFI_WP_CH(DT_F32, 1, 4), RFI_WP_CH(DT_F32, 1, 8),
    RFI_WPM_CH(DT_F32, 1, 2), RFI_WPM_CH(DT_F32, 1, 4), RFI_WPS_CH(DT_F32, 1, 0),
    RFI_WPW(DT_F32, 1, 2, 5, 0), RFI_WPW(DT_F32, 1, 4, 5, 0),
};

WpTable wp_instances_f32() { return {k_table, (int)(sizeof(k_table) / sizeof(k_table[0]))}; }

}  // namespace rfi
