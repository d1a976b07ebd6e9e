// rfi_inst_wp_f16.cu -- window-parallel kernels for binary16 input (two samples per
// 32-byte unit for even windows, one per 16-byte unit for odd windows).
#include "rfi_wpar.cuh"
#include "rfi_kernels.h"

namespace rfi {

static const WpInstance k_table[] = {
    RFI_WP_CH(DT_F16, 2, 2), RFI_WP_CH(DT_F16, 2, 4), RFI_WP_CH(DT_F16, 2, 8),
    RFI_WP_CH(DT_F16, 1, 2), RFI_WP_CH(DT_F16, 1, 4), RFI_WP_CH(DT_F16, 1, 8),
    RFI_WPM_CH(DT_F16, 2, 2), RFI_WPM_CH(DT_F16, 2, 4), RFI_WPM_CH(DT_F16, 1, 2),
    RFI_WPM_CH(DT_F16, 1, 4), RFI_WPS_CH(DT_F16, 2, 0), RFI_WPS_CH(DT_F16, 1, 0),
    RFI_WPS3_CH(DT_F16, 0), RFI_WPW3_CH(DT_F16, 0), RFI_WPW(DT_F16, 2, 4, 4, 0),
    RFI_WPW(DT_F16, 2, 2, 4, 0),
};

WpTable wp_instances_f16() { return {k_table, (int)(sizeof(k_table) / sizeof(k_table[0]))}; }

}  // namespace rfi
