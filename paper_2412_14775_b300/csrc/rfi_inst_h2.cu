// rfi_inst_h2.cu -- kernel instances of the binary16 Stokes arithmetic mode
// (precision = 2, binary16 input): lanes splitting each window (P = 1, 2, 4, 8; one
// lane per row for odd windows) and window-parallel lanes (P = 2, 4, 8).
#include "rfi_device.cuh"
#include "rfi_kernels.h"
#include "rfi_wpar.cuh"

namespace rfi {

static const Instance k_table[] = {
    RFI_INSTH_CH(DT_F16, 2, 1, 0), RFI_INSTH_CH(DT_F16, 2, 2, 0), RFI_INSTH_CH(DT_F16, 2, 4, 0),
    RFI_INSTH_CH(DT_F16, 2, 8, 0), RFI_INSTH_CH(DT_F16, 2, 1, 1), RFI_INSTH_CH(DT_F16, 2, 2, 1),
    RFI_INSTH_CH(DT_F16, 2, 4, 1), RFI_INSTH_CH(DT_F16, 2, 8, 1), RFI_INSTH_CH(DT_F16, 1, 1, 0),
    RFI_INSTH_CH(DT_F16, 1, 1, 1),
    RFI_INST3H_P(DT_F16, 2),
    RFI_INST3H(DT_F16, 1, 1, 1),
    RFI_INST3H(DT_F16, 1, 1, 2),
};

static const WpInstance wp_table[] = {
    RFI_WPH_CH(DT_F16, 2, 2), RFI_WPH_CH(DT_F16, 2, 4), RFI_WPH_CH(DT_F16, 2, 8),
    RFI_WPH_CH(DT_F16, 1, 2), RFI_WPH_CH(DT_F16, 1, 4), RFI_WPH_CH(DT_F16, 1, 8),
    RFI_WPS_CH(DT_F16, 2, 2), RFI_WPS_CH(DT_F16, 1, 2), RFI_WPS3_CH(DT_F16, 2),
    RFI_WPW3_CH(DT_F16, 2), RFI_WPW(DT_F16, 2, 4, 4, 2),
};

InstanceTable instances_f16_h2() { return {k_table, (int)(sizeof(k_table) / sizeof(k_table[0]))}; }
WpTable wp_instances_f16_h2() { return {wp_table, (int)(sizeof(wp_table) / sizeof(wp_table[0]))}; }

}  // namespace rfi
