// rfi_kernels.h -- the table of compiled kernel instances (internal).
//
// One entry per (input dtype, samples per load unit, lanes per row P, load units per
// chunk CH in {1, 2, 4, 5} (two chunks are in flight per lane), Kahan on/off, register budget LB).  The instances live in two translation
// units (complex64 and binary16) so that they compile in parallel.
#pragma once

namespace rfi {

struct Instance {
    int dt, spu, P, ch, kahan, lb, mixed, vs, pw, ad, pf;   // mixed: the precision mode
    const void *block_fn;   // k_block<...>
    const void *batch_fn;   // k_batch<...>; the register budget, the buffered stores and
                            // the prefetch do not change results, so all those share the
                            // plain batch kernel (null: take the plain sibling's)
};

struct InstanceTable {
    const Instance *items;
    int n;
};

InstanceTable instances_f32();
InstanceTable instances_f16();
InstanceTable instances_f32_pw();     // partial windows (rfi_inst_pw_f32.cu)
InstanceTable instances_f16_pw();     // partial windows (rfi_inst_pw_f16.cu)
InstanceTable instances_f32_ad();     // online SK thresholds (rfi_inst_ad_f32.cu)
InstanceTable instances_f16_ad();     // online SK thresholds (rfi_inst_ad_f16.cu)
InstanceTable instances_f32_pf();     // plain kernels with L2 prefetch (rfi_inst_pf_f32.cu)
InstanceTable instances_f16_pf();     // plain kernels with L2 prefetch (rfi_inst_pf_f16.cu)
InstanceTable instances_f16_h2();     // binary16 Stokes arithmetic (rfi_inst_h2.cu)
// State update of adaptive contexts after a flagging launch (rfi_adapt.cu): one thread
// per footprint row; k_adapt takes a StreamArgs, k_adapt_batch a BatchArgs.
const void *adapt_fn();
const void *adapt_batch_fn();

// The shared-memory (TMA) loader for one stream (batches use the direct loader).
struct TmaInstance {
    int dt, spu, P, ch, kahan, lb;
    const void *fn;         // k_tma<...>: one bulk copy per row and stage
    const void *fn2;        // k_tma2<...>: one tensor tile per warp and stage (no Kahan)
};
struct TmaTable {
    const TmaInstance *items;
    int n;
};
TmaTable tma_instances_f32();
TmaTable tma_instances_f16();

// Overlapping windows (rfi_sliding.cuh): L = M / H = 2 windows hold every sample (the
// registers of two more pending segments, L = 4, spill).
struct SwInstance {
    int dt, spu, P, ch, L;
    const void *fn;         // k_slide<...>
    const void *batch_fn;   // k_batch_sw<...>
};
struct SwTable {
    const SwInstance *items;
    int n;
};
SwTable sw_instances_f32();   // rfi_inst_sw_f32.cu
SwTable sw_instances_f16();   // rfi_inst_sw_f16.cu

// Window-parallel lanes (rfi_wpar.cuh): the P lanes of a row take whole windows in turn.
struct WpInstance {
    int dt, spu, P, ch, mixed;
    int fs;                 // 1: the whole-round flag-bit path (P M <= 32); 2: the same
                            // for launches whose rounds are all whole
    int lb;                 // register budget (0: 128, 3: 96); batches take the 128 kernel
    const void *fn;         // k_wpar<...>
    const void *batch_fn;   // k_batch_wp<...>
};
struct WpTable {
    const WpInstance *items;
    int n;
};
WpTable wp_instances_f32();   // rfi_inst_wp_f32.cu
WpTable wp_instances_f16();   // rfi_inst_wp_f16.cu
WpTable wp_instances_f16_h2();  // binary16 Stokes arithmetic (rfi_inst_h2.cu)

}  // namespace rfi

// Field `pf`: 1 = the kernel holds the L2 prefetch code (used when a launch asks for
// prefetch), 0 = it does not.  The plain 128-register kernels exist both ways; every
// other kind holds it.
// Entries for one (DT, SPU, P, CH, K): LB = 0 without prefetch code, and the batch
// kernel of every plain context (it holds the prefetch code, taken when the contexts
// ask for it; measured faster than the batch kernel without it, 514 against 552 us on
// the 8-subband batch).
#define RFI_INST0(DT, SPU, P, CH, K)                                                        \
    {DT, SPU, P, CH, K, 0, 0, 0, 0, 0, 0,                                                   \
     (const void *)&rfi::k_block<DT, SPU, P, CH, (bool)K, 0>,                               \
     (const void *)&rfi::k_batch<DT, SPU, P, CH, (bool)K, false, false, false, true>}
// The same with the L2 prefetch code (rfi_inst_pf_*.cu).  No batch kernel of its own: a
// batch of plain contexts runs the RFI_INST0 batch kernel, so that contexts with and
// without prefetch batch together.
#define RFI_INSTF(DT, SPU, P, CH, K)                                                        \
    {DT, SPU, P, CH, K, 0, 0, 0, 0, 0, 1,                                                   \
     (const void *)&rfi::k_block<DT, SPU, P, CH, (bool)K, 0, false, false, false, false,   \
                                 true>,                                                     \
     nullptr}
#define RFI_INSTF_CH(DT, SPU, P, K)                                                         \
    RFI_INSTF(DT, SPU, P, 1, K), RFI_INSTF(DT, SPU, P, 2, K), RFI_INSTF(DT, SPU, P, 4, K),  \
        RFI_INSTF(DT, SPU, P, 5, K)
#define RFI_INSTF_P(DT, SPU, K)                                                             \
    RFI_INSTF_CH(DT, SPU, 1, K), RFI_INSTF_CH(DT, SPU, 2, K), RFI_INSTF_CH(DT, SPU, 4, K),  \
        RFI_INSTF_CH(DT, SPU, 8, K), RFI_INSTF_CH(DT, SPU, 16, K),                         \
        RFI_INSTF_CH(DT, SPU, 32, K)
// A tighter register budget LB for the single-stream kernel (the batch kernel is the
// plain 128-register one).
#define RFI_INSTB(DT, SPU, P, CH, LB)                                                       \
    {DT, SPU, P, CH, 0, LB, 0, 0, 0, 0, 1,                                                  \
     (const void *)&rfi::k_block<DT, SPU, P, CH, false, LB, false, false, false, false,    \
                                 true>,                                                     \
     (const void *)&rfi::k_batch<DT, SPU, P, CH, false, false, false, false, true>}
// The paper-mixed precision mode (one lane per row).
#define RFI_INSTM(DT, SPU, CH)                                                              \
    {DT, SPU, 1, CH, 0, 0, 1, 0, 0, 0, 1,                                                   \
     (const void *)&rfi::k_block<DT, SPU, 1, CH, false, 0, true, false, false, false, true>, \
     (const void *)&rfi::k_batch<DT, SPU, 1, CH, false, true, false, false, true>}
// Buffered 16-byte output stores (for small windows); shares the batch kernel.
#define RFI_INSTV(DT, SPU, P, CH)                                                           \
    {DT, SPU, P, CH, 0, 0, 0, 1, 0, 0, 1,                                                   \
     (const void *)&rfi::k_block<DT, SPU, P, CH, false, 0, false, true, false, false,      \
                                 true>,                                                     \
     (const void *)&rfi::k_batch<DT, SPU, P, CH, false, false, false, false, true>}
#define RFI_INSTV_P(DT, SPU)                                                                \
    RFI_INSTV(DT, SPU, 1, 1), RFI_INSTV(DT, SPU, 1, 2), RFI_INSTV(DT, SPU, 1, 4),           \
        RFI_INSTV(DT, SPU, 2, 1), RFI_INSTV(DT, SPU, 2, 2), RFI_INSTV(DT, SPU, 2, 4),       \
        RFI_INSTV(DT, SPU, 4, 1), RFI_INSTV(DT, SPU, 4, 2), RFI_INSTV(DT, SPU, 4, 4)
// Partial windows (blocks of any length), 128-register budget.
#define RFI_INSTP(DT, SPU, P, CH, K)                                                        \
    {DT, SPU, P, CH, K, 0, 0, 0, 1, 0, 1,                                                   \
     (const void *)&rfi::k_block<DT, SPU, P, CH, (bool)K, 0, false, false, true, false,    \
                                 true>,                                                     \
     (const void *)&rfi::k_batch<DT, SPU, P, CH, (bool)K, false, true, false, true>}
#define RFI_INSTP_CH(DT, SPU, P, K)                                                         \
    RFI_INSTP(DT, SPU, P, 1, K), RFI_INSTP(DT, SPU, P, 2, K), RFI_INSTP(DT, SPU, P, 4, K),  \
        RFI_INSTP(DT, SPU, P, 5, K)
#define RFI_INSTP_P(DT, SPU, K)                                                             \
    RFI_INSTP_CH(DT, SPU, 1, K), RFI_INSTP_CH(DT, SPU, 2, K), RFI_INSTP_CH(DT, SPU, 4, K),  \
        RFI_INSTP_CH(DT, SPU, 8, K), RFI_INSTP_CH(DT, SPU, 16, K),                         \
        RFI_INSTP_CH(DT, SPU, 32, K)
// Online per-stream SK thresholds, 128-register budget.
#define RFI_INSTA(DT, SPU, P, CH, K)                                                        \
    {DT, SPU, P, CH, K, 0, 0, 0, 0, 1, 1,                                                   \
     (const void *)&rfi::k_block<DT, SPU, P, CH, (bool)K, 0, false, false, false, true,    \
                                 true>,                                                     \
     (const void *)&rfi::k_batch<DT, SPU, P, CH, (bool)K, false, false, true, true>}
#define RFI_INSTA_CH(DT, SPU, P, K)                                                         \
    RFI_INSTA(DT, SPU, P, 1, K), RFI_INSTA(DT, SPU, P, 2, K), RFI_INSTA(DT, SPU, P, 4, K),  \
        RFI_INSTA(DT, SPU, P, 5, K)
#define RFI_INSTA_P(DT, SPU, K)                                                             \
    RFI_INSTA_CH(DT, SPU, 1, K), RFI_INSTA_CH(DT, SPU, 2, K), RFI_INSTA_CH(DT, SPU, 4, K),  \
        RFI_INSTA_CH(DT, SPU, 8, K), RFI_INSTA_CH(DT, SPU, 16, K),                         \
        RFI_INSTA_CH(DT, SPU, 32, K)
#define RFI_INSTM_CH(DT, SPU)                                                               \
    RFI_INSTM(DT, SPU, 1), RFI_INSTM(DT, SPU, 2), RFI_INSTM(DT, SPU, 4), RFI_INSTM(DT, SPU, 5)
#define RFI_INST0_CH(DT, SPU, P, K)                                                         \
    RFI_INST0(DT, SPU, P, 1, K), RFI_INST0(DT, SPU, P, 2, K), RFI_INST0(DT, SPU, P, 4, K),  \
        RFI_INST0(DT, SPU, P, 5, K)
#define RFI_INSTB_CH(DT, SPU, P, LB)                                                        \
    RFI_INSTB(DT, SPU, P, 2, LB), RFI_INSTB(DT, SPU, P, 4, LB), RFI_INSTB(DT, SPU, P, 5, LB)
#define RFI_INST0_P(DT, SPU, K)                                                             \
    RFI_INST0_CH(DT, SPU, 1, K), RFI_INST0_CH(DT, SPU, 2, K), RFI_INST0_CH(DT, SPU, 4, K),  \
        RFI_INST0_CH(DT, SPU, 8, K), RFI_INST0_CH(DT, SPU, 16, K),                         \
        RFI_INST0_CH(DT, SPU, 32, K)
#define RFI_INSTB_P(DT, SPU, LB)                                                            \
    RFI_INSTB_CH(DT, SPU, 1, LB), RFI_INSTB_CH(DT, SPU, 2, LB), RFI_INSTB_CH(DT, SPU, 4, LB), \
        RFI_INSTB_CH(DT, SPU, 8, LB)
#define RFI_TMA(DT, SPU, P, CH, K, LB)                                                      \
    {DT, SPU, P, CH, K, LB, (const void *)&rfi::k_tma<DT, SPU, P, CH, (bool)K, LB>,         \
     rfi::tma2_fn<DT, SPU, P, CH, K, LB>()}
#define RFI_TMA_CH(DT, SPU, P, K, LB)                                                       \
    RFI_TMA(DT, SPU, P, 1, K, LB), RFI_TMA(DT, SPU, P, 2, K, LB),                           \
        RFI_TMA(DT, SPU, P, 4, K, LB), RFI_TMA(DT, SPU, P, 5, K, LB)
// lanes per row 1-8; Kahan with the 128-register budget, budgets 80 and 64 without
#define RFI_TMA_PB(DT, SPU, P)                                                              \
    RFI_TMA_CH(DT, SPU, P, 0, 0), RFI_TMA_CH(DT, SPU, P, 1, 0), RFI_TMA_CH(DT, SPU, P, 0, 1), \
        RFI_TMA_CH(DT, SPU, P, 0, 2)

#define RFI_SW(DT, SPU, P, CH, L)                                                           \
    {DT, SPU, P, CH, L, (const void *)&rfi::k_slide<DT, SPU, P, CH, L>,                     \
     (const void *)&rfi::k_batch_sw<DT, SPU, P, CH, L>}
// Chunks of 1, 2 or 4 units (5 would spill with the two pending-segment rings).
#define RFI_SW_CH(DT, SPU, P, L)                                                            \
    RFI_SW(DT, SPU, P, 1, L), RFI_SW(DT, SPU, P, 2, L), RFI_SW(DT, SPU, P, 4, L)

#define RFI_WP(DT, SPU, P, CH)                                                              \
    {DT, SPU, P, CH, 0, 0, 0, (const void *)&rfi::k_wpar<DT, SPU, P, CH>,                   \
     (const void *)&rfi::k_batch_wp<DT, SPU, P, CH>}
#define RFI_WPM(DT, SPU, P, CH)                                                             \
    {DT, SPU, P, CH, 1, 0, 0, (const void *)&rfi::k_wpar<DT, SPU, P, CH, true>,             \
     (const void *)&rfi::k_batch_wp<DT, SPU, P, CH, true>}
#define RFI_WP_CH(DT, SPU, P)                                                               \
    RFI_WP(DT, SPU, P, 1), RFI_WP(DT, SPU, P, 2), RFI_WP(DT, SPU, P, 4), RFI_WP(DT, SPU, P, 5)
// straddling windows (P M <= 32; 2 or 4 lanes per row, the footprints' splits)
#define RFI_WPS(DT, SPU, P, CH, PREC)                                                       \
    {DT, SPU, P, CH, PREC, 1, 0, (const void *)&rfi::k_wpar<DT, SPU, P, CH, PREC, true>,    \
     (const void *)&rfi::k_batch_wp<DT, SPU, P, CH, PREC, true>}
#define RFI_WPS_CH(DT, SPU, PREC)                                                           \
    RFI_WPS(DT, SPU, 2, 1, PREC), RFI_WPS(DT, SPU, 2, 2, PREC), RFI_WPS(DT, SPU, 2, 4, PREC), \
        RFI_WPS(DT, SPU, 2, 5, PREC), RFI_WPS(DT, SPU, 4, 1, PREC),                         \
        RFI_WPS(DT, SPU, 4, 2, PREC), RFI_WPS(DT, SPU, 4, 4, PREC), RFI_WPS(DT, SPU, 4, 5, PREC)
// the 96-register budget for binary16 odd windows (one sample per 16-byte unit) with
// the whole-round flag path, 2 lanes per row; batches run the 128-register kernel
#define RFI_WPS3(DT, P, CH, PREC)                                                           \
    {DT, 1, P, CH, PREC, 1, 3, (const void *)&rfi::k_wpar<DT, 1, P, CH, PREC, true, 3>,     \
     (const void *)&rfi::k_batch_wp<DT, 1, P, CH, PREC, true>}
#define RFI_WPS3_CH(DT, PREC)                                                               \
    RFI_WPS3(DT, 2, 1, PREC), RFI_WPS3(DT, 2, 2, PREC), RFI_WPS3(DT, 2, 4, PREC),            \
        RFI_WPS3(DT, 2, 5, PREC)
// the same for launches whose rounds are all whole (no per-window flag path compiled in)
#define RFI_WPW3(DT, P, CH, PREC)                                                           \
    {DT, 1, P, CH, PREC, 2, 3, (const void *)&rfi::k_wpar<DT, 1, P, CH, PREC, 2, 3>,        \
     (const void *)&rfi::k_batch_wp<DT, 1, P, CH, PREC, 1>}
// whole rounds only, the 128-register budget (binary16 M = 8 with 4 lanes, complex64
// 5 x 4 footprints with 2 or 4 lanes)
#define RFI_WPW(DT, SPU, P, CH, PREC)                                                       \
    {DT, SPU, P, CH, PREC, 2, 0, (const void *)&rfi::k_wpar<DT, SPU, P, CH, PREC, 2, 0>,    \
     (const void *)&rfi::k_batch_wp<DT, SPU, P, CH, PREC, 1>}
#define RFI_WPW3_CH(DT, PREC)                                                               \
    RFI_WPW3(DT, 2, 1, PREC), RFI_WPW3(DT, 2, 2, PREC), RFI_WPW3(DT, 2, 4, PREC),            \
        RFI_WPW3(DT, 2, 5, PREC)
#define RFI_WPM_CH(DT, SPU, P)                                                              \
    RFI_WPM(DT, SPU, P, 1), RFI_WPM(DT, SPU, P, 2), RFI_WPM(DT, SPU, P, 4),                  \
        RFI_WPM(DT, SPU, P, 5)

// Binary16 Stokes arithmetic (precision = 2; binary16 input), 128-register budget,
// without the prefetch code; a batch of such contexts runs its own batch kernel.
#define RFI_INSTH(DT, SPU, P, CH, K)                                                        \
    {DT, SPU, P, CH, K, 0, 2, 0, 0, 0, 0,                                                   \
     (const void *)&rfi::k_block<DT, SPU, P, CH, (bool)K, 0, 2>,                            \
     (const void *)&rfi::k_batch<DT, SPU, P, CH, (bool)K, 2, false, false, true>}
#define RFI_INSTH_CH(DT, SPU, P, K)                                                         \
    RFI_INSTH(DT, SPU, P, 1, K), RFI_INSTH(DT, SPU, P, 2, K), RFI_INSTH(DT, SPU, P, 4, K),  \
        RFI_INSTH(DT, SPU, P, 5, K)
#define RFI_WPH(DT, SPU, P, CH)                                                             \
    {DT, SPU, P, CH, 2, 0, 0, (const void *)&rfi::k_wpar<DT, SPU, P, CH, 2>,                \
     (const void *)&rfi::k_batch_wp<DT, SPU, P, CH, 2>}
#define RFI_WPH_CH(DT, SPU, P)                                                              \
    RFI_WPH(DT, SPU, P, 1), RFI_WPH(DT, SPU, P, 2), RFI_WPH(DT, SPU, P, 4),                  \
        RFI_WPH(DT, SPU, P, 5)

// The 96-register budget (LB = 3: 128-thread blocks, 5 per SM), two chunks of 1 or 2
// load units in flight per lane; float32 arithmetic with the prefetch code (like the
// other budgets), binary16 arithmetic without; plain batch kernels.
#define RFI_INST3(DT, SPU, P, CH)                                                           \
    {DT, SPU, P, CH, 0, 3, 0, 0, 0, 0, 1,                                                   \
     (const void *)&rfi::k_block<DT, SPU, P, CH, false, 3, 0, false, false, false, true>,  \
     (const void *)&rfi::k_batch<DT, SPU, P, CH, false, 0, false, false, true>}
#define RFI_INST3H(DT, SPU, P, CH)                                                          \
    {DT, SPU, P, CH, 0, 3, 2, 0, 0, 0, 0,                                                   \
     (const void *)&rfi::k_block<DT, SPU, P, CH, false, 3, 2>,                              \
     (const void *)&rfi::k_batch<DT, SPU, P, CH, false, 2, false, false, true>}
#define RFI_INST3_P(DT, SPU)                                                                \
    RFI_INST3(DT, SPU, 1, 1), RFI_INST3(DT, SPU, 1, 2), RFI_INST3(DT, SPU, 2, 1),           \
        RFI_INST3(DT, SPU, 2, 2), RFI_INST3(DT, SPU, 4, 1), RFI_INST3(DT, SPU, 4, 2),       \
        RFI_INST3(DT, SPU, 8, 1), RFI_INST3(DT, SPU, 8, 2)
#define RFI_INST3H_P(DT, SPU)                                                               \
    RFI_INST3H(DT, SPU, 1, 1), RFI_INST3H(DT, SPU, 1, 2), RFI_INST3H(DT, SPU, 2, 1),        \
        RFI_INST3H(DT, SPU, 2, 2), RFI_INST3H(DT, SPU, 4, 1), RFI_INST3H(DT, SPU, 4, 2),    \
        RFI_INST3H(DT, SPU, 8, 1), RFI_INST3H(DT, SPU, 8, 2)
