// rfi_api.cu -- C ABI of the online RFI flagging library (declared in include/rfi.h).
//
// Host responsibilities: argument and pointer validation (every device buffer is
// checked to be device memory of the context's GPU, aligned, and large enough for
// what the kernel will touch, before any launch), per-context state (thresholds,
// sample count, carry), launch-shape choice, the host-buffer pipeline and the
// persistent batch launch, optionally replayed from a CUDA graph.
#include "rfi.h"
#include "rfi_device.cuh"
#include "rfi_internal.h"
#include "rfi_kernels.h"
#include "rfi_sliding.cuh"
#include "rfi_wpar.cuh"

#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <set>
#include <vector>

using namespace rfi;

namespace {

thread_local char g_last_error[512] = "";

int fail(int status, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return status;
}

// ---- kernel instances (rfi_inst_f32.cu, rfi_inst_f16.cu) ----------------------
const Instance *find_instance(int dt, int spu, int P, int ch, int kahan, int lb, int mixed,
                              int vs, int pw, int ad, int pf) {
    const InstanceTable tabs[] = {instances_f32(),    instances_f16(),    instances_f32_pw(),
                                  instances_f16_pw(), instances_f32_ad(), instances_f16_ad(),
                                  instances_f32_pf(), instances_f16_pf(), instances_f16_h2()};
    for (const InstanceTable &t : tabs)
        for (int i = 0; i < t.n; ++i) {
            const Instance &in = t.items[i];
            if (in.dt == dt && in.spu == spu && in.P == P && in.ch == ch && in.kahan == kahan &&
                in.lb == lb && in.mixed == mixed && in.vs == vs && in.pw == pw && in.ad == ad &&
                in.pf == pf)
                return &in;
        }
    return nullptr;
}

const void *find_tma(int dt, int spu, int P, int ch, int kahan, int lb, int tile) {
    const TmaTable tabs[] = {tma_instances_f32(), tma_instances_f16()};
    for (const TmaTable &t : tabs)
        for (int i = 0; i < t.n; ++i) {
            const TmaInstance &in = t.items[i];
            if (in.dt == dt && in.spu == spu && in.P == P && in.ch == ch && in.kahan == kahan &&
                in.lb == lb)
                return tile ? in.fn2 : in.fn;
        }
    return nullptr;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link).
typedef CUresult (*PFN_encode)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                               const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                               const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                               CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
PFN_encode get_encode_fn() {
    static PFN_encode fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_encode>(p);
    });
    return fn;
}

const SwInstance *find_sw(int dt, int spu, int P, int ch, int L) {
    const SwTable tabs[] = {sw_instances_f32(), sw_instances_f16()};
    for (const SwTable &t : tabs)
        for (int i = 0; i < t.n; ++i) {
            const SwInstance &in = t.items[i];
            if (in.dt == dt && in.spu == spu && in.P == P && in.ch == ch && in.L == L)
                return &in;
        }
    return nullptr;
}

const WpInstance *find_wp(int dt, int spu, int P, int ch, int mixed, int fs, int lb) {
    const WpTable tabs[] = {wp_instances_f32(), wp_instances_f16(), wp_instances_f16_h2()};
    for (const WpTable &t : tabs)
        for (int i = 0; i < t.n; ++i) {
            const WpInstance &in = t.items[i];
            if (in.dt == dt && in.spu == spu && in.P == P && in.ch == ch && in.mixed == mixed &&
                in.fs == fs && in.lb == lb)
                return &in;
        }
    return nullptr;
}

int largest_chunk(int S) {
    static const int opts[] = {5, 4, 2, 1};
    for (int c : opts)
        if (S % c == 0) return c;
    return 1;
}

constexpr unsigned int CTX_MAGIC = 0x52464931u;  // "RFI1"
std::mutex g_live_mu;
std::set<const void *> g_live;                     // live contexts and graphs

bool is_live(const void *p) {
    std::lock_guard<std::mutex> lk(g_live_mu);
    return g_live.count(p) != 0;
}

// cuMemGetAddressRange through the runtime's driver entry point (no libcuda link).
typedef CUresult (*PFN_range)(CUdeviceptr *, size_t *, CUdeviceptr);
PFN_range get_range_fn() {
    static PFN_range fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_range>(p);
    });
    return fn;
}

}  // namespace

struct rfi_ctx {
    unsigned int magic;
    int device;
    int stations, channels, M, K;
    long long B, C, R;
    rfi_dtype dtype;
    rfi_thresholds thr;
    int P, spu, S, ch, kahan, wpb, lb;
    int wpb_auto;                       // warps_per_block was left to the library
    int F;                              // channels per window footprint
    int mixed;                          // 1: the paper's trained mixed precision
    int prec;                           // precision option: 0, 1 (mixed) or 2 (binary16
                                        // Stokes arithmetic)
    int loader;                         // 0: direct loads, 1: TMA staging in shared memory
                                        // (bulk copy per row), 2: the same with one tensor
                                        // tile per warp
    const void *tma_fn;
    int tma_G, tma_NS;                  // windows per stage, stages per warp
    unsigned tma_pitch;
    size_t tma_smem;                    // dynamic shared memory per block
    int inject;                         // fault injection: stage waits cannot complete
    int vs;                             // buffered 16-byte statistic and flag stores
    int pw;                             // partial windows: any T, open window carried
    char *hw;                           // [R][M] raw samples of each row's open window
    int ad;                             // online per-stream SK thresholds
    float *adapt;                       // [R/F][4]: n, mean, second moment of tau, unused
    rfi_adaptation adp;
    int pf_bytes, pf_groups;            // L2 prefetch group size and distance
    int ovl;                            // launch overlap: bytes per row requested early
    int indep;                          // independent_launches: a launch that shares no
                                        // buffer with the flagging launches that may still
                                        // run on the stream does not wait for them
    int last_launch;                    // how the last flagging launch was ordered (-1 none,
                                        // 0 plain, 1 waiting, 2 independent)
    int sw, H;                          // overlapping windows: a window every H samples
    const void *sw_fn;                  // k_slide<...>
    float *sw_buf;                      // [R][1][8] totals, [R][P][1][8] averaging sums of
                                        // the pending segment, [R] window flag history
    int wp;                             // window-parallel lanes (lane_split = 1)
    const void *wp_fn;                  // k_wpar<...>
    const void *wp_fn_whole;            // the same without the partial-round flag path (for
                                        // launches whose rounds are all whole), or null
    const Instance *inst;
    const void *batch_fn;               // persistent kernel of rfi_process_batch
    long long n_seen;
    int status;
    float *carry;                       // [R][P][9]
    unsigned long long *counter;        // [0] batch task counter, [1] blocks done,
                                        // [2] low word: device error word
    // host-buffer path
    int host_max_T, host_chunks;
    char *h_vis;
    uint32_t *h_flags;
    float *h_avg, *h_weight, *h_stats;
    cudaStream_t s_in, s_run, s_out;
    cudaEvent_t ev_start, ev_done;
    std::vector<cudaEvent_t> ev_in, ev_run;
};

struct rfi_batch_graph {
    int n;
    std::vector<rfi_ctx *> ctxs;
    std::vector<int> T;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    cudaGraphNode_t node;
    cudaGraphNode_t adapt_node;         // state update of adaptive contexts, or null
    const void *batch_fn;
    int grid, block;
};

namespace {

int sample_bytes(rfi_dtype dt) { return dt == RFI_C64 ? 32 : 16; }

// An NVTX range over one entry point (visible in Nsight timelines; a no-op without a
// tool attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
size_t adapt_bytes(const rfi_ctx *c) { return sizeof(float) * 4 * (size_t)(c->R / c->F); }

int check_ctx(const rfi_ctx *ctx) {
    if (!ctx) return fail(RFI_EINVAL, "null context");
    if (!is_live(ctx) || ctx->magic != CTX_MAGIC)
        return fail(RFI_ESTATE, "context was destroyed or is not a context");
    if (ctx->status != RFI_OK)
        return fail(RFI_ESTATE, "context is sticky-failed (%s); call rfi_reset",
                    rfi_status_str(ctx->status));
    return RFI_OK;
}

// A device buffer must be device (or managed) memory of `device`, aligned to
// `align`, and [p, p + bytes) must lie inside one allocation.
int check_dev(const void *p, size_t bytes, size_t align, int device, const char *what) {
    if (bytes == 0) return RFI_OK;
    if (!p) return fail(RFI_EINVAL, "%s: null pointer", what);
    if (reinterpret_cast<uintptr_t>(p) % align)
        return fail(RFI_EINVAL, "%s: pointer not %zu-byte aligned", what, align);
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(RFI_EINVAL, "%s: not a CUDA pointer (%s)", what, cudaGetErrorString(e));
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
        return fail(RFI_EINVAL, "%s: not device memory", what);
    if (at.type == cudaMemoryTypeDevice && at.device != device)
        return fail(RFI_EINVAL, "%s: memory of device %d, context on device %d", what,
                    at.device, device);
    PFN_range range = get_range_fn();
    if (range) {
        CUdeviceptr base = 0;
        size_t size = 0;
        if (range(&base, &size, reinterpret_cast<CUdeviceptr>(p)) == CUDA_SUCCESS) {
            const uintptr_t end = static_cast<uintptr_t>(base) + size;
            if (reinterpret_cast<uintptr_t>(p) + bytes > end)
                return fail(RFI_EINVAL, "%s: buffer holds %zu bytes from this pointer, need %zu",
                            what, (size_t)(end - reinterpret_cast<uintptr_t>(p)), bytes);
        }
    }
    return RFI_OK;
}

int check_thresholds(const rfi_thresholds *t) {
    if (!t) return fail(RFI_EINVAL, "null thresholds");
    if (std::isnan(t->d) || std::isnan(t->s_low) || std::isnan(t->s_high) ||
        std::isnan(t->gamma) || std::isnan(t->eps))
        return fail(RFI_EINVAL, "thresholds must not be NaN");
    if (!std::isfinite(t->d) || !std::isfinite(t->eps) || t->eps < 0)
        return fail(RFI_EINVAL, "d must be finite and eps finite and >= 0");
    if (t->s_low > t->s_high) return fail(RFI_EINVAL, "s_low > s_high");
    return RFI_OK;
}

int choose_shape(rfi_ctx *c, int P_req) {
    const int dt = c->dtype == RFI_C64 ? DT_F32 : DT_F16;
    // samples per 32-byte load unit: binary16 packs two samples when M is even
    if (c->wp) {
        // window-parallel lanes: each lane loads whole windows, so P need not divide M
        const int spu_w = (dt == DT_F16 && c->M % 2 == 0) ? 2 : 1;
        const int P = P_req ? P_req : 2;
        if (P != 2 && P != 4 && P != 8)
            return fail(RFI_EINVAL, "lane_split = 1 needs lanes_per_row 2, 4 or 8");
        if (P * c->F > 32)
            return fail(RFI_EINVAL, "lanes_per_row (%d) x window_F (%d) must not exceed 32", P,
                        c->F);
        if (c->K / c->M < P)
            return fail(RFI_EINVAL, "lane_split = 1 needs at least lanes_per_row = %d windows "
                                    "per averaging bin (K/M = %d)", P, c->K / c->M);
        c->P = P;
        c->spu = spu_w;
        c->S = c->M / spu_w;                   // load units per window, all in one lane
        c->ch = largest_chunk(c->S);
        if (c->mixed && c->F != 1)
            return fail(RFI_EINVAL, "precision = 1 supports time-only windows");
        // a round's P windows within 32 flag bits: the instances with the whole-round
        // flag path (measured 3-5 % faster for windows that straddle flag words, 2 % for
        // binary16 M = 8 with 4 lanes, where a round fills one word; the same bits)
        const bool whole_round = P * c->M <= 32;
        const WpInstance *wi =
            whole_round && c->prec != 1 ? find_wp(dt, spu_w, P, c->ch, c->prec, 1, c->lb)
                                        : nullptr;
        if (!wi) wi = find_wp(dt, spu_w, P, c->ch, c->prec, 0, c->lb);
        c->inst = nullptr;
        if (!wi && c->lb != 0)
            return fail(RFI_EUNSUPPORTED, "lane_split = 1 with max_registers = 96 is built for "
                                          "binary16 odd windows that straddle flag words, 2 "
                                          "lanes per row");
        if (!wi) return fail(RFI_EUNSUPPORTED, "no window-parallel kernel for this shape");
        c->wp_fn = wi->fn;
        c->batch_fn = wi->batch_fn;
        const WpInstance *ww =
            wi->fs == 1 ? find_wp(dt, spu_w, P, c->ch, c->prec, 2, c->lb) : nullptr;
        c->wp_fn_whole = ww ? ww->fn : nullptr;
        return RFI_OK;
    }
    // the run of samples the lanes of a row split: a window, or a hop of overlapping ones
    const int U = c->sw ? c->H : c->M;
    int spu = (dt == DT_F16 && U % 2 == 0) ? 2 : 1;
    int P = P_req;
    if (c->mixed) {
        // sums run sample after sample in one lane, as the tables order them
        if (P != 0 && P != 1) return fail(RFI_EINVAL, "precision = 1 needs lanes_per_row = 1");
        if (c->F != 1) return fail(RFI_EINVAL, "precision = 1 supports time-only windows");
        P = 1;
    }
    if (P == 0) {
        P = 2;
        while (P > 1 && (U % (P * spu)) != 0) P >>= 1;
    }
    if (P * c->F > 32)
        return fail(RFI_EINVAL, "lanes_per_row (%d) x window_F (%d) must not exceed 32", P, c->F);
    if (P != 1 && P != 2 && P != 4 && P != 8 && P != 16 && P != 32)
        return fail(RFI_EINVAL, "lanes_per_row must be a power of two <= 32");
    if (U % (P * spu) != 0) {
        if (dt == DT_F16 && spu == 2 && P_req != 0) {
            return fail(RFI_EINVAL, "%s %d is not a multiple of 2*lanes_per_row=%d",
                        c->sw ? "hop H" : "window M", U, 2 * P);
        }
        return fail(RFI_EINVAL, "%s %d is not a multiple of lanes_per_row=%d",
                    c->sw ? "hop H" : "window M", U, P);
    }
    if (dt == DT_F16 && spu == 1 && P != 1)
        return fail(RFI_EINVAL, "odd windows of binary16 input need lanes_per_row = 1");
    c->P = P;
    c->spu = spu;
    c->S = U / (P * spu);
    c->ch = largest_chunk(c->S);
    if (c->lb == 3) c->ch = c->S % 2 == 0 ? 2 : 1;   // two chunks of <= 2 units in 96 registers
    if (c->sw) {
        // overlapping windows: their own kernels, single-stream calls only
        c->ch = c->S % 4 == 0 ? 4 : (c->S % 2 == 0 ? 2 : 1);
        const SwInstance *si = find_sw(dt, spu, P, c->ch, c->M / c->H);
        c->inst = nullptr;
        if (!si)
            return fail(RFI_EUNSUPPORTED, "no overlapping-window kernel for lanes_per_row=%d "
                                          "(1, 2 or 4)", P);
        c->sw_fn = si->fn;
        c->batch_fn = si->batch_fn;
        return RFI_OK;
    }
    // the plain 128-register kernels exist with and without the prefetch code; the
    // other kinds always hold it
    const bool plain = c->lb == 0 && !c->prec && !c->vs && !c->pw && !c->ad;
    // the binary16 Stokes kernels are built without the prefetch code
    const int pf = plain ? (c->pf_groups > 0 ? 1 : 0) : (c->prec == 2 ? 0 : 1);
    c->inst = find_instance(dt, spu, P, c->ch, c->kahan, c->lb, c->prec, c->vs, c->pw, c->ad,
                            pf);
    if (c->inst) {
        c->batch_fn = c->inst->batch_fn;
        if (!c->batch_fn) {     // kernels with prefetch batch with the plain batch kernel
            const Instance *plain0 =
                find_instance(dt, spu, P, c->ch, c->kahan, 0, 0, 0, 0, 0, 0);
            c->batch_fn = plain0 ? plain0->batch_fn : nullptr;
        }
    }
    if (c->ad && (!c->inst || c->loader != 0))
        return fail(RFI_EUNSUPPORTED, "adaptive needs the direct loader, the 128-register "
                                      "budget and float32 arithmetic, without buffered_stores "
                                      "or partial_windows");
    if (c->pw && !c->inst)
        return fail(RFI_EUNSUPPORTED, "partial_windows needs the 128-register budget and "
                                      "float32 arithmetic, without buffered_stores");
    if (c->vs && (!c->inst || c->loader != 0))
        return fail(RFI_EUNSUPPORTED, "buffered_stores needs the direct loader, float32 "
                                      "arithmetic, the 128-register budget, no Kahan, "
                                      "lanes_per_row <= 4 and 1, 2 or 4 load units per chunk");
    if (c->loader == 1 || c->loader == 2) {
        c->tma_fn =
            c->prec ? nullptr : find_tma(dt, spu, P, c->ch, c->kahan, c->lb, c->loader == 2);
        if (!c->tma_fn)
            return fail(RFI_EUNSUPPORTED, "no shared-memory loader for this shape (float32 "
                                          "arithmetic, lanes_per_row <= 8, Kahan only with "
                                          "the 128-register budget and the row copies)");
        if (c->loader == 2 && !get_encode_fn())
            return fail(RFI_EUNSUPPORTED, "loader = 2 needs cuTensorMapEncodeTiled");
        // a tile copy's shared-memory destination (stage * rows * pitch, the pitch 16
        // mod 128 bytes) is 128-byte aligned only for a multiple of 8 rows per warp
        if (c->loader == 2 && (32 / P) % 8 != 0)
            return fail(RFI_EUNSUPPORTED, "loader = 2 needs lanes_per_row <= 4");
        const unsigned SR = (unsigned)(c->tma_G * c->M * (dt == DT_F32 ? 32 : 16));
        // row pitch = 16 mod 128 bytes: consecutive rows start 4 banks apart, so the
        // lanes' 16-byte shared-memory reads spread over all banks
        c->tma_pitch = ((SR + 111u) / 128u) * 128u + 16u;
        auto smem_for = [&](int wpb) {
            const size_t bars = (8u * c->tma_NS * wpb + 127u) & ~(size_t)127u;
            return bars + (size_t)wpb * c->tma_NS * (32 / P) * c->tma_pitch;
        };
        if (c->wpb_auto)      // the largest block that fits the shared memory
            while (c->wpb > 1 && smem_for(c->wpb) > 227 * 1024) c->wpb >>= 1;
        c->tma_smem = smem_for(c->wpb);
        if (c->loader == 2 && c->tma_pitch / 8 > 256)
            return fail(RFI_EINVAL, "loader = 2 copies at most 2048 bytes of a row per stage "
                                    "(%u): fewer windows per stage", c->tma_pitch);
        if (c->tma_smem > 227 * 1024)
            return fail(RFI_EINVAL, "shared-memory staging needs %zu bytes per block (max "
                                    "232448): fewer warps, stages or windows per stage",
                        c->tma_smem);
    }
    if (!c->inst)
        return fail(RFI_EUNSUPPORTED,
                    "no kernel for this launch shape (reduced register budgets exist for "
                    "lanes_per_row <= 8, 2-5 load units per chunk, no Kahan summation)");
    return RFI_OK;
}

// Samples of the open window carried into the next block, and the windows (hence
// statistics columns and M nwin flag bits) a block of T samples completes.
int phase_of(const rfi_ctx *c) { return c->pw ? (int)(c->n_seen % c->M) : 0; }
// Overlapping windows: windows complete once n samples of the stream have arrived.
long long sw_evaluated(const rfi_ctx *c, long long n) {
    return n >= c->M ? (n - c->M) / c->H + 1 : 0;
}
int windows_for(const rfi_ctx *c, int T) {
    if (c->sw) return (int)(sw_evaluated(c, c->n_seen + T) - sw_evaluated(c, c->n_seen));
    return (phase_of(c) + T) / c->M;
}
// Flag bits a completed window adds to a call's output (its samples that became final).
int bits_per_window(const rfi_ctx *c) { return c->sw ? c->H : c->M; }
// Stream index of the first sample whose flag the next call reports.
long long first_final(const rfi_ctx *c) {
    return c->sw ? sw_evaluated(c, c->n_seen) * c->H : c->n_seen - phase_of(c);
}
// Averaging bins the next call of T samples closes (bins close with final samples).
long long outputs_for_c(const rfi_ctx *c, int T) {
    if (c->sw) {
        const long long f0 = first_final(c);
        const long long f1 = sw_evaluated(c, c->n_seen + T) * c->H;
        return f1 / c->K - f0 / c->K;
    }
    return (c->n_seen + T) / c->K - c->n_seen / c->K;
}

// Overlapping-window state: the pending hop's totals [R][8] and the lanes' averaging
// sums [R][P][8], then the last window's flag [R].
size_t sw_tot_floats(const rfi_ctx *c) { return (size_t)c->R * 8; }
size_t sw_pend_floats(const rfi_ctx *c) { return (size_t)c->R * c->P * 8; }
size_t sw_bytes(const rfi_ctx *c) {
    return c->sw ? sizeof(float) * (sw_tot_floats(c) + sw_pend_floats(c)) + 4 * (size_t)c->R : 0;
}

StreamArgs make_args(const rfi_ctx *c, const void *vis, int T, uint32_t *flags, float *avg,
                     float *weight, float *stats, long long r0, long long nrows) {
    StreamArgs a = {};
    const int nwin = windows_for(c, T);
    const int Wpr = (nwin * bits_per_window(c) + 31) / 32;
    const long long n_out = outputs_for_c(c, T);
    a.vis = static_cast<const char *>(vis) + r0 * (long long)T * sample_bytes(c->dtype);
    a.flags = flags + r0 * Wpr;
    a.avg = avg ? avg + r0 * n_out * 8 : nullptr;
    a.weight = weight ? weight + r0 * n_out : nullptr;
    a.stats = stats + (r0 / c->F) * nwin;     // r0 is a multiple of F
    a.carry = c->carry + r0 * c->P * 9;
    a.hw = c->hw ? c->hw + r0 * c->M * sample_bytes(c->dtype) : nullptr;
    a.adapt = c->adapt ? c->adapt + (r0 / c->F) * 4 : nullptr;
    a.alpha = (float)c->adp.alpha;
    a.k_sigma = (float)c->adp.k_sigma;
    a.n_warm = (float)c->adp.n_warm;
    a.ovl_bytes = c->ovl;
    a.wphase = c->wp ? (int)((c->n_seen / c->M) % c->P) : 0;
    a.hop = c->H;
    if (c->sw) {
        a.warm = (int)std::min<long long>(c->n_seen / c->H, c->M / c->H - 1);
        a.sw_tot = c->sw_buf + r0 * 8;
        a.sw_pend = c->sw_buf + sw_tot_floats(c) + r0 * c->P * 8;
        a.sw_hist =
            reinterpret_cast<uint32_t *>(c->sw_buf + sw_tot_floats(c) + sw_pend_floats(c)) + r0;
    }
    a.phase = phase_of(c);
    a.R = nrows;
    a.stats_plane = (c->R / c->F) * nwin;
    a.F = c->F;
    a.d = (float)c->thr.d;
    a.stage_windows = c->tma_G;
    a.stages = c->tma_NS;
    a.pitch = c->tma_pitch;
    a.tx_extra = c->inject ? 16u : 0u;
    a.wait_limit = c->inject ? 2000000ll : 4000000000ll;   // ~1 ms / ~2 s at 2 GHz
    a.err = reinterpret_cast<int *>(c->counter + 2);
    a.T = T;
    a.M = c->M;
    a.K = c->K;
    a.Wpr = Wpr;
    a.nwin = nwin;
    a.n_out = (int)n_out;
    // samples of the open bin before window 0 (which may itself start in an earlier block;
    // with overlapping windows: final samples of the open bin)
    a.bin_pos0 = (int)(first_final(c) % c->K);
    const double Md = (double)c->M * c->F;     // W = M F samples per window
    a.c0 = (float)((Md * c->thr.d + 1.0) / (Md - 1.0));
    a.s_low = (float)c->thr.s_low;
    a.s_high = (float)c->thr.s_high;
    a.gamma = (float)c->thr.gamma;
    a.eps = (float)c->thr.eps;
    a.fM = (float)Md;
    a.fK = (float)c->K;
    a.invM = (float)(1.0 / Md);
    const int wbytes = c->M * sample_bytes(c->dtype);
    a.pf_windows = std::max(1, c->pf_bytes / wbytes);
    a.pf_groups = c->pf_groups;
    return a;
}

int check_T(const rfi_ctx *c, int T) {
    if (c->sw) {
        if (T <= 0 || T % c->H != 0)
            return fail(RFI_EINVAL, "T=%d must be a positive multiple of the hop H=%d", T, c->H);
        return RFI_OK;
    }
    if (c->pw) {
        if (T <= 0) return fail(RFI_EINVAL, "T=%d must be positive", T);
        if (T % c->spu != 0)
            return fail(RFI_EINVAL, "T=%d must be even (binary16 samples are loaded in pairs)", T);
        return RFI_OK;
    }
    if (T <= 0 || T % c->M != 0)
        return fail(RFI_EINVAL, "T=%d must be a positive multiple of M=%d (or create the "
                                "context with partial_windows = 1)", T, c->M);
    return RFI_OK;
}

int check_block_args(const rfi_ctx *c, const void *vis, int T, const uint32_t *flags,
                     const float *avg, const float *weight, const float *stats, bool device) {
    int rc0;
    if ((rc0 = check_T(c, T))) return rc0;
    if ((long long)T * c->R > (1ll << 40)) return fail(RFI_EINVAL, "block too large");
    const long long n_out = outputs_for_c(c, T);
    const size_t sb = sample_bytes(c->dtype);
    const size_t vis_align = (size_t)sb * c->spu;
    const size_t R = (size_t)c->R;
    const size_t nw = windows_for(c, T), wpr = (nw * bits_per_window(c) + 31) / 32;
    if (!device) {
        if (!vis || (nw > 0 && (!flags || !stats)) || (n_out > 0 && (!avg || !weight)))
            return fail(RFI_EINVAL, "null host buffer");
        return RFI_OK;
    }
    int rc;
    if ((rc = check_dev(vis, R * T * sb, vis_align, c->device, "vis"))) return rc;
    if ((rc = check_dev(flags, R * wpr * 4, 4, c->device, "flags"))) return rc;
    if ((rc = check_dev(stats, 3 * (R / c->F) * nw * 4, 4, c->device, "stats"))) return rc;
    if (n_out > 0) {
        if ((rc = check_dev(avg, R * n_out * 32, 16, c->device, "avg"))) return rc;
        if ((rc = check_dev(weight, R * n_out * 4, 4, c->device, "weight"))) return rc;
    }
    return RFI_OK;
}

int set_cuda_error(rfi_ctx *c, cudaError_t e, const char *where) {
    c->status = RFI_ECUDA;
    return fail(RFI_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

// Allow a kernel the dynamic shared memory it asks for (once per kernel and size).
cudaError_t allow_smem(const void *fn, size_t bytes) {
    static std::mutex mu;
    static std::vector<std::pair<const void *, size_t>> done;
    std::lock_guard<std::mutex> lk(mu);
    for (auto &d : done)
        if (d.first == fn && d.second >= bytes) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bytes);
    if (e == cudaSuccess) done.push_back({fn, bytes});
    return e;
}

// Launches recorded into a graph keep plain stream order.
bool capturing(cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return true;            // when in doubt, the plain launch
    }
    return cs != cudaStreamCaptureStatusNone;
}

// ---- launch ordering of the flagging kernels -----------------------------------------
// k_block, k_wpar and k_slide execute griddepcontrol.launch_dependents on entry, so a
// launch made after one of them with the programmatic-serialisation attribute may start
// once all of its blocks have started, while it (and, by the same rule, launches before
// it) still runs.  Per (device, stream) the host keeps the byte ranges that the flagging
// launches since the last fully ordered one read and write ("in flight": those that may
// still run when the next launch starts) and orders every new flagging launch:
//   independent (2): it reads nothing that a launch in flight writes and writes nothing
//       that one reads or writes, and the context allows it (independent_launches):
//       launched with the attribute, its blocks start at once;
//   waiting (1): otherwise, if every launch in flight waited for the one before it (so
//       the completion of the last implies that of all): launched with the attribute,
//       its blocks wait for the kernel before it (griddepcontrol.wait) first;
//   plain (0): otherwise (or overlap off, or more than kMaxInFlight in flight): a plain
//       launch, after everything before it on the stream.
// Kernels that do not trigger early (the staged loaders, the batch and state-update
// kernels, and graphs of them) are launched plain; after them nothing is in flight.
// rfi_process_block_noalloc may not allocate, so it does not touch the lists: it counts
// its launches (an epoch, under the same lock as its launch), and a flagging launch that
// finds the count changed since its stream's list was last brought up to date treats
// the stream as holding a launch in flight with unknown buffers.
// Work that other code puts on the stream between two calls is either a plain stream
// operation (ordered after everything before it) or a kernel of the caller's; the
// independent order assumes that no kernel of the caller's that triggers early writes
// a block's input or reads its outputs between two calls (the option's contract).
struct Span {
    uintptr_t lo, hi;                   // [lo, hi)
};
struct Footprint {
    int nr = 0, nw = 0;
    Span r[6], w[10];
    void read(const void *p, size_t bytes) { add(r, nr, 6, p, bytes); }
    void write(const void *p, size_t bytes) { add(w, nw, 10, p, bytes); }
    static void add(Span *s, int &n, int cap, const void *p, size_t bytes) {
        if (!p || !bytes) return;
        const uintptr_t lo = reinterpret_cast<uintptr_t>(p);
        if (n < cap) s[n++] = Span{lo, lo + bytes};
        else s[cap - 1] = Span{0, ~uintptr_t(0)};   // cannot happen; stay conservative
    }
    static Footprint everything() {
        Footprint f;
        f.r[f.nr++] = Span{0, ~uintptr_t(0)};
        f.w[f.nw++] = Span{0, ~uintptr_t(0)};
        return f;
    }
};
bool spans_meet(const Span *a, int na, const Span *b, int nb) {
    for (int i = 0; i < na; ++i)
        for (int k = 0; k < nb; ++k)
            if (a[i].lo < b[k].hi && b[k].lo < a[i].hi) return true;
    return false;
}
// x must wait for y: x reads what y writes, or writes what y reads or writes
bool clashes(const Footprint &x, const Footprint &y) {
    return spans_meet(x.r, x.nr, y.w, y.nw) || spans_meet(x.w, x.nw, y.r, y.nr) ||
           spans_meet(x.w, x.nw, y.w, y.nw);
}
struct InFlight {
    std::vector<Footprint> fp;
    bool all_waited = true;
    unsigned long long noalloc_seen = 0;   // no-allocation launches accounted for
};
constexpr size_t kMaxInFlight = 32;
std::mutex g_order_mu;
std::map<std::pair<int, uintptr_t>, InFlight> g_order;
std::atomic<unsigned long long> g_noalloc_launches{0};

InFlight &in_flight(int device, cudaStream_t st) {
    return g_order[{device, reinterpret_cast<uintptr_t>(st)}];
}

// The buffers one flagging launch reads and writes (rows r0 .. r0 + a.R of the stream).
Footprint footprint_of(const rfi_ctx *c, const StreamArgs &a) {
    Footprint f;
    const size_t R = (size_t)a.R, SB = (size_t)sample_bytes(c->dtype);
    f.read(a.vis, R * (size_t)a.T * SB);
    const size_t carry_bytes = R * (size_t)c->P * 9 * sizeof(float);
    if (c->sw) {
        // overlapping windows: the bin carry and the pending hop's state, both ways
        f.read(a.carry, carry_bytes);
        f.write(a.carry, carry_bytes);
        f.read(a.sw_tot, R * 8 * sizeof(float));
        f.write(a.sw_tot, R * 8 * sizeof(float));
        f.read(a.sw_pend, R * (size_t)c->P * 8 * sizeof(float));
        f.write(a.sw_pend, R * (size_t)c->P * 8 * sizeof(float));
        f.read(a.sw_hist, R * sizeof(uint32_t));
        f.write(a.sw_hist, R * sizeof(uint32_t));
    } else {
        // the open bin is read when the block starts inside one and written when it
        // ends inside one
        if (a.bin_pos0 != 0) f.read(a.carry, carry_bytes);
        if ((a.bin_pos0 / a.M + a.nwin) % (a.K / a.M) != 0) f.write(a.carry, carry_bytes);
    }
    if (c->pw) {
        f.read(a.hw, R * (size_t)a.M * SB);
        f.write(a.hw, R * (size_t)a.M * SB);
    }
    const size_t G = R / (size_t)c->F;              // footprint rows of the launch
    if (c->ad) f.read(a.adapt, G * 4 * sizeof(float));
    f.write(a.flags, R * (size_t)a.Wpr * sizeof(uint32_t));
    for (int k = 0; k < 3; ++k)
        f.write(a.stats + k * a.stats_plane, G * (size_t)a.nwin * sizeof(float));
    if (a.n_out > 0) {
        f.write(a.avg, R * (size_t)a.n_out * 8 * sizeof(float));
        f.write(a.weight, R * (size_t)a.n_out * sizeof(float));
    }
    return f;
}

// A plain launch of a kernel that does not trigger its successor early, made under the
// ordering lock: once it runs nothing launched before it is still running, and the
// launch after it waits for its completion, so the stream's list is emptied (the
// no-allocation count is left alone: a launch of rfi_process_block_noalloc between the
// list's last update and this one stays accounted for).  No bookkeeping while the
// stream is captured.
template <class Launch>
cudaError_t launch_plain(int device, cudaStream_t st, Launch &&launch) {
    std::lock_guard<std::mutex> lock(g_order_mu);
    const cudaError_t e = launch();
    if (e == cudaSuccess && !capturing(st)) {
        InFlight &fl = in_flight(device, st);
        fl.fp.clear();
        fl.all_waited = true;
    }
    return e;
}

// Synchronise the current device under the ordering lock, then empty its streams'
// lists: every launch made so far has completed, and no flagging launch can be made
// between the synchronisation and the clearing.  For the entry points that synchronise
// anyway (destroy, reset, restoring a saved state).
cudaError_t sync_device_and_forget() {
    std::lock_guard<std::mutex> lock(g_order_mu);
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) {
        const unsigned long long na = g_noalloc_launches.load();
        for (auto &kv : g_order) {
            if (kv.first.first != device) continue;
            kv.second.fp.clear();
            kv.second.all_waited = true;
            kv.second.noalloc_seen = na;
        }
    }
    return e;
}

int launch_block(rfi_ctx *c, const StreamArgs &a, cudaStream_t st) {
    if (a.R <= 0) return RFI_OK;
    const int RW = 32 / c->P;
    const long long groups = (a.R + RW - 1) / RW;
    const long long blocks = (groups + c->wpb - 1) / c->wpb;
    void *args[] = {const_cast<StreamArgs *>(&a)};
    // window-parallel lanes: a launch whose first window is lane 0's and whose window
    // count is a multiple of the lanes has whole rounds only
    const bool whole = c->wp && c->wp_fn_whole && a.wphase == 0 && a.nwin % c->P == 0;
    const void *fn = c->sw ? c->sw_fn
                           : (c->wp ? (whole ? c->wp_fn_whole : c->wp_fn)
                                    : (c->inst ? c->inst->block_fn : nullptr));
    cudaError_t e;
    if (c->loader == 2) {
        // the launch's rows as a 2-D tensor of 8-byte elements; one tile = the pitch of
        // a stage row (its G windows and the rest of the pitch) x the warp's rows
        const size_t SB = sample_bytes(c->dtype);
        alignas(64) CUtensorMap tmap;
        const cuuint64_t dims[2] = {(cuuint64_t)a.T * SB / 8, (cuuint64_t)a.R};
        const cuuint64_t strides[1] = {(cuuint64_t)a.T * SB};
        const cuuint32_t box[2] = {c->tma_pitch / 8, (cuuint32_t)RW};
        const cuuint32_t estr[2] = {1, 1};
        const CUresult r = get_encode_fn()(
            &tmap, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void *>(a.vis), dims, strides,
            box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS)
            return fail(RFI_EINVAL, "tensor map for the block (error %d): rows of %lld bytes "
                                    "must be a multiple of 16",
                        (int)r, (long long)(a.T * SB));
        void *args2[] = {const_cast<StreamArgs *>(&a), &tmap};
        e = allow_smem(c->tma_fn, c->tma_smem);
        if (e == cudaSuccess)
            e = launch_plain(c->device, st, [&] {
                return cudaLaunchKernel(c->tma_fn, dim3((unsigned)blocks), dim3(32 * c->wpb),
                                        args2, c->tma_smem, st);
            });
        c->last_launch = 0;
    } else if (c->loader == 1) {
        e = allow_smem(c->tma_fn, c->tma_smem);
        if (e == cudaSuccess)
            e = launch_plain(c->device, st, [&] {
                return cudaLaunchKernel(c->tma_fn, dim3((unsigned)blocks), dim3(32 * c->wpb),
                                        args, c->tma_smem, st);
            });
        c->last_launch = 0;
    } else {
        // a kernel that triggers its successor early: ordered against the flagging
        // launches in flight on the stream (see above); the decision and the launch
        // happen under one lock, so the bookkeeping follows the stream's order
        const bool cap = capturing(st);
        const Footprint fp = footprint_of(c, a);
        std::lock_guard<std::mutex> lock(g_order_mu);
        InFlight &fl = in_flight(c->device, st);
        const unsigned long long na = g_noalloc_launches.load();
        if (!cap && fl.noalloc_seen != na) {
            // a no-allocation launch (on this stream or another) since the list's last
            // update: it may still run here, with unknown buffers
            fl.fp.push_back(Footprint::everything());
            fl.noalloc_seen = na;
        }
        int order = 0;
        if (!cap && c->ovl > 0 && fl.fp.size() < kMaxInFlight) {
            bool clash = false;
            for (const Footprint &x : fl.fp) clash = clash || clashes(fp, x);
            if (c->indep && !clash) order = 2;
            else if (fl.all_waited) order = 1;
        }
        StreamArgs b = a;
        b.indep = order == 2;
        void *bargs[] = {&b};
        if (order > 0) {
            // programmatic dependent launch: the blocks may start while the kernel before
            // this one on the stream drains
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)blocks);
            cfg.blockDim = dim3(32 * c->wpb);
            cfg.stream = st;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            at[0].val.programmaticStreamSerializationAllowed = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            e = cudaLaunchKernelExC(&cfg, fn, bargs);
        } else {
            e = cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(32 * c->wpb), bargs, 0, st);
        }
        if (e == cudaSuccess && !cap) {
            if (order == 0) {
                fl.fp.clear();
                fl.all_waited = true;
            }
            if (order == 2) fl.all_waited = false;
            fl.fp.push_back(fp);
        }
        c->last_launch = cap ? -1 : order;
    }
    if (e == cudaSuccess && c->ad && a.nwin > 0) {     // advance the online thresholds
        const long long G = a.R / c->F;
        e = launch_plain(c->device, st, [&] {
            return cudaLaunchKernel(adapt_fn(), dim3((unsigned)((G + 255) / 256)), dim3(256),
                                    args, 0, st);
        });
    }
    if (e != cudaSuccess) return set_cuda_error(c, e, "kernel launch");
    return RFI_OK;
}

// Blocks of the batched state update of adaptive contexts: a grid-stride loop.
int adapt_batch_grid(int device) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    return std::max(sms, 1) * 4;
}

// Resident blocks of a batch kernel on the whole GPU (cached per kernel, block size
// and device).
int persistent_grid(const void *batch_fn, int wpb, int device) {
    struct Entry { const void *fn; int wpb, device, grid; };
    static std::mutex mu;
    static std::vector<Entry> cache;
    std::lock_guard<std::mutex> lk(mu);
    for (const Entry &e : cache)
        if (e.fn == batch_fn && e.wpb == wpb && e.device == device) return e.grid;
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_fn, 32 * wpb, 0) !=
            cudaSuccess ||
        per < 1) {
        cudaGetLastError();
        per = 1;
    }
    cache.push_back({batch_fn, wpb, device, std::max(sms, 1) * per});
    return cache.back().grid;
}

int build_batch(rfi_ctx *const *ctxs, int n, const void *const *vis, const int *T,
                uint32_t *const *flags, float *const *avg, float *const *weight,
                float *const *stats, bool validate_buffers, BatchArgs *b) {
    if (n < 1 || n > MAX_BATCH) return fail(RFI_EINVAL, "batch size %d not in [1, %d]", n, MAX_BATCH);
    if (!ctxs || !T) return fail(RFI_EINVAL, "null batch arrays");
    int rc;
    for (int i = 0; i < n; ++i) {
        if ((rc = check_ctx(ctxs[i]))) return rc;
        for (int k = 0; k < i; ++k)
            if (ctxs[k] == ctxs[i]) return fail(RFI_EINVAL, "context %d appears twice", i);
        if (!ctxs[i]->batch_fn || ctxs[i]->batch_fn != ctxs[0]->batch_fn ||
            ctxs[i]->device != ctxs[0]->device)
            return fail(RFI_EINVAL, "context %d differs in dtype, M or launch shape", i);
    }
    b->n = n;
    b->counter = ctxs[0]->counter;
    long long tot = 0;
    for (int i = 0; i < n; ++i) {
        const rfi_ctx *c = ctxs[i];
        if (validate_buffers) {
            if (!vis || !flags || !avg || !weight || !stats)
                return fail(RFI_EINVAL, "null batch buffer arrays");
            if ((rc = check_block_args(c, vis[i], T[i], flags[i], avg[i], weight[i], stats[i],
                                       true)))
                return rc;
            b->s[i] = make_args(c, vis[i], T[i], flags[i], avg[i], weight[i], stats[i], 0, c->R);
        } else {
            if ((rc = check_T(c, T[i]))) return rc;
            b->s[i] = make_args(c, nullptr, T[i], nullptr, nullptr, nullptr, nullptr, 0, c->R);
        }
        b->prefix[i] = tot;
        tot += (c->R + 32 / c->P - 1) / (32 / c->P);
    }
    b->prefix[n] = tot;
    for (int i = n + 1; i <= MAX_BATCH; ++i) b->prefix[i] = tot;
    b->total = tot;
    return RFI_OK;
}

void free_ctx(rfi_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    // the frees below synchronise the device as well; done first, explicitly, so the
    // launch-ordering lists of the device can be emptied
    if (sync_device_and_forget() != cudaSuccess) cudaGetLastError();
    if (c->carry) cudaFree(c->carry);
    if (c->hw) cudaFree(c->hw);
    if (c->adapt) cudaFree(c->adapt);
    if (c->sw_buf) cudaFree(c->sw_buf);
    if (c->counter) cudaFree(c->counter);
    if (c->h_vis) cudaFree(c->h_vis);
    if (c->h_flags) cudaFree(c->h_flags);
    if (c->h_avg) cudaFree(c->h_avg);
    if (c->h_weight) cudaFree(c->h_weight);
    if (c->h_stats) cudaFree(c->h_stats);
    for (cudaEvent_t e : c->ev_in) cudaEventDestroy(e);
    for (cudaEvent_t e : c->ev_run) cudaEventDestroy(e);
    if (c->ev_start) cudaEventDestroy(c->ev_start);
    if (c->ev_done) cudaEventDestroy(c->ev_done);
    if (c->s_in) cudaStreamDestroy(c->s_in);
    if (c->s_run) cudaStreamDestroy(c->s_run);
    if (c->s_out) cudaStreamDestroy(c->s_out);
    c->magic = 0;
    delete c;
}

}  // namespace

int rfi_internal_fail(int status, const char *msg) { return fail(status, "%s", msg); }

void rfi_internal_noalloc_launch_begin() {
    g_order_mu.lock();
    g_noalloc_launches.fetch_add(1);
}

void rfi_internal_noalloc_launch_end() { g_order_mu.unlock(); }

int rfi_internal_check_dev(const void *p, size_t bytes, size_t align, int device,
                           const char *what) {
    return check_dev(p, bytes, align, device, what);
}

extern "C" {

const char *rfi_status_str(int s) {
    switch (s) {
        case RFI_OK: return "RFI_OK";
        case RFI_EINVAL: return "RFI_EINVAL: invalid argument";
        case RFI_ENOMEM: return "RFI_ENOMEM: allocation failed";
        case RFI_ECUDA: return "RFI_ECUDA: CUDA error";
        case RFI_ETIMEOUT: return "RFI_ETIMEOUT: bounded device wait expired";
        case RFI_ESTATE: return "RFI_ESTATE: context failed, destroyed or misused";
        case RFI_EUNSUPPORTED: return "RFI_EUNSUPPORTED: no kernel for this request";
        default: return "unknown rfi status";
    }
}

const char *rfi_last_error(void) { return g_last_error; }

int rfi_create_ex(rfi_ctx **out, int stations, int channels, int window_M, int avg_K,
                  const rfi_thresholds *thr, rfi_dtype dtype, const rfi_options *opt) {
    NvtxRange nvtx("rfi_create");
    if (!out) return fail(RFI_EINVAL, "null output handle");
    *out = nullptr;
    if (stations < 1 || channels < 1) return fail(RFI_EINVAL, "stations and channels must be >= 1");
    if (window_M < 1 || (window_M < 2 && !(opt && opt->window_F > 1)))
        return fail(RFI_EINVAL, "a window needs at least 2 samples (tau divides by W-1)");
    // overlapping windows: a window every H = window_hop samples (0 or M: no overlap)
    const int hop = (opt && opt->window_hop > 0) ? opt->window_hop : window_M;
    if (opt && opt->window_hop < 0) return fail(RFI_EINVAL, "window_hop must be >= 0");
    if (hop != window_M) {
        if (hop > window_M || window_M % hop != 0 || window_M / hop != 2)
            return fail(RFI_EUNSUPPORTED, "window_hop must be M/2 (two windows hold every "
                                          "sample), got %d for M=%d", hop, window_M);
        if (avg_K < hop || avg_K % hop != 0)
            return fail(RFI_EINVAL, "averaging factor K=%d must be a positive multiple of the "
                                    "hop H=%d", avg_K, hop);
    } else if (avg_K < window_M || avg_K % window_M != 0) {
        return fail(RFI_EINVAL, "averaging factor K=%d must be a positive multiple of M=%d", avg_K,
                    window_M);
    }
    if (dtype != RFI_C64 && dtype != RFI_C32H) return fail(RFI_EINVAL, "unknown dtype");
    int rc;
    if ((rc = check_thresholds(thr))) return rc;
    rfi_options o = {};
    if (opt) o = *opt;
    if (o.warps_per_block < 0 || o.warps_per_block > 16 || o.host_max_T < 0 || o.host_chunks < 0 ||
        o.compensated < -1 || o.compensated > 1 || o.prefetch_bytes < 0 ||
        o.prefetch_bytes % 16 != 0 || o.prefetch_groups > 64 ||
        (o.max_registers != 0 && o.max_registers < 64) || o.window_F < 0 || o.precision < 0 ||
        o.precision > 2 || o.loader < 0 || o.loader > 2 || o.tma_stage_windows < 0 ||
        o.tma_stage_windows > 64 || o.tma_stages < 0 || o.tma_stages > 8 ||
        o.debug_inject_wait_timeout < 0 || o.debug_inject_wait_timeout > 1 ||
        o.overlap_bytes < -1 || (o.overlap_bytes > 0 && o.overlap_bytes % 128 != 0) ||
        o.lane_split < 0 || o.lane_split > 1 || o.independent_launches < 0 ||
        o.independent_launches > 1)
        return fail(RFI_EINVAL, "bad options");

    rfi_ctx *c = new (std::nothrow) rfi_ctx();
    if (!c) return fail(RFI_ENOMEM, "host allocation failed");
    c->magic = CTX_MAGIC;
    cudaError_t de = cudaGetDevice(&c->device);
    if (de != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return fail(RFI_ECUDA, "no usable CUDA device: %s", cudaGetErrorString(de));
    }
    c->stations = stations;
    c->channels = channels;
    c->M = window_M;
    c->K = avg_K;
    c->B = (long long)stations * (stations + 1) / 2;
    c->C = channels;
    c->R = c->B * c->C;
    c->dtype = dtype;
    c->thr = *thr;
    c->kahan = o.compensated == 1 || (o.compensated == 0 && window_M >= 64);
    c->wpb = o.warps_per_block ? o.warps_per_block : 8;
    c->wpb_auto = o.warps_per_block == 0;
    c->lb = o.max_registers == 0 || o.max_registers >= 128
                ? 0
                : (o.max_registers >= 96 ? 3 : (o.max_registers >= 80 ? 1 : 2));
    c->F = o.window_F ? o.window_F : 1;
    c->mixed = o.precision == 1;
    c->prec = o.precision;
    c->loader = o.loader;
    c->tma_G = o.tma_stage_windows ? o.tma_stage_windows : 1;
    c->tma_NS = o.tma_stages ? o.tma_stages : 2;
    c->inject = o.debug_inject_wait_timeout;
    c->vs = o.buffered_stores != 0;
    c->pw = o.partial_windows != 0;
    c->ad = o.adaptive != 0;
    c->adp.alpha = 1.0 / 64;
    c->adp.k_sigma = 3.0;
    c->adp.n_warm = 32;
    if (c->pw && c->loader != 0) {
        delete c;
        return fail(RFI_EUNSUPPORTED, "partial_windows needs the direct loader (loader = 0)");
    }
    if (c->mixed) {
        if (o.compensated == 1 || c->lb != 0) {
            delete c;
            return fail(RFI_EINVAL, "precision = 1 has no Kahan or register-budget variants");
        }
        c->kahan = 0;
    }
    if (c->prec == 2 && (dtype != RFI_C32H || (c->lb != 0 && c->lb != 3) || o.loader != 0 ||
                         o.buffered_stores != 0 || o.partial_windows != 0 || o.adaptive != 0 ||
                         o.prefetch_groups > 0)) {
        delete c;
        return fail(RFI_EUNSUPPORTED, "precision = 2 needs binary16 input (RFI_C32H), the "
                                      "direct loader and the 128- or 96-register budget, without "
                                      "buffered stores, partial windows, adaptive thresholds "
                                      "or prefetch");
    }
    if (c->F & (c->F - 1) || c->F > 32 || channels % c->F != 0 || c->M * c->F < 2) {
        delete c;
        return fail(RFI_EINVAL, "window_F must be a power of two <= 32 dividing channels=%d",
                    channels);
    }
    if (c->lb > 0 && c->wpb > 8) {
        delete c;
        return fail(RFI_EINVAL, "max_registers below 128 allows at most 8 warps per block");
    }
    if (c->lb == 3 && c->wpb > 4) {
        if (!c->wpb_auto) {
            delete c;
            return fail(RFI_EINVAL, "max_registers = 96 allows at most 4 warps per block");
        }
        c->wpb = 4;
    }
    c->pf_bytes = o.prefetch_bytes ? o.prefetch_bytes : 1024;
    c->pf_groups = o.prefetch_groups > 0 ? o.prefetch_groups : 0;
    c->ovl = o.overlap_bytes == 0 ? 512 : (o.overlap_bytes < 0 ? 0 : o.overlap_bytes);
    c->indep = o.independent_launches;
    c->last_launch = -1;
    c->H = hop;
    c->sw = hop != window_M;
    c->wp = o.lane_split == 1;
    if (c->wp && (c->sw || c->loader != 0 || (c->lb != 0 && c->lb != 3) || c->vs || c->pw ||
                  c->ad || o.compensated == 1)) {
        delete c;
        return fail(RFI_EUNSUPPORTED, "lane_split = 1 needs the direct loader, the 128- "
                                      "(or, for binary16 odd windows, 96-) register budget, "
                                      "plain stores and no Kahan summation, and excludes "
                                      "partial_windows, adaptive and window_hop");
    }
    if (c->wp) c->kahan = 0;
    if (c->sw) {
        if (c->F != 1 || c->prec || c->loader != 0 || c->lb != 0 || c->vs || c->pw || c->ad ||
            o.compensated == 1) {
            delete c;
            return fail(RFI_EUNSUPPORTED, "overlapping windows need time-only windows, float32 "
                                          "arithmetic, the direct loader, the 128-register "
                                          "budget, plain stores and no Kahan summation, and "
                                          "exclude partial_windows and adaptive");
        }
        c->kahan = 0;
    }
    c->status = RFI_OK;
    if ((rc = choose_shape(c, o.lanes_per_row))) {
        delete c;
        return rc;
    }
    cudaError_t e;
    if ((e = cudaMalloc(&c->carry, sizeof(float) * 9 * (size_t)c->P * c->R)) != cudaSuccess ||
        (e = cudaMalloc(&c->counter, 4 * sizeof(unsigned long long))) != cudaSuccess ||
        (e = cudaMemset(c->carry, 0, sizeof(float) * 9 * (size_t)c->P * c->R)) != cudaSuccess ||
        (e = cudaMemset(c->counter, 0, 4 * sizeof(unsigned long long))) != cudaSuccess ||
        (c->pw && (e = cudaMalloc(&c->hw, (size_t)c->R * c->M * sample_bytes(dtype))) !=
                      cudaSuccess) ||
        (c->ad && (e = cudaMalloc(&c->adapt, adapt_bytes(c))) != cudaSuccess) ||
        (c->ad && (e = cudaMemset(c->adapt, 0, adapt_bytes(c))) != cudaSuccess) ||
        (c->sw && (e = cudaMalloc(&c->sw_buf, sw_bytes(c))) != cudaSuccess) ||
        (c->sw && (e = cudaMemset(c->sw_buf, 0, sw_bytes(c))) != cudaSuccess)) {
        cudaGetLastError();
        free_ctx(c);
        return fail(e == cudaErrorMemoryAllocation ? RFI_ENOMEM : RFI_ECUDA,
                    "device allocation failed: %s", cudaGetErrorString(e));
    }
    c->host_max_T = o.host_max_T;
    c->host_chunks = o.host_chunks ? o.host_chunks : 4;
    if (c->host_max_T > 0) {
        const int unit = c->sw ? c->H : c->M;
        const int T = c->pw ? c->host_max_T : c->host_max_T - c->host_max_T % unit;
        if (T < (c->pw ? 1 : unit)) {
            free_ctx(c);
            return fail(RFI_EINVAL, "host_max_T smaller than M");
        }
        c->host_max_T = T;
        const size_t R = (size_t)c->R;
        const size_t n_out_max = (size_t)T / c->K + 1;
        // a carried partial window adds at most one completed window per block
        const size_t nw_max =
            c->sw ? (size_t)T / c->H : (size_t)(T + (c->pw ? c->M - 1 : 0)) / c->M;
        bool ok = cudaMalloc(&c->h_vis, R * T * sample_bytes(dtype)) == cudaSuccess &&
                  cudaMalloc(&c->h_flags, R * ((nw_max * bits_per_window(c) + 31) / 32) * 4) ==
                      cudaSuccess &&
                  cudaMalloc(&c->h_avg, R * n_out_max * 32) == cudaSuccess &&
                  cudaMalloc(&c->h_weight, R * n_out_max * 4) == cudaSuccess &&
                  cudaMalloc(&c->h_stats, 3 * R * nw_max * 4) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&c->s_in, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&c->s_run, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&c->s_out, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&c->ev_start, cudaEventDisableTiming) == cudaSuccess &&
                  cudaEventCreateWithFlags(&c->ev_done, cudaEventDisableTiming) == cudaSuccess;
        for (int i = 0; ok && i < c->host_chunks; ++i) {
            cudaEvent_t a, b;
            ok = cudaEventCreateWithFlags(&a, cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&b, cudaEventDisableTiming) == cudaSuccess;
            if (ok) {
                c->ev_in.push_back(a);
                c->ev_run.push_back(b);
            }
        }
        if (!ok) {
            cudaGetLastError();
            free_ctx(c);
            return fail(RFI_ENOMEM, "device staging allocation failed");
        }
    }
    {
        std::lock_guard<std::mutex> lk(g_live_mu);
        g_live.insert(c);
    }
    *out = c;
    return RFI_OK;
}

int rfi_create(rfi_ctx **out, int stations, int channels, int window_M, int avg_K,
               const rfi_thresholds *thr, rfi_dtype dtype) {
    return rfi_create_ex(out, stations, channels, window_M, avg_K, thr, dtype, nullptr);
}

int rfi_rows(const rfi_ctx *ctx, long long *rows) {
    if (!ctx || !is_live(ctx)) return fail(RFI_ESTATE, "not a live context");
    if (!rows) return fail(RFI_EINVAL, "null output");
    *rows = ctx->R;
    return RFI_OK;
}

int rfi_outputs_for(const rfi_ctx *ctx, int T, int *n_out) {
    if (!ctx || !is_live(ctx)) return fail(RFI_ESTATE, "not a live context");
    if (!n_out) return fail(RFI_EINVAL, "null output");
    if (T < 0 || (!ctx->pw && T % (ctx->sw ? ctx->H : ctx->M) != 0))
        return fail(RFI_EINVAL, "T must be a multiple of M (of the hop H with overlapping "
                                "windows)");
    *n_out = (int)outputs_for_c(ctx, T);
    return RFI_OK;
}

int rfi_windows_for(const rfi_ctx *ctx, int T, int *n_win, long long *first_sample) {
    if (!ctx || !is_live(ctx)) return fail(RFI_ESTATE, "not a live context");
    if (!n_win) return fail(RFI_EINVAL, "null output");
    if (T < 0 || (!ctx->pw && T % (ctx->sw ? ctx->H : ctx->M) != 0))
        return fail(RFI_EINVAL, "T must be a multiple of M (of the hop H with overlapping "
                                "windows)");
    *n_win = windows_for(ctx, T);
    if (first_sample) *first_sample = first_final(ctx);
    return RFI_OK;
}

int rfi_get_options(const rfi_ctx *ctx, rfi_options *opt) {
    if (!ctx || !is_live(ctx)) return fail(RFI_ESTATE, "not a live context");
    if (!opt) return fail(RFI_EINVAL, "null output");
    opt->lanes_per_row = ctx->P;
    opt->warps_per_block = ctx->wpb;
    opt->host_max_T = ctx->host_max_T;
    opt->host_chunks = ctx->host_chunks;
    opt->compensated = ctx->kahan ? 1 : -1;
    opt->prefetch_bytes = ctx->pf_bytes;
    opt->prefetch_groups = ctx->pf_groups;
    opt->max_registers = ctx->lb == 0 ? 128 : (ctx->lb == 1 ? 80 : (ctx->lb == 3 ? 96 : 64));
    opt->window_F = ctx->F;
    opt->precision = ctx->prec;
    opt->loader = ctx->loader;
    opt->tma_stage_windows = ctx->tma_G;
    opt->tma_stages = ctx->tma_NS;
    opt->debug_inject_wait_timeout = ctx->inject;
    opt->buffered_stores = ctx->vs;
    opt->partial_windows = ctx->pw;
    opt->adaptive = ctx->ad;
    opt->overlap_bytes = ctx->ovl > 0 ? ctx->ovl : -1;
    opt->window_hop = ctx->sw ? ctx->H : 0;
    opt->lane_split = ctx->wp;
    opt->independent_launches = ctx->indep;
    return RFI_OK;
}

int rfi_last_launch(const rfi_ctx *ctx, int *order) {
    if (!ctx || !is_live(ctx)) return fail(RFI_ESTATE, "not a live context");
    if (!order) return fail(RFI_EINVAL, "null output");
    *order = ctx->last_launch;
    return RFI_OK;
}

int rfi_set_thresholds(rfi_ctx *ctx, const rfi_thresholds *thr) {
    int rc;
    if ((rc = check_ctx(ctx))) return rc;
    if ((rc = check_thresholds(thr))) return rc;
    ctx->thr = *thr;
    return RFI_OK;
}

int rfi_set_adaptation(rfi_ctx *ctx, const rfi_adaptation *p) {
    int rc;
    if ((rc = check_ctx(ctx))) return rc;
    if (!ctx->ad) return fail(RFI_EINVAL, "context was created without adaptive = 1");
    if (!p || !(p->alpha >= 0.0 && p->alpha <= 1.0) || !(p->k_sigma >= 0.0) ||
        !std::isfinite(p->k_sigma) || p->n_warm < 1)
        return fail(RFI_EINVAL, "need 0 <= alpha <= 1, finite k_sigma >= 0, n_warm >= 1");
    ctx->adp = *p;
    return RFI_OK;
}

int rfi_adaptive_state(rfi_ctx *ctx, float *host, size_t n_floats, int write, void *stream) {
    int rc;
    if ((rc = check_ctx(ctx))) return rc;
    if (!ctx->ad) return fail(RFI_EINVAL, "context was created without adaptive = 1");
    const size_t need = adapt_bytes(ctx) / sizeof(float);
    if (!host || n_floats < need)
        return fail(RFI_EINVAL, "adaptive state needs %zu floats ([R/F][4])", need);
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e == cudaSuccess)
        e = write ? cudaMemcpy(ctx->adapt, host, adapt_bytes(ctx), cudaMemcpyHostToDevice)
                  : cudaMemcpy(host, ctx->adapt, adapt_bytes(ctx), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "rfi_adaptive_state");
    return RFI_OK;
}

int rfi_process_block(rfi_ctx *ctx, const void *vis, int T, uint32_t *flags, float *avg,
                      float *weight, float *stats, void *stream) {
    NvtxRange nvtx("rfi_process_block");
    int rc;
    if ((rc = check_ctx(ctx))) return rc;
    if ((rc = check_block_args(ctx, vis, T, flags, avg, weight, stats, true))) return rc;
    const StreamArgs a = make_args(ctx, vis, T, flags, avg, weight, stats, 0, ctx->R);
    if ((rc = launch_block(ctx, a, static_cast<cudaStream_t>(stream)))) return rc;
    ctx->n_seen += T;
    return RFI_OK;
}

int rfi_process_block_host(rfi_ctx *ctx, const void *vis, int T, uint32_t *flags, float *avg,
                           float *weight, float *stats, void *stream) {
    NvtxRange nvtx("rfi_process_block_host");
    int rc;
    if ((rc = check_ctx(ctx))) return rc;
    if ((rc = check_block_args(ctx, vis, T, flags, avg, weight, stats, false))) return rc;
    if (T > ctx->host_max_T)
        return fail(RFI_EINVAL, "T=%d exceeds the host staging (host_max_T=%d)", T, ctx->host_max_T);
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    const long long R = ctx->R;
    const int nch = (int)std::min<long long>(ctx->host_chunks, R);
    const int nwin = windows_for(ctx, T), wpr = (nwin * bits_per_window(ctx) + 31) / 32;
    const long long n_out = outputs_for_c(ctx, T);
    const size_t sb = sample_bytes(ctx->dtype);
    cudaError_t e;
    if ((e = cudaEventRecord(ctx->ev_start, user)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(ctx->s_in, ctx->ev_start, 0)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(ctx->s_run, ctx->ev_start, 0)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(ctx->s_out, ctx->ev_start, 0)) != cudaSuccess)
        return set_cuda_error(ctx, e, "host path setup");
    for (int k = 0; k < nch; ++k) {
        const long long F = ctx->F;
        const long long r0 = (R / F) * k / nch * F, r1 = (R / F) * (k + 1) / nch * F;
        const long long nr = r1 - r0;
        if (nr <= 0) continue;
        e = cudaMemcpyAsync(ctx->h_vis + r0 * T * sb, static_cast<const char *>(vis) + r0 * T * sb,
                            nr * T * sb, cudaMemcpyHostToDevice, ctx->s_in);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_in[k], ctx->s_in);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->s_run, ctx->ev_in[k], 0);
        if (e != cudaSuccess) return set_cuda_error(ctx, e, "host path copy-in");
        StreamArgs a = make_args(ctx, ctx->h_vis, T, ctx->h_flags, ctx->h_avg, ctx->h_weight,
                                 ctx->h_stats, r0, nr);
        if ((rc = launch_block(ctx, a, ctx->s_run))) return rc;
        e = cudaEventRecord(ctx->ev_run[k], ctx->s_run);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->s_out, ctx->ev_run[k], 0);
        if (e == cudaSuccess && nwin > 0)
            e = cudaMemcpyAsync(flags + r0 * wpr, ctx->h_flags + r0 * wpr, nr * wpr * 4,
                                cudaMemcpyDeviceToHost, ctx->s_out);
        if (e == cudaSuccess && nwin > 0)
            e = cudaMemcpy2DAsync(stats + (r0 / F) * nwin, (size_t)(R / F) * nwin * 4,
                                  ctx->h_stats + (r0 / F) * nwin, (size_t)(R / F) * nwin * 4,
                                  (nr / F) * nwin * 4, 3, cudaMemcpyDeviceToHost, ctx->s_out);
        if (e == cudaSuccess && n_out > 0)
            e = cudaMemcpyAsync(avg + r0 * n_out * 8, ctx->h_avg + r0 * n_out * 8,
                                nr * n_out * 32, cudaMemcpyDeviceToHost, ctx->s_out);
        if (e == cudaSuccess && n_out > 0)
            e = cudaMemcpyAsync(weight + r0 * n_out, ctx->h_weight + r0 * n_out, nr * n_out * 4,
                                cudaMemcpyDeviceToHost, ctx->s_out);
        if (e != cudaSuccess) return set_cuda_error(ctx, e, "host path copy-out");
    }
    if ((e = cudaEventRecord(ctx->ev_done, ctx->s_out)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(user, ctx->ev_done, 0)) != cudaSuccess ||
        (e = cudaEventSynchronize(ctx->ev_done)) != cudaSuccess)
        return set_cuda_error(ctx, e, "host path completion");
    ctx->n_seen += T;
    return RFI_OK;
}

int rfi_process_batch(rfi_ctx *const *ctxs, int n, const void *const *vis, const int *T,
                      uint32_t *const *flags, float *const *avg, float *const *weight,
                      float *const *stats, void *stream) {
    NvtxRange nvtx("rfi_process_batch");
    static thread_local BatchArgs tb;
    BatchArgs *b = &tb;
    int rc = build_batch(ctxs, n, vis, T, flags, avg, weight, stats, true, b);
    if (rc) return rc;
    rfi_ctx *c0 = ctxs[0];
    const int grid = persistent_grid(c0->batch_fn, c0->wpb, c0->device);
    void *args[] = {b};
    // the batch kernels do not trigger early: nothing before them is in flight after them
    const cudaStream_t bst = static_cast<cudaStream_t>(stream);
    cudaError_t e = launch_plain(c0->device, bst, [&] {
        cudaError_t r = cudaLaunchKernel(c0->batch_fn, dim3(grid), dim3(32 * c0->wpb), args, 0,
                                         bst);
        if (r == cudaSuccess && c0->ad)
            r = cudaLaunchKernel(adapt_batch_fn(), dim3(adapt_batch_grid(c0->device)),
                                 dim3(256), args, 0, bst);
        return r;
    });
    if (e != cudaSuccess) {
        for (int i = 0; i < n; ++i) ctxs[i]->status = RFI_ECUDA;
        return fail(RFI_ECUDA, "batch launch: %s", cudaGetErrorString(e));
    }
    for (int i = 0; i < n; ++i) ctxs[i]->n_seen += T[i];
    return RFI_OK;
}

int rfi_batch_graph_create(rfi_batch_graph **out, rfi_ctx *const *ctxs, int n, const int *T) {
    if (!out) return fail(RFI_EINVAL, "null output handle");
    *out = nullptr;
    BatchArgs *b = new (std::nothrow) BatchArgs;
    if (!b) return fail(RFI_ENOMEM, "host allocation failed");
    int rc = build_batch(ctxs, n, nullptr, T, nullptr, nullptr, nullptr, nullptr, false, b);
    if (rc) {
        delete b;
        return rc;
    }
    rfi_batch_graph *g = new (std::nothrow) rfi_batch_graph();
    if (!g) {
        delete b;
        return fail(RFI_ENOMEM, "host allocation failed");
    }
    g->n = n;
    g->ctxs.assign(ctxs, ctxs + n);
    g->T.assign(T, T + n);
    g->batch_fn = ctxs[0]->batch_fn;
    g->block = 32 * ctxs[0]->wpb;
    g->grid = persistent_grid(g->batch_fn, ctxs[0]->wpb, ctxs[0]->device);
    cudaKernelNodeParams kp = {};
    void *args[] = {b};
    kp.func = const_cast<void *>(g->batch_fn);
    kp.gridDim = dim3(g->grid);
    kp.blockDim = dim3(g->block);
    kp.kernelParams = args;
    cudaError_t e = cudaGraphCreate(&g->graph, 0);
    if (e == cudaSuccess) e = cudaGraphAddKernelNode(&g->node, g->graph, nullptr, 0, &kp);
    if (e == cudaSuccess && ctxs[0]->ad) {
        cudaKernelNodeParams ka = kp;
        ka.func = const_cast<void *>(adapt_batch_fn());
        ka.gridDim = dim3(adapt_batch_grid(ctxs[0]->device));
        ka.blockDim = dim3(256);
        e = cudaGraphAddKernelNode(&g->adapt_node, g->graph, &g->node, 1, &ka);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    delete b;
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (g->graph) cudaGraphDestroy(g->graph);
        delete g;
        return fail(RFI_ECUDA, "graph build: %s", cudaGetErrorString(e));
    }
    {
        std::lock_guard<std::mutex> lk(g_live_mu);
        g_live.insert(g);
    }
    *out = g;
    return RFI_OK;
}

int rfi_batch_graph_launch(rfi_batch_graph *g, const void *const *vis, uint32_t *const *flags,
                           float *const *avg, float *const *weight, float *const *stats,
                           void *stream) {
    NvtxRange nvtx("rfi_batch_graph_launch");
    if (!g || !is_live(g)) return fail(RFI_ESTATE, "not a live batch graph");
    static thread_local BatchArgs tb;
    BatchArgs *b = &tb;
    int rc = build_batch(g->ctxs.data(), g->n, vis, g->T.data(), flags, avg, weight, stats, true, b);
    if (rc) return rc;
    cudaKernelNodeParams kp = {};
    void *args[] = {b};
    kp.func = const_cast<void *>(g->batch_fn);
    kp.gridDim = dim3(g->grid);
    kp.blockDim = dim3(g->block);
    kp.kernelParams = args;
    cudaError_t e = cudaGraphExecKernelNodeSetParams(g->exec, g->node, &kp);
    if (e == cudaSuccess && g->adapt_node) {
        cudaKernelNodeParams ka = kp;
        ka.func = const_cast<void *>(adapt_batch_fn());
        ka.gridDim = dim3(adapt_batch_grid(g->ctxs[0]->device));
        ka.blockDim = dim3(256);
        e = cudaGraphExecKernelNodeSetParams(g->exec, g->adapt_node, &ka);
    }
    if (e == cudaSuccess)
        e = launch_plain(g->ctxs[0]->device, static_cast<cudaStream_t>(stream), [&] {
            return cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream));
        });
    if (e != cudaSuccess) {
        for (rfi_ctx *c : g->ctxs) c->status = RFI_ECUDA;
        return fail(RFI_ECUDA, "graph launch: %s", cudaGetErrorString(e));
    }
    for (int i = 0; i < g->n; ++i) g->ctxs[i]->n_seen += g->T[i];
    return RFI_OK;
}

int rfi_batch_graph_destroy(rfi_batch_graph *g) {
    if (!g) return RFI_OK;
    {
        std::lock_guard<std::mutex> lk(g_live_mu);
        if (!g_live.erase(g)) return fail(RFI_ESTATE, "not a live batch graph");
    }
    cudaGraphExecDestroy(g->exec);
    cudaGraphDestroy(g->graph);
    delete g;
    return RFI_OK;
}

namespace {
// Header of a saved stream state; followed by the carry, float[R][P][9], for contexts
// with partial windows the raw samples of the open windows, [R][M] samples, and for
// adaptive contexts the running moments of tau, float[R/F][4].
struct StateHeader {
    unsigned int magic, version;
    long long R, n_seen;
    int P, M, K, F, dtype, pw, ad, hop, split, prec;
    rfi_thresholds thr;
    rfi_adaptation adp;
};
size_t carry_bytes(const rfi_ctx *c) { return sizeof(float) * 9 * (size_t)c->P * c->R; }
size_t hw_bytes(const rfi_ctx *c) {
    return c->pw ? (size_t)c->R * c->M * sample_bytes(c->dtype) : 0;
}
constexpr unsigned int STATE_MAGIC = 0x52464953u;  // "RFIS"
}  // namespace

int rfi_state_size(const rfi_ctx *ctx, size_t *bytes) {
    if (!ctx || !is_live(ctx)) return fail(RFI_ESTATE, "not a live context");
    if (!bytes) return fail(RFI_EINVAL, "null output");
    *bytes = sizeof(StateHeader) + carry_bytes(ctx) + hw_bytes(ctx) +
             (ctx->ad ? adapt_bytes(ctx) : 0) + sw_bytes(ctx);
    return RFI_OK;
}

int rfi_get_state(rfi_ctx *ctx, void *buf, size_t bytes, void *stream) {
    int rc;
    if ((rc = check_ctx(ctx))) return rc;
    size_t need = 0;
    rfi_state_size(ctx, &need);
    if (!buf || bytes < need) return fail(RFI_EINVAL, "state buffer needs %zu bytes", need);
    StateHeader h = {};
    h.magic = STATE_MAGIC;
    h.version = 4;
    h.pw = ctx->pw;
    h.hop = ctx->H;
    h.split = ctx->wp;
    h.ad = ctx->ad;
    h.adp = ctx->adp;
    h.R = ctx->R;
    h.n_seen = ctx->n_seen;
    h.P = ctx->P;
    h.M = ctx->M;
    h.K = ctx->K;
    h.F = ctx->F;
    h.dtype = (int)ctx->dtype;
    h.prec = ctx->prec;
    h.thr = ctx->thr;
    std::memcpy(buf, &h, sizeof h);
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    char *dst = static_cast<char *>(buf) + sizeof h;
    if (e == cudaSuccess)
        e = cudaMemcpy(dst, ctx->carry, carry_bytes(ctx), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && ctx->pw)
        e = cudaMemcpy(dst + carry_bytes(ctx), ctx->hw, hw_bytes(ctx), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && ctx->ad)
        e = cudaMemcpy(dst + carry_bytes(ctx) + hw_bytes(ctx), ctx->adapt, adapt_bytes(ctx),
                       cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && ctx->sw)
        e = cudaMemcpy(dst + carry_bytes(ctx) + hw_bytes(ctx), ctx->sw_buf, sw_bytes(ctx),
                       cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "rfi_get_state");
    return RFI_OK;
}

int rfi_set_state(rfi_ctx *ctx, const void *buf, size_t bytes) {
    int rc;
    if ((rc = check_ctx(ctx))) return rc;
    size_t need = 0;
    rfi_state_size(ctx, &need);
    if (!buf || bytes < need) return fail(RFI_EINVAL, "state buffer holds %zu of %zu bytes",
                                          bytes, need);
    StateHeader h;
    std::memcpy(&h, buf, sizeof h);
    if (h.magic != STATE_MAGIC || h.version != 4)
        return fail(RFI_EINVAL, "not a saved stream state");
    if (h.R != ctx->R || h.P != ctx->P || h.M != ctx->M || h.K != ctx->K || h.F != ctx->F ||
        h.pw != ctx->pw || h.ad != ctx->ad || h.dtype != (int)ctx->dtype || h.hop != ctx->H ||
        h.split != ctx->wp || h.prec != ctx->prec)
        return fail(RFI_EINVAL, "saved state is for another geometry or launch shape "
                                "(rows %lld, lanes %d, M %d, K %d, F %d, partial windows %d, "
                                "adaptive %d, hop %d)",
                    h.R, h.P, h.M, h.K, h.F, h.pw, h.ad, h.hop);
    if ((rc = check_thresholds(&h.thr))) return rc;
    cudaError_t e = sync_device_and_forget();
    const char *src = static_cast<const char *>(buf) + sizeof h;
    if (e == cudaSuccess)
        e = cudaMemcpy(ctx->carry, src, carry_bytes(ctx), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && ctx->pw)
        e = cudaMemcpy(ctx->hw, src + carry_bytes(ctx), hw_bytes(ctx), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && ctx->ad)
        e = cudaMemcpy(ctx->adapt, src + carry_bytes(ctx) + hw_bytes(ctx), adapt_bytes(ctx),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess && ctx->sw)
        e = cudaMemcpy(ctx->sw_buf, src + carry_bytes(ctx) + hw_bytes(ctx), sw_bytes(ctx),
                       cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "rfi_set_state");
    ctx->n_seen = h.n_seen;
    ctx->thr = h.thr;
    if (ctx->ad) ctx->adp = h.adp;
    return RFI_OK;
}

int rfi_check(rfi_ctx *ctx, void *stream) {
    int rc;
    if ((rc = check_ctx(ctx))) return rc;
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    int err = 0;
    if (e == cudaSuccess)
        e = cudaMemcpy(&err, reinterpret_cast<int *>(ctx->counter + 2), sizeof(int),
                       cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "rfi_check");
    if (err & 4) {
        ctx->status = RFI_ESTATE;
        return fail(RFI_ESTATE, "a tensor tile's shared-memory destination was not 128-byte "
                                "aligned and its copy was skipped (error word %d); rfi_reset "
                                "clears it", err);
    }
    if (err & 1) {
        ctx->status = RFI_ETIMEOUT;
        return fail(RFI_ETIMEOUT, "a bounded wait in the kernel gave up (error word %d); "
                                  "results of that launch are incomplete; rfi_reset clears it",
                    err);
    }
    if (err) {
        ctx->status = RFI_ESTATE;
        return fail(RFI_ESTATE, "the debug-bounds build caught an access outside its buffer "
                                "(error word %d) and skipped it; rfi_reset clears it", err);
    }
    return RFI_OK;
}

int rfi_reset(rfi_ctx *ctx) {
    if (!ctx || !is_live(ctx) || ctx->magic != CTX_MAGIC)
        return fail(RFI_ESTATE, "not a live context");
    cudaSetDevice(ctx->device);
    cudaError_t e = sync_device_and_forget();
    if (e == cudaSuccess)
        e = cudaMemset(ctx->carry, 0, sizeof(float) * 9 * (size_t)ctx->P * ctx->R);
    if (e == cudaSuccess) e = cudaMemset(ctx->counter, 0, 4 * sizeof(unsigned long long));
    if (e == cudaSuccess && ctx->ad) e = cudaMemset(ctx->adapt, 0, adapt_bytes(ctx));
    if (e == cudaSuccess && ctx->sw) e = cudaMemset(ctx->sw_buf, 0, sw_bytes(ctx));
    if (e != cudaSuccess) {
        ctx->status = RFI_ECUDA;
        return fail(RFI_ECUDA, "reset: %s", cudaGetErrorString(e));
    }
    ctx->n_seen = 0;
    ctx->status = RFI_OK;
    return RFI_OK;
}

int rfi_destroy(rfi_ctx *ctx) {
    if (!ctx) return RFI_OK;
    {
        std::lock_guard<std::mutex> lk(g_live_mu);
        if (!g_live.erase(ctx)) return fail(RFI_ESTATE, "not a live context (double destroy?)");
    }
    free_ctx(ctx);
    return RFI_OK;
}

}  // extern "C"
