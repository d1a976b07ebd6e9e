// rfi_noalloc.cu -- rfi_process_block_noalloc: flag one block without a context and
// without allocating anything.
//
// Who needs it: code that runs where cudaMalloc must not be called -- for example a
// correlator stage whose device memory is entirely reserved up front by its own pool,
// a real-time thread that cannot afford the implicit device synchronisation an
// allocation may cause, or a plug-in loaded into a host that owns all allocation.
// Such callers already hold their input and output buffers; what they cannot obtain
// is the library's working memory.
//
// The working memory this entry point needs is the averaging carry: for every row the
// running sums (8 floats) and count of the averaging bin that is still open at the
// end of a block.  It lives here in a fixed file-scope device array of
// RFI_NOALLOC_SCRATCH_BYTES, which every GPU that loads the library holds until the
// process exits.  The kernel is the library's k_block with one lane per row, so its
// results are bit-identical to rfi_process_block on a context created with
// lanes_per_row = 1.
#include "rfi.h"
#include "rfi_device.cuh"
#include "rfi_internal.h"

#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>

using namespace rfi;

namespace {

// The carry of the open averaging bin: float[R][1][9].
static __device__ __align__(256) unsigned char g_noalloc_scratch[RFI_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch.  In host code the symbol is only a host-side
// stand-in, never a device address, so the kernel must receive the looked-up pointer.
// The address belongs to the CUDA context whose copy of this module it came from: the
// device's primary context, or a context the caller made current with the driver API,
// and after cudaDeviceReset a new primary context with a new copy.  So the lookup is
// cached per context, keyed by the context's unique id (cuCtxGetId, never reused in a
// process), and repeated for a context not seen before.
typedef CUresult (*PFN_ctx_current)(CUcontext *);
typedef CUresult (*PFN_ctx_id)(CUcontext, unsigned long long *);

struct CtxFns {
    PFN_ctx_current current = nullptr;
    PFN_ctx_id id = nullptr;
};

const CtxFns &ctx_fns() {
    static CtxFns f;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            f.current = reinterpret_cast<PFN_ctx_current>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            f.id = reinterpret_cast<PFN_ctx_id>(p);
    });
    return f;
}

// Id of the calling thread's current context; false when there is none yet (the
// runtime creates the device's primary context on its first call that needs one).
bool current_ctx_id(unsigned long long *id) {
    const CtxFns &f = ctx_fns();
    CUcontext c = nullptr;
    return f.current && f.id && f.current(&c) == CUDA_SUCCESS && c != nullptr &&
           f.id(c, id) == CUDA_SUCCESS;
}

constexpr int MAX_CONTEXTS = 64;
std::mutex g_mu;
unsigned long long g_ctx_id[MAX_CONTEXTS] = {};
void *g_ctx_addr[MAX_CONTEXTS] = {};
int g_n_ctx = 0;

int lookup_symbol(void **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        char msg[200];
        snprintf(msg, sizeof msg, "cudaGetSymbolAddress of the no-alloc scratch failed: %s",
                 cudaGetErrorString(e));
        return rfi_internal_fail(RFI_ECUDA, msg);
    }
    *out = p;
    return RFI_OK;
}

// The scratch's device address in the calling thread's current context (the current
// device's primary context unless the caller made another current).
int scratch_for_current_context(void **out) {
    unsigned long long id = 0;
    if (!current_ctx_id(&id)) {
        // no context yet, or no way to tell contexts apart: look the address up (this
        // also creates the primary context) and cache it under the context now current
        int rc = lookup_symbol(out);
        if (rc || !current_ctx_id(&id)) return rc;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    for (int i = 0; i < g_n_ctx; ++i)
        if (g_ctx_id[i] == id) {
            *out = g_ctx_addr[i];
            return RFI_OK;
        }
    void *p = nullptr;
    if (int rc = lookup_symbol(&p)) return rc;
    const int slot = g_n_ctx < MAX_CONTEXTS ? g_n_ctx++ : (int)(id % MAX_CONTEXTS);
    g_ctx_id[slot] = id;
    g_ctx_addr[slot] = p;
    *out = p;
    return RFI_OK;
}

typedef const void *KernelPtr;

template <int DT, int SPU, bool K>
KernelPtr pick_chunk(int ch) {
    switch (ch) {
        case 5: return (KernelPtr)&k_block<DT, SPU, 1, 5, K>;
        case 4: return (KernelPtr)&k_block<DT, SPU, 1, 4, K>;
        case 2: return (KernelPtr)&k_block<DT, SPU, 1, 2, K>;
        default: return (KernelPtr)&k_block<DT, SPU, 1, 1, K>;
    }
}

KernelPtr pick_kernel(int dt, int spu, int ch, bool kahan) {
    if (dt == DT_F32) return kahan ? pick_chunk<DT_F32, 1, true>(ch) : pick_chunk<DT_F32, 1, false>(ch);
    if (spu == 2) return kahan ? pick_chunk<DT_F16, 2, true>(ch) : pick_chunk<DT_F16, 2, false>(ch);
    return kahan ? pick_chunk<DT_F16, 1, true>(ch) : pick_chunk<DT_F16, 1, false>(ch);
}

int chunk_of(int S) {
    static const int opts[] = {5, 4, 2, 1};
    for (int c : opts)
        if (S % c == 0) return c;
    return 1;
}

}  // namespace

extern "C" int rfi_process_block_noalloc(int stations, int channels, int window_M, int avg_K,
                                         const rfi_thresholds *thr, rfi_dtype dtype,
                                         long long n_seen, const void *vis, int T,
                                         uint32_t *flags, float *avg, float *weight,
                                         float *stats, void *stream) {
    char msg[240];
    if (stations < 1 || channels < 1)
        return rfi_internal_fail(RFI_EINVAL, "stations and channels must be >= 1");
    if (window_M < 2) return rfi_internal_fail(RFI_EINVAL, "window M must be >= 2");
    if (avg_K < window_M || avg_K % window_M != 0)
        return rfi_internal_fail(RFI_EINVAL, "averaging factor K must be a positive multiple of M");
    if (T <= 0 || T % window_M != 0)
        return rfi_internal_fail(RFI_EINVAL, "T must be a positive multiple of M");
    if (n_seen < 0 || n_seen % window_M != 0)
        return rfi_internal_fail(RFI_EINVAL, "n_seen must be a non-negative multiple of M");
    if (dtype != RFI_C64 && dtype != RFI_C32H) return rfi_internal_fail(RFI_EINVAL, "unknown dtype");
    if (!thr || std::isnan(thr->d) || std::isnan(thr->s_low) || std::isnan(thr->s_high) ||
        std::isnan(thr->gamma) || !std::isfinite(thr->eps) || thr->eps < 0 ||
        !std::isfinite(thr->d) || thr->s_low > thr->s_high)
        return rfi_internal_fail(RFI_EINVAL, "invalid thresholds");
    const long long B = (long long)stations * (stations + 1) / 2;
    const long long R = B * channels;
    if ((long long)T * R > (1ll << 40)) return rfi_internal_fail(RFI_EINVAL, "block too large");
    const unsigned long long carry_bytes = (unsigned long long)R * 9 * sizeof(float);
    if (carry_bytes > RFI_NOALLOC_SCRATCH_BYTES) {
        snprintf(msg, sizeof msg,
                 "stream of %lld rows needs %llu bytes of carry; the no-alloc scratch holds %u "
                 "bytes (at most %u rows)",
                 R, carry_bytes, (unsigned)RFI_NOALLOC_SCRATCH_BYTES,
                 (unsigned)(RFI_NOALLOC_SCRATCH_BYTES / (9 * sizeof(float))));
        return rfi_internal_fail(RFI_EINVAL, msg);
    }
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return rfi_internal_fail(RFI_ECUDA, "no usable CUDA device");
    }
    const int dt = dtype == RFI_C64 ? DT_F32 : DT_F16;
    const int sb = dtype == RFI_C64 ? 32 : 16;
    const int spu = (dt == DT_F16 && window_M % 2 == 0) ? 2 : 1;
    const int nwin = T / window_M, wpr = (T + 31) / 32;
    const long long n_out = (n_seen + T) / avg_K - n_seen / avg_K;
    int rc;
    if ((rc = rfi_internal_check_dev(vis, (size_t)R * T * sb, (size_t)sb * spu, device, "vis")) ||
        (rc = rfi_internal_check_dev(flags, (size_t)R * wpr * 4, 4, device, "flags")) ||
        (rc = rfi_internal_check_dev(stats, (size_t)R * nwin * 12, 4, device, "stats")))
        return rc;
    if (n_out > 0 &&
        ((rc = rfi_internal_check_dev(avg, (size_t)R * n_out * 32, 16, device, "avg")) ||
         (rc = rfi_internal_check_dev(weight, (size_t)R * n_out * 4, 4, device, "weight"))))
        return rc;
    void *scratch = nullptr;
    if ((rc = scratch_for_current_context(&scratch))) return rc;

    // The kernel reads the carry only when this block continues an open bin
    // (n_seen % K != 0); that carry was written by the previous call for the same
    // stream.  Nothing in the scratch has to start at zero.
    StreamArgs a = {};
    a.vis = vis;
    a.flags = flags;
    a.avg = avg;
    a.weight = weight;
    a.stats = stats;
    a.carry = static_cast<float *>(scratch);
    a.R = R;
    a.stats_plane = R * nwin;
    a.T = T;
    a.M = window_M;
    a.K = avg_K;
    a.Wpr = wpr;
    a.nwin = nwin;
    a.n_out = (int)n_out;
    a.bin_pos0 = (int)(n_seen % avg_K);
    a.F = 1;
    a.d = (float)thr->d;
    a.pf_windows = std::max(1, 1024 / (window_M * sb));
    a.pf_groups = 0;
    const double Md = window_M;
    a.c0 = (float)((Md * thr->d + 1.0) / (Md - 1.0));
    a.s_low = (float)thr->s_low;
    a.s_high = (float)thr->s_high;
    a.gamma = (float)thr->gamma;
    a.eps = (float)thr->eps;
    a.fM = (float)window_M;
    a.fK = (float)avg_K;
    a.invM = (float)(1.0 / window_M);
    const int S = window_M / spu;
    const bool kahan = window_M >= 64;
    KernelPtr fn = pick_kernel(dt, spu, chunk_of(S), kahan);
    const int wpb = 8;
    const long long groups = (R + 31) / 32;
    const long long blocks = (groups + wpb - 1) / wpb;
    void *args[] = {&a};
    // the kernel lets the next launch on the stream start early: counted, so that a
    // flagging launch of a context after it is ordered as after a launch whose buffers
    // it does not know
    rfi_internal_noalloc_launch_begin();
    e = cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(32 * wpb), args, 0,
                         static_cast<cudaStream_t>(stream));
    rfi_internal_noalloc_launch_end();
    if (e != cudaSuccess) {
        snprintf(msg, sizeof msg, "kernel launch: %s", cudaGetErrorString(e));
        return rfi_internal_fail(RFI_ECUDA, msg);
    }
    return RFI_OK;
}
