// rfi_adapt.cu -- advance the online SK-threshold state of adaptive contexts.
//
// After a flagging launch has stored every window's tau and flag bits, one thread per
// footprint row walks the row's windows in order and, for each window that was not
// flagged, updates the row's {n, mean, second moment} of tau:
//   n += 1,  w = max(alpha, 1/n),  mean += w (tau - mean),  m2 += w (tau^2 - m2).
// The flagging kernel derives the next launch's SK interval from this state.
#include "rfi_device.cuh"
#include "rfi_kernels.h"

namespace rfi {
namespace {

__device__ void adapt_row(const StreamArgs &a, long long g) {
    float *st = a.adapt + g * 4;
    const float *tau_row = a.stats + g * a.nwin;                 // plane 0: tau
    const uint32_t *fl = a.flags + g * a.F * (long long)a.Wpr;   // first row of the footprint
    // debug-bounds build: the row's state, statistics and flag words lie in their buffers
    if (!rfi_in(st, 12, a.adapt, (a.R / a.F) * 16ll, a.err) ||
        !rfi_in(tau_row, 4ll * a.nwin, a.stats, (a.R / a.F) * a.nwin * 4ll, a.err) ||
        !rfi_in(fl, 4ll * a.Wpr, a.flags, a.R * a.Wpr * 4ll, a.err))
        return;
    float n = st[0], mu = st[1], m2 = st[2];
    // windows in groups of 8: the group's loads are issued together, then the state
    // runs over the group in window order
    for (int w0 = 0; w0 < a.nwin; w0 += 8) {
        float tau[8];
        uint32_t bit[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int w = min(w0 + k, a.nwin - 1);
            const int t = w * a.M;                               // first sample of window w
            tau[k] = tau_row[w];
            bit[k] = (fl[t >> 5] >> (t & 31)) & 1u;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (w0 + k >= a.nwin || bit[k]) continue;
            n += 1.f;
            const float wgt = fmaxf(a.alpha, __frcp_rn(n));
            mu = mu + wgt * (tau[k] - mu);
            m2 = m2 + wgt * (tau[k] * tau[k] - m2);
        }
    }
    st[0] = n;
    st[1] = mu;
    st[2] = m2;
}

__global__ void __launch_bounds__(256) k_adapt(const __grid_constant__ StreamArgs a) {
    const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (g < a.R / a.F) adapt_row(a, g);
}

__global__ void __launch_bounds__(256) k_adapt_batch(const __grid_constant__ BatchArgs b) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (int i = 0; i < b.n; ++i) {
        const StreamArgs &a = b.s[i];
        if (!a.adapt) continue;
        for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < a.R / a.F;
             g += stride)
            adapt_row(a, g);
    }
}

}  // namespace

const void *adapt_fn() { return (const void *)&k_adapt; }
const void *adapt_batch_fn() { return (const void *)&k_adapt_batch; }

}  // namespace rfi
