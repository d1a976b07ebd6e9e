// rfi_device.cuh -- sm_103a device code of the online RFI flagging path
// (arXiv 2412.14775, Sections 2, 2.1, 2.2; Tables 1 and 2).
//
// Work decomposition.  A warp owns RW = 32/P rows ("row group") and walks their
// windows in time order.  The P lanes of one row split every window of M samples:
// a window is a run of M*SB contiguous bytes, cut into 16- or 32-byte load units,
// and lane j of the row loads units j, j+P, j+2P, ... so one warp instruction reads
// P*UB contiguous bytes from each of RW rows (whole sectors, nothing wasted).
// Each lane keeps its own partial sums of the window; an xor-butterfly over the P
// lanes completes S1, S2 and the two resultant vectors, after which every lane of
// the row holds bit-identical totals (float addition is commutative), evaluates
// tau and r, and the window flag follows.  Per-row outputs (stats, flag words,
// averages) are written by lane 0 of the row.
//
// Averaging.  Each lane also sums its samples of the window (8 floats); when the
// window is not flagged that partial joins the lane's running bin sum.  When a bin
// of K samples closes, the P running sums are reduced and the mean of the unflagged
// samples and the weight (unflagged / K) are written.  An open bin at the end of a
// block is kept per lane in the context's carry, so splitting a stream into blocks
// at multiples of M gives bit-identical results.
#pragma once
#include <cuda.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace rfi {

enum { DT_F32 = 0, DT_F16 = 1 };
constexpr unsigned FULL = 0xffffffffu;
constexpr int MAX_BATCH = 64;

// One stream's work in one launch (passed by value in kernel parameter space).
struct StreamArgs {
    const void *vis;        // [R][T][4][2] of row 0 of this launch
    uint32_t *flags;        // [R][Wpr]
    float *avg;             // [R][n_out][8]
    float *weight;          // [R][n_out]
    float *stats;           // plane k at stats + k*stats_plane: [R][nwin]
    float *carry;           // [R][P][9]: per-lane open-bin sums (8) and count
    long long R;            // rows in this launch
    long long stats_plane;  // floats between the tau, r_Re and r_Im planes
    int T, M, K, Wpr, nwin, n_out;
    int bin_pos0;           // samples of the open bin before window 0 of this launch
    int F;                  // adjacent rows (channels) per window footprint (power of 2)
    float d;                // SK shape parameter (used by the mixed-precision mode)
    int pf_windows;         // windows per L2 prefetch group (>= 1)
    int pf_groups;          // prefetch distance in groups (0 = no prefetch)
    // shared-memory staging (TMA loader)
    int stage_windows;      // windows of every row per stage (G)
    int stages;             // stages per warp (NS)
    unsigned pitch;         // bytes per row in a stage (G*M*SB padded to an odd x 16)
    unsigned tx_extra;      // extra bytes expected per stage (fault injection only)
    long long wait_limit;   // cycles a stage wait may take before it gives up
    int *err;               // device error word: 1 = a bounded wait gave up, 2 = an
                            // access outside its buffer (debug-bounds build), 4 = a
                            // tensor tile copy skipped (unaligned destination)
    float c0;               // (W d + 1)/(W - 1), W = M F, Table 1 group 5
    float s_low, s_high, gamma, eps;
    float fM;               // W = M F as float (samples in one window)
    float fK;
    float invM;             // 1/W (exact when W is a power of two)
    // partial windows: a window may begin in an earlier block; its first `phase`
    // samples wait in hw, and the samples after this block's last whole window go there
    char *hw;               // [R][M] raw samples of each row's open window (or null)
    int phase;              // samples of window 0 already in hw (0 <= phase < M)
    // online SK thresholds: per footprint row {n, mean, second moment} of tau over the
    // unflagged windows seen so far (exponentially weighted), updated window by window
    float *adapt;           // [R/F][4] (or null)
    float alpha;            // weight of a new window once n >= 1/alpha
    float k_sigma;          // thresholds mean -/+ k_sigma * sd once n >= n_warm
    float n_warm;
    // launch overlap: bytes at the start of every row requested into L2 before the
    // kernel waits for the grid it depends on (0 = none); indep = 1: the host found
    // that nothing this launch reads is written, and nothing it writes is read or
    // written, by the flagging launches that may still run on the stream, so it
    // neither waits for the grid before it nor requests anything early
    int ovl_bytes;
    int indep;
    // overlapping windows (rfi_sliding.cuh): a window of M samples every hop samples;
    // warm = min(hops of the stream before this launch, M/hop - 1); the carried totals
    // [R][8] and the lane's averaging sums [R][P][8] of the pending hop, and the last
    // window's flag [R]
    int hop, warm;
    float *sw_tot, *sw_pend;
    uint32_t *sw_hist;
    // window-parallel lanes (rfi_wpar.cuh): the stream's window index of window 0 of
    // this launch, mod lanes_per_row
    int wphase;
};

struct BatchArgs {
    int n;
    long long total;                    // total row-group tasks
    long long prefix[MAX_BATCH + 1];    // first task of each stream
    unsigned long long *counter;        // [0] task counter, [1] low word: blocks done
    StreamArgs s[MAX_BATCH];
};

// ---- hardware approximations (PTX ISA: sqrt.approx / rcp.approx) --------------
// The .ftz forms are single MUFU operations; a subnormal argument (|I| or p below
// 1e-19) is read as 0, which changes a sum by less than the FP32 rounding of S1.
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// L2 prefetch of the 128-byte line holding p: a per-thread hint (no register, no wait,
// no memory clobber).  The bulk form (cp.async.bulk.prefetch.L2) takes warp-uniform
// operands, so with one address per row it was issued once per distinct address, about
// 100 instructions per prefetch and warp; the P lanes of a row instead split the range
// into lines.
__device__ __forceinline__ void prefetch_line(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
template <int P>
__device__ __forceinline__ void prefetch_rows(const char *p, long long bytes, int j) {
    const uintptr_t end = reinterpret_cast<uintptr_t>(p) + bytes;
    for (uintptr_t q = (reinterpret_cast<uintptr_t>(p) & ~uintptr_t(127)) + 128u * j; q < end;
         q += 128u * P)
        prefetch_line(reinterpret_cast<const void *>(q));
}

// ---- TMA bulk copies into shared memory, completed on an mbarrier --------------
__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; "
        "selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for a barrier phase for at most `limit` cycles; false when it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity, long long limit) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, unsigned bytes,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// One 2-D tile of a tensor map (rows x bytes of a row; 8-byte elements) into shared
// memory, completed on an mbarrier.  x (elements) times 8 is a multiple of 16 bytes by
// construction (the tile starts at a window boundary); rows and bytes beyond the
// tensor are filled with zeros and still counted.
__device__ __forceinline__ void tma_load_2d(void *dst, const void *tmap, int x, int y,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(tmap), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---- streaming loads of one 16- or 32-byte unit (read once: no L1 allocation) ---
template <int UB> struct Unit;
template <> struct Unit<32> { uint32_t r[8]; };
template <> struct Unit<16> { uint32_t r[4]; };

// Streaming loads: read-only path, no L1 allocation, and a 256-byte L2 fill per miss
// (.L2::256B; measured 5 % faster for binary16 M = 8 and the 5x4 footprints, the same
// elsewhere).
__device__ __forceinline__ void load_unit(const char *p, Unit<32> &u) {
    asm("ld.global.nc.L1::no_allocate.L2::256B.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(u.r[0]), "=r"(u.r[1]), "=r"(u.r[2]), "=r"(u.r[3]),
          "=r"(u.r[4]), "=r"(u.r[5]), "=r"(u.r[6]), "=r"(u.r[7])
        : "l"(p));
}
__device__ __forceinline__ void load_unit(const char *p, Unit<16> &u) {
    asm("ld.global.nc.L1::no_allocate.L2::256B.v4.b32 {%0,%1,%2,%3}, [%4];"
        : "=r"(u.r[0]), "=r"(u.r[1]), "=r"(u.r[2]), "=r"(u.r[3])
        : "l"(p));
}
// The window-parallel kernels give each lane whole windows, so with 16-byte units (odd
// binary16 windows: 80 bytes for M = 5) one warp instruction reads 16 bytes of each of
// 32 windows: half of every 32-byte sector.  Allocating those loads in L1 serves the
// other half to the lane's next load from L1 instead of L2 (binary16 5 x 4 footprints
// 136.8 -> 126.6 us, M = 5 216.2 -> 182.1 us, measured A/B).  32-byte units read whole
// sectors and stream past L1 as elsewhere.
__device__ __forceinline__ void load_unit_wp(const char *p, Unit<16> &u) {
    asm("ld.global.nc.L2::256B.v4.b32 {%0,%1,%2,%3}, [%4];"
        : "=r"(u.r[0]), "=r"(u.r[1]), "=r"(u.r[2]), "=r"(u.r[3])
        : "l"(p));
}
__device__ __forceinline__ void load_unit_wp(const char *p, Unit<32> &u) { load_unit(p, u); }

// ---- debug-bounds build (-DRFI_DEBUG_BOUNDS) -----------------------------------
// Every global access of the kernels is checked against the extent that the launch's
// own arguments give its buffer; an access outside it is skipped (a load reads zeros)
// and bit 1 of the context's error word is set, read by rfi_check.  In the normal build
// rfi_in is the constant true and the checks compile away.
__device__ __forceinline__ bool rfi_in(const void *p, long long n, const void *base,
                                       long long extent, int *err) {
#ifdef RFI_DEBUG_BOUNDS
    const char *c = static_cast<const char *>(p);
    const char *b = static_cast<const char *>(base);
    if (b != nullptr && c >= b && c + n <= b + extent) return true;
    if (err) atomicOr(err, 2);
    return false;
#else
    (void)p; (void)n; (void)base; (void)extent; (void)err;
    return true;
#endif
}

// The raw-sample carry of partial windows is read, then rewritten, by the same launch:
// coherent loads, ordered before the later stores.
__device__ __forceinline__ void load_unit_rw(const char *p, Unit<32> &u) {
    asm volatile("ld.global.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(u.r[0]), "=r"(u.r[1]), "=r"(u.r[2]), "=r"(u.r[3]),
                   "=r"(u.r[4]), "=r"(u.r[5]), "=r"(u.r[6]), "=r"(u.r[7])
                 : "l"(p) : "memory");
}
__device__ __forceinline__ void load_unit_rw(const char *p, Unit<16> &u) {
    asm volatile("ld.global.v4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(u.r[0]), "=r"(u.r[1]), "=r"(u.r[2]), "=r"(u.r[3])
                 : "l"(p) : "memory");
}

__device__ __forceinline__ void load_unit_smem(const unsigned char *p, Unit<32> &u) {
    const unsigned a = smem_u32(p);
    asm volatile("ld.shared.v4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(u.r[0]), "=r"(u.r[1]), "=r"(u.r[2]), "=r"(u.r[3]) : "r"(a));
    asm volatile("ld.shared.v4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(u.r[4]), "=r"(u.r[5]), "=r"(u.r[6]), "=r"(u.r[7]) : "r"(a + 16));
}
__device__ __forceinline__ void load_unit_smem(const unsigned char *p, Unit<16> &u) {
    asm volatile("ld.shared.v4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(u.r[0]), "=r"(u.r[1]), "=r"(u.r[2]), "=r"(u.r[3]) : "r"(smem_u32(p)));
}

// Sums of a binary16 and a float32 value (sm_100 mixed-precision add and subtract):
// the binary16 operand is widened exactly and the result rounded once to float32, so
// a + b of two binary16 values is the float32 sum of their exact widenings, as an
// FADD of two converted values gives it, with one instruction less.
__device__ __forceinline__ uint16_t lo16(uint32_t w) { return (uint16_t)(w & 0xffffu); }
__device__ __forceinline__ uint16_t hi16(uint32_t w) { return (uint16_t)(w >> 16); }
__device__ __forceinline__ float add_hf(uint16_t a, float c) {
    float d;
    asm("add.rn.f32.f16 %0, %1, %2;" : "=f"(d) : "h"(a), "f"(c));
    return d;
}
__device__ __forceinline__ float sub_hf(uint16_t a, float c) {
    float d;
    asm("sub.rn.f32.f16 %0, %1, %2;" : "=f"(d) : "h"(a), "f"(c));
    return d;
}

// Complex Stokes parameters (Sec. 2, Eq. IQUV) of sample k of a unit, each as a float2
// (re, im): I = xx + yy, Q = xx - yy, U = xy + yx, V = j (xy - yx), i.e.
// Re V = Im yx - Im xy and Im V = Re xy - Re yx.  Every component is the float32 sum
// of two input values.  Binary16 input: four of the eight halves are widened, and each
// component adds one of them to a half of another correlation with a mixed-precision
// add (the same float32 results as widening all eight; 1.5 % faster at M = 16).
struct Stokes { float2 I, Q, U, V; };

template <int DT, int UB>
__device__ __forceinline__ Stokes stokes_of(const Unit<UB> &u, int k) {
    Stokes s;
    if constexpr (DT == DT_F32) {
        const float2 xx = make_float2(__uint_as_float(u.r[0]), __uint_as_float(u.r[1]));
        const float2 xy = make_float2(__uint_as_float(u.r[2]), __uint_as_float(u.r[3]));
        const float2 yx = make_float2(__uint_as_float(u.r[4]), __uint_as_float(u.r[5]));
        const float2 yy = make_float2(__uint_as_float(u.r[6]), __uint_as_float(u.r[7]));
        s.I = __fadd2_rn(xx, yy);
        s.Q = __fadd2_rn(xx, make_float2(-yy.x, -yy.y));
        s.U = __fadd2_rn(xy, yx);
        s.V = make_float2(yx.y - xy.y, xy.x - yx.x);
    } else {
        const uint32_t wxx = u.r[4 * k + 0], wxy = u.r[4 * k + 1];
        const uint32_t wyx = u.r[4 * k + 2], wyy = u.r[4 * k + 3];
        const float2 yy = __half22float2(*reinterpret_cast<const __half2 *>(&wyy));
        const float yx_re = __low2float(*reinterpret_cast<const __half2 *>(&wyx));
        const float xy_im = __high2float(*reinterpret_cast<const __half2 *>(&wxy));
        s.I = make_float2(add_hf(lo16(wxx), yy.x), add_hf(hi16(wxx), yy.y));
        s.Q = make_float2(sub_hf(lo16(wxx), yy.x), sub_hf(hi16(wxx), yy.y));
        s.U = make_float2(add_hf(lo16(wxy), yx_re), add_hf(hi16(wyx), xy_im));
        s.V = make_float2(sub_hf(hi16(wyx), xy_im), sub_hf(lo16(wxy), yx_re));
    }
    return s;
}

// ---- packed FP32 pairs (Blackwell f32x2 pipes) -------------------------------
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    return __fadd2_rn(a, make_float2(-b.x, -b.y));
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// ---- per-lane window accumulators ------------------------------------------
// The real and imaginary parts of (Q, U, V) are carried side by side in float2
// pairs, so one packed instruction advances both directional statistics.
struct WinAcc {
    float2 s;        // (S1, S2): Table 1 groups 3, 4
    float2 c;        // Kahan compensation of (S1, S2) (when enabled)
    float2 q, u, v;  // (Re, Im) of the resultant sums, Table 2 group 4
    float2 a[4];     // sums of I, Q, U, V (averaging; converted back to correlations
                     // once per completed bin)
};

// One sample: Table 1 groups 1-4 and Table 2 groups 1-4 for the Re and Im parts of
// (Q, U, V) at once, plus the Stokes sums used for the averaged output.
template <bool KAHAN>
__device__ __forceinline__ void accumulate(WinAcc &A, const Stokes &x, float2 eps2) {
    const float2 I = x.I, Q = x.Q, U = x.U, V = x.V;
    const float2 I2 = mul2(I, I);
    const float y = I2.x + I2.y;                             // |I|^2
    const float z = sqrt_approx(y);                          // |I|
    if constexpr (KAHAN) {
        const float2 yk = sub2(make_float2(z, y), A.c);
        const float2 t = add2(A.s, yk);
        A.c = sub2(sub2(t, A.s), yk);
        A.s = t;
    } else {
        A.s = add2(A.s, make_float2(z, y));
    }
    float2 n = mul2(Q, Q);                                   // q^2 + u^2 + v^2, Re and Im
    n = fma2(U, U, n);
    n = fma2(V, V, n);
    const float2 p = add2(make_float2(sqrt_approx(n.x), sqrt_approx(n.y)), eps2);
    const float2 ip = make_float2(rcp_approx(p.x), rcp_approx(p.y));
    A.q = fma2(Q, ip, A.q);                                  // sum of q / p
    A.u = fma2(U, ip, A.u);
    A.v = fma2(V, ip, A.v);
    A.a[0] = add2(A.a[0], I);                                // sums of I, Q, U, V
    A.a[1] = add2(A.a[1], Q);
    A.a[2] = add2(A.a[2], U);
    A.a[3] = add2(A.a[3], V);
}

// ---- binary16 Stokes arithmetic (precision = 2) ----------------------------------
// The Stokes parameters of a binary16 sample are formed in binary16 (half2 adds and
// subtracts, round to nearest even: Eq. IQUV in the input's own precision).  Every
// product after that multiplies two binary16 values, which is exact in float32, and
// every sum is float32: S1 and S2 (Table 1 groups 3-4, Kahan when enabled), the
// polarisation-vector sums (Table 2 group 4) and the averaging sums.  The normalisation
// is q / sqrt(q^2 + u^2 + v^2 + eps^2) (one reciprocal square root per part instead of
// a square root, eps and a reciprocal; it differs from q / (sqrt(...) + eps) by a
// relative eps / |(q, u, v)|, below binary16 rounding for vectors longer than 2^-12,
// and a zero vector still contributes 0).  V is carried as (Re V, -Im V), the swapped
// halves of yx - xy: r depends on the squares of the resultant's components only, and
// a closed bin's averages undo the sign.
__device__ __forceinline__ __half2 as_h2(uint32_t w) { return *reinterpret_cast<const __half2 *>(&w); }

template <bool KAHAN>
__device__ __forceinline__ void accumulate_h2(WinAcc &A, const uint32_t *w, float e2) {
    const __half2 xx = as_h2(w[0]), xy = as_h2(w[1]), yx = as_h2(w[2]), yy = as_h2(w[3]);
    const float2 I = __half22float2(__hadd2(xx, yy));
    const float2 Q = __half22float2(__hsub2(xx, yy));
    const float2 U = __half22float2(__hadd2(xy, yx));
    const float2 V = __half22float2(__lowhigh2highlow(__hsub2(yx, xy)));   // (Re V, -Im V)
    const float2 I2 = mul2(I, I);
    const float y = I2.x + I2.y;                             // |I|^2
    const float z = sqrt_approx(y);                          // |I|
    if constexpr (KAHAN) {
        const float2 yk = sub2(make_float2(z, y), A.c);
        const float2 t = add2(A.s, yk);
        A.c = sub2(sub2(t, A.s), yk);
        A.s = t;
    } else {
        A.s = add2(A.s, make_float2(z, y));
    }
    float2 n = mul2(Q, Q);                                   // q^2 + u^2 + v^2 (+ eps^2)
    n = fma2(U, U, n);
    n = fma2(V, V, n);
    n = add2(n, make_float2(e2, e2));
    const float2 ip = make_float2(rsqrt_approx(n.x), rsqrt_approx(n.y));
    A.q = fma2(Q, ip, A.q);
    A.u = fma2(U, ip, A.u);
    A.v = fma2(V, ip, A.v);
    A.a[0] = add2(A.a[0], I);
    A.a[1] = add2(A.a[1], Q);
    A.a[2] = add2(A.a[2], U);
    A.a[3] = add2(A.a[3], V);
}

// ---- paper-mixed precision (Tables 3 and 4) -----------------------------------
// Binary16 values are carried in float registers; h16 rounds a float32 result to the
// nearest binary16 (ties to even).  Binary32 groups use correctly rounded operations
// without fused multiply-add, so every rounding matches the tables' operation order.
__device__ __forceinline__ float h16(float x) { return __half2float(__float2half_rn(x)); }

__device__ __forceinline__ void accumulate_mixed(WinAcc &A, const Stokes &x, float eps) {
    // Table 3, groups 1-4 (binary32): y = xr^2 + xi^2, z = sqrt(y), s1 += z, s2 += y
    const float y = __fadd_rn(__fmul_rn(x.I.x, x.I.x), __fmul_rn(x.I.y, x.I.y));
    const float z = __fsqrt_rn(y);
    A.s.x = __fadd_rn(A.s.x, z);
    A.s.y = __fadd_rn(A.s.y, y);
    // Table 4, groups 1-3 (binary32) and group 4 (binary16 sums), Re then Im part
    {
        const float n = __fadd_rn(__fadd_rn(__fmul_rn(x.Q.x, x.Q.x), __fmul_rn(x.U.x, x.U.x)),
                                  __fmul_rn(x.V.x, x.V.x));
        const float p = __fadd_rn(__fsqrt_rn(n), eps);
        A.q.x = h16(A.q.x + h16(__fdiv_rn(x.Q.x, p)));
        A.u.x = h16(A.u.x + h16(__fdiv_rn(x.U.x, p)));
        A.v.x = h16(A.v.x + h16(__fdiv_rn(x.V.x, p)));
    }
    {
        const float n = __fadd_rn(__fadd_rn(__fmul_rn(x.Q.y, x.Q.y), __fmul_rn(x.U.y, x.U.y)),
                                  __fmul_rn(x.V.y, x.V.y));
        const float p = __fadd_rn(__fsqrt_rn(n), eps);
        A.q.y = h16(A.q.y + h16(__fdiv_rn(x.Q.y, p)));
        A.u.y = h16(A.u.y + h16(__fdiv_rn(x.U.y, p)));
        A.v.y = h16(A.v.y + h16(__fdiv_rn(x.V.y, p)));
    }
    A.a[0] = add2(A.a[0], x.I);
    A.a[1] = add2(A.a[1], x.Q);
    A.a[2] = add2(A.a[2], x.U);
    A.a[3] = add2(A.a[3], x.V);
}

// Table 3 groups 5-7 and Table 4 groups 5-7 on one window's sums; returns the flag
// and the statistics (binary16 values).  Adding two binary16 values in float32 is
// exact, so h16(a + b) is the binary16 sum; products of two binary16 values are exact
// in float32 too; division and square root are correctly rounded in float32 first.
__device__ __forceinline__ bool finish_mixed(const StreamArgs &a, float S1, float S2, float qr,
                                             float ur, float vr, float qi, float ui, float vi,
                                             float &tau, float &r_re, float &r_im) {
    const float eps16 = 0.0009765625f;                       // 2^-10
    const float Wh = h16(a.fM), one = 1.0f;
    const float lead = h16(__fdiv_rn(h16(h16(Wh * h16(a.d)) + one), h16(Wh - one)));  // g5
    const float s12 = __fmul_rn(S1, S1);                                               // g6
    float t = h16(Wh * h16(S2));                                                       // g7
    t = h16(__fdiv_rn(t, h16(h16(s12) + eps16)));
    tau = h16(lead * h16(t - one));                  // Sec. 2.1: lead * (W s2/s12 - 1)
    const bool f_sk = !(tau >= h16(a.s_low) && tau <= h16(a.s_high));
    const float rre2 = h16(h16(h16(qr * qr) + h16(ur * ur)) + h16(vr * vr));           // g5
    const float rim2 = h16(h16(h16(qi * qi) + h16(ui * ui)) + h16(vi * vi));
    r_re = h16(__fdiv_rn(h16(__fsqrt_rn(rre2)), Wh));                                  // g6
    r_im = h16(__fdiv_rn(h16(__fsqrt_rn(rim2)), Wh));
    const float g = h16(a.gamma);
    return f_sk || !(r_re <= g) || !(r_im <= g);                                       // g7
}

template <int P>
__device__ __forceinline__ float allsum(float v) {
#pragma unroll
    for (int o = 1; o < P; o <<= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// Continue an allsum<P> over the F adjacent rows of a footprint (their lanes form one
// aligned block of P*F lanes); PF = P * F is warp-uniform.
template <int P>
__device__ __forceinline__ float rowsum(float v, int PF) {
#pragma unroll
    for (int o = P; o < 32; o <<= 1)
        if (o < PF) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// Packed pairs: both halves shuffled, then one f32x2 addition (the same additions, in
// the same order, as two scalar reductions).
__device__ __forceinline__ float2 shfl_xor2(float2 v, int o) {
    return make_float2(__shfl_xor_sync(FULL, v.x, o), __shfl_xor_sync(FULL, v.y, o));
}
template <int P>
__device__ __forceinline__ float2 allsum2(float2 v) {
#pragma unroll
    for (int o = 1; o < P; o <<= 1) v = add2(v, shfl_xor2(v, o));
    return v;
}

// The averaged output of one closed bin of one row (end of Sec. 2.1): tot holds the
// sums of (I, Q, U, V), re and im, over its unflagged samples and n their count; the
// correlations are xx = (I + Q)/2, yy = (I - Q)/2, xy = (U - jV)/2, yx = (U + jV)/2, and
// the weight is n / K (an empty bin gives zeros).
__device__ __forceinline__ void store_bin(const StreamArgs &a, long long row, int bin,
                                          const float (&tot)[8], float n) {
    float *const avp = a.avg + (row * a.n_out + bin) * 8;
    float *const wtp = a.weight + row * a.n_out + bin;
    if (!rfi_in(avp, 32, a.avg, a.R * a.n_out * 32ll, a.err) ||
        !rfi_in(wtp, 4, a.weight, a.R * a.n_out * 4ll, a.err))
        return;
    float4 *ap = reinterpret_cast<float4 *>(avp);
    const float h = n > 0.f ? 0.5f * __frcp_rn(n) : 0.f;
    const float Ir = tot[0], Ii = tot[1], Qr = tot[2], Qi = tot[3];
    const float Ur = tot[4], Ui = tot[5], Vr = tot[6], Vi = tot[7];
    ap[0] = make_float4((Ir + Qr) * h, (Ii + Qi) * h, (Ur + Vi) * h, (Ui - Vr) * h);
    ap[1] = make_float4((Ur - Vi) * h, (Ui + Vr) * h, (Ir - Qr) * h, (Ii - Qi) * h);
    *wtp = __fdiv_rn(n, a.fK);
}

// ---- one row group of one stream ---------------------------------------------
// DT: input dtype; SPU: samples per load unit (1 or 2); P: lanes per row;
// CH: load units issued together per lane; KAHAN: compensated S1, S2.
// DB: double-buffered loads (two chunks in flight per lane) or one chunk at a time
// (fewer registers, more resident warps).  The arithmetic is the same either way.
// PREC: 0 = float32 arithmetic throughout (binary16 input widened exactly); 1 = the
// paper's trained mixed precision (Tables 3 and 4; one lane per row, no footprint, no
// Kahan); 2 = binary16 Stokes parameters, exact products and float32 sums
// (accumulate_h2; binary16 input).
// TMA: every lane owns one row (P = 1) and reads it from shared memory, where the
// warp's rows are staged a few windows at a time by cp.async.bulk copies (one per row,
// issued by the row's lane) that complete on one mbarrier per stage.
// VS: statistics and flag words buffered in registers and written 16 bytes at a time
// (4 windows / 4 words) where the row layout allows; fewer, larger stores for small
// windows at the price of 16 live registers.
// PW: partial windows.  Window 0 may have begun in an earlier block (its first
// `phase` samples wait in the raw-sample carry), and the samples after the last whole
// window are put there for the next block.  A separate instance, so that the code of
// the head window and the tail copy does not cost the kernels that need neither.
// AD: online per-stream SK thresholds.  Each footprint row keeps a running estimate of
// the mean and second moment of tau over its unflagged windows (weight max(alpha, 1/n)
// for the n-th, so the first 1/alpha windows give the plain mean).  Once n >= n_warm
// the row's SK test uses [mean - k sd, mean + k sd] instead of [s_low, s_high]: the
// thresholds of the state at the start of the launch.  The state then advances window
// by window in k_adapt (rfi_adapt.cu), a light pass over the stored tau and flag bits.
// The DS threshold gamma stays fixed (its null, E r^2 = 1/W, does not depend on the
// data).
// PFT: the L2 prefetch code is compiled in (taken when the launch asks for it); the
// plain kernels come with and without it, since its mere presence changes how the
// compiler schedules the window loop.
// BAT: called from the persistent batch kernel (see the footprint sums below).
template <int DT, int SPU, int P, int CH, bool KAHAN, bool DB = true, int PREC = 0,
          int TMA = 0, bool VS = false, bool PW = false, bool AD = false,
          bool PFT = false, bool BAT = false>
__device__ __forceinline__ void process_group(const StreamArgs &a, long long group,
                                              const void *tmap = nullptr) {
    constexpr bool MIXED = PREC == 1, H2 = PREC == 2;
    static_assert(!MIXED || (P == 1 && !KAHAN), "mixed precision runs one lane per row");
    static_assert(!H2 || DT == DT_F16, "binary16 Stokes arithmetic needs binary16 input");
    constexpr int RW = 32 / P;
    constexpr int SB = (DT == DT_F32) ? 32 : 16;   // bytes per sample
    constexpr int UB = SB * SPU;                   // bytes per load unit
    const int lane = threadIdx.x & 31;
    const int j = lane & (P - 1);
    const long long row = group * RW + lane / P;
    const bool active = row < a.R;
    const long long rowc = active ? row : a.R - 1;  // inactive lanes re-read a valid row
    const int S = a.M / (P * SPU);                  // load units per lane per window
    const char *rp = static_cast<const char *>(a.vis) + rowc * (long long)a.T * SB;
    // window frame: sample 0 of window 0, `phase` samples before the block's first
    const char *fp = PW ? rp - (long long)a.phase * SB : rp;
    const bool head = PW && a.phase > 0 && a.nwin > 0;  // window 0 starts in the carry
    char *const hwp = PW ? a.hw + rowc * (long long)a.M * SB : nullptr;
    const int nbits = PW ? a.nwin * a.M : a.T;          // flagged samples of this call
    const bool lead = active && j == 0;     // writes the row's outputs
    // extents (bytes) of the launch's buffers, for the debug-bounds build
    const long long vis_ext = a.R * (long long)a.T * SB;
    const long long hw_ext = a.R * (long long)a.M * SB;
    const long long carry_ext = a.R * P * 9 * 4ll;
    const long long stats_ext = (2 * a.stats_plane + (a.R / a.F) * a.nwin) * 4ll;
    const long long flags_ext = a.R * a.Wpr * 4ll;
    const long long adapt_ext = (a.R / a.F) * 16ll;
    // the row's SK interval (set below, from the state at the start of the launch; the
    // state is advanced afterwards by k_adapt from the statistics and flags stored here)
    float slo = 0.f, shi = 0.f;

    float acc[8];            // running bin sums of (I, Q, U, V), re and im
    float cnt = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = 0.f;
    if (a.bin_pos0 != 0) {
        const float *cp = a.carry + (rowc * P + j) * 9;   // open-bin Stokes sums and count
        if (rfi_in(cp, 36, a.carry, carry_ext, a.err)) {
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[c] = cp[c];
            cnt = cp[8];
        }
    }
    // Per-row cursors and counters, set up once per task so that the per-window
    // bookkeeping is a handful of integer operations.
    // statistics are per footprint (F rows); the first row's lead lane writes them
    float *const st_row = a.stats + (rowc / a.F) * a.nwin;
    const bool st_lead = lead && (row % a.F) == 0;
    const int PF = P * a.F;
    uint32_t *const fl_row = a.flags + rowc * a.Wpr;
    const long long plane = a.stats_plane;
    const int wpbin = a.K / a.M;                              // windows per averaging bin
    int wib = a.bin_pos0 / a.M;                               // windows of the open bin seen
    int bin = 0;
    const float lane_samples = (float)(S * SPU);
    // flag words: mode 0 when M divides 32 (whole windows per word), 1 when 32 divides
    // M (whole words per window), 2 otherwise (windows straddle words)
    const int fmode = (32 % a.M == 0) ? 0 : ((a.M % 32 == 0) ? 1 : 2);
    const uint32_t wmask = a.M >= 32 ? FULL : ((1u << a.M) - 1u);
    const int words_per_window = a.M >> 5;
    uint32_t fword = 0;
    int fbit = 0, fwi = 0;
    const bool vec_stats = VS && (a.nwin & 3) == 0 && (a.stats_plane & 3) == 0 &&
                           (reinterpret_cast<uintptr_t>(a.stats) & 15) == 0;
    const bool vec_flags = VS && fmode == 0 && (a.Wpr & 3) == 0 && (nbits & 31) == 0 &&
                           (reinterpret_cast<uintptr_t>(a.flags) & 15) == 0;
    float4 tq = make_float4(0.f, 0.f, 0.f, 0.f), rq = tq, iq = tq;
    uint4 fq = make_uint4(0u, 0u, 0u, 0u);
    // L2 prefetch: the lanes of each row keep pf_groups groups of pf_windows windows
    // requested ahead of the window being loaded.
    const bool pf = PFT && a.pf_groups > 0 && active;
    const unsigned wbytes = (unsigned)a.M * SB;
    if (pf) {
        const int hi = min(a.nwin, (1 + a.pf_groups) * a.pf_windows);
        if (hi > 1 && rfi_in(fp + wbytes, (hi - 1) * (long long)wbytes, a.vis, vis_ext, a.err))
            prefetch_rows<P>(fp + wbytes, (hi - 1) * (long long)wbytes, j);
    }
    int pf_next = a.pf_windows;

    const float2 eps2 = make_float2(a.eps, a.eps);
    const float e2 = a.eps * a.eps;
    // The load units of a lane form one contiguous stream over the row: chunk q (CH
    // units) starts at rp + j*UB + q*CHB.  Two register buffers let the loads of chunk
    // q+1 be in flight while chunk q is consumed.
    constexpr int CHB = CH * P * UB;
    const int nch = S / CH;                       // chunks per window
    const int Q = a.nwin * nch;                   // chunks per lane in this block
    const char *cp_ = fp + j * UB;
    auto load_chunk = [&](int q, Unit<UB>(&u)[CH]) {
        if (PW && head && q < nch) {
            // window 0 began in an earlier block: its units before the block come from
            // the raw-sample carry (a warp-uniform branch, taken for window 0 only)
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const int off = q * CHB + c * (P * UB) + j * UB;
                if (off < a.phase * SB) {
                    if (rfi_in(hwp + off, UB, a.hw, hw_ext, a.err)) load_unit_rw(hwp + off, u[c]);
                    else u[c] = Unit<UB>{};
                } else {
                    if (rfi_in(fp + off, UB, a.vis, vis_ext, a.err)) load_unit(fp + off, u[c]);
                    else u[c] = Unit<UB>{};
                }
            }
            return;
        }
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const char *p = cp_ + (long long)q * CHB + c * (P * UB);
            if (rfi_in(p, UB, a.vis, vis_ext, a.err)) load_unit(p, u[c]);
            else u[c] = Unit<UB>{};
        }
    };
    WinAcc A;
    const float2 zero2 = make_float2(0.f, 0.f);
    A.s = A.c = A.q = A.u = A.v = zero2;
#pragma unroll
    for (int c = 0; c < 4; ++c) A.a[c] = zero2;
    int w = 0, cw = 0;
    Unit<UB> ua[CH], ub[DB ? CH : 1];
    if constexpr (!TMA && !PW) load_chunk(0, ua);
    if constexpr (AD) {
        // after the first loads are in flight, and without a branch, so that the wait
        // for the state overlaps them (requesting the state before the data loads, or
        // branching on it, measured 6-15 % slower)
        const float *const ad_row = a.adapt + (rowc / a.F) * 4;
        const bool ad_ok = rfi_in(ad_row, 12, a.adapt, adapt_ext, a.err);
        const float n0 = ad_ok ? ad_row[0] : 0.f, mu0 = ad_ok ? ad_row[1] : 0.f;
        const float m20 = ad_ok ? ad_row[2] : 0.f;
        const float sd = __fsqrt_rn(fmaxf(m20 - mu0 * mu0, 0.f));
        const bool warm = n0 >= a.n_warm;
        slo = warm ? mu0 - a.k_sigma * sd : a.s_low;
        shi = warm ? mu0 + a.k_sigma * sd : a.s_high;
    }

    auto consume = [&](const Unit<UB>(&u)[CH]) {
#pragma unroll
        for (int c = 0; c < CH; ++c) {
#pragma unroll
            for (int k = 0; k < SPU; ++k) {
                if constexpr (MIXED)
                    accumulate_mixed(A, stokes_of<DT, UB>(u[c], k), a.eps);
                else if constexpr (H2)
                    accumulate_h2<KAHAN>(A, &u[c].r[4 * k], e2);
                else
                    accumulate<KAHAN>(A, stokes_of<DT, UB>(u[c], k), eps2);
            }
        }
    };
    auto end_window = [&]() {
        if constexpr (KAHAN) A.s = sub2(A.s, A.c);
        // complete the window over the P lanes of the row (and the F rows of a footprint)
        float S1 = allsum<P>(A.s.x), S2 = allsum<P>(A.s.y);
        float qr = allsum<P>(A.q.x), ur = allsum<P>(A.u.x), vr = allsum<P>(A.v.x);
        float qi = allsum<P>(A.q.y), ui = allsum<P>(A.u.y), vi = allsum<P>(A.v.y);
        if (PF > P) {
            // continue the butterfly over the F adjacent rows of the footprint (their
            // lanes form one aligned block of P*F lanes).  The same additions in the
            // same order either way; the single-stream kernels test each step once for
            // all eight sums, the batch kernel once per sum: each form measured faster
            // in its kernel (a matter of how the compiler schedules the whole loop;
            // batch of 8 subbands 514 against 555 us, single-stream kernels 0-10 %).
            if constexpr (BAT) {
                S1 = rowsum<P>(S1, PF); S2 = rowsum<P>(S2, PF);
                qr = rowsum<P>(qr, PF); ur = rowsum<P>(ur, PF); vr = rowsum<P>(vr, PF);
                qi = rowsum<P>(qi, PF); ui = rowsum<P>(ui, PF); vi = rowsum<P>(vi, PF);
            } else {
#pragma unroll
                for (int o = P; o < 32; o <<= 1) {
                    if (o < PF) {
                        S1 += __shfl_xor_sync(FULL, S1, o);
                        S2 += __shfl_xor_sync(FULL, S2, o);
                        qr += __shfl_xor_sync(FULL, qr, o);
                        ur += __shfl_xor_sync(FULL, ur, o);
                        vr += __shfl_xor_sync(FULL, vr, o);
                        qi += __shfl_xor_sync(FULL, qi, o);
                        ui += __shfl_xor_sync(FULL, ui, o);
                        vi += __shfl_xor_sync(FULL, vi, o);
                    }
                }
            }
        }
        float tau, r_re, r_im;
        bool f;
        if constexpr (MIXED) {
            f = finish_mixed(a, S1, S2, qr, ur, vr, qi, ui, vi, tau, r_re, r_im);
        } else {
            // Table 1 groups 6-7 and Sec. 2.1: tau = c0 * (W S2 / (S1^2 + eps) - 1)
            const float s12 = S1 * S1;
            tau = a.c0 * (a.fM * S2 * rcp_approx(s12 + a.eps) - 1.0f);
            // Table 2 groups 5-6: r = sqrt(q^2 + u^2 + v^2) / W, per part
            r_re = sqrt_approx(qr * qr + ur * ur + vr * vr) * a.invM;
            r_im = sqrt_approx(qi * qi + ui * ui + vi * vi) * a.invM;
            // SK flag OR (DS Re OR DS Im); a NaN statistic fails its "inside" test
            if constexpr (AD)
                f = !(tau >= slo && tau <= shi) || !(r_re <= a.gamma) || !(r_im <= a.gamma);
            else
                f = !(tau >= a.s_low && tau <= a.s_high) || !(r_re <= a.gamma) ||
                    !(r_im <= a.gamma);
        }

        if (vec_stats) {
            tq = make_float4(tq.y, tq.z, tq.w, tau);
            rq = make_float4(rq.y, rq.z, rq.w, r_re);
            iq = make_float4(iq.y, iq.z, iq.w, r_im);
            if ((w & 3) == 3 && st_lead && rfi_in(st_row + w - 3, 16, a.stats, stats_ext, a.err) &&
                rfi_in(st_row + w - 3 + 2 * plane, 16, a.stats, stats_ext, a.err)) {
                *reinterpret_cast<float4 *>(st_row + w - 3) = tq;
                *reinterpret_cast<float4 *>(st_row + w - 3 + plane) = rq;
                *reinterpret_cast<float4 *>(st_row + w - 3 + 2 * plane) = iq;
            }
        } else if (st_lead && rfi_in(st_row + w, 4, a.stats, stats_ext, a.err) &&
                   rfi_in(st_row + w + 2 * plane, 4, a.stats, stats_ext, a.err)) {
            st_row[w] = tau;
            st_row[w + plane] = r_re;
            st_row[w + 2 * plane] = r_im;
        }
        // the flag covers every sample of the window: bits [w*M, w*M + M) of the row
        if (fmode == 0) {
            if (f) fword |= wmask << fbit;
            fbit += a.M;
            if (fbit == 32) {
                if (vec_flags) {
                    fq = make_uint4(fq.y, fq.z, fq.w, fword);
                    if ((fwi & 3) == 3 && lead &&
                        rfi_in(fl_row + fwi - 3, 16, a.flags, flags_ext, a.err))
                        *reinterpret_cast<uint4 *>(fl_row + fwi - 3) = fq;
                } else if (lead && rfi_in(fl_row + fwi, 4, a.flags, flags_ext, a.err)) {
                    fl_row[fwi] = fword;
                }
                ++fwi;
                fword = 0;
                fbit = 0;
            }
        } else if (fmode == 1) {
            if (lead && rfi_in(fl_row + fwi, 4ll * words_per_window, a.flags, flags_ext, a.err))
                for (int k = 0; k < words_per_window; ++k) fl_row[fwi + k] = f ? FULL : 0u;
            fwi += words_per_window;
        } else {
            int lo = w * a.M;
            const int hi = lo + a.M;
            while (lo < hi) {
                const int b0 = lo & 31;
                const int nb = min(hi - lo, 32 - b0);
                if (f) fword |= (nb == 32 ? FULL : ((1u << nb) - 1u)) << b0;
                lo += nb;
                if ((lo & 31) == 0) {
                    if (lead && rfi_in(fl_row + ((lo - 1) >> 5), 4, a.flags, flags_ext, a.err))
                        fl_row[(lo - 1) >> 5] = fword;
                    fword = 0;
                }
            }
        }
        // flagged samples are excluded from the average (end of Sec. 2.1)
        if (!f) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                acc[2 * c] += A.a[c].x;
                acc[2 * c + 1] += A.a[c].y;
            }
            cnt += lane_samples;
        }
        if (++wib == wpbin) {
            float tot[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) tot[c] = allsum<P>(acc[c]);
            const float n = allsum<P>(cnt);
            if constexpr (H2) tot[7] = -tot[7];      // V was carried as (Re V, -Im V)
            if (lead) store_bin(a, row, bin, tot, n);
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[c] = 0.f;
            cnt = 0.f;
            wib = 0;
            ++bin;
        }
        A.s = A.c = A.q = A.u = A.v = zero2;
#pragma unroll
        for (int c = 0; c < 4; ++c) A.a[c] = zero2;
        ++w;
        if (pf && w == pf_next) {
            const int g0 = w + a.pf_groups * a.pf_windows;
            const int g1 = min(a.nwin, g0 + a.pf_windows);
            if (g0 < g1 &&
                rfi_in(fp + (long long)g0 * wbytes, (g1 - g0) * (long long)wbytes, a.vis, vis_ext,
                       a.err))
                prefetch_rows<P>(fp + (long long)g0 * wbytes, (g1 - g0) * (long long)wbytes, j);
            pf_next += a.pf_windows;
        }
    };

    int q0 = 0;                                   // first chunk of the pipelined loop
    if constexpr (!TMA && PW) {
        if (Q > 0) load_chunk(0, ua);
    }

    if constexpr (TMA) {
        // stages of G windows for the warp's RW rows: [stage][row][pitch] bytes; the
        // row's first lane issues its copies, and its P lanes read their units (the
        // same units as the direct loader: j, j + P, ... of each window) from there
        extern __shared__ __align__(128) unsigned char smem_raw[];
        const int warp = threadIdx.x >> 5;
        const int NS = a.stages, G = a.stage_windows;
        const int r = lane / P;                       // the lane's row in the warp
        uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw) + warp * NS;
        const unsigned bar_bytes = (8u * NS * (blockDim.x >> 5) + 127u) & ~127u;
        unsigned char *wbuf = smem_raw + bar_bytes + (size_t)warp * NS * RW * a.pitch;
        const int ngroups = (a.nwin + G - 1) / G;
        const unsigned n_active = __popc(__ballot_sync(FULL, lead));   // rows with data
        if (lane == 0) {
            for (int st = 0; st < NS; ++st) mbar_init(&bars[st], 1);
            mbar_init_fence();
        }
        __syncwarp();
        auto issue = [&](int g) {
            const int st = g % NS;
            const int w0 = g * G;
            if constexpr (TMA == 2) {
                // one tile for the warp's RW rows: each row's G windows and the rest of
                // its pitch (the next samples, or zeros past the row), the whole box
                // counted whatever lies outside the tensor.  A tile copy needs a 128-byte
                // aligned destination (RW * pitch is one for RW a multiple of 8, which
                // the host requires); one that is not is skipped and flagged, and its
                // stage wait then gives up
                if (lane == 0) {
                    unsigned char *dst = wbuf + (size_t)st * RW * a.pitch;
                    mbar_arrive_expect_tx(&bars[st], RW * a.pitch + a.tx_extra);
                    if ((smem_u32(dst) & 127u) == 0)
                        tma_load_2d(dst, tmap, w0 * a.M * (SB / 8), (int)(group * RW),
                                    &bars[st]);
                    else
                        atomicOr(a.err, 4);
                }
                __syncwarp();
                return;
            }
            const unsigned bytes = (unsigned)(min(G, a.nwin - w0) * a.M * SB);
            if (lane == 0) mbar_arrive_expect_tx(&bars[st], bytes * n_active + a.tx_extra);
            __syncwarp();
            // (a copy skipped by the debug-bounds check leaves its stage wait to time out)
            if (lead && rfi_in(rp + (size_t)w0 * a.M * SB, bytes, a.vis, vis_ext, a.err))
                tma_load_1d(wbuf + ((size_t)st * RW + r) * a.pitch, rp + (size_t)w0 * a.M * SB,
                            bytes, &bars[st]);
        };
        for (int g = 0; g < min(NS, ngroups); ++g) issue(g);
        int g = 0;
        for (; g < ngroups; ++g) {
            const int st = g % NS;
            bool ok = mbar_wait_bounded(&bars[st], (unsigned)((g / NS) & 1), a.wait_limit);
            ok = __all_sync(FULL, ok);
            if (!ok) {
                if (lane == 0) atomicOr(a.err, 1);
                break;
            }
            const unsigned char *sp = wbuf + ((size_t)st * RW + r) * a.pitch + j * UB;
            const int nw = min(G, a.nwin - g * G);
            for (int wi = 0; wi < nw; ++wi) {
                for (int q = 0; q < nch; ++q) {
                    Unit<UB> u[CH];
#pragma unroll
                    for (int c = 0; c < CH; ++c)
                        load_unit_smem(sp + (q * CH + c) * (P * UB), u[c]);
                    consume(u);
                }
                end_window();
                sp += wbytes;
            }
            __syncwarp();
            fence_proxy_async();           // our reads of this stage precede its refill
            if (g + NS < ngroups) issue(g + NS);
        }
        if (g < ngroups) {
            // a wait gave up: let the copies still in flight land (again bounded)
            // before the warp leaves, so no copy targets shared memory of an exited CTA
            for (int h = g; h < min(ngroups, g + NS); ++h)
                mbar_wait_bounded(&bars[h % NS], (unsigned)((h / NS) & 1), a.wait_limit);
            return;
        }
    } else if constexpr (DB) {
        for (int q = q0; q < Q; q += 2) {
            if (q + 1 < Q) load_chunk(q + 1, ub);
            consume(ua);
            if (++cw == nch) { cw = 0; end_window(); }
            if (q + 1 >= Q) break;
            if (q + 2 < Q) load_chunk(q + 2, ua);
            consume(ub);
            if (++cw == nch) { cw = 0; end_window(); }
        }
    } else {
        for (int q = q0; q < Q; ++q) {
            if (q > q0) load_chunk(q, ua);
            consume(ua);
            if (++cw == nch) { cw = 0; end_window(); }
        }
    }
    // a last, partly filled flag word (nwin M not a multiple of 32)
    if (nbits & 31) {
        if (lead && rfi_in(fl_row + (nbits >> 5), 4, a.flags, flags_ext, a.err))
            fl_row[nbits >> 5] = fword;
    }
    // samples after the last whole window (window frame [max(nbits, phase), phase + T))
    // wait in the raw-sample carry for the next block; the window-0 loads above were
    // consumed before the row's lanes synchronised in end_window
    if (PW && !TMA && a.phase + a.T > nbits) {
        __syncwarp();
        const int s0 = max(nbits, a.phase);
        const uint4 *src = reinterpret_cast<const uint4 *>(fp + (long long)s0 * SB);
        uint4 *dst = reinterpret_cast<uint4 *>(hwp + (long long)(s0 - nbits) * SB);
        const int n16 = (a.phase + a.T - s0) * (SB / 16);
        if (active && rfi_in(src, 16ll * n16, a.vis, vis_ext, a.err) &&
            rfi_in(dst, 16ll * n16, a.hw, hw_ext, a.err))
            for (int k = j; k < n16; k += P) dst[k] = src[k];
    }
    if (wib != 0 && active && rfi_in(a.carry + (row * P + j) * 9, 36, a.carry, carry_ext, a.err)) {
        float *cp = a.carry + (row * P + j) * 9;
#pragma unroll
        for (int c = 0; c < 8; ++c) cp[c] = acc[c];
        cp[8] = cnt;
    }
}

// ---- kernels ---------------------------------------------------------------------
// Launch overlap (programmatic dependent launch).  Every flagging kernel executes
// griddepcontrol.launch_dependents on entry, so that the launch after it on the stream
// may begin once all of its blocks have started.  A launch made with the attribute
// calls this before anything else: until the grid before it has completed it only
// requests the first ovl_bytes of the warp's rows into L2 (a hint; L2 is where all of
// the GPU's writes meet, so this is safe whatever that grid writes); then it waits for
// that grid, after which its writes are visible.  For a launch without the attribute
// the wait returns at once.  A launch the host marked independent (a.indep) shares no
// buffer with the launches that may still be running and starts its work at once.
template <int DT, int P>
__device__ __forceinline__ void overlap_prologue(const StreamArgs &a, long long group) {
    if (a.indep) return;
    if (a.ovl_bytes > 0) {
        const int lane = threadIdx.x & 31;
        const int SB = DT == DT_F32 ? 32 : 16;
        const long long row = min(group * (32 / P) + lane / P, a.R - 1);
        const long long rb = (long long)a.T * SB;
        const char *rp = static_cast<const char *>(a.vis) + row * rb;
        const long long n = min((long long)a.ovl_bytes, rb);
        if (rfi_in(rp, n, a.vis, a.R * rb, a.err)) prefetch_rows<P>(rp, n, lane & (P - 1));
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// LB selects the register budget through the launch bounds: 0 -> at most 128
// registers (blocks up to 512 threads), 1 -> 80 (256 threads, 3 blocks per SM),
// 2 -> 64 (256 threads, 4 blocks per SM), 3 -> 96 (128 threads, 5 blocks per SM: 20
// resident warps with two chunks of at most 2 load units in flight per lane).  The
// arithmetic, hence every result, is the same for all budgets; only residency changes.
template <int LB> struct Bounds;
template <> struct Bounds<0> { static constexpr int threads = 512, blocks = 1; };
template <> struct Bounds<1> { static constexpr int threads = 256, blocks = 3; };
template <> struct Bounds<2> { static constexpr int threads = 256, blocks = 4; };
template <> struct Bounds<3> { static constexpr int threads = 128, blocks = 5; };

template <int DT, int SPU, int P, int CH, bool KAHAN, int LB = 0, int PREC = 0,
          bool VS = false, bool PW = false, bool AD = false, bool PFT = false>
__global__ void __launch_bounds__(Bounds<LB>::threads, Bounds<LB>::blocks)
    k_block(const __grid_constant__ StreamArgs a) {
    asm volatile("griddepcontrol.launch_dependents;");
    const long long group = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (group * (32 / P) >= a.R) return;     // whole warp leaves together
    overlap_prologue<DT, P>(a, group);
    // the 128- and 96-register budgets keep two chunks in flight; tighter budgets load
    // one chunk at a time and rely on more resident warps instead
    process_group<DT, SPU, P, CH, KAHAN, LB == 0 || LB == 3, PREC, false, VS, PW, AD, PFT>(a,
                                                                                       group);
}

// P lanes per row, rows staged in shared memory by TMA bulk copies; dynamic shared
// memory = round_up(8 * warps * stages, 128) + warps * stages * (32/P) * pitch bytes.
// Without register buffers for loads in flight, tighter register budgets (LB) leave
// room for more resident warps.
template <int DT, int SPU, int P, int CH, bool KAHAN, int LB = 0>
__global__ void __launch_bounds__(Bounds<LB>::threads, Bounds<LB>::blocks)
    k_tma(const __grid_constant__ StreamArgs a) {
    const long long group = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (group * (32 / P) >= a.R) return;     // whole warp leaves together
    process_group<DT, SPU, P, CH, KAHAN, false, false, 1>(a, group);
}

// The same staged loader with one TMA tile copy per warp and stage (tmap: the block's
// rows as a 2-D tensor of 8-byte elements, box = pitch bytes x 32/P rows), instead of
// one bulk copy per row; the same shared-memory layout, so the same results.
template <int DT, int SPU, int P, int CH, bool KAHAN, int LB = 0>
__global__ void __launch_bounds__(Bounds<LB>::threads, Bounds<LB>::blocks)
    k_tma2(const __grid_constant__ StreamArgs a, const __grid_constant__ CUtensorMap tmap) {
    const long long group = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (group * (32 / P) >= a.R) return;     // whole warp leaves together
    process_group<DT, SPU, P, CH, KAHAN, false, false, 2>(a, group, &tmap);
}

// The tile-copy variant of an instance of the staged loader (built without Kahan).
template <int DT, int SPU, int P, int CH, int K, int LB>
inline const void *tma2_fn() {
    if constexpr (K == 0) return (const void *)&k_tma2<DT, SPU, P, CH, false, LB>;
    else return nullptr;
}

// Persistent batch: every warp takes (stream, row group) tasks from a device counter
// until none is left, claiming its next task when it starts one; the last block to
// finish resets the counter for the next launch in stream order.
// The task loop of a persistent batch launch: every warp calls task(stream, group) for
// (stream, row group) tasks taken from the device counter until none is left.
template <class Task>
__device__ __forceinline__ void run_batch_tasks(const BatchArgs &b, Task &&task) {
    const int lane = threadIdx.x & 31;
    unsigned long long tn = 0;
    if (lane == 0) tn = atomicAdd(b.counter, 1ull);
    for (;;) {
        unsigned long long t = __shfl_sync(FULL, tn, 0);
        if ((long long)t >= b.total) break;
        // claim the next task now: the atomic's round trip hides behind this task
        // (measured on the 8-subband batch: 523 -> 501 us)
        if (lane == 0) tn = atomicAdd(b.counter, 1ull);
        // stream i = number of streams whose next-stream prefix is <= t
        int i = 0;
        for (int base = 0; base < b.n; base += 32) {
            const int k = base + lane;
            const bool le = k < b.n && b.prefix[k + 1] <= (long long)t;
            i += __popc(__ballot_sync(FULL, le));
        }
        task(b.s[i], (long long)t - b.prefix[i]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned int *done = reinterpret_cast<unsigned int *>(b.counter + 1);
        const unsigned int prev = atomicAdd(done, 1u);
        if (prev == gridDim.x - 1) {
            atomicExch(b.counter, 0ull);
            atomicExch(done, 0u);
        }
    }
}

template <int DT, int SPU, int P, int CH, bool KAHAN, int PREC = 0, bool PW = false,
          bool AD = false, bool PFT = false>
__global__ void __launch_bounds__(512, 1) k_batch(const __grid_constant__ BatchArgs b) {
    run_batch_tasks(b, [](const StreamArgs &a, long long group) {
        process_group<DT, SPU, P, CH, KAHAN, true, PREC, false, false, PW, AD, PFT, true>(a,
                                                                                      group);
    });
}

}  // namespace rfi
