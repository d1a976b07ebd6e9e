// rfi_wpar.cuh -- window-parallel lanes: the P lanes of a row take whole windows in
// turn (lane j evaluates the stream's windows g with g mod P = j) instead of splitting
// every window's load units.
//
// For small windows (few samples per lane per window) and T x F footprints this keeps
// the per-window work (butterfly, statistics, flag bits, stores) at one evaluation per
// window with no butterfly over the row's lanes, like one lane per row, while a warp
// holds 32/P rows instead of 32, so a launch is cut into P times more, shorter tasks
// (one lane per row left 1.65 waves of 32-row tasks on the LOFAR-scale block).  The
// arithmetic of a window is that of process_group with P = 1 (the same per-sample
// sums in the same order, then the footprint butterfly over the F rows, here on packed
// pairs: measured 12 % faster for the binary16-arithmetic 5 x 4 footprints; the sum of
// squares under r may round its last bit differently); the averaging sums of a bin
// are kept per lane (the lane's windows) and added over the P lanes when the bin
// closes, so results differ from the other lane splits only by the order of those
// additions (and r's rounding), and any split of a stream at multiples of M is
// bit-identical to one block (window ownership follows the stream's window index), as
// is a batch (k_batch_wp runs the same routine per task).
#pragma once
#include "rfi_device.cuh"

namespace rfi {

// PREC 1: the paper's trained mixed precision (Tables 3 and 4): each window is still
// summed sample by sample in one lane, in the tables' order, so statistics and flags
// are those of the one-lane-per-row mixed kernel bit for bit (time-only windows).
// PREC 2: binary16 Stokes arithmetic (accumulate_h2), as in process_group.
// FS: a round's P windows span at most 32 flag bits (P M <= 32): a whole round's flag
// bits are placed with one shift, across a word boundary where windows straddle flag
// words, and a round at an end of the block keeps only the bits of its windows inside
// the block (the host picks these instances for such shapes only; compiled into every
// kernel, the code cost the other shapes 2-3 %).  FS = 2: every round of the launch is
// whole (the host takes these instances for a launch whose first window is lane 0's and
// whose window count is a multiple of P), so the clamps at the block's ends are left out.
template <int DT, int SPU, int P, int CH, int PREC = 0, int FS = 0>
__device__ __forceinline__ void process_group_wp(const StreamArgs &a, long long group) {
    constexpr bool MIXED = PREC == 1, H2 = PREC == 2;
    static_assert(P >= 2, "one lane per row is the plain kernel");
    static_assert(!H2 || DT == DT_F16, "binary16 Stokes arithmetic needs binary16 input");
    constexpr int RW = 32 / P;
    constexpr int SB = (DT == DT_F32) ? 32 : 16;
    constexpr int UB = SB * SPU;
    const int lane = threadIdx.x & 31;
    const int j = lane & (P - 1);
    const int r = lane / P;                          // the lane's row in the warp
    const long long row = group * RW + r;
    const bool active = row < a.R;
    const long long rowc = active ? row : a.R - 1;
    const int MU = a.M / SPU;                        // load units per window
    const long long WB = (long long)a.M * SB;        // bytes per window of one row
    const char *rp = static_cast<const char *>(a.vis) + rowc * (long long)a.T * SB;
    const long long vis_ext = a.R * (long long)a.T * SB;
    const long long carry_ext = a.R * P * 9 * 4ll;
    const long long stats_ext = (2 * a.stats_plane + (a.R / a.F) * a.nwin) * 4ll;
    const long long flags_ext = a.R * a.Wpr * 4ll;

    // windows of this launch are local indices 0..nwin-1, global g0 + i; lane j owns the
    // windows with g mod P = j.  Round k covers the P windows kP - s .. kP - s + P - 1
    // (s = g0 mod P, from the host), lane j the window kP - s + j.
    const int s = a.wphase;
    const int NR = (a.nwin + s + P - 1) / P;                  // rounds
    const int wpbin = a.K / a.M;                              // windows per bin (>= P)
    int wib = a.bin_pos0 / a.M;                               // windows of the open bin seen
    int bin = 0;

    float2 acc[4];
    float cnt = 0.f;
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[c] = make_float2(0.f, 0.f);
    if (a.bin_pos0 != 0) {
        const float *cp = a.carry + (rowc * P + j) * 9;
        if (rfi_in(cp, 36, a.carry, carry_ext, a.err)) {
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[c] = make_float2(cp[2 * c], cp[2 * c + 1]);
            cnt = cp[8];
        }
    }
    float *const st_row = a.stats + (rowc / a.F) * a.nwin;
    const bool st_lead = active && (row % a.F) == 0;
    const int PF = P * a.F;
    uint32_t *const fl_row = a.flags + rowc * a.Wpr;
    const bool lead = active && j == 0;
    const long long plane = a.stats_plane;
    const int fmode = (32 % a.M == 0) ? 0 : ((a.M % 32 == 0) ? 1 : 2);
    const uint32_t wmask = a.M >= 32 ? FULL : ((1u << a.M) - 1u);
    const int words_per_window = a.M >> 5;
    uint32_t fword = 0;
    const int nbits = a.T;
    const float2 eps2 = make_float2(a.eps, a.eps);
    const float e2 = a.eps * a.eps;

    // the lane's load stream: chunk c of round k reads units c*CH .. c*CH + CH-1 of its
    // window kP - s + j (nothing for a window outside this launch)
    const int nch = MU / CH;
    const int Q = NR * nch;
    auto load_chunk = [&](int k, int c, Unit<UB>(&u)[CH]) {
        const int i = k * P - s + j;
        const bool ok = i >= 0 && i < a.nwin;
        const char *p0 = rp + (long long)i * WB + (long long)c * CH * UB;
#pragma unroll
        for (int e = 0; e < CH; ++e) {
            const char *p = p0 + e * UB;
            if (ok && rfi_in(p, UB, a.vis, vis_ext, a.err)) load_unit_wp(p, u[e]);
            else u[e] = Unit<UB>{};
        }
    };
    WinAcc A;
    const float2 zero2 = make_float2(0.f, 0.f);
    A.s = A.c = A.q = A.u = A.v = zero2;
#pragma unroll
    for (int c = 0; c < 4; ++c) A.a[c] = zero2;
    auto consume = [&](const Unit<UB>(&u)[CH]) {
#pragma unroll
        for (int c = 0; c < CH; ++c)
#pragma unroll
            for (int k = 0; k < SPU; ++k) {
                if constexpr (MIXED)
                    accumulate_mixed(A, stokes_of<DT, UB>(u[c], k), a.eps);
                else if constexpr (H2)
                    accumulate_h2<false>(A, &u[c].r[4 * k], e2);
                else
                    accumulate<false>(A, stokes_of<DT, UB>(u[c], k), eps2);
            }
    };
    auto end_round = [&](int k) {
        const int i = k * P - s + j;                 // this lane's window
        const bool ok = i >= 0 && i < a.nwin;
        float2 ws = A.s, wq = A.q, wu = A.u, wv = A.v;
        if (!MIXED && PF > P) {                      // the footprint's F rows
#pragma unroll
            for (int o = P; o < 32; o <<= 1) {
                if (o < PF) {
                    ws = add2(ws, shfl_xor2(ws, o));
                    wq = add2(wq, shfl_xor2(wq, o));
                    wu = add2(wu, shfl_xor2(wu, o));
                    wv = add2(wv, shfl_xor2(wv, o));
                }
            }
        }
        const float S1 = ws.x, S2 = ws.y;
        float tau, r_re, r_im;
        bool f;
        if constexpr (MIXED) {
            f = finish_mixed(a, S1, S2, wq.x, wu.x, wv.x, wq.y, wu.y, wv.y, tau, r_re, r_im);
        } else {
            // Table 1 groups 6-7 / Sec. 2.1 and Table 2 groups 5-6 / Sec. 2.2
            tau = a.c0 * (a.fM * S2 * rcp_approx(S1 * S1 + a.eps) - 1.0f);
            const float2 n2 = fma2(wv, wv, fma2(wu, wu, mul2(wq, wq)));
            r_re = sqrt_approx(n2.x) * a.invM;
            r_im = sqrt_approx(n2.y) * a.invM;
            f = !(tau >= a.s_low && tau <= a.s_high) || !(r_re <= a.gamma) ||
                !(r_im <= a.gamma);
        }
        if (ok && st_lead && rfi_in(st_row + i, 4, a.stats, stats_ext, a.err) &&
            rfi_in(st_row + i + 2 * plane, 4, a.stats, stats_ext, a.err)) {
            st_row[i] = tau;
            st_row[i + plane] = r_re;
            st_row[i + 2 * plane] = r_im;
        }
        // the row's P window flags of this round, in window order, to its lead lane
        const unsigned fb = __ballot_sync(FULL, ok && f);
        const unsigned rowbits = (fb >> (r * P)) & ((1u << P) - 1u);
        auto flag_each = [&]() {
#pragma unroll
            for (int e = 0; e < P; ++e) {
                const int wi = k * P - s + e;            // window of lane e of the row
                if (wi < 0 || wi >= a.nwin) continue;
                const bool fe = (rowbits >> e) & 1u;
                if (fmode == 0) {
                    const int b0 = (wi * a.M) & 31;
                    if (fe) fword |= wmask << b0;
                    if (b0 + a.M == 32) {
                        uint32_t *w = fl_row + ((wi * a.M) >> 5);
                        if (lead && rfi_in(w, 4, a.flags, flags_ext, a.err)) *w = fword;
                        fword = 0;
                    }
                } else if (fmode == 1) {
                    const int w0 = (wi * a.M) >> 5;
                    if (lead &&
                        rfi_in(fl_row + w0, 4ll * words_per_window, a.flags, flags_ext, a.err))
                        for (int q = 0; q < words_per_window; ++q) fl_row[w0 + q] = fe ? FULL : 0u;
                } else {
                    int lo = wi * a.M;
                    const int hi = lo + a.M;
                    while (lo < hi) {
                        const int b0 = lo & 31;
                        const int nb = min(hi - lo, 32 - b0);
                        if (fe) fword |= (nb == 32 ? FULL : ((1u << nb) - 1u)) << b0;
                        lo += nb;
                        if ((lo & 31) == 0) {
                            uint32_t *w = fl_row + ((lo - 1) >> 5);
                            if (lead && rfi_in(w, 4, a.flags, flags_ext, a.err)) *w = fword;
                            fword = 0;
                        }
                    }
                }
            }
        };
        if constexpr (FS != 0) {
            // a round's P windows, P M <= 32 bits spread from the P flags, placed with one
            // shift (they straddle at most one word boundary).  A round at either end of
            // the block keeps only its windows inside the block: before window 0 the
            // bits are shifted out, after the block's last sample the word is left open
            // for the store after the loop (FS = 2: every round is whole)
            uint32_t m = 0;
#pragma unroll
            for (int e = 0; e < P; ++e)
                if ((rowbits >> e) & 1u) m |= wmask << (e * a.M);
            int lo = (k * P - s) * a.M;
            int span = P * a.M;
            if constexpr (FS == 1) {
                if (lo < 0) {
                    m >>= -lo;
                    span += lo;
                    lo = 0;
                }
                span = min(span, nbits - lo);
            }
            const int b0 = lo & 31;
            const unsigned long long m64 = (unsigned long long)m << b0;
            fword |= (uint32_t)m64;
            if (b0 + span >= 32) {
                if (lead && rfi_in(fl_row + (lo >> 5), 4, a.flags, flags_ext, a.err))
                    fl_row[lo >> 5] = fword;
                fword = (uint32_t)(m64 >> 32);
            }
        } else {
            flag_each();
        }
        // flagged samples leave the average (end of Sec. 2.1).  The open bin needs
        // wpbin - wib more windows: the round's windows [first, e) belong to it; if the
        // bin closes in this round (at most once: a bin holds at least P windows), the
        // rest open the next one
        const bool add = ok && !f;
        auto add_window = [&]() {
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[c] = add2(acc[c], A.a[c]);
            cnt += (float)a.M;
        };
        const int first = max(k * P - s, 0), last = min(k * P - s + P, a.nwin);
        const int e = first + (wpbin - wib);
        if (last < e) {
            if (add) add_window();
            wib += last - first;
        } else {
            if (add && i < e) add_window();
            float tot[8];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float2 t = allsum2<P>(acc[c]);
                tot[2 * c] = t.x;
                tot[2 * c + 1] = t.y;
            }
            const float n = allsum<P>(cnt);
            if constexpr (H2) tot[7] = -tot[7];      // V was carried as (Re V, -Im V)
            if (lead) store_bin(a, row, bin, tot, n);
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[c] = make_float2(0.f, 0.f);
            cnt = 0.f;
            ++bin;
            if (add && i >= e) add_window();
            wib = last - e;
        }
        A.s = A.q = A.u = A.v = zero2;
#pragma unroll
        for (int c = 0; c < 4; ++c) A.a[c] = zero2;
    };

    Unit<UB> ua[CH], ub[CH];
    int kl = 0, cl = 0;                              // next chunk to load (round, chunk)
    int kc = 0, cc = 0;                              // chunk being consumed
    auto advance = [&](int &k, int &c) {
        if (++c == nch) { c = 0; ++k; }
    };
    if (Q > 0) { load_chunk(kl, cl, ua); advance(kl, cl); }
    for (int q = 0; q < Q; q += 2) {
        if (q + 1 < Q) { load_chunk(kl, cl, ub); advance(kl, cl); }
        consume(ua);
        if (cc + 1 == nch) end_round(kc);
        advance(kc, cc);
        if (q + 1 >= Q) break;
        if (q + 2 < Q) { load_chunk(kl, cl, ua); advance(kl, cl); }
        consume(ub);
        if (cc + 1 == nch) end_round(kc);
        advance(kc, cc);
    }
    if (nbits & 31) {
        if (lead && rfi_in(fl_row + (nbits >> 5), 4, a.flags, flags_ext, a.err))
            fl_row[nbits >> 5] = fword;
    }
    if (wib != 0 && active && rfi_in(a.carry + (row * P + j) * 9, 36, a.carry, carry_ext, a.err)) {
        float *cp = a.carry + (row * P + j) * 9;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            cp[2 * c] = acc[c].x;
            cp[2 * c + 1] = acc[c].y;
        }
        cp[8] = cnt;
    }
}

// LB: the register budget (Bounds in rfi_device.cuh): 0 = 128 registers, 3 = 96 (20
// resident warps per SM; built for the binary16 odd windows, which fit it unspilled).
template <int DT, int SPU, int P, int CH, int PREC = 0, int FS = 0, int LB = 0>
__global__ void __launch_bounds__(Bounds<LB>::threads, Bounds<LB>::blocks)
    k_wpar(const __grid_constant__ StreamArgs a) {
    asm volatile("griddepcontrol.launch_dependents;");
    const long long group = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (group * (32 / P) >= a.R) return;     // whole warp leaves together
    overlap_prologue<DT, P>(a, group);
    process_group_wp<DT, SPU, P, CH, PREC, FS>(a, group);
}

// The persistent batch over window-parallel contexts (same task loop as k_batch).
template <int DT, int SPU, int P, int CH, int PREC = 0, int FS = 0>
__global__ void __launch_bounds__(512, 1) k_batch_wp(const __grid_constant__ BatchArgs b) {
    run_batch_tasks(b, [](const StreamArgs &a, long long group) {
        process_group_wp<DT, SPU, P, CH, PREC, FS>(a, group);
    });
}

}  // namespace rfi
