// rfi_sliding.cuh -- overlapping (sliding) windows on sm_103a.
//
// An extension of the method: the paper's windows (Sec. 2) are consecutive and do not
// overlap.  Here a window of M samples starts every H samples (H divides M), so every
// sample lies in L = M / H windows.  Each window's statistics and flag are those of
// Secs. 2.1 and 2.2 on its M samples; a sample is flagged when any window that holds it
// is flagged, and becomes final (flag known, averaged) once the last window holding it
// has been evaluated, M - H samples after it.
//
// Work split and loads are those of process_group with the window replaced by a
// segment of H samples: lane j of a row loads units j, j+P, ... of each segment.  At
// the end of every segment the P lanes complete the segment's eight statistic sums with
// the xor butterfly (the same cost as one butterfly per window, since a window ends with
// every segment), and the window that ends there is the sum of the last L segment
// totals, oldest first.  The totals of the L-1 segments before the current one, and the
// lane's averaging sums of those segments (their flags are not known yet), live in
// registers and, at the end of a block, in the context's carry, so any split of a
// stream at multiples of H gives bit-identical results, alone or in a batch.
#pragma once
#include "rfi_device.cuh"

namespace rfi {

template <int DT, int SPU, int P, int CH, int L>
__device__ __forceinline__ void process_group_sw(const StreamArgs &a, long long group) {
    static_assert(L >= 2, "overlapping windows need at least two windows per sample");
    constexpr int LM = L - 1;
    constexpr int RW = 32 / P;
    constexpr int SB = (DT == DT_F32) ? 32 : 16;
    constexpr int UB = SB * SPU;
    const int lane = threadIdx.x & 31;
    const int j = lane & (P - 1);
    const long long row = group * RW + lane / P;
    const bool active = row < a.R;
    const long long rowc = active ? row : a.R - 1;
    const bool lead = active && j == 0;
    const int H = a.hop;
    const int S = H / (P * SPU);                    // load units per lane per segment
    const char *rp = static_cast<const char *>(a.vis) + rowc * (long long)a.T * SB;
    const long long vis_ext = a.R * (long long)a.T * SB;
    const long long carry_ext = a.R * P * 9 * 4ll;
    const long long stats_ext = (2 * a.stats_plane + a.R * a.nwin) * 4ll;
    const long long flags_ext = a.R * a.Wpr * 4ll;
    const long long tot_ext = a.R * LM * 32ll;
    const long long pend_ext = a.R * P * LM * 32ll;
    const long long hist_ext = a.R * 4ll;

    // carried state: segment totals and the lane's averaging sums of the pending
    // segments (oldest first), and the flags of the last L-1 windows
    float rt[LM][8], ra[LM][8];
    uint32_t hist = 0;
    {
        const float *tp = a.sw_tot + rowc * (LM * 8);
        const float *pp = a.sw_pend + (rowc * P + j) * (LM * 8);
        const bool ok = rfi_in(tp, LM * 32, a.sw_tot, tot_ext, a.err) &&
                        rfi_in(pp, LM * 32, a.sw_pend, pend_ext, a.err) &&
                        rfi_in(a.sw_hist + rowc, 4, a.sw_hist, hist_ext, a.err);
#pragma unroll
        for (int k = 0; k < LM; ++k)
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                rt[k][c] = ok ? tp[k * 8 + c] : 0.f;
                ra[k][c] = ok ? pp[k * 8 + c] : 0.f;
            }
        hist = ok ? a.sw_hist[rowc] : 0u;
    }
    float acc[8];
    float cnt = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = 0.f;
    if (a.bin_pos0 != 0) {
        const float *cp = a.carry + (rowc * P + j) * 9;
        if (rfi_in(cp, 36, a.carry, carry_ext, a.err)) {
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[c] = cp[c];
            cnt = cp[8];
        }
    }
    float *const st_row = a.stats + rowc * a.nwin;
    uint32_t *const fl_row = a.flags + rowc * a.Wpr;
    const long long plane = a.stats_plane;
    const int spb = a.K / H;                        // segments per averaging bin
    int wib = a.bin_pos0 / H;                       // final segments of the open bin
    int bin = 0;
    const float lane_samples = (float)(S * SPU);
    // flag words, as for windows but per segment of H samples
    const int fmode = (32 % H == 0) ? 0 : ((H % 32 == 0) ? 1 : 2);
    const uint32_t hmask = H >= 32 ? FULL : ((1u << H) - 1u);
    const int words_per_seg = H >> 5;
    uint32_t fword = 0;
    int fbit = 0, fwi = 0;
    const int nbits = a.nwin * H;
    int seen = a.warm;                              // segments before, up to L - 1
    int w = 0;                                      // windows completed in this launch

    const float2 eps2 = make_float2(a.eps, a.eps);
    constexpr int CHB = CH * P * UB;
    const int nch = S / CH;
    const int Q = (a.T / H) * nch;
    const char *cp_ = rp + j * UB;
    auto load_chunk = [&](int q, Unit<UB>(&u)[CH]) {
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
    auto consume = [&](const Unit<UB>(&u)[CH]) {
#pragma unroll
        for (int c = 0; c < CH; ++c)
#pragma unroll
            for (int k = 0; k < SPU; ++k) accumulate<false>(A, stokes_of<DT, UB>(u[c], k), eps2);
    };
    auto end_segment = [&]() {
        // the segment's totals over the row's P lanes (bit-identical on every lane)
        float tot[8] = {allsum<P>(A.s.x), allsum<P>(A.s.y), allsum<P>(A.q.x), allsum<P>(A.u.x),
                        allsum<P>(A.v.x), allsum<P>(A.q.y), allsum<P>(A.u.y), allsum<P>(A.v.y)};
        float as[8];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            as[2 * c] = A.a[c].x;
            as[2 * c + 1] = A.a[c].y;
        }
        if (seen >= LM) {
            // the window of the last L segments is complete: sums oldest first
            float ws[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                float v = rt[0][c];
#pragma unroll
                for (int k = 1; k < LM; ++k) v += rt[k][c];
                ws[c] = v + tot[c];
            }
            const float S1 = ws[0], S2 = ws[1];
            // Sec. 2.1 / Table 1 groups 5-7, Sec. 2.2 / Table 2 groups 5-6, as for a window
            // that does not overlap another
            const float tau = a.c0 * (a.fM * S2 * rcp_approx(S1 * S1 + a.eps) - 1.0f);
            const float r_re = sqrt_approx(ws[2] * ws[2] + ws[3] * ws[3] + ws[4] * ws[4]) * a.invM;
            const float r_im = sqrt_approx(ws[5] * ws[5] + ws[6] * ws[6] + ws[7] * ws[7]) * a.invM;
            const bool fw = !(tau >= a.s_low && tau <= a.s_high) || !(r_re <= a.gamma) ||
                            !(r_im <= a.gamma);
            if (lead && rfi_in(st_row + w, 4, a.stats, stats_ext, a.err) &&
                rfi_in(st_row + w + 2 * plane, 4, a.stats, stats_ext, a.err)) {
                st_row[w] = tau;
                st_row[w + plane] = r_re;
                st_row[w + 2 * plane] = r_im;
            }
            // the oldest pending segment is final: flagged if any of its L windows is
            const bool fs = fw || (hist & ((1u << LM) - 1u)) != 0u;
            hist = (hist << 1) | (fw ? 1u : 0u);
            if (fmode == 0) {
                if (fs) fword |= hmask << fbit;
                fbit += H;
                if (fbit == 32) {
                    if (lead && rfi_in(fl_row + fwi, 4, a.flags, flags_ext, a.err))
                        fl_row[fwi] = fword;
                    ++fwi;
                    fword = 0;
                    fbit = 0;
                }
            } else if (fmode == 1) {
                if (lead && rfi_in(fl_row + fwi, 4ll * words_per_seg, a.flags, flags_ext, a.err))
                    for (int k = 0; k < words_per_seg; ++k) fl_row[fwi + k] = fs ? FULL : 0u;
                fwi += words_per_seg;
            } else {
                int lo = w * H;
                const int hi = lo + H;
                while (lo < hi) {
                    const int b0 = lo & 31;
                    const int nb = min(hi - lo, 32 - b0);
                    if (fs) fword |= (nb == 32 ? FULL : ((1u << nb) - 1u)) << b0;
                    lo += nb;
                    if ((lo & 31) == 0) {
                        if (lead && rfi_in(fl_row + ((lo - 1) >> 5), 4, a.flags, flags_ext, a.err))
                            fl_row[(lo - 1) >> 5] = fword;
                        fword = 0;
                    }
                }
            }
            // flagged samples are left out of the average (end of Sec. 2.1)
            if (!fs) {
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[c] += ra[0][c];
                cnt += lane_samples;
            }
            if (++wib == spb) {
                float t8[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) t8[c] = allsum<P>(acc[c]);
                const float n = allsum<P>(cnt);
                if (lead) store_bin(a, row, bin, t8, n);
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[c] = 0.f;
                cnt = 0.f;
                wib = 0;
                ++bin;
            }
            ++w;
        } else {
            ++seen;
        }
        // this segment joins the pending ones
#pragma unroll
        for (int k = 0; k + 1 < LM; ++k)
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                rt[k][c] = rt[k + 1][c];
                ra[k][c] = ra[k + 1][c];
            }
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            rt[LM - 1][c] = tot[c];
            ra[LM - 1][c] = as[c];
        }
        A.s = A.q = A.u = A.v = zero2;
#pragma unroll
        for (int c = 0; c < 4; ++c) A.a[c] = zero2;
    };

    Unit<UB> ua[CH], ub[CH];
    int cw = 0;
    if (Q > 0) load_chunk(0, ua);
    for (int q = 0; q < Q; q += 2) {
        if (q + 1 < Q) load_chunk(q + 1, ub);
        consume(ua);
        if (++cw == nch) { cw = 0; end_segment(); }
        if (q + 1 >= Q) break;
        if (q + 2 < Q) load_chunk(q + 2, ua);
        consume(ub);
        if (++cw == nch) { cw = 0; end_segment(); }
    }
    if (nbits & 31) {
        if (lead && rfi_in(fl_row + (nbits >> 5), 4, a.flags, flags_ext, a.err))
            fl_row[nbits >> 5] = fword;
    }
    // carry for the next block
    if (active) {
        float *tp = a.sw_tot + row * (LM * 8);
        float *pp = a.sw_pend + (row * P + j) * (LM * 8);
        if (j == 0 && rfi_in(tp, LM * 32, a.sw_tot, tot_ext, a.err)) {
#pragma unroll
            for (int k = 0; k < LM; ++k)
#pragma unroll
                for (int c = 0; c < 8; ++c) tp[k * 8 + c] = rt[k][c];
        }
        if (rfi_in(pp, LM * 32, a.sw_pend, pend_ext, a.err)) {
#pragma unroll
            for (int k = 0; k < LM; ++k)
#pragma unroll
                for (int c = 0; c < 8; ++c) pp[k * 8 + c] = ra[k][c];
        }
        if (j == 0 && rfi_in(a.sw_hist + row, 4, a.sw_hist, hist_ext, a.err))
            a.sw_hist[row] = hist & ((1u << LM) - 1u);
        if (wib != 0 && rfi_in(a.carry + (row * P + j) * 9, 36, a.carry, carry_ext, a.err)) {
            float *cp = a.carry + (row * P + j) * 9;
#pragma unroll
            for (int c = 0; c < 8; ++c) cp[c] = acc[c];
            cp[8] = cnt;
        }
    }
}

template <int DT, int SPU, int P, int CH, int L>
__global__ void __launch_bounds__(512, 1) k_slide(const __grid_constant__ StreamArgs a) {
    asm volatile("griddepcontrol.launch_dependents;");
    const long long group = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (group * (32 / P) >= a.R) return;     // whole warp leaves together
    overlap_prologue<DT, P>(a, group);
    process_group_sw<DT, SPU, P, CH, L>(a, group);
}

// The persistent batch over overlapping-window contexts (same task loop as k_batch).
template <int DT, int SPU, int P, int CH, int L>
__global__ void __launch_bounds__(512, 1) k_batch_sw(const __grid_constant__ BatchArgs b) {
    run_batch_tasks(b, [](const StreamArgs &a, long long group) {
        process_group_sw<DT, SPU, P, CH, L>(a, group);
    });
}

}  // namespace rfi
