/*
 * rfi_oracle.c -- plain, slow FP64 CPU oracle for the online RFI flagging path of
 * "Energy and polarization based online interference mitigation in radio
 * interferometry" (Yatawatta, Boonstra, Broekema; arXiv 2412.14775).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file: only the tests, the smoke check and the bench's CPU-baseline leg use
 * it.  It shares no code, header, table or constant with the CUDA path.
 *
 * Every quantity is evaluated in double precision, in the order the paper states
 * it, one window at a time, with plain sequential summation (or, on request, a
 * Neumaier-compensated sum used only to bound the oracle's own rounding error).
 *
 * Paper notation: a window holds W samples (called M in the library API).  For one
 * baseline, one channel and time sample i the correlator delivers the 2x2 matrix
 * V_i = [[xx_i, xy_i], [yx_i, yy_i]] (Section 2, Eq. V).
 *
 * Readings of points the paper leaves open (each is listed in the design notes):
 *  - tau follows Section 2.1's equation, (Wd+1)/(W-1) * (W*S2/(S1^2+eps) - 1), with
 *    the eps of Table 1 (group 7) in the denominator.  Table 1's row 7 prints the
 *    "-1" outside the product; only the equation's form has mean 1 under the null.
 *  - eps is one absolute constant, added to S1^2 (Table 1) and to p (Table 2).
 *  - comparisons are strict as printed (tau < s_low, tau > s_high, r > gamma); a
 *    statistic that is NaN is flagged (the comparisons are written in the negated
 *    form "not inside the accepted interval").
 *  - a window flag applies to every sample of the window and to all 4 correlations.
 *  - the output is the mean of the unflagged samples of each averaging bin of K
 *    samples; the weight is (number of unflagged samples) / K; an empty bin gives
 *    value 0 and weight 0.
 *  - windows are consecutive, non-overlapping runs of W samples of one (baseline,
 *    channel) stream, counted from the stream's first sample across blocks.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- Summation (plain sequential, or Neumaier-compensated) -------------------- */
typedef struct { double s, c; } acc_t;

static void acc_add(acc_t *a, double x, int compensated)
{
    if (!compensated) { a->s += x; return; }
    /* Neumaier's improvement of Kahan summation: the rounding error of each add is
     * recovered exactly (TwoSum) and accumulated in c. */
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else                       a->c += (x - t) + a->s;
    a->s = t;
}
static double acc_val(const acc_t *a) { return a->s + a->c; }

/* ---- Section 2, Eq. IQUV: complex Stokes parameters of one sample ------------ */
/* v[8] = re/im of xx, xy, yx, yy (the layout of Eq. V read row by row).
 * s[8] = re/im of I, Q, U, V with
 *   I = xx + yy,  Q = xx - yy,  U = xy + yx,  V = j (xy - yx).                      */
void oracle_stokes(const double v[8], double s[8])
{
    const double xx_re = v[0], xx_im = v[1], xy_re = v[2], xy_im = v[3];
    const double yx_re = v[4], yx_im = v[5], yy_re = v[6], yy_im = v[7];
    s[0] = xx_re + yy_re;            /* Re I */
    s[1] = xx_im + yy_im;            /* Im I */
    s[2] = xx_re - yy_re;            /* Re Q */
    s[3] = xx_im - yy_im;            /* Im Q */
    s[4] = xy_re + yx_re;            /* Re U */
    s[5] = xy_im + yx_im;            /* Im U */
    /* j * (a + jb) = -b + ja, with a + jb = xy - yx */
    s[6] = -(xy_im - yx_im);         /* Re V */
    s[7] = (xy_re - yx_re);          /* Im V */
}

/* ---- Section 2.1 and Table 1: spectral kurtosis of one window ---------------- */
/* stokes: W samples x 8 doubles (output of oracle_stokes).  Returns tau_SK and the
 * moments S1 = sum |I_i|, S2 = sum |I_i|^2. */
double oracle_sk_window(const double *stokes, int W, double d, double eps,
                        int compensated, double *S1_out, double *S2_out)
{
    acc_t S1 = {0, 0}, S2 = {0, 0};
    for (int i = 0; i < W; ++i) {
        const double xr = stokes[8 * i + 0], xi = stokes[8 * i + 1];
        const double y = xr * xr + xi * xi;     /* Table 1 group 1: y = |I|^2 */
        const double z = sqrt(y);               /* Table 1 group 2: z = |I|   */
        acc_add(&S1, z, compensated);           /* Table 1 group 3            */
        acc_add(&S2, y, compensated);           /* Table 1 group 4            */
    }
    const double s1 = acc_val(&S1), s2 = acc_val(&S2);
    if (S1_out) *S1_out = s1;
    if (S2_out) *S2_out = s2;
    const double Wd = (double)W;
    const double lead = (Wd * d + 1.0) / (Wd - 1.0);  /* Table 1 group 5 */
    const double s12 = s1 * s1;                       /* Table 1 group 6 */
    return lead * (Wd * s2 / (s12 + eps) - 1.0);      /* Sec. 2.1 tau_SK, eps of group 7 */
}

/* ---- Section 2.2 and Table 2: directional statistic of one part --------------- */
/* part = 0 uses the real parts of Q, U, V; part = 1 the imaginary parts. */
double oracle_ds_window(const double *stokes, int W, int part, double eps,
                        int compensated, double sums_out[3])
{
    acc_t qs = {0, 0}, us = {0, 0}, vs = {0, 0};
    for (int i = 0; i < W; ++i) {
        const double q = stokes[8 * i + 2 + part];
        const double u = stokes[8 * i + 4 + part];
        const double v = stokes[8 * i + 6 + part];
        const double a = q * q, b = u * u, c = v * v;   /* Table 2 group 1           */
        const double p = sqrt(a + b + c) + eps;         /* group 2: vector length p  */
        acc_add(&qs, q / p, compensated);               /* group 3 (normalise) and   */
        acc_add(&us, u / p, compensated);               /* group 4 (sum over window) */
        acc_add(&vs, v / p, compensated);
    }
    const double q = acc_val(&qs), u = acc_val(&us), v = acc_val(&vs);
    if (sums_out) { sums_out[0] = q; sums_out[1] = u; sums_out[2] = v; }
    const double qb = q * q, ub = u * u, vb = v * v;    /* group 5 */
    return sqrt(qb + ub + vb) / (double)W;              /* group 6: r */
}

/* ---- Flag rule: Sec. 2.1 (SK), Sec. 2.2 (DS, Re OR Im), OR of both ------------- */
int oracle_flag(double tau, double r_re, double r_im,
                double s_low, double s_high, double gamma)
{
    const int f_sk = !(tau >= s_low && tau <= s_high);  /* tau < s_low OR tau > s_high */
    const int f_re = !(r_re <= gamma);                   /* r > gamma (Re part)         */
    const int f_im = !(r_im <= gamma);                   /* r > gamma (Im part)         */
    return f_sk | (f_re | f_im);
}

/* Number of completed averaging bins when a block of T samples follows n_seen. */
long long oracle_outputs_for(long long n_seen, int T, int K)
{
    return (n_seen + T) / K - n_seen / K;
}

/* ---- One block of one stream ----------------------------------------------------
 * vis      [R][T][8] doubles: rows are (baseline, channel) streams, 8 = re/im of
 *          xx, xy, yx, yy.  Rows are mitigated separately (Sec. 2), except that a
 *          window may span F adjacent rows (F channels of one baseline): the paper's
 *          windows are time-frequency footprints of W = T x F samples (Secs. 3.2, 4).
 * Mt       samples per row in a window (the time extent); W = Mt * F.
 * thr      {d, s_low, s_high, gamma, eps}
 * n_seen   samples of this stream already consumed by earlier blocks (multiple of Mt)
 * carry_sum [R][8], carry_cnt [R]: running sum of unflagged samples and their count
 *          in the open averaging bin of every row; read at entry, written at exit.
 * Outputs (caller-allocated):
 *   tau, r_re, r_im, wflag  [R/F][T/Mt]
 *   flagbits                [R][ceil(T/32)]  bit (t mod 32) of word t/32 = flag of sample t
 *   avg                     [R][n_out][8]    mean of unflagged samples of each completed bin
 *   weight                  [R][n_out]       unflagged count / K
 * Returns 0, or -1 on invalid sizes.  */
static int process_block_impl(const double *vis, int R, int T, int Mt, int F, int K,
                              const double thr[5], int compensated, long long n_seen,
                              double *carry_sum, double *carry_cnt, const uint8_t *given,
                              double *tau, double *r_re, double *r_im, uint8_t *wflag,
                              uint32_t *flagbits, double *avg, double *weight)
{
    if (R < 0 || T < 0 || Mt < 1 || F < 1 || Mt * F < 2 || R % F != 0 || K < Mt ||
        T % Mt != 0 || K % Mt != 0 || n_seen % Mt != 0)
        return -1;
    const double d = thr[0], s_low = thr[1], s_high = thr[2], gamma = thr[3], eps = thr[4];
    const int W = Mt * F;                     /* samples in one window */
    const int nwin = T / Mt;
    const int nwords = (T + 31) / 32;
    const int G = R / F;                      /* window rows (channel groups) */
    const long long n_out = oracle_outputs_for(n_seen, T, K);
    const long long first_bin = n_seen / K;
    double *stokes = (double *)malloc(sizeof(double) * 8 * (size_t)W);
    acc_t *bins = (acc_t *)malloc(sizeof(acc_t) * 8 * (size_t)F);
    double *bins_n = (double *)malloc(sizeof(double) * (size_t)F);
    if (!stokes || !bins || !bins_n) {
        free(stokes); free(bins); free(bins_n);
        return -1;
    }

    for (int g = 0; g < G; ++g) {
        for (int k = 0; k < F; ++k) {
            const int row = g * F + k;
            uint32_t *fb = flagbits + (size_t)row * nwords;
            for (int q = 0; q < nwords; ++q) fb[q] = 0;
            /* open-bin running sums continue from the previous block (Kahan state not
             * carried: the carry is the plain value) */
            acc_t *bin = bins + 8 * k;
            for (int c = 0; c < 8; ++c) { bin[c].s = carry_sum[(size_t)row * 8 + c]; bin[c].c = 0; }
            bins_n[k] = carry_cnt[row];
        }
        for (int w = 0; w < nwin; ++w) {
            /* the window's W samples: Mt samples of each of the F rows, row by row */
            for (int k = 0; k < F; ++k) {
                const double *vw = vis + ((size_t)(g * F + k) * T + (size_t)w * Mt) * 8;
                for (int i = 0; i < Mt; ++i) oracle_stokes(vw + 8 * i, stokes + 8 * (k * Mt + i));
            }
            const double t  = oracle_sk_window(stokes, W, d, eps, compensated, 0, 0);
            const double rr = oracle_ds_window(stokes, W, 0, eps, compensated, 0);
            const double ri = oracle_ds_window(stokes, W, 1, eps, compensated, 0);
            const size_t o = (size_t)g * nwin + w;
            /* the window's flag: from its statistics, or the caller's (the flags of
             * another arithmetic, whose averages are wanted) */
            const int f = given ? (given[o] != 0) : oracle_flag(t, rr, ri, s_low, s_high, gamma);

            tau[o] = t; r_re[o] = rr; r_im[o] = ri; wflag[o] = (uint8_t)f;

            const long long g_end = n_seen + (long long)(w + 1) * Mt;   /* stream index */
            for (int k = 0; k < F; ++k) {
                const int row = g * F + k;
                const double *vw = vis + ((size_t)row * T + (size_t)w * Mt) * 8;
                uint32_t *fb = flagbits + (size_t)row * nwords;
                acc_t *bin = bins + 8 * k;
                /* every sample of a flagged window is flagged (Sec. 2.1, last sentence) */
                for (int i = 0; i < Mt; ++i) {
                    const int ts = w * Mt + i;
                    if (f) fb[ts / 32] |= (uint32_t)1u << (ts % 32);
                }
                /* flagged samples are left out of the time average (Sec. 2.1) */
                if (!f) {
                    for (int i = 0; i < Mt; ++i)
                        for (int c = 0; c < 8; ++c) acc_add(&bin[c], vw[8 * i + c], compensated);
                    bins_n[k] += Mt;
                }
                if (g_end % K == 0) {
                    const long long b = g_end / K - 1 - first_bin;          /* output slot */
                    double *ao = avg + ((size_t)row * n_out + b) * 8;
                    const double bin_n = bins_n[k];
                    for (int c = 0; c < 8; ++c) ao[c] = bin_n > 0 ? acc_val(&bin[c]) / bin_n : 0.0;
                    weight[(size_t)row * n_out + b] = bin_n / (double)K;
                    for (int c = 0; c < 8; ++c) { bin[c].s = 0; bin[c].c = 0; }
                    bins_n[k] = 0;
                }
            }
        }
        for (int k = 0; k < F; ++k) {
            const int row = g * F + k;
            for (int c = 0; c < 8; ++c) carry_sum[(size_t)row * 8 + c] = acc_val(&bins[8 * k + c]);
            carry_cnt[row] = bins_n[k];
        }
    }
    free(stokes); free(bins); free(bins_n);
    return 0;
}

int oracle_process_block_tf(const double *vis, int R, int T, int Mt, int F, int K,
                            const double thr[5], int compensated, long long n_seen,
                            double *carry_sum, double *carry_cnt,
                            double *tau, double *r_re, double *r_im, uint8_t *wflag,
                            uint32_t *flagbits, double *avg, double *weight)
{
    return process_block_impl(vis, R, T, Mt, F, K, thr, compensated, n_seen, carry_sum,
                              carry_cnt, 0, tau, r_re, r_im, wflag, flagbits, avg, weight);
}

/* As oracle_process_block_tf, with the window flags given by the caller (given
 * [R/F][T/Mt], nonzero = flagged) instead of taken from the statistics: flag bits and
 * averages follow them (Sec. 2.1: flagged samples leave the time average), and wflag
 * echoes them; the statistics are still those of this oracle. */
int oracle_process_block_given_flags(const double *vis, int R, int T, int Mt, int F, int K,
                                     const double thr[5], int compensated, long long n_seen,
                                     double *carry_sum, double *carry_cnt, const uint8_t *given,
                                     double *tau, double *r_re, double *r_im, uint8_t *wflag,
                                     uint32_t *flagbits, double *avg, double *weight)
{
    if (!given) return -1;
    return process_block_impl(vis, R, T, Mt, F, K, thr, compensated, n_seen, carry_sum,
                              carry_cnt, given, tau, r_re, r_im, wflag, flagbits, avg, weight);
}

/* Time-only windows of W samples per row (F = 1). */
int oracle_process_block(const double *vis, int R, int T, int W, int K,
                         const double thr[5], int compensated, long long n_seen,
                         double *carry_sum, double *carry_cnt,
                         double *tau, double *r_re, double *r_im, uint8_t *wflag,
                         uint32_t *flagbits, double *avg, double *weight)
{
    if (W < 2) return -1;
    return oracle_process_block_tf(vis, R, T, W, 1, K, thr, compensated, n_seen, carry_sum,
                                   carry_cnt, tau, r_re, r_im, wflag, flagbits, avg, weight);
}

/* ---- Overlapping windows (an extension: the paper's windows do not overlap) -------
 * Windows of W samples that start every H samples (H divides W), aligned to the
 * buffer's first sample: window k covers buffer samples [kH, kH + W).  For every row
 * of vis [R][Tb][8] and every window that fits in the buffer, the statistics of
 * Secs. 2.1 and 2.2 and the window's flag, exactly as for a window that does not
 * overlap another (the same W samples, the same order).
 * Outputs tau, r_re, r_im, wflag [R][nk] with nk = Tb >= W ? (Tb - W) / H + 1 : 0, which
 * must equal nk_capacity.  Returns nk, or -1 on invalid sizes (nothing written). */
int oracle_window_stats_hop(const double *vis, int R, int Tb, int W, int H,
                            const double thr[5], int compensated, int nk_capacity,
                            double *tau, double *r_re, double *r_im, uint8_t *wflag)
{
    if (R < 0 || Tb < 0 || W < 2 || H < 1 || W % H != 0) return -1;
    const double d = thr[0], s_low = thr[1], s_high = thr[2], gamma = thr[3], eps = thr[4];
    const int nk = Tb >= W ? (Tb - W) / H + 1 : 0;
    if (nk != nk_capacity) return -1;           /* the caller sized the outputs for nk */
    double *stokes = (double *)malloc(sizeof(double) * 8 * (size_t)(Tb > 0 ? Tb : 1));
    if (!stokes) return -1;
    for (int row = 0; row < R; ++row) {
        const double *v = vis + (size_t)row * Tb * 8;
        for (int i = 0; i < Tb; ++i) oracle_stokes(v + 8 * i, stokes + 8 * (size_t)i);
        for (int k = 0; k < nk; ++k) {
            const double *sw = stokes + 8 * (size_t)k * H;      /* the window's W samples */
            const double t  = oracle_sk_window(sw, W, d, eps, compensated, 0, 0);
            const double rr = oracle_ds_window(sw, W, 0, eps, compensated, 0);
            const double ri = oracle_ds_window(sw, W, 1, eps, compensated, 0);
            const size_t o = (size_t)row * nk + k;
            tau[o] = t; r_re[o] = rr; r_im[o] = ri;
            wflag[o] = (uint8_t)oracle_flag(t, rr, ri, s_low, s_high, gamma);
        }
    }
    free(stokes);
    return nk;
}
