"""Emulation of the paper's trained mixed-precision flagging (TEST INFRASTRUCTURE ONLY).

Tables 3 and 4 of the paper (Section 4.1) list, for every group of operations of
Tables 1 and 2, the precision its reinforcement-learning agent chose:

  spectral kurtosis (Table 3)        directional statistics (Table 4), per Re/Im part
  g1 y = xr^2 + xi^2      binary32    g1 a, b, c = q^2, u^2, v^2        binary32
  g2 z = sqrt(y)          binary32    g2 p = sqrt(a + b + c) + eps      binary32
  g3 s1 = sum z           binary32    g3 q/p, u/p, v/p                  binary32
  g4 s2 = sum y           binary32    g4 sums of the normalised terms   binary16
  g5 lead = (Wd+1)/(W-1)  binary16    g5 squares of the sums            binary16
  g6 s12 = s1^2           binary32    g6 r = sqrt(sum of squares) / W   binary16
  g7 tau, and its test    binary16    g7 r > gamma                      binary16

(Table 3 prints action 0.497 for g5 yet labels it 16 bit; its "Precision" column is
followed.  Group 7 evaluates the equation of Section 2.1, lead * (W s2/(s12+eps) - 1),
as everywhere in this build, not the printed row's lead * W s2/(s12+eps) - 1.)

The map is the table PRECISION below; every group reads its format from it.  Every
operation of a group rounds its result to the group's format (IEEE round to nearest
even), values entering a group are converted to its format first, and sums run sample
after sample in window order.  eps is the machine epsilon of the group's format, as
the captions of Tables 1 and 2 describe it: the caller's eps in binary32 groups and
2^-10 in binary16 groups.  The parameters (d, thresholds, eps) are binary32 values,
as the library stores them.  The Stokes parameters (Section 2) and the averaged
output are not part of the tables and are computed in binary32.

numpy's binary16 operations round a correctly rounded binary32 result to binary16,
which equals direct binary16 rounding for +, -, *, / and sqrt (binary32 has at least
2 * 11 + 2 significand bits).

Pins: tests/test_oracle_mixed.py evaluates the same windows exactly (rationals,
IEEE rounding from its definition) with the tables' map, on inputs chosen so that
every single-group change of the map that can change a result does so.
"""
import numpy as np

F32 = np.float32
F16 = np.float16

# Tables 3 and 4, "Precision" column, one entry per group of Tables 1 and 2.
PRECISION = {
    "sk": {1: F32, 2: F32, 3: F32, 4: F32, 5: F16, 6: F32, 7: F16},
    "ds": {1: F32, 2: F32, 3: F32, 4: F16, 5: F16, 6: F16, 7: F16},
}


def _param(x, fmt):
    """A parameter as the library stores it (binary32), then in a group's format
    (out-of-range values become +-inf, as in a conversion)."""
    with np.errstate(over="ignore"):
        return fmt(F32(x))


def _eps(fmt, eps):
    """eps of a group: binary16's machine epsilon in binary16, the caller's eps in
    binary32 (captions of Tables 1 and 2)."""
    return F16(2.0 ** -10) if fmt is F16 else F32(eps)


def stokes32(v8):
    """Eq. IQUV in binary32 on rows [..., 8] (re/im of xx, xy, yx, yy): returns the 8
    components (I, Q, U, V; re, im)."""
    v = v8.astype(F32)
    xxr, xxi, xyr, xyi, yxr, yxi, yyr, yyi = (v[..., k] for k in range(8))
    return np.stack([xxr + yyr, xxi + yyi, xxr - yyr, xxi - yyi,
                     xyr + yxr, xyi + yxi, yxi - xyi, xyr - yxr], axis=-1)


def sk_mixed(st, W, d, s_low, s_high, eps=2.0 ** -23, prec=None):
    """Table 1 with the groups' precisions on windows st [n, W, 8]: (tau, flag)."""
    g = (prec or PRECISION)["sk"]
    with np.errstate(over="ignore", invalid="ignore", divide="ignore"):
        xr, xi = st[..., 0].astype(g[1]), st[..., 1].astype(g[1])
        y = xr * xr + xi * xi                            # g1
        z = np.sqrt(y.astype(g[2]))                      # g2
        s1 = np.zeros(st.shape[0], g[3])
        s2 = np.zeros(st.shape[0], g[4])
        for i in range(W):                               # g3, g4: sequential sums
            s1 = s1 + z[:, i].astype(g[3])
            s2 = s2 + y[:, i].astype(g[4])
        f5 = g[5]
        Wf, one5 = f5(W), f5(1)
        lead = (Wf * _param(d, f5) + one5) / (Wf - one5)  # g5
        s1_6 = s1.astype(g[6])
        s12 = s1_6 * s1_6                                 # g6
        f7 = g[7]
        one7 = f7(1)
        t = f7(W) * s2.astype(f7)                         # g7
        t = t / (s12.astype(f7) + _eps(f7, eps))
        tau = f7(lead) * (t - one7)                       # Sec. 2.1: lead * (W s2/s12 - 1)
        flag = ~((tau >= _param(s_low, f7)) & (tau <= _param(s_high, f7)))
    return tau, flag


def ds_mixed(st, W, part, eps, gamma, prec=None):
    """Table 2 with the groups' precisions on windows st [n, W, 8] for part 0 (Re) or
    1 (Im): (r, flag)."""
    g = (prec or PRECISION)["ds"]
    with np.errstate(over="ignore", invalid="ignore", divide="ignore"):
        q32, u32, v32 = st[..., 2 + part], st[..., 4 + part], st[..., 6 + part]
        q, u, v = q32.astype(g[1]), u32.astype(g[1]), v32.astype(g[1])
        a, b, c = q * q, u * u, v * v                     # g1
        f2 = g[2]
        p = np.sqrt((a.astype(f2) + b.astype(f2)) + c.astype(f2)) + _eps(f2, eps)   # g2
        f3 = g[3]
        p3 = p.astype(f3)
        qn, un, vn = q32.astype(f3) / p3, u32.astype(f3) / p3, v32.astype(f3) / p3  # g3
        f4 = g[4]
        Q = np.zeros(st.shape[0], f4)
        U = np.zeros(st.shape[0], f4)
        V = np.zeros(st.shape[0], f4)
        for i in range(W):                                # g4: sequential sums
            Q = Q + qn[:, i].astype(f4)
            U = U + un[:, i].astype(f4)
            V = V + vn[:, i].astype(f4)
        f5 = g[5]
        Q5, U5, V5 = Q.astype(f5), U.astype(f5), V.astype(f5)
        qb, ub, vb = Q5 * Q5, U5 * U5, V5 * V5            # g5
        f6 = g[6]
        r = np.sqrt((qb.astype(f6) + ub.astype(f6)) + vb.astype(f6)) / f6(W)         # g6
        f7 = g[7]
        flag = ~(r.astype(f7) <= _param(gamma, f7))       # g7
    return r, flag


def process_block_mixed(vis_rows, M, d, s_low, s_high, gamma, eps, prec=None):
    """Window statistics and flags of a block [R, T, 8] (float32 or float16 values) with
    time-only windows of M samples.  Returns dict of tau, r_re, r_im (in the format of
    the group that produced them, as float64) and wflag [R, T/M]."""
    R, T = vis_rows.shape[0], vis_rows.shape[1]
    nw = T // M
    st = stokes32(vis_rows.reshape(R * nw, M, 8))
    tau, f_sk = sk_mixed(st, M, d, s_low, s_high, eps, prec)
    r_re, f_re = ds_mixed(st, M, 0, eps, gamma, prec)
    r_im, f_im = ds_mixed(st, M, 1, eps, gamma, prec)
    shape = (R, nw)
    return dict(tau=tau.astype(np.float64).reshape(shape),
                r_re=r_re.astype(np.float64).reshape(shape),
                r_im=r_im.astype(np.float64).reshape(shape),
                wflag=(f_sk | f_re | f_im).reshape(shape).astype(np.uint8))
