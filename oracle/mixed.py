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

Every operation of a group rounds its result to the group's format (IEEE
round to nearest even), values entering a group are converted to its format first,
and sums run sample after sample in window order.  eps is the machine epsilon of the
group's format, as the captions of Tables 1 and 2 describe it: the caller's eps in
binary32 groups and 2^-10 in binary16 groups.  The Stokes parameters (Section 2) and
the averaged output are not part of the tables and are computed in binary32.

numpy's binary16 operations round a correctly rounded binary32 result to binary16,
which equals direct binary16 rounding for +, -, *, / and sqrt (binary32 has at least
2 * 11 + 2 significand bits).
"""
import numpy as np

F32 = np.float32
F16 = np.float16
EPS16 = F16(2.0 ** -10)


def _f16(x):
    """A threshold in binary16 (out-of-range values become +-inf, as in a conversion)."""
    with np.errstate(over="ignore"):
        return F16(x)


def stokes32(v8):
    """Eq. IQUV in binary32 on rows [..., 8] (re/im of xx, xy, yx, yy): returns the 8
    components (I, Q, U, V; re, im)."""
    v = v8.astype(F32)
    xxr, xxi, xyr, xyi, yxr, yxi, yyr, yyi = (v[..., k] for k in range(8))
    return np.stack([xxr + yyr, xxi + yyi, xxr - yyr, xxi - yyi,
                     xyr + yxr, xyi + yxi, yxi - xyi, xyr - yxr], axis=-1)


def sk_mixed(st, W, d, s_low, s_high):
    """Table 3 on windows st [n, W, 8]: returns (tau as binary16, flag)."""
    xr, xi = st[..., 0], st[..., 1]
    y = xr * xr + xi * xi                        # g1, binary32 (two products, one sum)
    z = np.sqrt(y)                               # g2, binary32
    s1 = np.zeros(st.shape[0], F32)
    s2 = np.zeros(st.shape[0], F32)
    for i in range(W):                           # g3, g4: sequential binary32 sums
        s1 = s1 + z[:, i]
        s2 = s2 + y[:, i]
    Wh, one = F16(W), F16(1)
    lead = (Wh * F16(d) + one) / (Wh - one)      # g5, binary16
    s12 = s1 * s1                                # g6, binary32
    t = Wh * s2.astype(F16)                      # g7, binary16 from here on
    t = t / (s12.astype(F16) + EPS16)
    tau = lead * (t - one)                       # the equation of Sec. 2.1 (reading 1)
    flag = ~((tau >= _f16(s_low)) & (tau <= _f16(s_high)))
    return tau, flag


def ds_mixed(st, W, part, eps, gamma):
    """Table 4 on windows st [n, W, 8] for part 0 (Re) or 1 (Im): (r as binary16, flag)."""
    q, u, v = st[..., 2 + part], st[..., 4 + part], st[..., 6 + part]
    a, b, c = q * q, u * u, v * v                # g1, binary32
    p = np.sqrt(a + b + c) + F32(eps)            # g2, binary32: (a + b) + c
    qn, un, vn = q / p, u / p, v / p             # g3, binary32
    Q = np.zeros(st.shape[0], F16)
    U = np.zeros(st.shape[0], F16)
    V = np.zeros(st.shape[0], F16)
    for i in range(W):                           # g4, binary16 sums
        Q = Q + qn[:, i].astype(F16)
        U = U + un[:, i].astype(F16)
        V = V + vn[:, i].astype(F16)
    qb, ub, vb = Q * Q, U * U, V * V             # g5, binary16
    r = np.sqrt(qb + ub + vb) / F16(W)           # g6, binary16
    flag = ~(r <= _f16(gamma))                   # g7
    return r, flag


def process_block_mixed(vis_rows, M, d, s_low, s_high, gamma, eps):
    """Window statistics and flags of a block [R, T, 8] (float32 or float16 values) with
    time-only windows of M samples.  Returns dict of tau, r_re, r_im (binary16 values
    as float64) and wflag [R, T/M]."""
    R, T = vis_rows.shape[0], vis_rows.shape[1]
    nw = T // M
    st = stokes32(vis_rows.reshape(R * nw, M, 8))
    tau, f_sk = sk_mixed(st, M, d, s_low, s_high)
    r_re, f_re = ds_mixed(st, M, 0, eps, gamma)
    r_im, f_im = ds_mixed(st, M, 1, eps, gamma)
    shape = (R, nw)
    return dict(tau=tau.astype(np.float64).reshape(shape),
                r_re=r_re.astype(np.float64).reshape(shape),
                r_im=r_im.astype(np.float64).reshape(shape),
                wflag=(f_sk | f_re | f_im).reshape(shape).astype(np.uint8))
