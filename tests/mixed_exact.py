"""Exact evaluation of the paper's mixed-precision flagging (test infrastructure).

Tables 1 and 2 of the paper (Sec. 3) split the two statistics into 7 groups of
operations each; Tables 3 and 4 (Sec. 4.1) give the precision the trained agent chose
for every group.  This module evaluates one window with each operation done exactly
on rationals and rounded once to its group's format (ieee_exact), the operations in
the tables' order, a value entering a group converted to that group's format first,
and the group-to-format map passed in, so that the same evaluator also gives the
result of any other map (a flipped group).  It shares no code with oracle/mixed.py.

Parameters (d, s_low, s_high, gamma, eps) enter as binary32 values, as the library
stores them, and are converted to a group's format where the group uses them.

eps: the captions of Tables 1 and 2 tie it to the word length of the group that uses
it: the caller's eps in a binary32 group, binary16's machine epsilon 2^-10 in a
binary16 group.  Group 7 of Table 1 evaluates lead * (W s2/(s12 + eps) - 1), the
equation of Sec. 2.1.  The Stokes parameters (Sec. 2, Eq. IQUV) are not in the
tables; they are formed in binary32 from the stored values.
"""
from fractions import Fraction

import ieee_exact as X

# Tables 3 and 4, the "Precision" column, one entry per group of Tables 1 and 2
# (Table 3 prints action 0.497 for group 5 and labels it 16 bit; the printed label is
# taken).
TABLES_3_4 = {
    ("sk", 1): 32, ("sk", 2): 32, ("sk", 3): 32, ("sk", 4): 32,
    ("sk", 5): 16, ("sk", 6): 32, ("sk", 7): 16,
    ("ds", 1): 32, ("ds", 2): 32, ("ds", 3): 32, ("ds", 4): 16,
    ("ds", 5): 16, ("ds", 6): 16, ("ds", 7): 16,
}


def _fmt(bits):
    return X.B16 if bits == 16 else X.B32


def _param(x):
    """A threshold or parameter as the library holds it: a binary32 value."""
    return X.rnd(X.from_float(float(x)), X.B32)


def _eps(bits, eps):
    return Fraction(1, 1024) if bits == 16 else _param(eps)


def stokes_b32(s8):
    """Eq. IQUV in binary32 on one sample's 8 stored values (re/im of xx, xy, yx, yy):
    (Ir, Ii, Qr, Qi, Ur, Ui, Vr, Vi)."""
    f = X.B32
    xxr, xxi, xyr, xyi, yxr, yxi, yyr, yyi = (X.from_float(float(v)) for v in s8)
    return (X.add(xxr, yyr, f), X.add(xxi, yyi, f), X.sub(xxr, yyr, f), X.sub(xxi, yyi, f),
            X.add(xyr, yxr, f), X.add(xyi, yxi, f), X.sub(yxi, xyi, f), X.sub(xyr, yxr, f))


def sk_exact(st, W, d, s_low, s_high, eps, prec):
    """Table 1 on one window of Stokes tuples; returns (tau, flag)."""
    g = {k: _fmt(prec[("sk", k)]) for k in range(1, 8)}
    s1 = Fraction(0)
    s2 = Fraction(0)
    for x in st:
        xr, xi = X.to_fmt(x[0], g[1]), X.to_fmt(x[1], g[1])
        y = X.add(X.mul(xr, xr, g[1]), X.mul(xi, xi, g[1]), g[1])       # group 1
        z = X.sqrt(X.to_fmt(y, g[2]), g[2])                               # group 2
        s1 = X.add(s1, X.to_fmt(z, g[3]), g[3])                           # group 3
        s2 = X.add(s2, X.to_fmt(y, g[4]), g[4])                           # group 4
    f5 = g[5]
    Wf, one = X.to_fmt(W, f5), Fraction(1)
    lead = X.div(X.add(X.mul(Wf, X.to_fmt(_param(d), f5), f5), one, f5),
                 X.sub(Wf, one, f5), f5)                                  # group 5
    s1_6 = X.to_fmt(s1, g[6])
    s12 = X.mul(s1_6, s1_6, g[6])                                         # group 6
    f7 = g[7]
    t = X.mul(X.to_fmt(W, f7), X.to_fmt(s2, f7), f7)                      # group 7
    t = X.div(t, X.add(X.to_fmt(s12, f7), _eps(prec[("sk", 7)], eps), f7), f7)
    tau = X.mul(X.to_fmt(lead, f7), X.sub(t, one, f7), f7)
    lo = X.to_fmt(_param(s_low), f7)
    hi = X.to_fmt(_param(s_high), f7)
    flag = not (X.ge(tau, lo) and X.le(tau, hi))
    return tau, flag


def ds_exact(st, W, part, eps, gamma, prec):
    """Table 2 on one window for part 0 (Re) or 1 (Im); returns (r, flag)."""
    g = {k: _fmt(prec[("ds", k)]) for k in range(1, 8)}
    sums = [Fraction(0)] * 3
    for x in st:
        q, u, v = (X.to_fmt(x[2 + part], g[1]), X.to_fmt(x[4 + part], g[1]),
                   X.to_fmt(x[6 + part], g[1]))
        a, b, c = X.mul(q, q, g[1]), X.mul(u, u, g[1]), X.mul(v, v, g[1])   # group 1
        f2 = g[2]
        n = X.add(X.add(X.to_fmt(a, f2), X.to_fmt(b, f2), f2), X.to_fmt(c, f2), f2)
        p = X.add(X.sqrt(n, f2), _eps(prec[("ds", 2)], eps), f2)            # group 2
        f3 = g[3]
        p3 = X.to_fmt(p, f3)
        hats = [X.div(X.to_fmt(w, f3), p3, f3) for w in (x[2 + part], x[4 + part], x[6 + part])]
        # group 3 divides the binary32 Stokes components (its inputs) by p
        sums = [X.add(s, X.to_fmt(h, g[4]), g[4]) for s, h in zip(sums, hats)]   # group 4
    f5 = g[5]
    sq = [X.mul(X.to_fmt(s, f5), X.to_fmt(s, f5), f5) for s in sums]        # group 5
    f6 = g[6]
    tot = X.add(X.add(X.to_fmt(sq[0], f6), X.to_fmt(sq[1], f6), f6), X.to_fmt(sq[2], f6), f6)
    r = X.div(X.sqrt(tot, f6), X.to_fmt(W, f6), f6)                          # group 6
    f7 = g[7]
    flag = not X.le(X.to_fmt(r, f7), X.to_fmt(_param(gamma), f7))      # group 7
    return r, flag


def window_exact(vis8, d, s_low, s_high, gamma, eps, prec=TABLES_3_4):
    """One window of stored samples vis8 [W, 8] -> (tau, r_re, r_im, flag) as floats
    (statistics) and bool (flag)."""
    W = len(vis8)
    st = [stokes_b32(s) for s in vis8]
    tau, f_sk = sk_exact(st, W, d, s_low, s_high, eps, prec)
    r_re, f_re = ds_exact(st, W, 0, eps, gamma, prec)
    r_im, f_im = ds_exact(st, W, 1, eps, gamma, prec)
    return float(tau), float(r_re), float(r_im), bool(f_sk or f_re or f_im)
