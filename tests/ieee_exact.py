"""Exact IEEE 754 binary arithmetic on rationals (test infrastructure).

Values are fractions.Fraction (or +-inf / nan as floats).  Every operation is done
exactly and then rounded once to the target format, round to nearest, ties to even,
with gradual underflow and overflow to infinity, as IEEE 754 defines a correctly
rounded operation.  Nothing here uses the host's floating-point arithmetic for the
values themselves, so it is an independent route to what numpy's float16 / float32
(or a GPU's correctly rounded instructions) must produce.

Formats: binary16 (11 significand bits, emin -14, emax 15) and binary32 (24, -126,
127).
"""
from fractions import Fraction
from math import isqrt

INF = float("inf")
NAN = float("nan")


class Fmt:
    def __init__(self, name, p, emin, emax):
        self.name, self.p, self.emin, self.emax = name, p, emin, emax
        self.max = Fraction(2 ** p - 1, 2 ** (p - 1)) * Fraction(2) ** emax

    def __repr__(self):
        return self.name


B16 = Fmt("binary16", 11, -14, 15)
B32 = Fmt("binary32", 24, -126, 127)


def _is_special(x):
    return isinstance(x, float)


def _floor_log2(n: int, d: int) -> int:
    """floor(log2(n/d)) for integers n, d > 0, exactly."""
    e = n.bit_length() - d.bit_length()
    # 2^e <= n/d < 2^(e+1) after at most one correction step
    if (n << -e if e < 0 else n) < (d << e if e > 0 else d):
        e -= 1
    return e


def rnd(x, fmt: Fmt):
    """Round x (Fraction, int or special float) to fmt."""
    if _is_special(x):
        return x
    x = Fraction(x)
    n, d = x.numerator, x.denominator
    if n == 0:
        return Fraction(0)
    s = -1 if n < 0 else 1
    n = abs(n)
    qe = max(_floor_log2(n, d), fmt.emin) - fmt.p + 1   # exponent of the quantum (ulp)
    num, den = (n, d << qe) if qe >= 0 else (n << -qe, d)
    m, r = divmod(num, den)
    if 2 * r > den or (2 * r == den and m & 1):          # to nearest, ties to even
        m += 1
    v = Fraction(m << qe) if qe >= 0 else Fraction(m, 1 << -qe)
    if v > fmt.max:
        return s * INF
    return s * v


def from_float(x: float):
    """Exact value of a Python float (binary64), inf / nan kept as floats."""
    if x != x or x in (INF, -INF):
        return x
    return Fraction(x)


def add(a, b, fmt):
    if _is_special(a) or _is_special(b):
        return float(a) + float(b)
    return rnd(a + b, fmt)


def sub(a, b, fmt):
    if _is_special(a) or _is_special(b):
        return float(a) - float(b)
    return rnd(a - b, fmt)


def mul(a, b, fmt):
    if _is_special(a) or _is_special(b):
        return float(a) * float(b)
    return rnd(a * b, fmt)


def div(a, b, fmt):
    if _is_special(a) or _is_special(b):
        fa, fb = float(a), float(b)
        if fb == 0.0:
            return NAN if fa == 0.0 or fa != fa else (INF if fa > 0 else -INF)
        return fa / fb
    if b == 0:
        return NAN if a == 0 else (INF if a > 0 else -INF)
    return rnd(Fraction(a) / Fraction(b), fmt)


def sqrt(a, fmt):
    """Correctly rounded square root of a >= 0 (a Fraction)."""
    if _is_special(a):
        return a if a == INF else NAN
    a = Fraction(a)
    if a < 0:
        return NAN
    if a == 0:
        return Fraction(0)
    # s = floor(sqrt(a) * 2^k) with enough bits that every tie point of fmt is an
    # integer multiple of >= 2 units: sqrt(a) * 2^k lies in [s, s + 1), and it equals s
    # exactly only if a * 4^k is the perfect square s^2
    k = fmt.p + 8 - _floor_log2(a.numerator, a.denominator) // 2
    num = a * Fraction(4) ** k
    n = num.numerator // num.denominator
    s = isqrt(n)
    exact = (num.denominator == 1) and s * s == n
    approx = Fraction(s) if exact else Fraction(2 * s + 1, 2)
    return rnd(approx / Fraction(2) ** k, fmt)


def to_fmt(x, fmt):
    """Convert a value entering a group to that group's format."""
    return rnd(x, fmt)


def le(a, b):
    """IEEE a <= b (False when either is NaN)."""
    fa, fb = (float(a) if _is_special(a) else a), (float(b) if _is_special(b) else b)
    if (isinstance(fa, float) and fa != fa) or (isinstance(fb, float) and fb != fb):
        return False
    if isinstance(fa, float) or isinstance(fb, float):
        return float(fa) <= float(fb)
    return fa <= fb


def ge(a, b):
    return le(b, a)


def as_float(x) -> float:
    return float(x)
