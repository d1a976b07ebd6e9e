"""Thresholds from a target false-alarm probability (Section 2.3; the paper fixes no
values).

The paper determines d, s_low, s_high and gamma from a desired false-alarm probability
and then fine-tunes them because its windows are too small for the large-W theory.
Here the small-W null distributions are used directly:

  * SK (Section 2.1).  tau = (W d + 1)/(W - 1) (W S2/S1^2 - 1) with S1 = sum |I|,
    S2 = sum |I|^2.  The null model is interference-free correlator noise: I a
    circular complex Gaussian, so |I|^2 is exponential and |I| Rayleigh ("rayleigh"),
    for which d = pi/(4 - pi) centres tau at 1 for large W (W S2/S1^2 -> 4/pi); or
    |I| ~ Gamma(d) ("gamma"), the generalised SK of Nita & Gary (2010, cited in
    Section 2.1), under which E[tau] = 1 exactly.  tau's distribution at small W is
    skewed, so 1 -/+ k sigma misses a two-sided target (at W = 16, 1 -/+ 3 sigma flags
    about 1.1 % of null windows above and none below, against 0.135 % each); the
    interval is therefore taken at the fa/2 and 1 - fa/2 quantiles of tau over 2^20
    (fewer for W > 16) null windows drawn from a fixed seed, exactly as the statistic
    is defined, so its false-alarm probability is fa up to the sampling error of those
    quantiles (about 3 % relative at fa = 0.0027).
  * DS (Section 2.2).  Under isotropic noise the W unit vectors of one part are
    uniform on the sphere, and r = |sum u_i| / W is a 3-D random flight (Rayleigh,
    1919).  The projection of a uniform unit vector on an axis is uniform on [-1, 1]
    (Archimedes), so the projection of the sum has the Irwin-Hall density g, and for
    an isotropic vector P(|S| > rho) = 2 rho g(rho) + 2 P(X > rho).  gamma solves
    P(r > gamma) = alpha exactly (rational arithmetic), per part, for W <= 128; for
    larger W, 3 W r^2 is chi-square with 3 degrees of freedom to within 0.2 %.
"""
import math
from fractions import Fraction
from functools import lru_cache

import numpy as np

EPS32 = 2.0 ** -23
D_RAYLEIGH = math.pi / (4.0 - math.pi)
# two-sided probability outside +-3 standard deviations of a normal distribution
FA_3SIGMA = math.erfc(3.0 / math.sqrt(2.0))
_SEED = 20241477


def sk_sigma(W, d):
    """Standard deviation of tau for Gamma(d) magnitudes (closed form)."""
    return math.sqrt(2.0 * d * (d + 1.0) * W * W / ((W - 1.0) * (W * d + 2.0) * (W * d + 3.0)))


def sk_null_tau(W, d, null="rayleigh", n=1 << 16, seed=_SEED):
    """n values of tau for windows of W null samples (see the module docstring)."""
    rng = np.random.default_rng([seed, W, 0 if null == "rayleigh" else 1])
    if null == "rayleigh":
        y = rng.standard_exponential((n, W))          # |I|^2
        z = np.sqrt(y)
    elif null == "gamma":
        z = rng.gamma(d, size=(n, W))                 # |I|
        y = z * z
    else:
        raise ValueError(f"unknown null model {null!r}")
    S1, S2 = z.sum(axis=1), y.sum(axis=1)
    return (W * d + 1.0) / (W - 1.0) * (W * S2 / (S1 * S1) - 1.0)


@lru_cache(maxsize=256)
def sk_interval(W, fa, d=D_RAYLEIGH, null="rayleigh"):
    """(s_low, s_high) with P(tau < s_low) = P(tau > s_high) = fa/2 under the null."""
    if not 0.0 < fa < 1.0 or W < 2:
        raise ValueError("need 0 < fa < 1 and W >= 2")
    n_total = int(min(1 << 20, max(1 << 15, (1 << 24) // W)))
    chunks = []
    done, part = 0, 0
    while done < n_total:
        n = min(1 << 16, n_total - done)
        chunks.append(sk_null_tau(W, d, null, n, seed=_SEED + part))
        done += n
        part += 1
    tau = np.concatenate(chunks)
    lo, hi = np.quantile(tau, [fa / 2.0, 1.0 - fa / 2.0])
    return float(lo), float(hi)


def _irwin_hall(n, s):
    """Density and distribution function of a sum of n uniform(0, 1) variables at the
    rational point s, exactly."""
    f = Fraction(0)
    F = Fraction(0)
    for k in range(0, min(n, math.floor(s)) + 1):
        c = (-1) ** k * math.comb(n, k)
        t = s - k
        f += c * t ** (n - 1)
        F += c * t ** n
    return f / math.factorial(n - 1), F / math.factorial(n)


def flight_survival(W, rho):
    """P(|u_1 + ... + u_W| > rho) for W independent unit vectors uniform on the sphere
    (exact; rho a float or Fraction in [0, W])."""
    rho = Fraction(rho)
    if rho <= 0:
        return Fraction(1)
    if rho >= W:
        return Fraction(0)
    s = (rho + W) / 2              # X = 2 S - W with S Irwin-Hall: X > rho <=> S > s
    f, F = _irwin_hall(W, s)
    # g_X(rho) = f(s)/2, P(X > rho) = 1 - F(s)
    return rho * f + 2 * (1 - F)


# 0.95, 0.99, 0.999 quantiles of the chi-square distribution with 3 degrees of freedom
_CHI2_3 = {0.05: 7.814727903251178, 0.01: 11.344866730144373, 0.001: 16.26623619623813}
EXACT_FLIGHT_MAX_W = 128


@lru_cache(maxsize=256)
def ds_gamma(W, alpha):
    """gamma with P(r > gamma) = alpha for one part of a W-sample isotropic window:
    exact for W <= 128; above, 3 W r^2 ~ chi-square(3) (at W = 64 the two differ by
    0.2 %)."""
    if not 0.0 < alpha < 1.0 or W < 1:
        raise ValueError("need 0 < alpha < 1 and W >= 1")
    if W > EXACT_FLIGHT_MAX_W:
        q = _CHI2_3.get(alpha)
        if q is None:
            from scipy.stats import chi2
            q = float(chi2.ppf(1.0 - alpha, 3))
        return math.sqrt(q / (3.0 * W))
    lo, hi = 0.0, float(W)
    target = Fraction(alpha)
    for _ in range(64):            # bisection on rho = W gamma
        mid = 0.5 * (lo + hi)
        if flight_survival(W, mid) > target:
            lo = mid
        else:
            hi = mid
    return hi / W


def default_thresholds(M, d=D_RAYLEIGH, fa=FA_3SIGMA, alpha=0.05, eps=EPS32, null="rayleigh",
                       k_sigma=None):
    """Thresholds for windows of W = M samples (pass M * F for T x F footprints).

    fa: two-sided SK false-alarm probability under the null (default: that of +-3
    sigma of a normal); alpha: DS false-alarm probability of each part (Re, Im).
    k_sigma: if given, the SK interval 1 -/+ k_sigma sigma (Gamma(d) sigma) instead."""
    if k_sigma is not None:
        sig = sk_sigma(M, d)
        s_low, s_high = 1.0 - k_sigma * sig, 1.0 + k_sigma * sig
    else:
        s_low, s_high = sk_interval(int(M), float(fa), float(d), null)
    return dict(d=d, s_low=s_low, s_high=s_high, gamma=ds_gamma(int(M), float(alpha)),
                eps=eps)
