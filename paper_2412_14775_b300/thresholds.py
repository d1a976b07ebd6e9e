"""Default thresholds for a window of M samples (a build choice; the paper fixes none).

The paper determines d, s_low, s_high and gamma from a desired false-alarm
probability and then fine-tunes them (Section 2.3).  The defaults here follow that
recipe with two closed forms:
  * SK: d = pi / (4 - pi) centres tau at 1 for complex Gaussian visibilities with
    Rayleigh-distributed |I| (M S2/S1^2 -> 4/pi); [s_low, s_high] = 1 -/+ k sigma with
    sigma^2 = 2 d (d+1) M^2 / ((M-1)(Md+2)(Md+3)), the variance of the generalised
    SK for Gamma(d) magnitudes (Nita & Gary 2010, cited in Section 2.1).
  * DS: under isotropic noise 3 M r^2 is asymptotically chi-square with 3 degrees of
    freedom (Rayleigh test), so gamma = sqrt(chi2_3(1 - alpha) / (3 M)).
"""
import math

EPS32 = 2.0 ** -23
# 0.95 quantile of the chi-square distribution with 3 degrees of freedom
_CHI2_3 = {0.05: 7.814727903251178, 0.01: 11.344866730144373, 0.001: 16.26623619623813}


def sk_sigma(M, d):
    return math.sqrt(2.0 * d * (d + 1.0) * M * M / ((M - 1.0) * (M * d + 2.0) * (M * d + 3.0)))


def default_thresholds(M, d=math.pi / (4.0 - math.pi), k_sigma=3.0, alpha=0.05, eps=EPS32):
    sig = sk_sigma(M, d)
    q = _CHI2_3.get(alpha)
    if q is None:
        from scipy.stats import chi2
        q = float(chi2.ppf(1.0 - alpha, 3))
    return dict(d=d, s_low=1.0 - k_sigma * sig, s_high=1.0 + k_sigma * sig,
                gamma=math.sqrt(q / (3.0 * M)), eps=eps)
