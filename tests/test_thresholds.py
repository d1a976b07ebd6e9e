"""Thresholds from a target false-alarm probability (Section 2.3) against the FP64
oracle on null windows, and the random-flight distribution against closed forms.

The oracle runs on windows drawn from each null model; the fraction of windows its
tests flag must match the target within 5 standard errors of a binomial count."""
import math

import numpy as np
import pytest

import oracle
from paper_2412_14775_b300 import thresholds as T


def _sk_flags(z, phase, thr, W):
    """The oracle's SK statistic on windows with xx = z e^{j phase} (others 0), so
    |I| = z; returns (below s_low, above s_high) fractions."""
    n = z.shape[0]
    v = np.zeros((n, W, 4), np.complex128)
    v[:, :, 0] = z * np.exp(1j * phase)
    o = oracle.OracleStream(n, W, W, thr["d"], -1e300, 1e300, 1e300, thr["eps"]).process(v)
    tau = o["tau"][:, 0]
    return float((tau < thr["s_low"]).mean()), float((tau > thr["s_high"]).mean())


def _within(frac, p, n, k=5.0):
    return abs(frac - p) <= k * math.sqrt(p * (1 - p) / n)


@pytest.mark.parametrize("W", [8, 16, 20])
def test_sk_false_alarm_rayleigh_null(W):
    """Circular complex Gaussian I (interference-free noise): each tail flags fa/2."""
    n = 200_000
    fa = 0.01
    thr = T.default_thresholds(W, fa=fa)
    rng = np.random.default_rng(100 + W)
    I = rng.standard_normal((n, W)) + 1j * rng.standard_normal((n, W))
    lo, hi = _sk_flags(np.abs(I), np.angle(I), thr, W)
    assert _within(lo, fa / 2, n) and _within(hi, fa / 2, n), (lo, hi)


@pytest.mark.parametrize("d", [1.0, 2.0])
def test_sk_false_alarm_gamma_null(d):
    """|I| ~ Gamma(d), the generalised SK model (Nita & Gary 2010)."""
    W, n, fa = 16, 200_000, 0.01
    lo_t, hi_t = T.sk_interval(W, fa, d, "gamma")
    thr = dict(d=d, s_low=lo_t, s_high=hi_t, eps=0.0)
    rng = np.random.default_rng(7 + int(d))
    z = rng.gamma(d, size=(n, W))
    lo, hi = _sk_flags(z, rng.uniform(0, 2 * np.pi, (n, W)), thr, W)
    assert _within(lo, fa / 2, n) and _within(hi, fa / 2, n), (lo, hi)


def test_sk_interval_is_not_symmetric_at_small_w():
    """The Gaussian interval 1 -/+ 3 sigma misses the skewed small-W null; the quantile
    interval sits higher on both sides."""
    lo, hi = T.sk_interval(16, T.FA_3SIGMA)
    sig = T.sk_sigma(16, T.D_RAYLEIGH)
    assert lo > 1 - 3 * sig and hi > 1 + 3 * sig


@pytest.mark.parametrize("W", [5, 16, 20])
def test_ds_false_alarm_isotropic_null(W):
    """Isotropic polarisation (independent circular Gaussian correlations): each part's
    r exceeds gamma in a fraction alpha of windows."""
    n, alpha = 100_000, 0.05
    thr = T.default_thresholds(W, alpha=alpha)
    rng = np.random.default_rng(300 + W)
    v = (rng.standard_normal((n, W, 4)) + 1j * rng.standard_normal((n, W, 4))) / math.sqrt(2)
    o = oracle.OracleStream(n, W, W, thr["d"], -1e300, 1e300, 1e300, thr["eps"]).process(v)
    for key in ("r_re", "r_im"):
        frac = float((o[key][:, 0] > thr["gamma"]).mean())
        assert _within(frac, alpha, n), (key, frac)


def test_flight_survival_closed_forms():
    # one vector: |u| = 1; two vectors: |u1 + u2|^2 = 2 + 2 cos(angle), cos ~ U(-1, 1)
    for rho in (0.1, 0.5, 0.99):
        assert T.flight_survival(1, rho) == 1
    for rho in (0.3, 1.0, 1.7):
        assert abs(float(T.flight_survival(2, rho)) - (1 - rho * rho / 4)) < 1e-15
    # large W: 3 W r^2 -> chi-square(3); and P(|S| > 0) = 1, P(|S| > W) = 0
    from scipy.stats import chi2
    W = 100
    g = T.ds_gamma(W, 0.05)
    assert abs(3 * W * g * g - chi2.ppf(0.95, 3)) / chi2.ppf(0.95, 3) < 0.01
    assert T.flight_survival(7, 0) == 1 and T.flight_survival(7, 7) == 0
