"""Thresholds from a desired false-alarm probability (Section 2.3).

The paper derives d, s_low, s_high and gamma from a target false-alarm probability and
then fine-tunes them, because its windows are too small for the large-W theory.  This
helper takes the empirical route on interference-free data: it runs the flagging kernel
with permissive thresholds, collects the window statistics it returns, and places the
thresholds at their quantiles:

  s_low, s_high = the fa/2 and 1 - fa/2 quantiles of tau (two-sided SK test),
  gamma         = the 1 - fa quantile of max(r_Re, r_Im) (one-sided DS test),

so each test alone flags a fraction fa of clean windows.  d only scales tau (through
(Wd+1)/(W-1)), so the quantiles absorb it; it is kept as given.
"""
import math

import numpy as np


def permissive(d=1.0, eps=2.0 ** -23):
    """Thresholds that flag nothing finite (for collecting statistics)."""
    return dict(d=d, s_low=-math.inf, s_high=math.inf, gamma=math.inf, eps=eps)


def _host(x):
    """A statistics buffer as a float64 numpy array [3, n] (a device tensor is copied to
    host memory; torch is used only for that copy)."""
    if hasattr(x, "detach"):
        x = x.detach().cpu().numpy()
    return np.asarray(x, dtype=np.float64).reshape(3, -1)


def thresholds_for_false_alarm(stats, fa=0.05, d=1.0, eps=2.0 ** -23):
    """stats: array or device tensor [3, ..., n_windows] (tau, r_Re, r_Im) from clean
    data, or a list of them.  Returns a thresholds dict."""
    if isinstance(stats, (list, tuple)):
        s = np.concatenate([_host(x) for x in stats], axis=1)
    else:
        s = _host(stats)
    tau = s[0][np.isfinite(s[0])]
    r = np.maximum(s[1], s[2])
    r = r[np.isfinite(r)]

    def q(x, p):
        k = min(max(int(round(p * (x.size - 1))), 0), x.size - 1)
        return float(np.partition(x, k)[k])

    return dict(d=d, s_low=q(tau, fa / 2), s_high=q(tau, 1 - fa / 2), gamma=q(r, 1 - fa),
                eps=eps)
