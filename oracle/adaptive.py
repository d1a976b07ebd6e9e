"""Online per-stream SK thresholds, evaluated in float64 (TEST INFRASTRUCTURE ONLY).

Section 5 of the paper names online adaptation of the thresholds as future work and
gives no rule.  The rule this build implements, stated here so that it can be checked
by eye:

  * every footprint row g keeps (n_g, mu_g, m2_g): the number of its windows that were
    not flagged, and running estimates of the mean of tau and of tau^2 over them;
  * when a window is not flagged, n += 1, w = max(alpha, 1/n), mu += w (tau - mu),
    m2 += w (tau^2 - m2)  (the plain mean for the first 1/alpha windows, then an
    exponential average); flagged windows leave the state alone;
  * a block is flagged with the thresholds of the state at its start: once
    n_g >= n_warm, the SK test of row g accepts [mu - k sd, mu + k sd] with
    sd = sqrt(max(m2 - mu^2, 0)); before that it accepts the fixed [s_low, s_high];
    the DS threshold gamma never changes;
  * everything else (statistics, flag bits, averaging) is the method of Sections 2.1
    and 2.2, computed by the FP64 oracle (oracle_process_block_tf) with the row's
    thresholds.
"""
import numpy as np

from .oracle import OracleStream, to_f64_rows


class AdaptiveOracleStream:
    """R rows (R/F footprint rows) with per-row SK thresholds that follow the data."""

    def __init__(self, R, M, K, d, s_low, s_high, gamma, eps, alpha=1.0 / 64, k_sigma=3.0,
                 n_warm=32, F=1, compensated=False):
        if R % F:
            raise ValueError("R must be a multiple of F")
        self.R, self.M, self.K, self.F = R, M, K, F
        self.G = R // F
        self.s_low, self.s_high, self.gamma = float(s_low), float(s_high), float(gamma)
        self.alpha, self.k_sigma, self.n_warm = float(alpha), float(k_sigma), int(n_warm)
        self.groups = [OracleStream(F, M, K, d, s_low, s_high, gamma, eps, compensated, F)
                       for _ in range(self.G)]
        self.state = np.zeros((self.G, 3))      # n, mean of tau, mean of tau^2

    def thresholds(self):
        """The SK interval [lo, hi] each footprint row uses for the next block."""
        n, mu, m2 = self.state[:, 0], self.state[:, 1], self.state[:, 2]
        sd = np.sqrt(np.maximum(m2 - mu * mu, 0.0))
        warm = n >= self.n_warm
        lo = np.where(warm, mu - self.k_sigma * sd, self.s_low)
        hi = np.where(warm, mu + self.k_sigma * sd, self.s_high)
        return lo, hi

    def process(self, vis):
        v = to_f64_rows(vis)
        if v.shape[0] != self.R:
            raise ValueError(f"expected {self.R} rows, got {v.shape[0]}")
        lo, hi = self.thresholds()
        parts = []
        for g, st in enumerate(self.groups):
            st.thr[1], st.thr[2] = lo[g], hi[g]
            parts.append(st.process(v[g * self.F:(g + 1) * self.F]))
        out = {k: np.concatenate([p[k] for p in parts], axis=0) for k in parts[0]}
        out["s_low_used"], out["s_high_used"] = lo, hi
        # advance every row's moments over its windows, in window order
        for g in range(self.G):
            n, mu, m2 = self.state[g]
            for tau, f in zip(out["tau"][g], out["wflag"][g]):
                if f:
                    continue
                n += 1.0
                w = max(self.alpha, 1.0 / n)
                mu += w * (tau - mu)
                m2 += w * (tau * tau - m2)
            self.state[g] = (n, mu, m2)
        return out


__all__ = ["AdaptiveOracleStream"]
