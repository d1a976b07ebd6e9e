"""Overlapping (sliding) windows, evaluated in float64 (TEST INFRASTRUCTURE ONLY).

The paper's windows are consecutive and do not overlap (Sec. 2); sliding windows are
an extension.  The rule this build implements, stated here so that it can be checked
by eye:

  * a window holds M consecutive samples of one (baseline, channel) stream and a new
    window starts every H samples (H divides M), counted from the stream's first
    sample: window w covers samples [w H, w H + M), so every sample lies in L = M / H
    windows (fewer in the stream's first M - H samples);
  * each window's statistics and flag are those of Secs. 2.1 and 2.2 on its M samples
    (the C oracle's window functions), evaluated once all M samples have arrived;
  * a sample is flagged when any window that holds it is flagged (the OR of Sec. 2's
    per-window flags), and it is final once the last window holding it has been
    evaluated: sample t after window floor(t / H), i.e. M - H samples later;
  * the averages of Sec. 2.1 are taken over final samples, bins of K samples of the
    stream (K a multiple of H), flagged samples left out, weight = unflagged / K.

A call therefore reports the windows it completes, the flags of the samples that
became final (the first ones up to M - H samples before the block) and the bins that
closed.  With H = M this is the plain non-overlapping method.
"""
import numpy as np

from .oracle import _load, to_f64_rows


class SlidingOracleStream:
    def __init__(self, R, M, H, K, d, s_low, s_high, gamma, eps, compensated=False):
        if M < 2 or H < 1 or M % H or K % H:
            raise ValueError("need M >= 2, H dividing M and K a multiple of H")
        self.R, self.M, self.H, self.K, self.L = int(R), int(M), int(H), int(K), M // H
        self.thr = np.array([d, s_low, s_high, gamma, eps], dtype=np.float64)
        self.compensated = bool(compensated)
        self.n_seen = 0
        self.pending = np.zeros((self.R, 0, 8))          # samples not final yet
        # flags of the last L - 1 evaluated windows (the only ones that can hold a
        # sample that is not final yet); windows before the stream count as clean
        self.history = np.zeros((self.R, self.L - 1), dtype=bool)
        self.carry_sum = np.zeros((self.R, 8))
        self.carry_cnt = np.zeros(self.R)

    def evaluated(self, n):
        """Windows complete once n samples of the stream have arrived."""
        return max(0, (n - self.M) // self.H + 1)

    def windows_for(self, T):
        """(windows the next T samples complete, stream index of the first sample whose
        flag the call reports)."""
        e0, e1 = self.evaluated(self.n_seen), self.evaluated(self.n_seen + T)
        return e1 - e0, e0 * self.H

    def outputs_for(self, T):
        e0, e1 = self.evaluated(self.n_seen), self.evaluated(self.n_seen + T)
        return (e1 * self.H) // self.K - (e0 * self.H) // self.K

    def process(self, vis):
        v = to_f64_rows(vis)
        R, T = v.shape[0], v.shape[1]
        if R != self.R:
            raise ValueError(f"expected {self.R} rows, got {R}")
        if T % self.H:
            raise ValueError("T must be a multiple of the hop H")
        M, H, K, L = self.M, self.H, self.K, self.L
        e0, e1 = self.evaluated(self.n_seen), self.evaluated(self.n_seen + T)
        nk = e1 - e0
        buf = np.ascontiguousarray(np.concatenate([self.pending, v], axis=1))  # from e0 H
        Tb = buf.shape[1]
        tau, r_re, r_im = (np.zeros((R, nk)) for _ in range(3))
        wflag = np.zeros((R, nk), dtype=np.uint8)
        got = _load().oracle_window_stats_hop(buf.ctypes.data, R, Tb, M, H,
                                              self.thr.ctypes.data, int(self.compensated), nk,
                                              tau.ctypes.data, r_re.ctypes.data,
                                              r_im.ctypes.data, wflag.ctypes.data)
        if got != nk:
            raise ValueError("window count mismatch")
        # windows e0 - L + 1 .. e1 - 1, oldest first
        allw = np.concatenate([self.history, wflag.astype(bool)], axis=1)
        # sample run (segment) s = e0 .. e1 - 1 of H samples lies in windows s - L + 1 .. s
        seg = np.zeros((R, nk), dtype=bool)
        for i in range(nk):
            seg[:, i] = allw[:, i:i + L].any(axis=1)
        sflag = np.repeat(seg, H, axis=1)                 # samples e0 H .. e1 H - 1
        nbits = nk * H
        flagbits = np.zeros((R, (nbits + 31) // 32), dtype=np.uint32)
        for i in range(nbits):
            flagbits[sflag[:, i], i // 32] |= np.uint32(1 << (i % 32))
        # bins over the final samples, in stream order
        n_out = (e1 * H) // K - (e0 * H) // K
        avg, weight = np.zeros((R, n_out, 8)), np.zeros((R, n_out))
        b = 0
        for i in range(nbits):
            t = e0 * H + i
            keep = ~sflag[:, i]
            self.carry_sum[keep] += buf[keep, i]
            self.carry_cnt[keep] += 1.0
            if (t + 1) % K == 0:
                n = self.carry_cnt
                avg[:, b] = np.where(n[:, None] > 0, self.carry_sum / np.where(n > 0, n, 1.0)[:, None],
                                     0.0)
                weight[:, b] = n / K
                self.carry_sum[:] = 0.0
                self.carry_cnt[:] = 0.0
                b += 1
        self.pending = buf[:, nbits:].copy()
        if L > 1:
            self.history = allw[:, allw.shape[1] - (L - 1):].copy()
        self.n_seen += T
        return dict(tau=tau, r_re=r_re, r_im=r_im, wflag=wflag, flagbits=flagbits, avg=avg,
                    weight=weight, first_sample=e0 * H)


__all__ = ["SlidingOracleStream"]
