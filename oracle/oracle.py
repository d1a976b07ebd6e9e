"""ctypes wrapper around the FP64 C oracle (test infrastructure only).

Inputs are widened exactly to float64 before the oracle sees them: complex64,
float32 and float16 values are all exactly representable in double, so the oracle
evaluates the method on the very values the GPU path stores.
"""
import ctypes

import numpy as np

from . import build as _build

_lib = None
_lib_path = None


def use_library(path=None):
    """Point the wrapper at another build of rfi_oracle.c (None = the default build).

    Used only by the tests that plant a mistake in a copy of the oracle source to
    show that the pins detect it."""
    global _lib, _lib_path
    _lib, _lib_path = None, path


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(_lib_path or _build.build())
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_stokes.argtypes = [dp, dp]
        lib.oracle_stokes.restype = None
        lib.oracle_sk_window.argtypes = [dp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_int, dp, dp]
        lib.oracle_sk_window.restype = ctypes.c_double
        lib.oracle_ds_window.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_int, dp]
        lib.oracle_ds_window.restype = ctypes.c_double
        lib.oracle_flag.argtypes = [ctypes.c_double] * 6
        lib.oracle_flag.restype = ctypes.c_int
        lib.oracle_outputs_for.argtypes = [ctypes.c_longlong, ctypes.c_int, ctypes.c_int]
        lib.oracle_outputs_for.restype = ctypes.c_longlong
        lib.oracle_process_block.argtypes = [
            ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
            ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong,
            ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.oracle_process_block.restype = ctypes.c_int
        lib.oracle_process_block_tf.argtypes = [
            ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
            ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong,
            ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.oracle_process_block_tf.restype = ctypes.c_int
        lib.oracle_process_block_given_flags.argtypes = [
            ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
            ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong,
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.oracle_process_block_given_flags.restype = ctypes.c_int
        lib.oracle_window_stats_hop.argtypes = [
            ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
            ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.oracle_window_stats_hop.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def to_f64_rows(vis):
    """Widen visibilities exactly to float64 rows of shape [R, T, 8].

    Accepted layouts: [..., T, 4] complex (pol order xx, xy, yx, yy), or
    [..., T, 4, 2] / [..., T, 8] real (re, im interleaved) in float16/32/64.
    """
    a = np.asarray(vis)
    if np.iscomplexobj(a):
        if a.shape[-1] != 4:
            raise ValueError("complex input must end in 4 polarisations")
        a = np.stack([a.real, a.imag], axis=-1)
    if a.shape[-2:] == (4, 2):
        a = a.reshape(a.shape[:-2] + (8,))
    if a.shape[-1] != 8:
        raise ValueError(f"unsupported visibility shape {a.shape}")
    T = a.shape[-2]
    return np.ascontiguousarray(a.reshape(-1, T, 8).astype(np.float64))


def outputs_for(n_seen, T, K):
    """Completed averaging bins when T samples follow n_seen samples."""
    return (n_seen + T) // K - n_seen // K


def stokes(v8):
    """Eq. IQUV for one sample: 8 doubles (xx, xy, yx, yy) -> (I, Q, U, V) re/im."""
    v = np.ascontiguousarray(np.asarray(v8, dtype=np.float64).reshape(8))
    out = np.zeros(8)
    _load().oracle_stokes(_ptr(v), _ptr(out))
    return out


def sk_window(stokes_w, d, eps, compensated=False):
    """Section 2.1 on one window of Stokes samples [W, 8]: returns (tau, S1, S2)."""
    s = np.ascontiguousarray(np.asarray(stokes_w, dtype=np.float64))
    S1 = ctypes.c_double()
    S2 = ctypes.c_double()
    tau = _load().oracle_sk_window(_ptr(s), s.shape[0], d, eps, int(compensated),
                                   ctypes.byref(S1), ctypes.byref(S2))
    return tau, S1.value, S2.value


def ds_window(stokes_w, part, eps, compensated=False):
    """Section 2.2 on one window of Stokes samples [W, 8]: returns (r, (q, u, v))."""
    s = np.ascontiguousarray(np.asarray(stokes_w, dtype=np.float64))
    sums = np.zeros(3)
    r = _load().oracle_ds_window(_ptr(s), s.shape[0], part, eps, int(compensated), _ptr(sums))
    return r, tuple(sums)


def flag(tau, r_re, r_im, s_low, s_high, gamma):
    """Combined flag: SK outside [s_low, s_high] OR r_re > gamma OR r_im > gamma."""
    return bool(_load().oracle_flag(tau, r_re, r_im, s_low, s_high, gamma))


class OracleStream:
    """One stream (a set of R independent (baseline, channel) rows) fed block by block.

    Holds the open averaging bin of every row between blocks, exactly (float64),
    so that any split of the stream at multiples of the window gives the same
    results as one long block.  With `partial`, blocks may have any length: the
    samples after a block's last whole window are kept and put in front of the next
    block, so every window is evaluated whole, on consecutive samples of the stream
    (Sec. 2), and a call reports the windows it completes.
    """

    def __init__(self, R, M, K, d, s_low, s_high, gamma, eps, compensated=False, F=1,
                 partial=False):
        """M: samples per row in a window; F: adjacent rows (channels) per window, so
        a window holds W = M * F samples; R must be a multiple of F."""
        if M * F < 2 or K % M != 0 or R % F != 0:
            raise ValueError("need M*F >= 2, K a multiple of M and R a multiple of F")
        self.R, self.M, self.K, self.F = int(R), int(M), int(K), int(F)
        self.thr = np.array([d, s_low, s_high, gamma, eps], dtype=np.float64)
        self.compensated = bool(compensated)
        self.n_seen = 0
        self.carry_sum = np.zeros((self.R, 8))
        self.carry_cnt = np.zeros(self.R)
        self.partial = bool(partial)
        self.pending = np.zeros((self.R, 0, 8))     # samples of the open window

    def outputs_for(self, T):
        """Averaging bins completed by the next block of T samples (bins end at window
        ends, so the samples of an open window do not change this count)."""
        return outputs_for(self.n_seen + self.pending.shape[1], T, self.K)

    def windows_for(self, T):
        """(windows completed, stream index of their first sample) for T samples."""
        return (self.pending.shape[1] + T) // self.M, self.n_seen

    def process(self, vis, wflag=None):
        """Process one block; vis is any layout accepted by to_f64_rows with R rows.

        wflag: optional window flags [R/F][windows of the block] to use instead of the
        oracle's own (e.g. those of another arithmetic); flag bits and averages then
        follow them.  Not with `partial`."""
        v = to_f64_rows(vis)
        R = v.shape[0]
        if R != self.R:
            raise ValueError(f"expected {self.R} rows, got {R}")
        if self.partial:
            v = np.concatenate([self.pending, v], axis=1)
            whole = (v.shape[1] // self.M) * self.M
            v, self.pending = np.ascontiguousarray(v[:, :whole]), v[:, whole:].copy()
        T = v.shape[1]
        if T % self.M != 0:
            raise ValueError("T must be a multiple of M")
        nw = T // self.M
        nwords = (T + 31) // 32
        n_out = self.outputs_for(T)
        G = R // self.F
        if T == 0:          # the block only extends the open window
            return dict(tau=np.zeros((G, 0)), r_re=np.zeros((G, 0)), r_im=np.zeros((G, 0)),
                        wflag=np.zeros((G, 0), dtype=np.uint8),
                        flagbits=np.zeros((R, 0), dtype=np.uint32),
                        avg=np.zeros((R, 0, 8)), weight=np.zeros((R, 0)))
        out = dict(
            tau=np.zeros((G, nw)), r_re=np.zeros((G, nw)), r_im=np.zeros((G, nw)),
            wflag=np.zeros((G, nw), dtype=np.uint8),
            flagbits=np.zeros((R, nwords), dtype=np.uint32),
            avg=np.zeros((R, n_out, 8)), weight=np.zeros((R, n_out)))
        common = (v.ctypes.data, R, T, self.M, self.F, self.K, self.thr.ctypes.data,
                  int(self.compensated),
                  self.n_seen, self.carry_sum.ctypes.data, self.carry_cnt.ctypes.data)
        outs = (out["tau"].ctypes.data, out["r_re"].ctypes.data, out["r_im"].ctypes.data,
                out["wflag"].ctypes.data, out["flagbits"].ctypes.data,
                out["avg"].ctypes.data, out["weight"].ctypes.data)
        if wflag is None:
            rc = _load().oracle_process_block_tf(*common, *outs)
        else:
            if self.partial:
                raise ValueError("given window flags need whole windows (partial=False)")
            given = np.ascontiguousarray(np.asarray(wflag).astype(np.uint8).reshape(G, nw))
            rc = _load().oracle_process_block_given_flags(*common, given.ctypes.data, *outs)
        if rc != 0:
            raise ValueError("oracle rejected the block sizes")
        self.n_seen += T
        return out


__all__ = ["OracleStream", "outputs_for", "stokes", "sk_window", "ds_window", "flag",
           "to_f64_rows"]
