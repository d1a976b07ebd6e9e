"""Shared helpers of the GPU parity tests: run the CUDA path and the FP64 oracle on the
same seeded input and compare them element by element.

Tolerances (FP32 path, written here once and used by every parity test):
  * statistics: |gpu - oracle| <= 1e-5 * max(|oracle|, floor), floor = 1 for tau (its
    null mean) and M^-1/2 for r_Re, r_Im (their null RMS);
  * flags: identical, except windows where some statistic of the oracle lies within
    1e-4 * max(|threshold|, floor) of its threshold (those may fall either way);
  * averages: |gpu - oracle| <= 1e-5 * max(|oracle|, 1) per component and weights
    exactly equal, in every bin none of whose windows is exempt from flag equality.
The GPU flag words must also equal, bit for bit, the flag rule applied in float32 to
the GPU's own statistics (self-consistency of the packing).
"""
import numpy as np
import torch

STAT_RTOL = 1e-5
BAND = 1e-4
AVG_RTOL = 1e-5


def to_device_rows(vis_np, dtype):
    """[..., T, 4, 2] numpy float32 -> contiguous CUDA tensor [R, T, 4, 2] of `dtype`."""
    v = vis_np.reshape(-1, *vis_np.shape[-3:])
    t = torch.from_numpy(np.ascontiguousarray(v))
    if dtype == "f16":
        t = t.to(torch.float16)
    return t.cuda()


def run_gpu(stream, vis_dev, out=None):
    o = stream.process(vis_dev, out=out)
    torch.cuda.synchronize()
    return gpu_to_numpy(o)


def gpu_to_numpy(o):
    st = o["stats"].cpu().numpy()
    return dict(tau=st[0].astype(np.float64), r_re=st[1].astype(np.float64),
                r_im=st[2].astype(np.float64),
                flagbits=o["flags"].cpu().numpy().view(np.uint32),
                avg=o["avg"].cpu().numpy().reshape(o["avg"].shape[0], -1, 8).astype(np.float64),
                weight=o["weight"].cpu().numpy().astype(np.float64))


def expand_window_flags(flagbits, M, T):
    """Window flags from packed per-sample bits (requires all M bits equal)."""
    R = flagbits.shape[0]
    t = np.arange(T)
    bits = (flagbits[:, t // 32] >> (t % 32).astype(np.uint32)) & 1
    w = bits.reshape(R, T // M, M)
    assert np.all(w == w[:, :, :1]), "flag bits differ inside one window"
    # bits past T in the last word must be zero
    if T % 32:
        tail = flagbits[:, -1] >> np.uint32(T % 32)
        assert np.all(tail == 0), "flag bits set past the end of the block"
    return w[:, :, 0].astype(bool)


def flag_rule_f32(tau, r_re, r_im, thr):
    f = np.float32
    tau, r_re, r_im = tau.astype(f), r_re.astype(f), r_im.astype(f)
    inside = (tau >= f(thr["s_low"])) & (tau <= f(thr["s_high"]))
    return ~inside | ~(r_re <= f(thr["gamma"])) | ~(r_im <= f(thr["gamma"]))


def near_threshold(orc, thr, M):
    """Windows whose oracle statistics lie within BAND of a threshold."""
    def near(x, t, floor):
        if not np.isfinite(t):
            return np.zeros_like(x, bool)
        return np.abs(x - t) <= BAND * max(abs(t), floor)
    return (near(orc["tau"], thr["s_low"], 1.0) | near(orc["tau"], thr["s_high"], 1.0) |
            near(orc["r_re"], thr["gamma"], M ** -0.5) | near(orc["r_im"], thr["gamma"], M ** -0.5))


def rel_err(x, ref, floor):
    return np.abs(x - ref) / np.maximum(np.abs(ref), floor)


def compare(gpu, orc, thr, M, K, n_seen=0, stat_rtol=STAT_RTOL, avg_rtol=AVG_RTOL,
            check_flags=True, F=1):
    """Assert parity; return a dict of the observed worst errors and counts.

    With a T x F footprint (F > 1) the statistics are per footprint [R/F, T/M] while
    flags and averages are per row; W = M F is the window size."""
    T = gpu["tau"].shape[1] * M
    W = M * F
    rep = {}
    for key, floor in (("tau", 1.0), ("r_re", W ** -0.5), ("r_im", W ** -0.5)):
        both_nan = np.isnan(gpu[key]) & np.isnan(orc[key])
        e = np.where(both_nan, 0.0, rel_err(gpu[key], orc[key], floor))
        rep[key] = float(np.nanmax(e)) if e.size else 0.0
        if stat_rtol is not None:
            assert not np.isnan(e).any(), f"{key}: NaN on one side only"
            assert rep[key] <= stat_rtol, f"{key}: worst relative error {rep[key]:.3g}"
    wflag = expand_window_flags(gpu["flagbits"], M, T)                 # per row
    self_rule = np.repeat(flag_rule_f32(gpu["tau"], gpu["r_re"], gpu["r_im"], thr), F, axis=0)
    assert np.array_equal(wflag, self_rule), "packed flags disagree with the GPU's own statistics"
    exempt = np.repeat(near_threshold(orc, thr, W), F, axis=0)
    diff = wflag != np.repeat(orc["wflag"].astype(bool), F, axis=0)
    rep["flag_disagree"] = int(diff.sum())
    rep["flag_disagree_frac"] = float(diff.mean()) if diff.size else 0.0
    rep["exempt"] = int(exempt.sum())
    if check_flags:
        bad = diff & ~exempt
        assert not bad.any(), f"{int(bad.sum())} window flags differ outside the threshold band"
    # averages: bins whose windows are all clear of the threshold band
    n_out = gpu["weight"].shape[1]
    rep["avg"] = 0.0
    if n_out:
        wpb = K // M
        first_open = (n_seen % K) // M       # windows of the first bin seen in earlier blocks
        R = exempt.shape[0]
        ok = np.ones((R, n_out), bool)
        for b in range(n_out):
            lo = max(0, b * wpb - first_open)
            hi = min(exempt.shape[1], (b + 1) * wpb - first_open)
            ok[:, b] = ~(exempt[:, lo:hi].any(axis=1) | diff[:, lo:hi].any(axis=1))
        ea = rel_err(gpu["avg"], orc["avg"], 1.0).max(axis=2)
        rep["avg"] = float(ea[ok].max()) if ok.any() else 0.0
        if avg_rtol is not None:
            assert rep["avg"] <= avg_rtol, f"avg: worst relative error {rep['avg']:.3g}"
            # weight = n/K: float32 division on the GPU, double in the oracle
            assert np.allclose(gpu["weight"][ok], orc["weight"][ok], rtol=1.2e-7, atol=0), \
                "weights differ"
    return rep


# ---- binary16 Stokes arithmetic (precision = 2) ----------------------------------
# Each Stokes component is one binary16 rounding (relative u = 2^-11) of the exact sum
# of two binary16 inputs; everything after it is exact products and float32 sums.  So:
#   |I| is off by at most u relative, S1 by u and S2 by 2u, and t = W S2/S1^2 by 4u:
#     |d tau| <= 4u (tau + c0) (tau + c0 = c0 t >= 0, c0 = (Wd+1)/(W-1));
#   each unit polarisation vector moves by at most 2u (a relative u error per
#     component), so |d r| <= 2u (plus the normalisation's eps^2 form, negligible for
#     vectors longer than 2^-12, and the float32 terms);
#   an averaged correlation xx = (I + Q)/2 is off by at most u (|I| + |Q|)/2 <=
#     u (|xx| + |yy|) per re/im part per sample (xy, yx: u (|xy| + |yx|)).
# The float32 path's own tolerance (STAT_RTOL, AVG_RTOL) is added to each bound.
U16 = 2.0 ** -11


def _pair_bound(vis_rows, keep, K, n_out):
    """u * mean over a bin's unflagged samples of |a| + |b| for the pair of correlations
    each output component mixes ((xx, yy) or (xy, yx), same re/im part): [R, n_out, 8]
    (bins counted from the block's first sample)."""
    x = np.abs(vis_rows)                                   # [R, T, 8]
    pair = np.empty_like(x)
    for a, b in ((0, 6), (1, 7), (2, 4), (3, 5)):
        pair[..., a] = pair[..., b] = x[..., a] + x[..., b]
    out = np.zeros((x.shape[0], n_out, 8))
    for b in range(n_out):
        k = keep[:, b * K:(b + 1) * K, None]
        n = np.maximum(k.sum(axis=1), 1)
        out[:, b] = U16 * (pair[:, b * K:(b + 1) * K] * k).sum(axis=1) / n
    return out


def compare_h2(gpu, orc, vis_rows, thr, M, K, F=1):
    """Assert the bounds above for one block that starts a stream (n_seen = 0);
    vis_rows [R, T, 8] are the binary16 input values as float64.  Returns the worst
    errors relative to each bound and the flag disagreement."""
    W = M * F
    c0 = (W * thr["d"] + 1.0) / (W - 1.0)
    rep = {}
    b_tau = 4.02 * U16 * np.maximum(orc["tau"] + c0, 0.0) + STAT_RTOL * np.maximum(np.abs(orc["tau"]), 1.0)
    b_r = {k: 2.5 * U16 + STAT_RTOL * np.maximum(orc[k], W ** -0.5) for k in ("r_re", "r_im")}
    for key, bound in (("tau", b_tau), ("r_re", b_r["r_re"]), ("r_im", b_r["r_im"])):
        err = np.abs(gpu[key] - orc[key])
        rep[key + "_abs"] = float(err.max()) if err.size else 0.0
        rep[key + "_of_bound"] = float((err / bound).max()) if err.size else 0.0
        assert np.all(err <= bound), f"{key}: error {rep[key + '_abs']:.3g} beyond its bound"
    T = gpu["tau"].shape[1] * M
    wflag = expand_window_flags(gpu["flagbits"], M, T)
    self_rule = np.repeat(flag_rule_f32(gpu["tau"], gpu["r_re"], gpu["r_im"], thr), F, axis=0)
    assert np.array_equal(wflag, self_rule), "packed flags disagree with the GPU's own statistics"
    # windows whose oracle statistic lies within its bound of a threshold may flip
    near = ((np.abs(orc["tau"] - thr["s_low"]) <= b_tau) | (np.abs(orc["tau"] - thr["s_high"]) <= b_tau) |
            (np.abs(orc["r_re"] - thr["gamma"]) <= b_r["r_re"]) |
            (np.abs(orc["r_im"] - thr["gamma"]) <= b_r["r_im"]))
    near = np.repeat(near, F, axis=0)
    diff = wflag != np.repeat(orc["wflag"].astype(bool), F, axis=0)
    assert not (diff & ~near).any(), "window flags differ outside the error bounds"
    rep["flag_disagree_frac"] = float(diff.mean()) if diff.size else 0.0
    n_out = gpu["weight"].shape[1]
    rep["avg_of_bound"] = 0.0
    if n_out:
        keep = ~np.repeat(np.repeat(orc["wflag"].astype(bool), F, axis=0), M, axis=1)
        bnd = _pair_bound(vis_rows, keep, K, n_out) + AVG_RTOL * np.maximum(np.abs(orc["avg"]), 1.0)
        wpb = K // M
        ok = np.ones((wflag.shape[0], n_out), bool)
        for b in range(n_out):
            ok[:, b] = ~(near[:, b * wpb:(b + 1) * wpb].any(axis=1) | diff[:, b * wpb:(b + 1) * wpb].any(axis=1))
        err = np.abs(gpu["avg"] - orc["avg"])
        assert np.all(err[ok] <= bnd[ok]), "averages beyond their bound"
        rep["avg_of_bound"] = float((err[ok] / bnd[ok]).max()) if ok.any() else 0.0
        assert np.allclose(gpu["weight"][ok], orc["weight"][ok], rtol=1.2e-7, atol=0)
    return rep
