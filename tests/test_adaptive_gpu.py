"""Online per-stream SK thresholds on the GPU against the FP64 oracle
(oracle/adaptive.py states the rule).

Each block is checked as one step of the state machine: the oracle starts from the
GPU's own state (float32 values widened exactly), both flag the block, and then the
statistics, flags, averages and the advanced state are compared.  Flags may differ
only where a statistic lies within 1e-4 of the row's threshold; rows with such a
window are left out of the state comparison (their clean-window sets may differ).
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2412_14775_b300 import RfiStream, binding, default_thresholds
from paper_2412_14775_b300.binding import RfiError
from parity import gpu_to_numpy, rel_err, to_device_rows

pytestmark = pytest.mark.gpu

BAND = 1e-4


def _rows(d, dtype):
    v = d.reshape(-1, *d.shape[-3:])
    return v.astype(np.float16) if dtype == "f16" else v


def _window_flags(flagbits, M, F, nw):
    R = flagbits.shape[0]
    t = np.arange(nw * M)
    bits = (flagbits[:, t // 32] >> (t % 32).astype(np.uint32)) & 1
    w = bits.reshape(R, nw, M)
    assert np.all(w == w[:, :, :1])
    return w[::F, :, 0].astype(bool)          # one row per footprint


def _step(st, orc, blk_dev, blk_host, thr, M, K, F):
    gpu_state = st.adaptive_state()
    orc.state[:] = gpu_state[:, :3].astype(np.float64)
    n_seen = orc.groups[0].n_seen
    g = gpu_to_numpy(st.process(blk_dev))
    o = orc.process(blk_host)
    W = M * F
    for key, floor in (("tau", 1.0), ("r_re", W ** -0.5), ("r_im", W ** -0.5)):
        e = rel_err(g[key], o[key], floor)
        assert float(np.max(e)) <= 1e-5, (key, float(np.max(e)))
    lo, hi = o["s_low_used"][:, None], o["s_high_used"][:, None]

    def near(x, t, floor):
        return np.abs(x - t) <= BAND * np.maximum(np.abs(t), floor)
    exempt = (near(o["tau"], lo, 1.0) | near(o["tau"], hi, 1.0) |
              near(o["r_re"], thr["gamma"], W ** -0.5) | near(o["r_im"], thr["gamma"], W ** -0.5))
    nw = g["tau"].shape[1]
    gf = _window_flags(g["flagbits"], M, F, nw)
    diff = gf != o["wflag"].astype(bool)
    assert not (diff & ~exempt).any(), f"{int((diff & ~exempt).sum())} flags differ"
    # averages in bins clear of the band
    n_out = g["weight"].shape[1]
    if n_out:
        wpb, first_open = K // M, (n_seen % K) // M
        ex_rows = np.repeat(exempt | diff, F, axis=0)
        for b in range(n_out):
            lo_w, hi_w = max(0, b * wpb - first_open), min(nw, (b + 1) * wpb - first_open)
            ok = ~ex_rows[:, lo_w:hi_w].any(axis=1)
            ea = rel_err(g["avg"][ok, b], o["avg"][ok, b], 1.0)
            assert ea.size == 0 or float(ea.max()) <= 1e-5
    # the advanced state
    new = st.adaptive_state()
    clean = ~(exempt | diff).any(axis=1)
    assert np.array_equal(new[clean, 0], orc.state[clean, 0]), "clean-window counts differ"
    for c in (1, 2):
        e = rel_err(new[clean, c].astype(np.float64), orc.state[clean, c], 1.0)
        assert e.size == 0 or float(e.max()) <= 2e-5, (c, float(e.max()))
    return gf, o


@pytest.mark.parametrize("dtype,M,K,F,P", [("f32", 16, 64, 1, 4), ("f16", 8, 32, 1, 2),
                                           ("f32", 10, 20, 2, 2), ("f16", 5, 10, 1, 1),
                                           ("f32", 64, 128, 1, 8)])
def test_online_thresholds_match_oracle(dtype, M, K, F, P):
    N, C, T, nblk = 6, 8, 8 * M, 6
    thr = default_thresholds(M * F)
    d = synth.tiny_block(seed=51, stations=N, channels=C, T=T * nblk, duty=0.05)["vis"]
    st = RfiStream(N, C, M, K, thr, dtype, lanes_per_row=P, window_F=F, adaptive=1)
    st.set_adaptation(alpha=1.0 / 16, k_sigma=3.0, n_warm=6)
    R = st.R
    orc = oracle.AdaptiveOracleStream(R, M, K, **thr, alpha=1.0 / 16, k_sigma=3.0, n_warm=6, F=F,
                                      compensated=st.options["compensated"] == 1)
    warm = 0
    for k in range(nblk):
        blk = d[:, :, k * T:(k + 1) * T]
        _, o = _step(st, orc, to_device_rows(blk, dtype), _rows(blk, dtype), thr, M, K, F)
        warm = max(warm, int((o["s_low_used"] != thr["s_low"]).sum()))
    assert warm > 0, "no row reached its own thresholds"
    st.close()


def test_before_warm_up_equals_fixed_thresholds():
    """Until n_warm clean windows, the adaptive kernels give the fixed kernels' outputs
    bit for bit (and the batch kernel the single-stream kernel's)."""
    M, K, T = 16, 64, 256
    thr = default_thresholds(M)
    d = synth.tiny_block(seed=53, stations=7, channels=9, T=2 * T)["vis"]
    v = to_device_rows(d, "f32")
    a = RfiStream(7, 9, M, K, thr, "f32", lanes_per_row=4)
    b = RfiStream(7, 9, M, K, thr, "f32", lanes_per_row=4, adaptive=1)
    c = RfiStream(7, 9, M, K, thr, "f32", lanes_per_row=4, adaptive=1)
    b.set_adaptation(n_warm=10 ** 6)
    c.set_adaptation(n_warm=10 ** 6)
    for k in range(2):
        blk = v[:, k * T:(k + 1) * T].contiguous()
        x, y = a.process(blk), b.process(blk)
        z = c.alloc_outputs(T)
        binding.rfi_process_batch([c.ctx], [blk], [T], [z["flags"]], [z["avg"]], [z["weight"]],
                                  [z["stats"]])
        torch.cuda.synchronize()
        for key in ("flags", "avg", "weight", "stats"):
            assert torch.equal(x[key], y[key]), key
            assert torch.equal(x[key], z[key]), key
    assert np.array_equal(b.adaptive_state(), c.adaptive_state())


def test_adaptation_follows_a_mistuned_stream():
    """Thresholds set for the wrong SK shape flag much of a clean stream; the online
    thresholds bring the rate down once they have learned the stream."""
    M, K, T = 16, 256, 256
    thr = dict(default_thresholds(M))
    thr["s_low"], thr["s_high"] = 1.1, 1.6          # centred away from the clean tau
    d = synth.tiny_block(seed=57, stations=8, channels=16, T=8 * T, duty=0.0)["vis"]
    fixed = RfiStream(8, 16, M, K, thr, "f32")
    ad = RfiStream(8, 16, M, K, thr, "f32", adaptive=1)
    ad.set_adaptation(alpha=1.0 / 32, k_sigma=3.0, n_warm=8)
    rates_f, rates_a = [], []
    for k in range(8):
        blk = to_device_rows(d[:, :, k * T:(k + 1) * T], "f32")
        for st, rates in ((fixed, rates_f), (ad, rates_a)):
            g = gpu_to_numpy(st.process(blk))
            rates.append(_window_flags(g["flagbits"], M, 1, T // M).mean())
    # the fixed thresholds flag about 73 % of the windows throughout; the online ones
    # learn the clean distribution (from the windows they accept) and widen block by block
    assert min(rates_f) > 0.6
    assert rates_a[7] < rates_a[5] < rates_a[3] < rates_a[1], rates_a
    assert rates_a[7] < 0.3 * rates_f[7], (rates_a, rates_f)


def test_state_checkpoint_reset_and_arguments():
    M, K, T = 16, 64, 128
    thr = default_thresholds(M)
    d = synth.tiny_block(seed=59, stations=5, channels=6, T=4 * T)["vis"]
    v = to_device_rows(d, "f32")
    a = RfiStream(5, 6, M, K, thr, "f32", adaptive=1)
    a.set_adaptation(alpha=0.1, k_sigma=2.0, n_warm=3)
    for k in range(2):
        a.process(v[:, k * T:(k + 1) * T].contiguous())
    blob = binding.rfi_get_state(a.ctx)
    b = RfiStream(5, 6, M, K, thr, "f32", adaptive=1)
    binding.rfi_set_state(b.ctx, blob)             # state and parameters both move
    for k in range(2, 4):
        x = a.process(v[:, k * T:(k + 1) * T].contiguous())
        y = b.process(v[:, k * T:(k + 1) * T].contiguous())
        torch.cuda.synchronize()
        for key in ("flags", "avg", "weight", "stats"):
            assert torch.equal(x[key], y[key]), key
    assert np.array_equal(a.adaptive_state(), b.adaptive_state())
    assert a.adaptive_state()[:, 0].max() > 0
    a.reset()
    assert not a.adaptive_state().any()
    with pytest.raises(RfiError):
        a.set_adaptation(alpha=1.5)
    with pytest.raises(RfiError):
        a.set_adaptation(n_warm=0)
    with pytest.raises(RfiError):          # a context without the option
        RfiStream(5, 6, M, K, thr, "f32").set_adaptation()
    for bad in (dict(loader=1), dict(max_registers=64), dict(precision=1),
                dict(buffered_stores=1), dict(partial_windows=1)):
        with pytest.raises(RfiError):
            RfiStream(5, 6, M, K, thr, "f32", adaptive=1, **bad)
