"""Overlapping (sliding) windows on the GPU against the FP64 oracle (oracle/sliding.py
states the rule: a window of M samples every H = M/2 samples, a sample flagged when
any window holding it is, final M - H samples after it).

A stream is fed to both block by block; the windows, the flag bits of the samples that
became final and the closed bins of every call are concatenated and compared with the
tolerances of tests/parity.py.  Samples held by a window whose statistic lies within
the threshold band may be flagged either way; bins holding such samples are left out
of the average comparison.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2412_14775_b300 import RfiStream, binding, default_thresholds
from paper_2412_14775_b300.binding import RfiError
from parity import AVG_RTOL, BAND, STAT_RTOL, rel_err, to_device_rows

pytestmark = pytest.mark.gpu


def _bits(words, n):
    w = np.asarray(words).view(np.uint32).astype(np.uint64)
    t = np.arange(n)
    return ((w[..., t // 32] >> (t % 32).astype(np.uint64)) & 1).astype(bool)


def _run(st, orc, vis_np, cuts, dtype):
    """Feed both the blocks vis[:, a:b]; return the concatenated outputs of each."""
    g_parts, o_parts = [], []
    edges = (0,) + tuple(cuts) + (vis_np.shape[-3],)
    for a, b in zip(edges[:-1], edges[1:]):
        blk = vis_np[:, :, a:b]
        nwin, f0 = st.windows_for(b - a)
        o_nwin, o_f0 = orc.windows_for(b - a)
        assert (nwin, f0) == (o_nwin, o_f0)
        assert st.outputs_for(b - a) == orc.outputs_for(b - a)
        g = st.process(to_device_rows(blk, dtype))
        torch.cuda.synchronize()
        rows = blk.reshape(-1, *blk.shape[-3:])
        o = orc.process(rows.astype(np.float16) if dtype == "f16" else rows)
        st_np = g["stats"].cpu().numpy()
        g_parts.append(dict(tau=st_np[0], r_re=st_np[1], r_im=st_np[2],
                            bits=_bits(g["flags"].cpu().numpy(), nwin * st.bits_per_window),
                            avg=g["avg"].cpu().numpy().reshape(st.R, -1, 8),
                            weight=g["weight"].cpu().numpy()))
        o_parts.append(dict(tau=o["tau"], r_re=o["r_re"], r_im=o["r_im"], wflag=o["wflag"],
                            bits=_bits(o["flagbits"], nwin * orc.H), avg=o["avg"],
                            weight=o["weight"]))

    def cat(parts):
        return {k: np.concatenate([p[k] for p in parts], axis=1) for k in parts[0]}
    return cat(g_parts), cat(o_parts)


def _compare(g, o, thr, M, H, K):
    W = M
    for key, floor in (("tau", 1.0), ("r_re", W ** -0.5), ("r_im", W ** -0.5)):
        x = g[key].astype(np.float64)
        both_nan = np.isnan(x) & np.isnan(o[key])
        assert not (np.isnan(x) ^ np.isnan(o[key])).any(), f"{key}: NaN on one side only"
        e = np.where(both_nan, 0.0, rel_err(x, o[key], floor))
        assert e.size == 0 or float(e.max()) <= STAT_RTOL, (key, float(e.max()))

    def near(x, t, floor):
        return np.abs(x - t) <= BAND * np.maximum(np.abs(t), floor)
    nearw = (near(o["tau"], thr["s_low"], 1.0) | near(o["tau"], thr["s_high"], 1.0) |
             near(o["r_re"], thr["gamma"], W ** -0.5) | near(o["r_im"], thr["gamma"], W ** -0.5))
    R, E = nearw.shape
    n = g["bits"].shape[1]
    assert n == E * H
    # sample t lies in windows t//H - 1 and t//H (those that exist)
    seg_ex = nearw.copy()
    seg_ex[:, 1:] |= nearw[:, :-1]
    ex = np.repeat(seg_ex, H, axis=1)
    diff = g["bits"] != o["bits"]
    assert not (diff & ~ex).any(), f"{int((diff & ~ex).sum())} sample flags differ"
    nb = g["weight"].shape[1]
    for b in range(nb):
        ok = ~(ex[:, b * K:(b + 1) * K] | diff[:, b * K:(b + 1) * K]).any(axis=1)
        e = rel_err(g["avg"][ok, b].astype(np.float64), o["avg"][ok, b], 1.0)
        assert e.size == 0 or float(e.max()) <= AVG_RTOL, (b, float(e.max()))
        # weight = n/K: float32 division on the GPU, double in the oracle
        assert np.allclose(g["weight"][ok, b].astype(np.float64), o["weight"][ok, b],
                           rtol=1.2e-7, atol=0), b
    return int(ex.sum()), int(o["wflag"].sum())


@pytest.mark.parametrize("dtype,M,K,P,cuts,T", [
    ("f32", 16, 64, 4, (64, 128, 192), 256),      # bins inside blocks
    ("f32", 16, 24, 2, (40, 96, 200), 256),       # bins straddle blocks, uneven blocks
    ("f16", 16, 32, 2, (24, 120), 192),
    ("f16", 8, 12, 1, (4, 8, 60), 96),            # blocks of one hop
    ("f32", 10, 20, 1, (15, 35, 100), 160),       # odd hop
    ("f16", 10, 30, 1, (45,), 120),               # odd hop, one sample per 16-byte load
], ids=["f32_M16", "f32_M16_straddle", "f16_M16", "f16_M8_small_blocks", "f32_M10",
        "f16_M10"])
def test_sliding_windows_match_oracle(dtype, M, K, P, cuts, T):
    H = M // 2
    N, C = 7, 12
    thr = default_thresholds(M)
    d = synth.tiny_block(seed=81, stations=N, channels=C, T=T, duty=0.06)["vis"]
    st = RfiStream(N, C, M, K, thr, dtype, lanes_per_row=P, window_hop=H)
    assert st.options["window_hop"] == H and st.bits_per_window == H
    orc = oracle.SlidingOracleStream(st.R, M, H, K, **thr)
    g, o = _run(st, orc, d, cuts, dtype)
    exempt, flagged = _compare(g, o, thr, M, H, K)
    assert flagged > 0 and o["bits"].any()
    st.close()


def test_sliding_block_splits_bit_identical():
    """Any split of the stream at multiples of H gives the outputs of one block, bit for
    bit (the pending segment's totals and averaging sums are carried exactly)."""
    M, H, K, T = 16, 8, 32, 512
    thr = default_thresholds(M)
    d = synth.tiny_block(seed=83, stations=9, channels=8, T=T, duty=0.08)["vis"]
    v = to_device_rows(d, "f32")
    for P in (1, 2, 4):
        one = RfiStream(9, 8, M, K, thr, "f32", lanes_per_row=P, window_hop=H)
        a = one.process(v)
        st = RfiStream(9, 8, M, K, thr, "f32", lanes_per_row=P, window_hop=H)
        parts = []
        for lo, hi in ((0, 8), (8, 24), (24, 160), (160, 168), (168, 512)):
            parts.append(st.process(v[:, lo:hi].contiguous()))
        torch.cuda.synchronize()
        for key in ("avg", "weight"):
            assert torch.equal(torch.cat([p[key] for p in parts], dim=1), a[key]), (P, key)
        got = torch.cat([p["stats"] for p in parts], dim=2)
        assert torch.equal(got, a["stats"]), P
        bits = np.concatenate([_bits(p["flags"].cpu().numpy(), p["stats"].shape[2] * H)
                               for p in parts], axis=1)
        assert np.array_equal(bits, _bits(a["flags"].cpu().numpy(), a["stats"].shape[2] * H))
        one.close(); st.close()


def test_sliding_host_path_and_state():
    """The host-buffer entry point and a saved/restored state give the device path's
    results."""
    M, H, K, T = 16, 8, 48, 96
    thr = default_thresholds(M)
    d = synth.tiny_block(seed=85, stations=6, channels=8, T=4 * T, duty=0.08)["vis"]
    v = to_device_rows(d, "f32")
    dev = RfiStream(6, 8, M, K, thr, "f32", window_hop=H)
    host = RfiStream(6, 8, M, K, thr, "f32", window_hop=H, host_max_T=T, host_chunks=3)
    for k in range(2):
        blk = v[:, k * T:(k + 1) * T].contiguous()
        x = dev.process(blk)
        y = host.process_host(blk.cpu().pin_memory())
        torch.cuda.synchronize()
        for key in ("flags", "avg", "weight", "stats"):
            assert torch.equal(x[key].cpu(), y[key]), (k, key)
    blob = binding.rfi_get_state(dev.ctx)
    other = RfiStream(6, 8, M, K, thr, "f32", window_hop=H)
    binding.rfi_set_state(other.ctx, blob)
    for k in range(2, 4):
        blk = v[:, k * T:(k + 1) * T].contiguous()
        x, z = dev.process(blk), other.process(blk)
        torch.cuda.synchronize()
        for key in ("flags", "avg", "weight", "stats"):
            assert torch.equal(x[key], z[key]), (k, key)
    dev.reset()
    assert dev.windows_for(T) == ((T - M) // H + 1, 0)
    dev.close(); host.close(); other.close()


def test_sliding_option_checks():
    thr = default_thresholds(16)
    for bad in (dict(window_hop=4), dict(window_hop=5), dict(window_hop=8, adaptive=1),
                dict(window_hop=8, partial_windows=1), dict(window_hop=8, window_F=2),
                dict(window_hop=8, loader=1), dict(window_hop=8, max_registers=64),
                dict(window_hop=8, lanes_per_row=8)):
        with pytest.raises(RfiError):
            RfiStream(4, 4, 16, 32, thr, "f32", **bad)
    with pytest.raises(RfiError):                   # K must be a multiple of H
        RfiStream(4, 4, 16, 12, thr, "f32", window_hop=8)
    a = RfiStream(4, 4, 16, 24, thr, "f32", window_hop=8)   # K = 24: a multiple of H only
    b = RfiStream(4, 4, 16, 32, thr, "f32")
    with pytest.raises(RfiError):                   # T must be a multiple of H
        a.process(torch.zeros((a.R, 12, 4, 2), device="cuda"))
    with pytest.raises(RfiError):                   # a batch does not mix kinds
        z = [s.alloc_outputs(32) for s in (a, b)]
        v = torch.zeros((a.R, 32, 4, 2), device="cuda")
        binding.rfi_process_batch([a.ctx, b.ctx], [v, v], [32, 32], [o["flags"] for o in z],
                                  [o["avg"] for o in z], [o["weight"] for o in z],
                                  [o["stats"] for o in z])
    a.close(); b.close()


@pytest.mark.parametrize("seed", range(8))
def test_sliding_random_combinations_match_oracle(seed):
    """Seeded random geometry, window, lanes per row, bin length and block lengths."""
    rng = np.random.default_rng(2000 + seed)
    ran = 0
    while ran < 3:
        dtype = str(rng.choice(["f32", "f16"]))
        M = int(rng.choice([4, 6, 8, 10, 12, 16, 20, 24, 32, 64]))
        H = M // 2
        spu = 2 if (dtype == "f16" and H % 2 == 0) else 1
        ps = [p for p in (1, 2, 4) if H % (p * spu) == 0]
        if dtype == "f16" and spu == 1:
            ps = [1]
        P = int(rng.choice(ps))
        K = H * int(rng.integers(1, 7))
        N, C = int(rng.integers(2, 8)), int(rng.integers(1, 9))
        nblk = int(rng.integers(1, 5))
        lens = [H * int(rng.integers(1, 8)) for _ in range(nblk)]
        T = sum(lens)
        cuts = tuple(np.cumsum(lens)[:-1].tolist())
        thr = dict(d=1.0, s_low=float(rng.uniform(0.2, 0.7)), s_high=float(rng.uniform(1.3, 2.5)),
                   gamma=float(rng.uniform(0.3, 0.9)), eps=2.0 ** -23)
        d = synth.tiny_block(seed=int(rng.integers(1, 1 << 30)), stations=N, channels=C, T=T,
                             duty=0.08)["vis"]
        st = RfiStream(N, C, M, K, thr, dtype, lanes_per_row=P, window_hop=H)
        orc = oracle.SlidingOracleStream(st.R, M, H, K, **thr)
        g, o = _run(st, orc, d, cuts, dtype)
        _compare(g, o, thr, M, H, K)
        st.close()
        ran += 1


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_sliding_non_finite_samples(dtype):
    """A NaN or an infinity makes both windows that hold it flagged, so every sample of
    them is flagged and left out of the averages, which stay finite."""
    M, H, K, T = 16, 8, 32, 96
    thr = default_thresholds(M)
    d = synth.tiny_block(seed=87, stations=3, channels=4, T=T)["vis"].copy()
    d[0, 0] = 0.0
    d[1, 1, 5, 2, 0] = np.nan
    d[2, 3, 40, 0, 1] = np.inf
    d[3, 2, 17, 3, 0] = -np.inf
    st = RfiStream(3, 4, M, K, thr, dtype, window_hop=H)
    orc = oracle.SlidingOracleStream(st.R, M, H, K, **thr)
    g, o = _run(st, orc, d, (48,), dtype)
    _compare(g, o, thr, M, H, K)
    rows = d.reshape(st.R, T, 4, 2)
    for r in range(st.R):
        bad = np.flatnonzero(~np.isfinite(rows[r]).all(axis=(1, 2)))
        for t in bad:                # windows t//H - 1 and t//H hold it
            lo, hi = max(0, (t // H - 1) * H), min(t // H * H + M, g["bits"].shape[1])
            assert g["bits"][r, lo:hi].all(), (r, t)
    assert np.isfinite(g["avg"]).all() and np.isfinite(g["weight"]).all()
    st.close()


def test_sliding_batch_bit_identical():
    """Uneven overlapping-window streams in one persistent launch, and from a CUDA graph,
    give each stream's single-launch results bit for bit, block after block (the pending
    hop carried between blocks either way)."""
    M, H, K, T = 16, 8, 48, 72
    thr = default_thresholds(M)
    geo = [(5, 8), (9, 4), (3, 12), (7, 8)]
    data = [synth.tiny_block(seed=89 + i, stations=n, channels=c, T=3 * T, duty=0.08)["vis"]
            for i, (n, c) in enumerate(geo)]
    solo = [RfiStream(n, c, M, K, thr, "f32", window_hop=H, lanes_per_row=2) for n, c in geo]
    bat = [RfiStream(n, c, M, K, thr, "f32", window_hop=H, lanes_per_row=2) for n, c in geo]
    g = binding.rfi_batch_graph_create([s.ctx for s in bat[2:]], [T, T])
    for k in range(3):
        vis = [to_device_rows(d[:, :, k * T:(k + 1) * T], "f32") for d in data]
        outs = [s.alloc_outputs(T) for s in bat]
        binding.rfi_process_batch([s.ctx for s in bat[:2]], vis[:2], [T, T],
                                  [o["flags"] for o in outs[:2]], [o["avg"] for o in outs[:2]],
                                  [o["weight"] for o in outs[:2]], [o["stats"] for o in outs[:2]])
        binding.rfi_batch_graph_launch(g, vis[2:], [o["flags"] for o in outs[2:]],
                                       [o["avg"] for o in outs[2:]],
                                       [o["weight"] for o in outs[2:]],
                                       [o["stats"] for o in outs[2:]])
        exp = [s.process(v) for s, v in zip(solo, vis)]
        torch.cuda.synchronize()
        for e, o in zip(exp, outs):
            for key in ("flags", "avg", "weight", "stats"):
                assert torch.equal(e[key], o[key]), (k, key)
    binding.rfi_batch_graph_destroy(g)
    for s in solo + bat:
        s.close()
