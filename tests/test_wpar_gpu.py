"""Window-parallel lanes (lane_split = 1): the lanes of a row take whole windows in turn.

Every block of a stream against the FP64 oracle (the tolerances of tests/parity.py),
including windows of odd length, T x F footprints, bins that straddle blocks (so a
block starts in the middle of a round of windows), and bit-identity of any split of a
stream at multiples of M with one block.
"""
import numpy as np
import pytest
import torch

import synth
from paper_2412_14775_b300 import RfiStream, binding, default_thresholds
from paper_2412_14775_b300.binding import RfiError
from parity import to_device_rows
from test_parity_gpu import _check_stream

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,M,K,P,F,Ts", [
    ("f16", 5, 250, 2, 4, [250, 250]),          # the paper's 5 x 4 footprint
    ("f32", 5, 20, 2, 4, [35, 45, 20]),         # bins straddle blocks, odd M
    ("f32", 5, 20, 4, 4, [15, 65]),
    ("f16", 10, 40, 2, 2, [50, 70]),            # 10 x 2 footprint
    ("f16", 8, 32, 2, 1, [64, 24, 40]),
    ("f16", 8, 32, 4, 1, [96, 32]),
    ("f32", 16, 64, 4, 1, [48, 80]),
    ("f16", 3, 12, 2, 1, [9, 15, 12]),          # odd M, one sample per 16-byte load
    ("f32", 64, 128, 2, 1, [128, 64]),          # long windows: 16 chunks per window
    ("f32", 4, 32, 8, 1, [40, 24]),
    ("f16", 10, 250, 2, 2, [250, 250]),         # 25 windows per bin: rounds straddle bins
    ("f32", 8, 24, 2, 1, [40, 56, 24]),         # 3 windows per bin
    ("f16", 5, 15, 2, 4, [35, 45]),
    ("f32", 4, 20, 4, 1, [28, 36]),             # 5 windows per bin, 4 lanes
], ids=["f16_5x4", "f32_5x4_straddle", "f32_5x4_P4", "f16_10x2", "f16_M8", "f16_M8_P4",
        "f32_M16_P4", "f16_M3", "f32_M64", "f32_M4_P8", "f16_10x2_K250", "f32_M8_K3M",
        "f16_5x4_K3M", "f32_M4_K5M_P4"])
def test_window_parallel_matches_oracle(dtype, M, K, P, F, Ts):
    reps = _check_stream(7, 8, M, K, Ts, dtype, seed=91, lanes_per_row=P,
                         window_F=F, lane_split=1)
    assert reps


def test_window_parallel_splits_bit_identical():
    M, K, T = 5, 20, 400
    thr = default_thresholds(5 * 4)
    d = synth.tiny_block(seed=93, stations=8, channels=8, T=T, duty=0.08)["vis"]
    v = to_device_rows(d, "f16")
    for P in (2, 4):
        opts = dict(lanes_per_row=P, window_F=4, lane_split=1)
        one = RfiStream(8, 8, M, K, thr, "f16", **opts)
        assert one.options["lane_split"] == 1
        a = one.process(v)
        st = RfiStream(8, 8, M, K, thr, "f16", **opts)
        parts = [st.process(v[:, lo:hi].contiguous())
                 for lo, hi in ((0, 5), (5, 35), (35, 200), (200, 215), (215, 400))]
        torch.cuda.synchronize()
        for key in ("avg", "weight"):
            assert torch.equal(torch.cat([p[key] for p in parts], dim=1), a[key]), (P, key)
        assert torch.equal(torch.cat([p["stats"] for p in parts], dim=2), a["stats"]), P
        # flag bits: concatenate the blocks' bit streams
        bits = []
        for p in parts:
            n = p["stats"].shape[2] * M
            w = p["flags"].cpu().numpy().view(np.uint32).astype(np.uint64)
            t = np.arange(n)
            bits.append(((w[:, t // 32] >> (t % 32).astype(np.uint64)) & 1).astype(bool))
        w = a["flags"].cpu().numpy().view(np.uint32).astype(np.uint64)
        t = np.arange(T)
        ref = ((w[:, t // 32] >> (t % 32).astype(np.uint64)) & 1).astype(bool)
        assert np.array_equal(np.concatenate(bits, axis=1), ref), P
        one.close(); st.close()


@pytest.mark.parametrize("prec", [0, 2])
def test_window_parallel_96_registers_bit_identical(prec):
    """The 96-register budget of binary16 odd windows changes residency only: the bits
    of the 128-register kernel, alone and in a batch with it."""
    M, K, T = 5, 20, 200
    thr = default_thresholds(5 * 4)
    d = synth.tiny_block(seed=94, stations=8, channels=8, T=T, duty=0.08)["vis"]
    v = to_device_rows(d, "f16")
    opts = dict(lanes_per_row=2, window_F=4, lane_split=1, precision=prec, warps_per_block=4)
    a = RfiStream(8, 8, M, K, thr, "f16", **opts)
    b = RfiStream(8, 8, M, K, thr, "f16", max_registers=96, **opts)
    assert b.options["max_registers"] == 96
    x, y = a.process(v), b.process(v)
    torch.cuda.synchronize()
    for key in ("flags", "avg", "weight", "stats"):
        assert torch.equal(x[key], y[key]), key
    outs = [s.alloc_outputs(T) for s in (a, b)]
    binding.rfi_process_batch([a.ctx, b.ctx], [v, v], [T, T], [o["flags"] for o in outs],
                              [o["avg"] for o in outs], [o["weight"] for o in outs],
                              [o["stats"] for o in outs])
    c = RfiStream(8, 8, M, K, thr, "f16", **opts)
    c.process(v)
    z = c.process(v)
    torch.cuda.synchronize()
    for o in outs:
        for key in ("flags", "avg", "weight", "stats"):
            assert torch.equal(o[key], z[key]), key
    with pytest.raises(RfiError):            # built for binary16 odd windows only
        RfiStream(8, 8, 8, 32, default_thresholds(8), "f16", lanes_per_row=2, lane_split=1,
                  max_registers=96)
    a.close(); b.close(); c.close()


def test_window_parallel_option_checks():
    thr = default_thresholds(8)
    for bad in (dict(lane_split=1, lanes_per_row=1), dict(lane_split=1, lanes_per_row=16),
                dict(lane_split=2), dict(lane_split=1, adaptive=1),
                dict(lane_split=1, partial_windows=1), dict(lane_split=1, window_hop=4),
                dict(lane_split=1, loader=1), dict(lane_split=1, max_registers=64),
                dict(lane_split=1, lanes_per_row=4, window_F=16)):
        with pytest.raises(RfiError):
            RfiStream(4, 16, 8, 32, thr, "f32", **bad)
    with pytest.raises(RfiError):            # a bin of one window, fewer than 2 lanes' worth
        RfiStream(4, 4, 8, 8, thr, "f32", lane_split=1)
    a = RfiStream(4, 4, 8, 32, thr, "f32", lane_split=1)
    b = RfiStream(4, 4, 8, 32, thr, "f32")
    with pytest.raises(RfiError):            # a batch does not mix lane splits
        z = [s.alloc_outputs(32) for s in (a, b)]
        v = torch.zeros((a.R, 32, 4, 2), device="cuda")
        binding.rfi_process_batch([a.ctx, b.ctx], [v, v], [32, 32], [o["flags"] for o in z],
                                  [o["avg"] for o in z], [o["weight"] for o in z],
                                  [o["stats"] for o in z])
    blob = binding.rfi_get_state(a.ctx)
    with pytest.raises(RfiError):            # the carry means something else per lane
        binding.rfi_set_state(b.ctx, blob)
    a.close(); b.close()


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_window_parallel_edge_values(dtype):
    """All-zero windows and non-finite samples, as for the default lane split."""
    from test_parity_gpu import _oracle_input, compare, run_gpu
    import oracle
    M, K, T = 8, 32, 64
    thr = default_thresholds(M)
    d = synth.tiny_block(seed=95, stations=3, channels=4, T=T)["vis"].copy()
    d[0, 0] = 0.0
    d[1, 1, 5, 2, 0] = np.nan
    d[2, 3, 40, 0, 1] = np.inf
    d[3, 2, 17, 3, 0] = -np.inf
    st = RfiStream(3, 4, M, K, thr, dtype, lanes_per_row=4, lane_split=1)
    g = run_gpu(st, to_device_rows(d, dtype))
    o = oracle.OracleStream(st.R, M, K, **thr).process(_oracle_input(d, dtype))
    assert g["tau"][0, 0] == np.float32(-(M * thr["d"] + 1) / (M - 1))
    compare(g, o, thr, M, K)
    assert np.isfinite(g["avg"]).all() and np.isfinite(g["weight"]).all()
    st.close()


def test_window_parallel_batch_bit_identical():
    """Uneven window-parallel streams in one persistent launch (and from a CUDA graph)
    give each stream's single-launch results bit for bit, block after block."""
    M, K, T = 5, 20, 100
    thr = default_thresholds(5 * 4)
    geo = [(5, 8), (9, 4), (3, 12), (7, 8)]
    opts = dict(lanes_per_row=2, window_F=4, lane_split=1)
    data = [synth.tiny_block(seed=97 + i, stations=n, channels=c, T=2 * T, duty=0.08)["vis"]
            for i, (n, c) in enumerate(geo)]
    solo = [RfiStream(n, c, M, K, thr, "f16", **opts) for n, c in geo]
    bat = [RfiStream(n, c, M, K, thr, "f16", **opts) for n, c in geo]
    g = binding.rfi_batch_graph_create([s.ctx for s in bat[2:]], [T, T])
    for k in range(2):
        vis = [to_device_rows(d[:, :, k * T:(k + 1) * T], "f16") for d in data]
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


@pytest.mark.parametrize("seed", range(6))
def test_window_parallel_random_combinations(seed):
    """Seeded random window, footprint, lanes per row, bin and block lengths."""
    rng = np.random.default_rng(3000 + seed)
    ran = 0
    while ran < 3:
        dtype = str(rng.choice(["f32", "f16"]))
        M = int(rng.choice([2, 3, 4, 5, 6, 8, 10, 12, 16, 20, 32]))
        F = int(rng.choice([1, 1, 2, 4]))
        P = int(rng.choice([2, 4, 8]))
        if P * F > 32 or M * F < 2:
            continue
        K = M * int(rng.integers(P, 3 * P + 1))
        Ts = [M * int(rng.integers(1, 3 * P + 1)) for _ in range(int(rng.integers(1, 4)))]
        _check_stream(int(rng.integers(2, 7)), F * int(rng.integers(1, 4)), M, K, Ts, dtype,
                      seed=int(rng.integers(1, 1 << 30)), lanes_per_row=P, window_F=F,
                      lane_split=1)
        ran += 1


def test_window_parallel_host_path_and_state():
    """The host-buffer entry point (rows staged in chunks) and a saved / restored state
    give the device path's results bit for bit."""
    M, K, T = 8, 32, 48
    thr = default_thresholds(M)
    d = synth.tiny_block(seed=99, stations=6, channels=8, T=4 * T, duty=0.08)["vis"]
    v = to_device_rows(d, "f32")
    opts = dict(lanes_per_row=4, lane_split=1)
    dev = RfiStream(6, 8, M, K, thr, "f32", **opts)
    host = RfiStream(6, 8, M, K, thr, "f32", host_max_T=T, host_chunks=3, **opts)
    for k in range(2):
        blk = v[:, k * T:(k + 1) * T].contiguous()
        x = dev.process(blk)
        y = host.process_host(blk.cpu().pin_memory())
        torch.cuda.synchronize()
        for key in ("flags", "avg", "weight", "stats"):
            assert torch.equal(x[key].cpu(), y[key]), (k, key)
    other = RfiStream(6, 8, M, K, thr, "f32", **opts)
    binding.rfi_set_state(other.ctx, binding.rfi_get_state(dev.ctx))
    for k in range(2, 4):
        blk = v[:, k * T:(k + 1) * T].contiguous()
        x, z = dev.process(blk), other.process(blk)
        torch.cuda.synchronize()
        for key in ("flags", "avg", "weight", "stats"):
            assert torch.equal(x[key], z[key]), (k, key)
    dev.close(); host.close(); other.close()
