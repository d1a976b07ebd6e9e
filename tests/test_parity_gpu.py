"""Parity of the sm_103a path (through the C ABI) with the FP64 oracle.

Every case runs the CUDA kernels and the oracle on the same seeded input and compares
them element by element with the tolerances stated in tests/parity.py.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2412_14775_b300 import RfiStream, autotune, binding, default_thresholds
from paper_2412_14775_b300.binding import RfiError
from parity import compare, gpu_to_numpy, run_gpu, to_device_rows

pytestmark = pytest.mark.gpu


def _oracle_input(vis_np, dtype):
    """The exact values the GPU reads: float32 as is, or rounded to binary16."""
    v = vis_np.reshape(-1, *vis_np.shape[-3:])
    return v.astype(np.float16) if dtype == "f16" else v


def _check_stream(stations, channels, M, K, Ts, dtype, thr=None, seed=3, **opts):
    """Run blocks of lengths Ts through one context and one oracle stream; compare
    every block."""
    F = opts.get("window_F", 1)
    thr = thr or default_thresholds(M * F)
    data = synth.tiny_block(seed=seed, stations=stations, channels=channels, T=sum(Ts),
                            duty=0.08)["vis"]
    R = data.shape[0] * data.shape[1]
    st = RfiStream(stations, channels, M, K, thr, dtype, **opts)
    orc = oracle.OracleStream(R, M, K, **thr, F=F, partial=bool(opts.get("partial_windows")))
    t0 = 0
    reps = []
    for T in Ts:
        blk = data[:, :, t0:t0 + T]
        n_seen = orc.n_seen
        g = run_gpu(st, to_device_rows(blk, dtype))
        o = orc.process(_oracle_input(blk, dtype))
        reps.append(compare(g, o, thr, M, K, n_seen=n_seen, F=F))
        t0 += T
    binding.rfi_check(st.ctx)           # no error word (in the debug-bounds build: no
    st.close()                          # access outside its buffer)
    return reps


def test_tiny_fp32_reference():
    """6 stations, 16 channels, T = 1024, M = 16, K = 64, one block."""
    d = synth.tiny_block(seed=1)
    M, K = 16, 64
    thr = default_thresholds(M)
    st = RfiStream(6, 16, M, K, thr, "f32")
    g = run_gpu(st, to_device_rows(d["vis"], "f32"))
    o = oracle.OracleStream(st.R, M, K, **thr).process(d["vis"].reshape(st.R, 1024, 4, 2))
    rep = compare(g, o, thr, M, K)
    assert o["wflag"].mean() > 0.01          # the bursts do raise flags
    print("tiny fp32", rep)


def test_tiny_fp16_storage():
    """Same block stored as binary16: FP32 arithmetic on exactly widened values."""
    d = synth.tiny_block(seed=1)
    M, K = 16, 64
    thr = default_thresholds(M)
    st = RfiStream(6, 16, M, K, thr, "f16")
    g = run_gpu(st, to_device_rows(d["vis"], "f16"))
    R = st.R
    o16 = oracle.OracleStream(R, M, K, **thr).process(
        d["vis"].reshape(R, 1024, 4, 2).astype(np.float16))
    compare(g, o16, thr, M, K)
    # against the oracle on the unrounded input: quantisation only, reported
    o32 = oracle.OracleStream(R, M, K, **thr).process(d["vis"].reshape(R, 1024, 4, 2))
    rep = compare(g, o32, thr, M, K, stat_rtol=None, avg_rtol=None, check_flags=False)
    assert rep["flag_disagree_frac"] <= 1e-3, rep
    print("tiny fp16 vs fp32 input", rep)


SHAPES = [
    # dtype, stations, channels, M, K, blocks, options
    ("f32", 5, 3, 16, 64, [1024], {}),
    ("f32", 3, 7, 16, 48, [48, 96, 16, 64], {"lanes_per_row": 4}),
    ("f32", 4, 5, 2, 6, [6, 10, 2, 30], {}),
    ("f32", 4, 5, 2, 4, [8, 4], {"lanes_per_row": 2}),
    ("f32", 3, 4, 3, 9, [9, 27, 6], {}),
    ("f32", 6, 3, 20, 40, [40, 60, 100], {"lanes_per_row": 4}),
    ("f32", 6, 3, 20, 20, [40, 20], {"lanes_per_row": 1}),
    ("f32", 5, 4, 64, 128, [128, 64, 192], {}),
    ("f32", 5, 4, 64, 64, [128], {"lanes_per_row": 8, "compensated": -1}),
    ("f32", 4, 6, 32, 32, [64, 96], {"lanes_per_row": 32}),
    ("f32", 4, 6, 16, 32, [64, 32], {"lanes_per_row": 16}),
    ("f32", 4, 6, 16, 16, [64], {"lanes_per_row": 8, "warps_per_block": 3}),
    ("f32", 4, 6, 8, 8, [40, 24], {"lanes_per_row": 1, "warps_per_block": 1}),
    ("f32", 10, 8, 16, 256, [256], {}),
    ("f16", 5, 3, 16, 64, [256, 128], {}),
    ("f16", 4, 5, 5, 10, [10, 20, 5], {}),
    ("f16", 4, 5, 3, 6, [6, 12, 3], {}),
    ("f16", 4, 5, 8, 16, [32, 48], {"lanes_per_row": 4}),
    ("f16", 4, 5, 64, 64, [128], {"lanes_per_row": 8}),
    ("f16", 6, 3, 20, 60, [60, 40, 20], {"lanes_per_row": 2}),
    ("f16", 4, 6, 32, 64, [96, 32], {"lanes_per_row": 16}),
    ("f16", 7, 5, 16, 32, [48], {"lanes_per_row": 1, "compensated": 1}),
    ("f32", 5, 6, 16, 32, [64, 32], {"lanes_per_row": 4, "max_registers": 64}),
    ("f16", 5, 6, 20, 40, [40, 80], {"lanes_per_row": 2, "max_registers": 80}),
    ("f16", 4, 5, 5, 10, [10, 20], {"max_registers": 64}),
    # the 96-register budget (two chunks of at most 2 load units in flight)
    ("f32", 5, 6, 16, 64, [64, 192], {"lanes_per_row": 4, "max_registers": 96}),
    ("f32", 4, 5, 10, 20, [40, 20], {"lanes_per_row": 1, "max_registers": 96}),
    ("f16", 5, 6, 16, 32, [64, 96], {"lanes_per_row": 2, "max_registers": 96}),
    ("f16", 4, 5, 5, 10, [10, 20], {"max_registers": 96}),
    # time-frequency footprints: the paper's 10 x 2 and 5 x 4 windows (W = 20)
    ("f32", 5, 4, 10, 20, [20, 40, 60], {"window_F": 2}),
    ("f16", 5, 4, 10, 30, [40, 20, 60], {"window_F": 2}),
    ("f32", 4, 8, 5, 10, [10, 20, 40], {"window_F": 4}),
    ("f16", 4, 8, 5, 20, [20, 40], {"window_F": 4}),
    ("f32", 3, 16, 16, 32, [48, 16], {"window_F": 8, "lanes_per_row": 4}),
    ("f16", 3, 16, 8, 16, [32, 32], {"window_F": 16, "lanes_per_row": 2}),
    ("f32", 3, 4, 1, 4, [8, 4], {"window_F": 4}),
    # rows staged in shared memory by TMA bulk copies (one lane per row)
    ("f32", 5, 4, 16, 64, [256, 128], {"loader": 1}),
    ("f16", 5, 4, 16, 32, [96, 64], {"loader": 1, "tma_stage_windows": 3, "tma_stages": 3}),
    ("f16", 4, 5, 5, 10, [10, 20, 40], {"loader": 1, "tma_stage_windows": 2}),
    ("f32", 6, 3, 20, 40, [40, 60, 100], {"loader": 1, "tma_stages": 1, "warps_per_block": 2}),
    ("f16", 5, 4, 10, 20, [20, 40], {"loader": 1, "window_F": 2}),
    ("f32", 5, 4, 64, 128, [128, 64, 192], {"loader": 1}),
    ("f32", 5, 6, 16, 64, [256, 128], {"loader": 1, "lanes_per_row": 4}),
    ("f16", 6, 4, 16, 32, [96, 64], {"loader": 1, "lanes_per_row": 2, "max_registers": 64}),
    ("f32", 4, 5, 20, 40, [40, 80], {"loader": 1, "lanes_per_row": 2, "max_registers": 80,
                                     "tma_stage_windows": 2}),
    ("f16", 5, 4, 32, 64, [128, 64], {"loader": 1, "lanes_per_row": 8, "tma_stages": 3}),
    ("f32", 5, 4, 10, 20, [20, 40], {"loader": 1, "lanes_per_row": 2, "window_F": 2}),
    # the same with one TMA tensor tile per warp and stage (rows past the last one read
    # as zeros: 60 rows are 2 warps of 32 at one lane per row)
    ("f32", 5, 4, 16, 64, [256, 128], {"loader": 2}),
    ("f16", 5, 4, 16, 32, [96, 64], {"loader": 2, "tma_stage_windows": 3, "tma_stages": 3}),
    ("f16", 4, 5, 5, 10, [10, 20, 40], {"loader": 2, "tma_stage_windows": 2}),
    ("f32", 6, 3, 20, 40, [40, 60, 100], {"loader": 2, "tma_stages": 1, "warps_per_block": 2}),
    ("f16", 5, 4, 10, 20, [20, 40], {"loader": 2, "window_F": 2}),
    ("f32", 5, 6, 16, 64, [256, 128], {"loader": 2, "lanes_per_row": 4}),
    ("f16", 6, 4, 16, 32, [96, 64], {"loader": 2, "lanes_per_row": 2, "max_registers": 64}),
    ("f16", 5, 4, 32, 64, [128, 64], {"loader": 2, "lanes_per_row": 4, "tma_stages": 3}),
    ("f32", 5, 4, 10, 20, [20, 40], {"loader": 2, "lanes_per_row": 2, "window_F": 2}),
    # statistics and flag words written 16 bytes at a time (falls back to plain
    # stores where T/M or the flag words per row are not multiples of 4)
    ("f16", 5, 4, 8, 32, [128, 64, 32], {"buffered_stores": 1, "lanes_per_row": 2}),
    ("f32", 4, 5, 8, 16, [64, 40], {"buffered_stores": 1, "lanes_per_row": 4}),
    ("f16", 4, 6, 16, 64, [512, 192], {"buffered_stores": 1}),
    ("f32", 5, 4, 4, 8, [128, 8, 256], {"buffered_stores": 1, "lanes_per_row": 1}),
    ("f32", 5, 4, 8, 16, [64, 32], {"buffered_stores": 1, "window_F": 2}),
    # long windows and long blocks
    ("f32", 3, 4, 1024, 2048, [2048, 1024], {"lanes_per_row": 8}),
    ("f16", 3, 4, 256, 512, [1024, 512], {"lanes_per_row": 4}),
    ("f32", 3, 2, 250, 500, [1000, 500], {"lanes_per_row": 2}),
    ("f16", 3, 2, 16, 8192, [8192, 4096], {}),
    # blocks of any length: windows left open by a block are completed by the next
    ("f32", 5, 4, 16, 64, [250, 7, 1, 100, 300], {"partial_windows": 1, "lanes_per_row": 4}),
    ("f16", 4, 5, 8, 32, [50, 6, 2, 100], {"partial_windows": 1, "lanes_per_row": 2}),
    ("f16", 4, 5, 5, 10, [7, 3, 11, 20], {"partial_windows": 1}),
    ("f32", 5, 4, 10, 20, [33, 17, 50], {"partial_windows": 1, "window_F": 2}),
    ("f32", 4, 6, 16, 32, [40, 24, 100], {"partial_windows": 1, "lanes_per_row": 2}),
    ("f16", 5, 4, 16, 64, [90, 38], {"partial_windows": 1, "compensated": 1,
                                     "lanes_per_row": 1}),
    ("f32", 4, 5, 8, 16, [20, 12, 64], {"partial_windows": 1, "lanes_per_row": 4}),
    ("f32", 4, 5, 64, 128, [100, 60, 200], {"partial_windows": 1, "lanes_per_row": 8}),
]


@pytest.mark.parametrize("dtype,N,C,M,K,Ts,opts", SHAPES,
                         ids=[f"{s[0]}-N{s[1]}-C{s[2]}-M{s[3]}-K{s[4]}-{len(s[5])}blk-"
                              f"{'-'.join(f'{k[:3]}{v}' for k, v in s[6].items())}"
                              for s in SHAPES])
def test_shapes(dtype, N, C, M, K, Ts, opts):
    _check_stream(N, C, M, K, Ts, dtype, **opts)


@pytest.mark.parametrize("dtype,opts", [("f32", dict(lanes_per_row=4, loader=2,
                                                     tma_stage_windows=2)),
                                        ("f16", dict(lanes_per_row=2, loader=2,
                                                     tma_stage_windows=2))])
def test_lofar_scale_tensor_tile_loader(dtype, opts):
    """The full-size block through the tensor-tile staged loader (1953 or 3906 warps,
    tensor maps over 124,992 rows): bit-identical to the direct loader of the same
    lanes per row, and the oracle on a seeded sample of 1024 rows."""
    M, K = 16, 256
    thr = default_thresholds(M)
    d = synth.lofar_block(seed=3)
    vis = to_device_rows(d["vis"], dtype)
    st = RfiStream(62, 64, M, K, thr, dtype, warps_per_block=4, **opts)
    ref = RfiStream(62, 64, M, K, thr, dtype, warps_per_block=4,
                    lanes_per_row=opts["lanes_per_row"])
    a, b = st.process(vis), ref.process(vis)
    torch.cuda.synchronize()
    for k in ("flags", "avg", "weight", "stats"):
        assert torch.equal(a[k], b[k]), k
    binding.rfi_check(st.ctx)
    g = run_gpu(st, vis)
    del vis
    rows = np.sort(np.random.default_rng(19).choice(st.R, size=1024, replace=False))
    v = d["vis"].reshape(st.R, 256, 4, 2)[rows]
    orc = oracle.OracleStream(len(rows), M, K, **thr)
    orc.process(_oracle_input(v, dtype))                 # the first block, as above
    o = orc.process(_oracle_input(v, dtype))
    compare({k: val[rows] for k, val in g.items()}, o, thr, M, K, n_seen=256)
    st.close(); ref.close()


@pytest.mark.parametrize("dtype,M", [("f32", 16), ("f16", 8), ("f16", 16), ("f16", 32),
                                     ("f16", 64)])
def test_lofar_scale_sampled_rows(dtype, M):
    """62 stations (1953 baselines), 64 channels, T = 256, K = 256 in the launch shape
    the bench times (the committed tuning table); the oracle checks a seeded sample of
    2048 rows one by one."""
    K = 256
    thr = default_thresholds(M)
    d = synth.lofar_block(seed=2)
    vis = to_device_rows(d["vis"], dtype)
    best, _ = autotune.tune(62, 64, M, K, thr, dtype, vis, cache_path=autotune.TUNED_PATH,
                            write_cache=False)
    st = RfiStream(62, 64, M, K, thr, dtype, **autotune.options_of(best))
    g = run_gpu(st, vis)
    del vis
    rows = np.sort(np.random.default_rng(17).choice(st.R, size=2048, replace=False))
    v = d["vis"].reshape(st.R, 256, 4, 2)[rows]
    o = oracle.OracleStream(len(rows), M, K, **thr).process(_oracle_input(v, dtype))
    gs = {k: val[rows] for k, val in g.items()}
    rep = compare(gs, o, thr, M, K)
    print(f"lofar {dtype} M={M}", rep)
    if dtype == "f16":      # against the unrounded input: binary16 quantisation, reported
        o32 = oracle.OracleStream(len(rows), M, K, **thr).process(v)
        rep32 = compare(gs, o32, thr, M, K, stat_rtol=None, avg_rtol=None, check_flags=False)
        assert rep32["flag_disagree_frac"] <= 1e-3, rep32      # spec bound: 0.1 %
        print(f"lofar f16 M={M} vs float32 input", rep32)
    st.close()


@pytest.mark.parametrize("dtype,M,F", [("f32", 10, 2), ("f32", 5, 4), ("f16", 10, 2),
                                       ("f16", 5, 4)])
def test_footprints_full_size_sampled(dtype, M, F):
    """The paper's 10 x 2 and 5 x 4 footprints on 62 stations, 64 channels, T = K = 250,
    in the launch shape the bench times (the committed tuning table); the oracle checks
    a seeded sample of 512 footprint rows (F adjacent channels of one baseline each)."""
    T = K = 250
    thr = default_thresholds(M * F)
    d = synth.lofar_block(seed=4, T=T)
    vis = to_device_rows(d["vis"], dtype)
    best, _ = autotune.tune(62, 64, M, K, thr, dtype, vis, fixed={"window_F": F},
                            cache_path=autotune.TUNED_PATH, write_cache=False)
    st = RfiStream(62, 64, M, K, thr, dtype, **autotune.options_of(best))
    g = run_gpu(st, vis)
    del vis
    groups = np.sort(np.random.default_rng(19).choice(st.R // F, size=512, replace=False))
    rows = (groups[:, None] * F + np.arange(F)).ravel()
    v = d["vis"].reshape(st.R, T, 4, 2)[rows]
    o = oracle.OracleStream(len(rows), M, K, **thr, F=F).process(_oracle_input(v, dtype))
    gs = {k: (val[groups] if k in ("tau", "r_re", "r_im") else val[rows])
          for k, val in g.items()}
    rep = compare(gs, o, thr, M, K, F=F)
    print(f"footprint {M}x{F} {dtype}", autotune.options_of(best), rep)
    binding.rfi_check(st.ctx)
    st.close()


def test_batched_uneven_full_size_sampled():
    """The batched workload at full size: 8 binary16 subbands (stations 24..76,
    channels 16..128, T = 256) in one persistent launch replayed from a CUDA graph, in
    the launch shape the bench times; 256 seeded rows of every subband against the
    oracle, and the second replay equal to the streams launched one by one."""
    M, K, T = 16, 256, 256
    thr = default_thresholds(M)
    geo = list(zip(synth.BATCH_STATIONS, synth.BATCH_CHANNELS))
    vis = [synth.generate.device_block(n, c, T, seed=300 + i) for i, (n, c) in enumerate(geo)]
    best, _ = autotune.tune(62, 64, M, K, thr, "f16", vis[3], cache_path=autotune.TUNED_PATH,
                            write_cache=False)
    opts = {k: v for k, v in autotune.options_of(best).items() if k != "max_registers"}
    streams = [RfiStream(n, c, M, K, thr, "f16", **opts) for n, c in geo]
    solo = [RfiStream(n, c, M, K, thr, "f16", **opts) for n, c in geo]
    outs = [s.alloc_outputs(T) for s in streams]
    g = binding.rfi_batch_graph_create([s.ctx for s in streams], [T] * len(streams))
    binding.rfi_batch_graph_launch(g, vis, [o["flags"] for o in outs], [o["avg"] for o in outs],
                                   [o["weight"] for o in outs], [o["stats"] for o in outs])
    torch.cuda.synchronize()
    rng = np.random.default_rng(23)
    for i, (s, o) in enumerate(zip(streams, outs)):
        rows = np.sort(rng.choice(s.R, size=256, replace=False))
        gs = {k: v[rows] for k, v in gpu_to_numpy(o).items()}
        host = vis[i][torch.from_numpy(rows).cuda()].cpu().numpy()       # float16 values
        orc = oracle.OracleStream(len(rows), M, K, **thr).process(host)
        compare(gs, orc, thr, M, K)
    # a second replay (the blocks continue the streams) against one launch per stream
    for st, v in zip(solo, vis):
        st.process(v)
    outs2 = [s.alloc_outputs(T) for s in streams]
    binding.rfi_batch_graph_launch(g, vis, [o["flags"] for o in outs2], [o["avg"] for o in outs2],
                                   [o["weight"] for o in outs2], [o["stats"] for o in outs2])
    exp = [st.process(v) for st, v in zip(solo, vis)]
    torch.cuda.synchronize()
    for e, o in zip(exp, outs2):
        for k in ("flags", "avg", "weight", "stats"):
            assert torch.equal(e[k], o[k]), k
    binding.rfi_batch_graph_destroy(g)
    for s in streams + solo:
        s.close()


def test_block_split_bit_identical():
    """One block versus the same samples split at multiples of M: identical bits."""
    M, K = 16, 64
    thr = default_thresholds(M)
    data = synth.tiny_block(seed=4, stations=5, channels=6, T=448)["vis"]
    whole_s = RfiStream(5, 6, M, K, thr, "f32")
    whole = gpu_to_numpy(whole_s.process(to_device_rows(data, "f32")))
    for cuts in ((16, 224), (48, 64, 400), (208,)):
        st = RfiStream(5, 6, M, K, thr, "f32")
        parts = []
        edges = (0,) + cuts + (448,)
        for a, b in zip(edges[:-1], edges[1:]):
            parts.append(gpu_to_numpy(st.process(to_device_rows(data[:, :, a:b], "f32"))))
        for key in ("tau", "r_re", "r_im"):
            assert np.array_equal(np.concatenate([p[key] for p in parts], 1), whole[key]), key
        assert np.array_equal(np.concatenate([p["avg"] for p in parts], 1), whole["avg"])
        assert np.array_equal(np.concatenate([p["weight"] for p in parts], 1), whole["weight"])
        st.close()


def _batch_setup(dtype, geoms, M, K, T, seed=9, regs=None):
    thr = default_thresholds(M)
    streams, vis, datas = [], [], []
    for i, (N, C) in enumerate(geoms):
        d = synth.tiny_block(seed=seed + i, stations=N, channels=C, T=T, duty=0.06)["vis"]
        datas.append(d)
        opts = {"max_registers": regs[i]} if regs else {}
        streams.append(RfiStream(N, C, M, K, thr, dtype, **opts))
        vis.append(to_device_rows(d, dtype))
    return thr, streams, vis, datas


def _alloc(streams, T):
    return [s.alloc_outputs(T) for s in streams]


def test_batch_matches_solo_bit_identical():
    """Uneven streams in one persistent launch give the same bits as alone."""
    M, K, T = 16, 64, 128
    geoms = [(5, 3), (9, 7), (3, 2), (12, 5)]
    for dtype in ("f32", "f16"):
        # the batch mixes register budgets; the solo runs use other budgets again:
        # the budget changes residency only, never a result
        thr, bs, vis, _ = _batch_setup(dtype, geoms, M, K, T, regs=[0, 64, 80, 0])
        _, ss, _, _ = _batch_setup(dtype, geoms, M, K, T, regs=[64, 0, 0, 80])
        for step in range(2):
            outs = _alloc(bs, T)
            binding.rfi_process_batch([s.ctx for s in bs], vis, [T] * len(bs),
                                      [o["flags"] for o in outs], [o["avg"] for o in outs],
                                      [o["weight"] for o in outs], [o["stats"] for o in outs])
            torch.cuda.synchronize()
            for s, v, o in zip(ss, vis, outs):
                solo = s.process(v)
                torch.cuda.synchronize()
                for k in ("flags", "avg", "weight", "stats"):
                    assert torch.equal(solo[k], o[k]), (dtype, step, k)


def test_batch_graph_replay_matches_solo():
    """The batch captured in a CUDA graph and replayed for three blocks."""
    M, K, T = 16, 32, 48
    geoms = [(4, 3), (7, 2), (2, 9)]
    thr, bs, vis, _ = _batch_setup("f16", geoms, M, K, T)
    _, ss, _, _ = _batch_setup("f16", geoms, M, K, T)
    g = binding.rfi_batch_graph_create([s.ctx for s in bs], [T] * len(bs))
    try:
        for step in range(3):
            outs = _alloc(bs, T)
            binding.rfi_batch_graph_launch(g, vis, [o["flags"] for o in outs],
                                           [o["avg"] for o in outs], [o["weight"] for o in outs],
                                           [o["stats"] for o in outs])
            torch.cuda.synchronize()
            for s, v, o in zip(ss, vis, outs):
                solo = s.process(v)
                torch.cuda.synchronize()
                for k in ("flags", "avg", "weight", "stats"):
                    assert torch.equal(solo[k], o[k]), (step, k)
    finally:
        binding.rfi_batch_graph_destroy(g)


def test_footprints_in_batch_and_host_path():
    """Streams with 10 x 2 footprints next to time-only streams in one persistent
    launch, and the chunked host path with a footprint: identical to the device path."""
    M, K, T = 10, 20, 40
    thr = default_thresholds(M * 2)
    geoms = [(4, 6, 2), (5, 4, 1), (3, 8, 2)]
    datas = [synth.tiny_block(seed=40 + i, stations=n, channels=c, T=T)["vis"]
             for i, (n, c, _) in enumerate(geoms)]
    mk = lambda: [RfiStream(n, c, M, K, thr, "f32", window_F=f) for n, c, f in geoms]
    bs, ss = mk(), mk()
    vis = [to_device_rows(d, "f32") for d in datas]
    outs = [s.alloc_outputs(T) for s in bs]
    binding.rfi_process_batch([s.ctx for s in bs], vis, [T] * 3, [o["flags"] for o in outs],
                              [o["avg"] for o in outs], [o["weight"] for o in outs],
                              [o["stats"] for o in outs])
    torch.cuda.synchronize()
    for s, v, o in zip(ss, vis, outs):
        solo = s.process(v)
        torch.cuda.synchronize()
        for k in ("flags", "avg", "weight", "stats"):
            assert torch.equal(solo[k], o[k]), k
    n, c, f = geoms[0]
    host = RfiStream(n, c, M, K, thr, "f32", window_F=f, host_max_T=T, host_chunks=3)
    dev = RfiStream(n, c, M, K, thr, "f32", window_F=f)
    want = dev.process(vis[0])
    torch.cuda.synchronize()
    got = host.process_host(torch.from_numpy(datas[0].reshape(-1, T, 4, 2).copy()).pin_memory())
    for k in ("flags", "avg", "weight", "stats"):
        assert torch.equal(want[k].cpu(), got[k]), k


def test_host_path_matches_device_path():
    M, K, T = 16, 64, 256
    thr = default_thresholds(M)
    d = synth.tiny_block(seed=6, stations=8, channels=5, T=T)["vis"]
    dev = RfiStream(8, 5, M, K, thr, "f32")
    host = RfiStream(8, 5, M, K, thr, "f32", host_max_T=T, host_chunks=3)
    want = dev.process(to_device_rows(d, "f32"))
    torch.cuda.synchronize()
    hv = torch.from_numpy(d.reshape(-1, T, 4, 2).copy()).pin_memory()
    got = host.process_host(hv)
    for k in ("flags", "avg", "weight", "stats"):
        assert torch.equal(want[k].cpu(), got[k]), k
    # pageable host memory works too (copies are staged by the runtime)
    got2 = RfiStream(8, 5, M, K, thr, "f32", host_max_T=T).process_host(
        torch.from_numpy(d.reshape(-1, T, 4, 2).copy()))
    for k in ("flags", "avg", "weight", "stats"):
        assert torch.equal(want[k].cpu(), got2[k]), k
    # both staged loaders in chunks of rows: the tensor-tile loader's map starts at the
    # chunk's first row (180 rows in 3 chunks of 60: 4 warps of 16 rows at 2 lanes per
    # row, the last one partly empty)
    for loader in (1, 2):
        got3 = RfiStream(8, 5, M, K, thr, "f32", host_max_T=T, host_chunks=3,
                         loader=loader).process_host(hv)
        for k in ("flags", "avg", "weight", "stats"):
            assert torch.equal(want[k].cpu(), got3[k]), (loader, k)


def test_edge_values():
    """All-zero windows (tau = -(Md+1)/(M-1), finite) and non-finite samples (flagged,
    excluded from the averages)."""
    M, K, T = 16, 32, 64
    thr = default_thresholds(M)
    d = synth.tiny_block(seed=8, stations=3, channels=4, T=T)["vis"].copy()
    d[0, 0] = 0.0                                # one row all zero
    d[1, 1, 5, 2, 0] = np.nan                    # NaN in window 0
    d[2, 3, 40, 0, 1] = np.inf                   # +inf in window 2
    d[3, 2, 17, 3, 0] = -np.inf                  # -inf in window 1
    R = 6 * 4
    for dtype in ("f32", "f16"):
        st = RfiStream(3, 4, M, K, thr, dtype)
        g = run_gpu(st, to_device_rows(d, dtype))
        o = oracle.OracleStream(R, M, K, **thr).process(_oracle_input(d, dtype))
        assert g["tau"][0, 0] == np.float32(-(M * thr["d"] + 1) / (M - 1))
        compare(g, o, thr, M, K)
        rows = d.reshape(R, T, 4, 2)
        for r in range(R):
            bad = ~np.isfinite(rows[r]).all(axis=(1, 2))
            for w in np.flatnonzero(bad.reshape(-1, M).any(axis=1)):
                assert (g["flagbits"][r, (w * M) // 32] >> np.uint32((w * M) % 32)) & 1
        assert np.isfinite(g["avg"]).all() and np.isfinite(g["weight"]).all()


def test_binary16_range_extremes():
    """Binary16 input across its whole range: rows scaled from the smallest subnormal
    (2^-24) to the largest finite value (65504), and a row whose xx + yy (131008)
    exceeds binary16 but not float32.  The Stokes sums of two binary16 values are
    formed in float32 (one rounding each), so statistics, flags and averages match the
    FP64 oracle on the same binary16 values within the usual tolerances."""
    M, K, T = 16, 32, 64
    thr = default_thresholds(M)
    S, C = 3, 4
    R = S * (S + 1) // 2 * C
    rng = np.random.default_rng(77)
    scales = [2.0 ** -24, 2.0 ** -20, 2.0 ** -14, 2.0 ** -6, 1.0, 16.0, 256.0, 4096.0, 32768.0]
    rows = np.empty((R, T, 4, 2), np.float32)
    for r in range(R):
        mag = rng.uniform(0.5, 1.0, (T, 4, 2)) * scales[r % len(scales)]
        rows[r] = (mag * rng.choice([-1.0, 1.0], (T, 4, 2))).astype(np.float16)
    rows[R - 1] = np.float16(65504.0)            # xx + yy = 131008: float32 only
    rows[R - 2, :, :, 1] = 0.0
    rows[R - 2, :, 0, 0] = np.float16(65504.0)   # xx = 65504 and yy = -65504 (I = 0)
    rows[R - 2, :, 3, 0] = np.float16(-65504.0)
    rows[R - 3, ::3] = np.float16(2.0 ** -24)    # subnormal samples among normal ones
    rows[R - 3, 1::3] = np.float16(-(2.0 ** -24))
    assert np.isfinite(rows).all() and np.abs(rows).max() == 65504.0
    st = RfiStream(S, C, M, K, thr, "f16")
    g = run_gpu(st, to_device_rows(rows, "f16"))
    o = oracle.OracleStream(R, M, K, **thr).process(rows.astype(np.float16))
    compare(g, o, thr, M, K)
    assert np.isfinite(g["tau"]).all() and np.isfinite(g["avg"]).all()
    st.close()


def test_threshold_update():
    M, K, T = 16, 64, 128
    thr = default_thresholds(M)
    d = synth.tiny_block(seed=10, stations=4, channels=4, T=T)["vis"]
    st = RfiStream(4, 4, M, K, thr, "f32")
    v = to_device_rows(d, "f32")
    a = run_gpu(st, v)
    never = dict(thr, s_low=-1e30, s_high=1e30, gamma=2.0)
    binding.rfi_set_thresholds(st.ctx, never)
    b = run_gpu(st, v)
    assert a["flagbits"].any() and not b["flagbits"].any()
    assert np.all(b["weight"] == 1.0)


def test_invalid_arguments():
    M, K, T = 16, 64, 128
    thr = default_thresholds(M)
    st = RfiStream(4, 4, M, K, thr, "f32")
    v = torch.zeros((st.R, T, 4, 2), device="cuda")
    out = st.alloc_outputs(T)
    ctx = st.ctx
    args = lambda **kw: dict(dict(vis=v, T=T, flags=out["flags"], avg=out["avg"],
                                  weight=out["weight"], stats=out["stats"]), **kw)

    def call(**kw):
        a = args(**kw)
        binding.rfi_process_block(ctx, a["vis"], a["T"], a["flags"], a["avg"], a["weight"],
                                  a["stats"])

    def status(**kw):
        with pytest.raises(RfiError) as ei:
            call(**kw)
        return ei.value.status

    assert status(T=120) == 1                                   # not a multiple of M
    assert status(T=0) == 1
    vv = torch.zeros(st.R * T * 8 + 8, device="cuda")
    assert status(vis=vv[4:].data_ptr()) == 1                   # 16-byte misaligned
    assert status(vis=v.cpu()) == 1                             # host memory
    # a raw allocation 4 KB shorter than the block: the range check must refuse it
    # (sub-blocks of torch's caching allocator sit inside larger allocations)
    from cuda.bindings import runtime as rt
    need = st.R * T * 32
    err, raw = rt.cudaMalloc(need - 4096)
    assert err == rt.cudaError_t.cudaSuccess
    try:
        assert status(vis=int(raw)) == 1                        # too small
    finally:
        rt.cudaFree(raw)
    assert status(flags=None) == 1
    assert status(avg=None) == 1
    call()                                                      # the valid call works
    torch.cuda.synchronize()
    with pytest.raises(RfiError):
        binding.rfi_create(0, 4, M, K, thr, "f32")
    with pytest.raises(RfiError):
        binding.rfi_create(4, 4, 1, K, thr, "f32")               # M < 2
    with pytest.raises(RfiError):
        binding.rfi_create(4, 4, 16, 24, thr, "f32")             # K not a multiple of M
    with pytest.raises(RfiError):
        binding.rfi_create(4, 4, 16, 32, dict(thr, s_low=3.0, s_high=1.0), "f32")
    with pytest.raises(RfiError):
        binding.rfi_create_ex(4, 4, 16, 32, thr, "f32", lanes_per_row=3)
    with pytest.raises(RfiError):
        binding.rfi_create_ex(4, 4, 3, 3, thr, "f16", lanes_per_row=2)   # odd M, f16
    st.close()
    with pytest.raises(RfiError) as ei:
        call()
    assert ei.value.status == 5                                 # destroyed context
    with pytest.raises(RfiError) as ei:
        binding.rfi_destroy(ctx)
    assert ei.value.status == 5                                 # double destroy
    binding.rfi_destroy(None)                                   # no-op


def test_tma_loader_bit_identical_to_direct_loads():
    """The shared-memory loader and the direct loader with the same lanes per row
    perform the same arithmetic in the same order."""
    M, K, T = 16, 64, 256
    thr = default_thresholds(M)
    d = synth.tiny_block(seed=31, stations=9, channels=11, T=T)["vis"]
    for dtype, P in (("f32", 1), ("f16", 1), ("f32", 4), ("f16", 2), ("f32", 8)):
        v = to_device_rows(d, dtype)
        a = RfiStream(9, 11, M, K, thr, dtype, lanes_per_row=P).process(v)
        b = RfiStream(9, 11, M, K, thr, dtype, lanes_per_row=P, loader=1, tma_stage_windows=2,
                      max_registers=64 if P > 1 else 0).process(v)
        # tensor tiles: lanes_per_row <= 4 (a tile of at least 8 rows)
        b2 = RfiStream(9, 11, M, K, thr, dtype, lanes_per_row=P, loader=2, tma_stage_windows=2,
                       max_registers=80 if P > 1 else 0).process(v) if P <= 4 else b
        torch.cuda.synchronize()
        for k in ("flags", "avg", "weight", "stats"):
            assert torch.equal(a[k], b[k]), (dtype, P, k)
            assert torch.equal(a[k], b2[k]), (dtype, P, "tensor tiles", k)
        # a staged-loader context batches with direct-loader ones (the batch kernel
        # loads directly): same bits again
        c = RfiStream(9, 11, M, K, thr, dtype, lanes_per_row=P, loader=1)
        e = RfiStream(9, 11, M, K, thr, dtype, lanes_per_row=P, max_registers=80 if P <= 8 else 0)
        bat = [c, e] + ([RfiStream(9, 11, M, K, thr, dtype, lanes_per_row=P, loader=2)]
                        if P <= 4 else [])
        outs = [x.alloc_outputs(T) for x in bat]
        binding.rfi_process_batch([x.ctx for x in bat], [v] * len(bat), [T] * len(bat),
                                  [o["flags"] for o in outs], [o["avg"] for o in outs],
                                  [o["weight"] for o in outs], [o["stats"] for o in outs])
        torch.cuda.synchronize()
        for o in outs:
            for k in ("flags", "avg", "weight", "stats"):
                assert torch.equal(a[k], o[k]), (dtype, P, "batch", k)


def test_buffered_stores_bit_identical_to_plain_stores():
    """Buffering four windows' outputs per store changes only how they are written."""
    thr8 = default_thresholds(8)
    d = synth.tiny_block(seed=37, stations=10, channels=13, T=512)["vis"]
    for dtype, P in (("f32", 2), ("f32", 4), ("f16", 2), ("f16", 1)):
        v = to_device_rows(d, dtype)
        a = RfiStream(10, 13, 8, 64, thr8, dtype, lanes_per_row=P).process(v)
        st = RfiStream(10, 13, 8, 64, thr8, dtype, lanes_per_row=P, buffered_stores=1)
        assert st.options["buffered_stores"] == 1
        b = st.process(v)
        torch.cuda.synchronize()
        for k in ("flags", "avg", "weight", "stats"):
            assert torch.equal(a[k], b[k]), (dtype, P, k)
    with pytest.raises(binding.RfiError):      # no buffered variant of the staged loader
        RfiStream(4, 4, 8, 64, thr8, "f32", loader=1, buffered_stores=1)
    with pytest.raises(binding.RfiError):      # tensor tiles of 4 rows: not 128-B aligned
        RfiStream(4, 4, 16, 64, thr8, "f32", loader=2, lanes_per_row=8)
    with pytest.raises(binding.RfiError):      # nor of the reduced register budgets
        RfiStream(4, 4, 8, 64, thr8, "f32", max_registers=64, buffered_stores=1)


def _bit_stream(flags, n):
    """The first n flag bits of every row, [R, n] uint8."""
    f = flags.cpu().numpy().view(np.uint32).astype(np.uint64)
    t = np.arange(n)
    return ((f[:, t // 32] >> (t % 32).astype(np.uint64)) & 1).astype(np.uint8)


@pytest.mark.parametrize("dtype,M,P,F", [("f32", 16, 4, 1), ("f16", 8, 2, 1), ("f16", 5, 1, 1),
                                         ("f32", 10, 2, 2)])
def test_partial_windows_bit_identical_to_one_block(dtype, M, P, F):
    """A stream cut into blocks of any length gives, bit for bit, the outputs of the
    unsplit stream (every window is evaluated whole, in the same lane order)."""
    N, C, K, T = 7, 8, 4 * M, 40 * M
    thr = default_thresholds(M * F)
    d = synth.tiny_block(seed=41, stations=N, channels=C, T=T, duty=0.08)["vis"]
    v = to_device_rows(d, dtype)
    opts = dict(lanes_per_row=P, window_F=F)
    one = RfiStream(N, C, M, K, thr, dtype, **opts).process(v)
    rng = np.random.default_rng(5)
    st = RfiStream(N, C, M, K, thr, dtype, partial_windows=1, **opts)
    cuts = sorted(set(int(x) for x in rng.integers(1, T, size=12)))
    if dtype == "f16" and M % 2 == 0:
        cuts = sorted(set(c - c % 2 for c in cuts) - {0})
    edges = [0] + cuts + [T]
    parts = [st.process(v[:, a:b].contiguous()) for a, b in zip(edges[:-1], edges[1:])]
    torch.cuda.synchronize()
    for k in ("stats", "avg", "weight"):
        assert torch.equal(torch.cat([p[k] for p in parts], dim=-1 if k == "stats" else 1),
                           one[k]), k
    bits = np.concatenate([_bit_stream(p["flags"], p["stats"].shape[-1] * M) for p in parts],
                          axis=1)
    assert np.array_equal(bits, _bit_stream(one["flags"], T))


def test_partial_windows_batch_host_and_checkpoint():
    """Partial windows through the persistent batch (contexts at different phases),
    the host-buffer path and a checkpoint taken while a window is open."""
    M, K = 16, 64
    thr = default_thresholds(M)
    d = synth.tiny_block(seed=43, stations=6, channels=8, T=512)["vis"]
    v = to_device_rows(d, "f32")
    solo = [RfiStream(6, 8, M, K, thr, "f32", partial_windows=1, lanes_per_row=2)
            for _ in range(2)]
    bat = [RfiStream(6, 8, M, K, thr, "f32", partial_windows=1, lanes_per_row=2)
           for _ in range(2)]
    # phases: stream 0 advanced by 5 samples, stream 1 by 22
    for ss in (solo, bat):
        ss[0].process(v[:, :5].contiguous())
        ss[1].process(v[:, :22].contiguous())
    Ts = [37, 90]
    blocks = [v[:, 5:42].contiguous(), v[:, 22:112].contiguous()]
    exp = [s.process(b) for s, b in zip(solo, blocks)]
    outs = [s.alloc_outputs(T) for s, T in zip(bat, Ts)]
    binding.rfi_process_batch([s.ctx for s in bat], blocks, Ts,
                              [o["flags"] for o in outs], [o["avg"] for o in outs],
                              [o["weight"] for o in outs], [o["stats"] for o in outs])
    torch.cuda.synchronize()
    for e, o in zip(exp, outs):
        for k in ("flags", "avg", "weight", "stats"):
            assert torch.equal(e[k], o[k]), k
    # host path: the same stream, block by block, in host memory
    a = RfiStream(6, 8, M, K, thr, "f32", partial_windows=1, host_max_T=200)
    b = RfiStream(6, 8, M, K, thr, "f32", partial_windows=1)
    h = v.cpu()
    t0 = 0
    for T in (13, 200, 51, 3):
        ga = a.process_host(h[:, t0:t0 + T].contiguous())
        gb = b.process(v[:, t0:t0 + T].contiguous())
        torch.cuda.synchronize()
        for k in ("flags", "avg", "weight", "stats"):
            assert torch.equal(ga[k], gb[k].cpu()), (T, k)
        t0 += T
    # checkpoint with a window open, resume in a new context
    blob = binding.rfi_get_state(b.ctx)
    c = RfiStream(6, 8, M, K, thr, "f32", partial_windows=1)
    binding.rfi_set_state(c.ctx, blob)
    x = b.process(v[:, t0:t0 + 77].contiguous())
    y = c.process(v[:, t0:t0 + 77].contiguous())
    torch.cuda.synchronize()
    for k in ("flags", "avg", "weight", "stats"):
        assert torch.equal(x[k], y[k]), k
    # argument checks
    with pytest.raises(RfiError):        # pairs of binary16 samples: T must be even
        RfiStream(4, 4, 8, 32, default_thresholds(8), "f16", partial_windows=1).process(
            torch.zeros(10, 7, 4, 2, dtype=torch.float16, device="cuda"))
    for bad in (dict(loader=1), dict(max_registers=64), dict(precision=1),
                dict(buffered_stores=1)):      # instances exist for the default kernel only
        with pytest.raises(RfiError):
            RfiStream(4, 4, 16, 64, thr, "f32", partial_windows=1, **bad)
    with pytest.raises(RfiError):        # without the option, T must be a multiple of M
        RfiStream(4, 4, 16, 64, thr, "f32").process(
            torch.zeros(10, 24, 4, 2, device="cuda"))


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_symmetries_bit_exact(dtype):
    """The kernels' Stokes wiring under the symmetries of pin P12, exactly: swapping the
    polarisation feeds, negating or conjugating every correlation leave every statistic
    and flag bit unchanged (each is the same operations on operands that differ only in
    sign or order of a commutative addition); multiplying by j swaps r_Re and r_Im."""
    M, K, T = 16, 64, 256
    thr = default_thresholds(M)
    d = synth.tiny_block(seed=61, stations=6, channels=8, T=T)["vis"]
    v = to_device_rows(d, dtype)                             # [R, T, 4, 2]

    def run(x):
        st = RfiStream(6, 8, M, K, thr, dtype, lanes_per_row=2)
        o = st.process(x.contiguous())
        torch.cuda.synchronize()
        st.close()
        return o
    base = run(v)
    conj = v.clone()
    conj[..., 1] = -conj[..., 1]
    jv = torch.stack([-v[..., 1], v[..., 0]], dim=-1)
    for name, x in (("feed swap", v[:, :, [3, 2, 1, 0], :]), ("negation", -v),
                    ("conjugation", conj)):
        o = run(x)
        assert torch.equal(o["stats"], base["stats"]), name
        assert torch.equal(o["flags"], base["flags"]), name
    o = run(jv)
    assert torch.equal(o["stats"][0], base["stats"][0])
    assert torch.equal(o["stats"][1], base["stats"][2])
    assert torch.equal(o["stats"][2], base["stats"][1])
    assert torch.equal(o["flags"], base["flags"])


def test_process_block_captures_in_a_cuda_graph():
    """rfi_process_block allocates nothing and never synchronises, so it can be captured
    in a CUDA graph; with K = T every block's launch arguments are the same, and each
    replay equals a direct call on the same block."""
    M, K, T = 16, 256, 256
    thr = default_thresholds(M)
    d = synth.tiny_block(seed=67, stations=8, channels=8, T=T)["vis"]
    v = to_device_rows(d, "f32")
    st = RfiStream(8, 8, M, K, thr, "f32", lanes_per_row=4)
    ref = RfiStream(8, 8, M, K, thr, "f32", lanes_per_row=4)
    out = st.alloc_outputs(T)
    st.process(v, out=out)                     # warm-up outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            st.process(v, out=out, stream=s)
    for _ in range(3):
        for k in out:
            out[k].zero_()
        g.replay()
        e = ref.process(v)
        torch.cuda.synchronize()
        for k in ("flags", "avg", "weight", "stats"):
            assert torch.equal(out[k], e[k]), k
    st.close()
    ref.close()


@pytest.mark.parametrize("loader", [1, 2])
def test_bounded_wait_reports_timeout_and_gpu_stays_usable(loader):
    """Failure detection without a GPU fault: with the injection option the staged
    loader (row copies or tensor tiles) expects more bytes than it copies, so every
    stage wait gives up after about 1 ms; rfi_check reports RFI_ETIMEOUT, and the
    device keeps working."""
    M, K, T = 16, 64, 128
    thr = default_thresholds(M)
    d = synth.tiny_block(seed=32, stations=6, channels=4, T=T)["vis"]
    v = to_device_rows(d, "f32")
    bad = RfiStream(6, 4, M, K, thr, "f32", loader=loader, debug_inject_wait_timeout=1)
    bad.process(v)
    with pytest.raises(RfiError) as ei:
        binding.rfi_check(bad.ctx)
    assert ei.value.status == 4                                   # RFI_ETIMEOUT
    with pytest.raises(RfiError):                                 # sticky until reset
        bad.process(v)
    binding.rfi_reset(bad.ctx)
    good = RfiStream(6, 4, M, K, thr, "f32", loader=loader)
    out = good.process(v)
    binding.rfi_check(good.ctx)
    want = RfiStream(6, 4, M, K, thr, "f32",
                     lanes_per_row=good.options["lanes_per_row"]).process(v)
    torch.cuda.synchronize()
    for k in ("flags", "avg", "weight", "stats"):
        assert torch.equal(out[k], want[k]), k


def test_checkpoint_resume_bit_identical():
    """Save a stream's state after a block whose last averaging bin is open, load it
    into a new context, and continue: identical to the uninterrupted stream."""
    M, K = 16, 96
    thr = default_thresholds(M)
    d = synth.tiny_block(seed=50, stations=6, channels=5, T=256)["vis"]
    blocks = [d[:, :, 0:64], d[:, :, 64:160], d[:, :, 160:256]]
    ref = RfiStream(6, 5, M, K, thr, "f32")
    want = [ref.process(to_device_rows(b, "f32")) for b in blocks]
    a = RfiStream(6, 5, M, K, thr, "f32")
    a.process(to_device_rows(blocks[0], "f32"))
    state = binding.rfi_get_state(a.ctx)
    assert len(state) == binding.rfi_state_size(a.ctx)
    b = RfiStream(6, 5, M, K, dict(thr, s_low=-9.0), "f32")   # thresholds come with the state
    binding.rfi_set_state(b.ctx, state)
    assert binding.rfi_outputs_for(b.ctx, 96) == binding.rfi_outputs_for(a.ctx, 96)
    for blk, w in zip(blocks[1:], want[1:]):
        got = b.process(to_device_rows(blk, "f32"))
        torch.cuda.synchronize()
        for k in ("flags", "avg", "weight", "stats"):
            assert torch.equal(got[k], w[k]), k
    other = RfiStream(6, 5, M, 64, thr, "f32")                 # another K: refused
    with pytest.raises(RfiError):
        binding.rfi_set_state(other.ctx, state)
    with pytest.raises(RfiError):
        binding.rfi_set_state(other.ctx, state[:10])


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_degenerate_thresholds_and_geometries(dtype):
    """Every window flagged (averages 0, weight 0); nothing flagged (plain means); a
    single-row stream; K spanning many blocks."""
    M, K, T = 16, 64, 128
    d = synth.tiny_block(seed=51, stations=3, channels=4, T=T)["vis"]
    v = to_device_rows(d, dtype)
    rows = d.reshape(-1, T, 8).astype(np.float16 if dtype == "f16" else np.float32)
    every = dict(d=1.0, s_low=1e30, s_high=2e30, gamma=2.0, eps=2 ** -23)
    o = RfiStream(3, 4, M, K, every, dtype).process(v)
    torch.cuda.synchronize()
    assert torch.all(o["flags"] == -1) and torch.all(o["weight"] == 0) and torch.all(o["avg"] == 0)
    none = dict(d=1.0, s_low=-1e30, s_high=1e30, gamma=2.0, eps=2 ** -23)
    o = RfiStream(3, 4, M, K, none, dtype).process(v)
    torch.cuda.synchronize()
    assert torch.all(o["flags"] == 0) and torch.all(o["weight"] == 1)
    mean = rows.astype(np.float64).reshape(-1, T // K, K, 8).mean(axis=2)
    got = o["avg"].cpu().numpy().reshape(-1, T // K, 8)
    assert np.all(np.abs(got - mean) <= 1e-5 * np.maximum(np.abs(mean), 1.0))
    # one station, one channel: a single row
    _check_stream(1, 1, 16, 32, [64, 32], dtype)
    # averaging bins of 512 samples over blocks of 48
    _check_stream(2, 3, 16, 512, [48] * 12, dtype)
