"""Continuous batching: every stream's results in the serving mix equal, bit for bit,
the results of the same blocks processed alone."""
import numpy as np
import pytest
import torch

import synth
from paper_2412_14775_b300 import RfiStream, default_thresholds
from paper_2412_14775_b300.serve import DevicePool, ServingLoop

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("options,T", [({}, 48), ({"adaptive": 1}, 48),
                                       ({"partial_windows": 1}, 40),
                                       ({"window_hop": 8, "lanes_per_row": 2}, 40),
                                       ({"lane_split": 1, "lanes_per_row": 2}, 48)],
                         ids=["fixed", "online_thresholds", "partial_windows",
                              "overlapping_windows", "window_parallel"])
def test_serving_mix_equals_solo(options, T):
    """With online thresholds the per-stream threshold state lives on the device too and
    advances with every block; with partial windows blocks of 40 samples leave windows
    of 16 open between blocks; with overlapping windows the pending half-window waits on
    the device between blocks.  In the mix exactly as alone."""
    M, K = 16, 32                 # bins of 32 straddle the blocks: the carry is exercised
    cfgs = [dict(stations=n, channels=c, rho=r) for n, c, r in
            ((5, 4, 3.0), (9, 8, 2.0), (7, 16, 4.0), (12, 4, 1.5), (4, 8, 3.5), (8, 16, 2.5))]
    thr = default_thresholds(M)
    blocks = [[synth.generate.device_block(c["stations"], c["channels"], T, seed=100 + 7 * i + k)
               for k in range(3)] for i, c in enumerate(cfgs)]
    loop = ServingLoop(cfgs, M=M, K=K, T=T, thresholds=thr, dtype="f16", block_seconds=0.01,
                       max_batch=4, cuda_streams=3, record_outputs=True, blocks=blocks,
                       hbm_budget_bytes=1 << 30, options=options)
    if options.get("adaptive"):
        for s in loop.streams:
            s.st.set_adaptation(alpha=1.0 / 16, k_sigma=3.0, n_warm=4)
    stats = loop.run(1.0, seed=3)
    assert stats["blocks"] > 200
    assert stats["mean_batch"] > 1.0, stats          # blocks were batched together
    opts = loop.streams[0].st.options
    for i, cfg in enumerate(cfgs):
        got = sorted(loop.outputs[i], key=lambda t: t[0])
        assert [k for k, _ in got] == list(range(len(got)))
        kw = dict(lanes_per_row=opts["lanes_per_row"], warps_per_block=opts["warps_per_block"])
        kw.update(options)
        solo = RfiStream(cfg["stations"], cfg["channels"], M, K, thr, "f16", **kw)
        if options.get("adaptive"):
            solo.set_adaptation(alpha=1.0 / 16, k_sigma=3.0, n_warm=4)
        for k, mixed in got:
            o = solo.process(blocks[i][k % 3].contiguous())
            torch.cuda.synchronize()
            for name in ("flags", "avg", "weight", "stats"):
                assert np.array_equal(o[name].cpu().numpy(), mixed[name]), (i, k, name)
        solo.close()
    loop.close()


def test_serving_in_place_equals_solo():
    """Blocks read where they arrived in device memory (no copy into the pool; slots
    hold the outputs only): the same bits as the blocks processed alone."""
    M, K, T = 16, 32, 48
    cfgs = [dict(stations=n, channels=c, rho=r) for n, c, r in
            ((5, 4, 3.0), (9, 8, 2.0), (7, 16, 4.0), (12, 4, 1.5))]
    thr = default_thresholds(M)
    blocks = [[synth.generate.device_block(c["stations"], c["channels"], T, seed=400 + 7 * i + k)
               for k in range(3)] for i, c in enumerate(cfgs)]
    loop = ServingLoop(cfgs, M=M, K=K, T=T, thresholds=thr, dtype="f16", block_seconds=0.01,
                       max_batch=4, cuda_streams=3, record_outputs=True, blocks=blocks,
                       hbm_budget_bytes=1 << 30, copy_in=False)
    assert loop.streams[0].parts[0] == ("vis", 0)
    stats = loop.run(0.5, seed=6)
    assert stats["blocks"] > 100
    opts = loop.streams[0].st.options
    for i, cfg in enumerate(cfgs):
        solo = RfiStream(cfg["stations"], cfg["channels"], M, K, thr, "f16",
                         lanes_per_row=opts["lanes_per_row"],
                         warps_per_block=opts["warps_per_block"])
        for k, mixed in sorted(loop.outputs[i], key=lambda t: t[0]):
            o = solo.process(blocks[i][k % 3].contiguous())
            torch.cuda.synchronize()
            for name in ("flags", "avg", "weight", "stats"):
                assert np.array_equal(o[name].cpu().numpy(), mixed[name]), (i, k, name)
        solo.close()
    loop.close()
    with pytest.raises(ValueError):           # host blocks must be copied to the device
        ServingLoop(cfgs[:1], M=M, K=K, T=T, dtype="f16", source="host", copy_in=False)


def test_serving_admission_respects_memory_budget():
    """With a block pool that holds one block at a time, batches hold a single block
    and every block is still served."""
    M, K, T = 16, 16, 32
    cfgs = [dict(stations=6, channels=8, rho=4.0), dict(stations=6, channels=8, rho=4.0)]
    s = DevicePool.rounded(1)
    loop = ServingLoop(cfgs, M=M, K=K, T=T, dtype="f16", block_seconds=0.01, max_batch=8,
                       pool_blocks=1)
    slot = loop.streams[0].slot_bytes
    loop.pool = DevicePool(slot + s, "cuda")          # room for exactly one block
    stats = loop.run(0.3, seed=1)
    assert stats["blocks"] > 0 and stats["mean_batch"] == 1.0
    assert stats["admission_waits"] > 0 and loop.pool.used == 0
    loop.close()


def test_serving_host_fed_equals_solo():
    """Blocks arriving in pinned host memory, copied into the device pool per batch,
    results copied back: the same bits as the blocks processed alone."""
    M, K, T = 16, 32, 48
    cfgs = [dict(stations=n, channels=c, rho=r) for n, c, r in
            ((5, 4, 3.0), (9, 8, 2.0), (7, 16, 4.0))]
    thr = default_thresholds(M)
    blocks = [[synth.generate.device_block(c["stations"], c["channels"], T, seed=200 + 7 * i + k)
               for k in range(2)] for i, c in enumerate(cfgs)]
    loop = ServingLoop(cfgs, M=M, K=K, T=T, thresholds=thr, dtype="f16", block_seconds=0.01,
                       max_batch=4, record_outputs=True, blocks=blocks, source="host")
    stats = loop.run(0.5, seed=4)
    assert stats["blocks"] > 50 and stats["h2d_bytes"] > 0 and stats["d2h_bytes"] > 0
    opts = loop.streams[0].st.options
    for i, cfg in enumerate(cfgs):
        solo = RfiStream(cfg["stations"], cfg["channels"], M, K, thr, "f16",
                         lanes_per_row=opts["lanes_per_row"],
                         warps_per_block=opts["warps_per_block"])
        for k, mixed in sorted(loop.outputs[i], key=lambda t: t[0]):
            o = solo.process(blocks[i][k % 2].contiguous())
            torch.cuda.synchronize()
            for name in ("flags", "avg", "weight", "stats"):
                assert np.array_equal(o[name].cpu().numpy(), mixed[name]), (i, k, name)
        solo.close()
    loop.close()
