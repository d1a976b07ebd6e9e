"""The entry point that allocates nothing, against the context-based entry point and
the FP64 oracle.

rfi_process_block_noalloc exists for callers that may not allocate device memory
(their GPU memory is reserved up front by another pool, or they run on a real-time
thread that must not risk an allocation's implicit synchronisation).  Its working
memory -- the carry of each row's open averaging bin -- sits in a fixed array inside
the library.  Its kernel is the library's one-lane-per-row kernel, so every output
equals, bit for bit, rfi_process_block on a context with lanes_per_row = 1.  This file
is collected last on purpose (it is named so): a run that stops at the first failure
has run every other test before it.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2412_14775_b300 import RfiStream, binding, default_thresholds
from paper_2412_14775_b300.binding import RfiError
from parity import compare, gpu_to_numpy

pytestmark = pytest.mark.gpu


def _rows(vis_np, dtype):
    v = torch.from_numpy(np.ascontiguousarray(vis_np.reshape(-1, *vis_np.shape[-3:]))).cuda()
    return v.half() if dtype == "f16" else v


def _noalloc(stations, channels, M, K, thr, dtype, n_seen, blk, T, like):
    got = {k: torch.empty_like(v) for k, v in like.items()}
    n_out = got["weight"].shape[1]
    binding.rfi_process_block_noalloc(
        stations, channels, M, K, thr, dtype, n_seen, blk, T, got["flags"],
        got["avg"] if n_out else None, got["weight"] if n_out else None, got["stats"])
    return got


# (M, K, T): K a multiple of M, T not a multiple of K, so averaging bins straddle the
# two calls and the second call continues the carry the first left in the scratch.
# The windows cover every kernel branch: odd M (binary16 one sample per load unit),
# load-unit chunks of 5, 4 and 2, and Kahan-compensated moments (M >= 64).
SHAPES = [(15, 45, 30), (16, 64, 48), (20, 60, 40), (64, 128, 192)]


@pytest.mark.parametrize("dtype", ["f32", "f16"])
@pytest.mark.parametrize("M,K,T", SHAPES, ids=[f"M{m}" for m, _, _ in SHAPES])
def test_noalloc_equals_context_entry_point_on_two_calls(dtype, M, K, T):
    stations, channels = 10, 12
    thr = default_thresholds(M)
    data = synth.tiny_block(seed=21 + M, stations=stations, channels=channels, T=2 * T,
                            duty=0.08)["vis"]
    ref = RfiStream(stations, channels, M, K, thr, dtype, lanes_per_row=1)
    n_seen = 0
    for call in range(2):
        blk = _rows(data[:, :, call * T:(call + 1) * T], dtype)
        want = ref.process(blk)
        got = _noalloc(stations, channels, M, K, thr, dtype, n_seen, blk, T, want)
        torch.cuda.synchronize()
        for k in ("flags", "stats", "avg", "weight"):
            assert torch.equal(got[k], want[k]), (call, k)
        n_seen += T
    ref.close()


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_noalloc_matches_oracle_on_two_calls(dtype):
    stations, channels, M, K, T = 8, 16, 16, 64, 48
    thr = default_thresholds(M)
    data = synth.tiny_block(seed=33, stations=stations, channels=channels, T=2 * T,
                            duty=0.08)["vis"]
    R = data.shape[0] * data.shape[1]
    orc = oracle.OracleStream(R, M, K, **thr)
    n_seen = 0
    for call in range(2):
        part = data[:, :, call * T:(call + 1) * T]
        blk = _rows(part, dtype)
        n_out = (n_seen + T) // K - n_seen // K
        like = dict(flags=torch.empty((R, (T + 31) // 32), dtype=torch.int32, device="cuda"),
                    stats=torch.empty((3, R, T // M), device="cuda"),
                    avg=torch.empty((R, n_out, 4, 2), device="cuda"),
                    weight=torch.empty((R, n_out), device="cuda"))
        got = _noalloc(stations, channels, M, K, thr, dtype, n_seen, blk, T, like)
        torch.cuda.synchronize()
        ref_in = part.astype(np.float16) if dtype == "f16" else part
        compare(gpu_to_numpy(got), orc.process(ref_in.reshape(R, T, 4, 2)), thr, M, K,
                n_seen=n_seen)
        n_seen += T


def test_noalloc_rejects_streams_larger_than_its_scratch():
    M, K, T = 16, 256, 256
    thr = default_thresholds(M)
    rows = 1953 * 64                      # 62 stations x 64 channels: 4.5 MB of carry
    assert rows * 36 > binding.RFI_NOALLOC_SCRATCH_BYTES
    vis = torch.zeros((rows, T, 4, 2), device="cuda", dtype=torch.float16)
    out = dict(flags=torch.empty((rows, T // 32), dtype=torch.int32, device="cuda"),
               avg=torch.empty((rows, 1, 4, 2), device="cuda"),
               weight=torch.empty((rows, 1), device="cuda"),
               stats=torch.empty((3, rows, T // M), device="cuda"))
    with pytest.raises(RfiError) as ei:
        binding.rfi_process_block_noalloc(62, 64, M, K, thr, "f16", 0, vis, T, out["flags"],
                                          out["avg"], out["weight"], out["stats"])
    assert ei.value.status == 1
    assert "scratch" in str(ei.value)
