"""The entry point that allocates nothing, against the context-based entry point.

rfi_process_block_noalloc exists for callers that may not allocate device memory
(their GPU memory is reserved up front by another pool, or they run on a real-time
thread that must not risk an allocation's implicit synchronisation).  Its working
memory -- the carry of each row's open averaging bin -- sits in a fixed array inside
the library.  This file is collected last on purpose (it is named so): a run that
stops at the first failure has run every other test before it.
"""
import numpy as np
import pytest
import torch

import synth
from paper_2412_14775_b300 import RfiStream, binding, default_thresholds
from paper_2412_14775_b300.binding import RfiError

pytestmark = pytest.mark.gpu


def _rows(vis_np, dtype):
    v = torch.from_numpy(np.ascontiguousarray(vis_np.reshape(-1, *vis_np.shape[-3:]))).cuda()
    return v.half() if dtype == "f16" else v


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_noalloc_matches_context_entry_point_on_two_calls(dtype):
    # bins of K = 64 straddle blocks of T = 48, so the second call continues the bin
    # whose carry the first call left in the library's scratch array
    stations, channels, M, K, T = 10, 12, 16, 64, 48
    thr = default_thresholds(M)
    data = synth.tiny_block(seed=21, stations=stations, channels=channels, T=2 * T)["vis"]
    ref = RfiStream(stations, channels, M, K, thr, dtype, lanes_per_row=1)
    n_seen = 0
    for call in range(2):
        blk = _rows(data[:, :, call * T:(call + 1) * T], dtype)
        want = ref.process(blk)
        got = {k: torch.empty_like(v) for k, v in want.items()}
        n_out = got["weight"].shape[1]
        binding.rfi_process_block_noalloc(
            stations, channels, M, K, thr, dtype, n_seen, blk, T, got["flags"],
            got["avg"] if n_out else None, got["weight"] if n_out else None, got["stats"])
        torch.cuda.synchronize()
        assert torch.equal(got["flags"], want["flags"]), call
        for k in ("stats", "avg", "weight"):
            assert torch.allclose(got[k], want[k], rtol=1e-5, atol=1e-6), (call, k)
        n_seen += T
    ref.close()


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
