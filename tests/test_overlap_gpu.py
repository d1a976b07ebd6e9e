"""Launch overlap (programmatic dependent launch) of consecutive single-stream calls.

A flagging launch may start while the launch before it on the stream finishes; until
that one has completed it only requests its first bytes into L2.  Every result must be
what the same calls give with the overlap off: outputs of one call that are overwritten
by the next hold the later call's values, and carries (open averaging bin, open
window, threshold state) pass from call to call in order.
"""
import numpy as np
import pytest
import torch

import synth
from paper_2412_14775_b300 import RfiStream, binding, default_thresholds
from paper_2412_14775_b300.binding import RfiError
from parity import to_device_rows

pytestmark = pytest.mark.gpu


def _blocks(n, stations, channels, T, dtype, seed):
    d = synth.tiny_block(seed=seed, stations=stations, channels=channels, T=n * T,
                         duty=0.05)["vis"]
    return [to_device_rows(d[:, :, k * T:(k + 1) * T], dtype) for k in range(n)]


@pytest.mark.parametrize("dtype,M,K,T,opts", [
    ("f32", 16, 32, 48, {}),                                # bins straddle calls
    ("f16", 16, 64, 64, {}),
    ("f32", 16, 32, 40, {"partial_windows": 1}),            # windows straddle calls
    ("f32", 16, 64, 64, {"adaptive": 1}),                   # threshold state in order
    ("f16", 8, 16, 48, {"buffered_stores": 1}),
    ("f32", 10, 20, 40, {"window_F": 2}),
], ids=["f32", "f16", "partial_windows", "adaptive", "buffered_stores", "footprint"])
def test_overlap_equals_plain_stream_order(dtype, M, K, T, opts):
    N, C = 9, 16
    thr = default_thresholds(M * opts.get("window_F", 1))
    blocks = _blocks(6, N, C, T, dtype, seed=71)
    on = RfiStream(N, C, M, K, thr, dtype, lanes_per_row=2, **opts)
    off = RfiStream(N, C, M, K, thr, dtype, lanes_per_row=2, overlap_bytes=-1, **opts)
    assert on.options["overlap_bytes"] == 512 and off.options["overlap_bytes"] == -1
    if opts.get("adaptive"):
        for s in (on, off):
            s.set_adaptation(alpha=1.0 / 8, k_sigma=3.0, n_warm=2)
    for rep in range(2):
        # back-to-back calls, no host synchronisation between them
        got, ref = [], []
        for blk in blocks:
            got.append(on.process(blk))          # fresh outputs per call, no copies between
        for blk in blocks:
            o = off.process(blk)
            ref.append(o)
        torch.cuda.synchronize()
        for g, r in zip(got, ref):
            for k in ("flags", "avg", "weight", "stats"):
                assert torch.equal(g[k], r[k]), (rep, k)
    if opts.get("adaptive"):
        assert np.array_equal(on.adaptive_state(), off.adaptive_state())
    on.close(); off.close()


def test_overlapped_calls_into_shared_outputs_keep_the_last_call():
    """Two inputs alternate into the same output buffers: the values left are those of
    the last call, exactly (the overlapping launch writes only after the one before it
    has completed)."""
    M, K, T = 16, 256, 256
    thr = default_thresholds(M)
    a, b = _blocks(2, 12, 32, T, "f32", seed=73)
    st = RfiStream(12, 32, M, K, thr, "f32", lanes_per_row=4)
    ref = RfiStream(12, 32, M, K, thr, "f32", lanes_per_row=4, overlap_bytes=-1)
    rb = ref.process(b)
    out = st.alloc_outputs(T)
    for _ in range(20):
        st.process(a, out=out)
        st.process(b, out=out)
    torch.cuda.synchronize()
    for k in ("flags", "avg", "weight", "stats"):
        assert torch.equal(out[k], rb[k]), k
    st.close(); ref.close()


def test_overlap_after_a_foreign_kernel_that_writes_the_input():
    """Each call follows one of torch's kernels that writes the call's input: the early
    L2 requests may see the old values, the kernel itself reads only the new ones.
    (Capture into a CUDA graph, where launches keep plain stream order, is tested with
    the default options in test_parity_gpu.py.)"""
    M, K, T = 16, 64, 64
    thr = default_thresholds(M)
    src = _blocks(3, 7, 8, T, "f32", seed=79)
    st = RfiStream(7, 8, M, K, thr, "f32", lanes_per_row=4)
    ref = RfiStream(7, 8, M, K, thr, "f32", lanes_per_row=4, overlap_bytes=-1)
    buf = torch.zeros_like(src[0])
    for k in range(3):
        buf.mul_(0.0).add_(src[k])          # a foreign kernel writes the input just before
        o = st.process(buf)
        r = ref.process(src[k])
        torch.cuda.synchronize()
        for name in ("flags", "avg", "weight", "stats"):
            assert torch.equal(o[name], r[name]), (k, name)
    st.close(); ref.close()


def test_overlap_option_checks():
    thr = default_thresholds(16)
    for bad in (100, -2):
        with pytest.raises(RfiError):
            RfiStream(3, 4, 16, 32, thr, "f32", overlap_bytes=bad)
    st = RfiStream(3, 4, 16, 32, thr, "f32", overlap_bytes=1024)
    assert st.options["overlap_bytes"] == 1024
    st.close()
    assert binding.rfi_options.overlap_bytes.offset > binding.rfi_options.adaptive.offset
