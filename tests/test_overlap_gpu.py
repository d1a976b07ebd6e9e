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


# ---- independent launches (option independent_launches) ------------------------------
# A launch that shares no byte with the flagging launches that may still run on the
# stream starts without waiting for the kernel before it.  The library decides per
# launch (rfi_last_launch); these tests check both the decision and that every result
# equals the same calls made one at a time with the overlap off.

def _order(st):
    return binding.rfi_last_launch(st.ctx)


@pytest.mark.parametrize("dtype,opts", [("f32", {}), ("f16", {}),
                                        ("f16", {"lane_split": 1, "lanes_per_row": 2}),
                                        ("f32", {"window_F": 2})],
                         ids=["f32", "f16", "lane_split", "footprint"])
def test_independent_blocks_overlap_and_match(dtype, opts):
    """Blocks that close their bins (K = T) into a ring of eight output sets: every call
    runs independent of the calls still in flight, except one that writes the output
    set of a call since the last plain launch (launch i + 8 writes what launch i wrote,
    and launch i may in principle still run): that one runs in plain stream order.
    The results are those of plain calls."""
    M, K, T = 16, 64, 64
    N, C = 9, 16
    thr = default_thresholds(M * opts.get("window_F", 1))
    blocks = _blocks(6, N, C, T, dtype, seed=81)
    on = RfiStream(N, C, M, K, thr, dtype, independent_launches=1, **opts)
    off = RfiStream(N, C, M, K, thr, dtype, overlap_bytes=-1, **opts)
    assert on.options["independent_launches"] == 1 and off.options["independent_launches"] == 0
    ref = []
    for blk in blocks:
        ref.append(off.process(blk))
        torch.cuda.synchronize()
    assert _order(off) == "plain"
    ring = [on.alloc_outputs(T) for _ in range(8)]
    orders = []
    n = 3 * len(blocks)
    for i in range(n):
        on.process(blocks[i % len(blocks)], out=ring[i % 8])
        orders.append(_order(on))
        if i % 8 == 7 or i == n - 1:            # compare the ring before it is reused
            torch.cuda.synchronize()
            for j in range(i - i % 8, i + 1):
                for k in ("flags", "avg", "weight", "stats"):
                    assert torch.equal(ring[j % 8][k], ref[j % len(blocks)][k]), (j, k)
    want = ["plain" if i > 0 and i % 8 == 0 else "independent" for i in range(n)]
    assert orders == want, orders
    binding.rfi_check(on.ctx)                    # no device error (and, in the checked
    on.close(); off.close()                      # build, no access outside a buffer)


def test_independent_launches_wait_for_what_they_share():
    """Shared output buffers and an open bin carried between calls make launches wait
    (or run in plain stream order when an independent launch is still in flight); the
    results are those of plain calls."""
    M, T = 16, 48
    N, C = 9, 16
    thr = default_thresholds(M)
    blocks = _blocks(6, N, C, T, "f32", seed=83)
    # K = 32 does not divide T = 48: bins straddle calls, so the open bin's carry
    # passes from call to call (written by one, read by the next)
    on = RfiStream(N, C, M, 32, thr, "f32", independent_launches=1)
    off = RfiStream(N, C, M, 32, thr, "f32", overlap_bytes=-1)
    got, orders = [], []
    for blk in blocks:
        got.append(on.process(blk))
        orders.append(_order(on))
    torch.cuda.synchronize()
    for g, blk in zip(got, blocks):
        r = off.process(blk)
        torch.cuda.synchronize()
        for k in ("flags", "avg", "weight", "stats"):
            assert torch.equal(g[k], r[k]), k
    assert "independent" not in orders[1:], orders
    binding.rfi_check(on.ctx)
    on.close(); off.close()
    # shared outputs: the second call writes what the first writes
    M, K, T = 16, 64, 64
    a, b = _blocks(2, N, C, T, "f32", seed=85)
    st = RfiStream(N, C, M, K, thr, "f32", independent_launches=1)
    ref = RfiStream(N, C, M, K, thr, "f32", overlap_bytes=-1)
    rb = ref.process(b)
    out = st.alloc_outputs(T)
    for _ in range(10):
        st.process(a, out=out)
        st.process(b, out=out)
        assert _order(st) in ("plain", "waiting")
    torch.cuda.synchronize()
    for k in ("flags", "avg", "weight", "stats"):
        assert torch.equal(out[k], rb[k]), k
    binding.rfi_check(st.ctx)
    st.close(); ref.close()


def test_independent_launches_across_contexts_and_the_no_alloc_path():
    """Two contexts on one stream writing the same output buffers are ordered; a
    launch after rfi_process_block_noalloc (whose buffers the library does not track)
    waits for it; at most 32 launches stay in flight."""
    M, K, T = 16, 64, 64
    N, C = 9, 16
    thr = default_thresholds(M)
    a, b = _blocks(2, N, C, T, "f32", seed=87)
    s1 = RfiStream(N, C, M, K, thr, "f32", independent_launches=1)
    s2 = RfiStream(N, C, M, K, thr, "f32", independent_launches=1, lanes_per_row=2)
    ref = RfiStream(N, C, M, K, thr, "f32", lanes_per_row=2, overlap_bytes=-1)
    rb = ref.process(b)
    out = s1.alloc_outputs(T)
    for _ in range(5):
        s1.process(a, out=out)
        s2.process(b, out=out)                  # the same outputs, another context
        assert _order(s2) in ("plain", "waiting")
    torch.cuda.synchronize()
    for k in ("flags", "avg", "weight", "stats"):
        assert torch.equal(out[k], rb[k]), k
    # after the no-allocation entry point: waiting, never independent
    o2 = s1.alloc_outputs(T)
    binding.rfi_process_block_noalloc(N, C, M, K, thr, binding.RFI_C64, 0, a, T,
                                      o2["flags"], o2["avg"], o2["weight"], o2["stats"])
    s2.process(b)
    assert _order(s2) == "waiting"
    # a plain launch empties the list of launches in flight; then 31 independent
    # launches fill it to 32 and the next runs in plain stream order (references from a
    # context of s1's shape with the overlap off)
    ref1 = RfiStream(N, C, M, K, thr, "f32", overlap_bytes=-1)
    rb = ref1.process(b)
    ra = ref1.process(a)
    assert _order(ref1) == "plain"
    ring = [s1.alloc_outputs(T) for _ in range(40)]
    orders = []
    for i in range(70):
        s1.process(a if i % 2 else b, out=ring[i % 40])
        orders.append(_order(s1))
    torch.cuda.synchronize()
    want = ["plain" if i in (31, 63) else "independent" for i in range(70)]
    assert orders == want, orders
    for i in (0, 31, 32, 63, 69):
        exp = ra if i % 2 else rb
        for k in ("flags", "avg", "weight", "stats"):
            assert torch.equal(ring[i % 40][k], exp[k]), (i, k)
    binding.rfi_check(s1.ctx)
    binding.rfi_check(s2.ctx)
    s1.close(); s2.close(); ref.close(); ref1.close()


def test_independent_launches_option_checks():
    thr = default_thresholds(16)
    for bad in (2, -1):
        with pytest.raises(RfiError):
            RfiStream(3, 4, 16, 32, thr, "f32", independent_launches=bad)
    st = RfiStream(3, 4, 16, 32, thr, "f32")
    assert st.options["independent_launches"] == 0 and _order(st) == "none"
    st.close()


def test_independent_launches_random_sequences():
    """A seeded random sequence of calls of three contexts on one stream (one carries its
    open bin from call to call, one is binary16 with window-parallel lanes), each call
    into one of a few output sets that later calls, of the same or another context of
    the same shape, may write again: the sets' final contents and every context's saved
    state equal those of the same sequence with the overlap off."""
    rng = np.random.default_rng(91)
    N, C = 7, 8
    specs = [dict(M=16, K=64, T=64, dtype="f32", opts={}),
             dict(M=16, K=32, T=48, dtype="f32", opts={"lanes_per_row": 2}),
             dict(M=8, K=64, T=64, dtype="f16", opts={"lane_split": 1, "lanes_per_row": 4})]
    on, off, inputs, sets_on, sets_off = [], [], [], [], []
    for i, sp in enumerate(specs):
        thr = default_thresholds(sp["M"])
        on.append(RfiStream(N, C, sp["M"], sp["K"], thr, sp["dtype"], independent_launches=1,
                            **sp["opts"]))
        off.append(RfiStream(N, C, sp["M"], sp["K"], thr, sp["dtype"], overlap_bytes=-1,
                             **sp["opts"]))
        inputs.append(_blocks(3, N, C, sp["T"], sp["dtype"], seed=93 + i))
    # three output sets per context, taken at random by its calls; context 1's output
    # sizes depend on the stream position (its bins straddle calls), so its calls take
    # fresh outputs
    for i, sp in enumerate(specs):
        if i == 1:
            sets_on.append(None); sets_off.append(None)
        else:
            sets_on.append([on[i].alloc_outputs(sp["T"]) for _ in range(3)])
            sets_off.append([off[i].alloc_outputs(sp["T"]) for _ in range(3)])
    # the sequence runs back to back with independent launches, then again with the
    # overlap off (so that no plain launch of the reference breaks the first run's chains)
    seq = [(int(rng.integers(3)), int(rng.integers(3)), int(rng.integers(3))) for _ in range(60)]
    fresh_on, fresh_off, orders = [], [], []
    for i, blk, k in seq:
        if i == 1:
            fresh_on.append(on[1].process(inputs[1][blk]))
        else:
            on[i].process(inputs[i][blk], out=sets_on[i][k])
        orders.append(_order(on[i]))
    for i, blk, k in seq:
        if i == 1:
            fresh_off.append(off[1].process(inputs[1][blk]))
        else:
            off[i].process(inputs[i][blk], out=sets_off[i][k])
    torch.cuda.synchronize()
    for i in (0, 2):
        for a, b in zip(sets_on[i], sets_off[i]):
            for name in ("flags", "avg", "weight", "stats"):
                assert torch.equal(a[name], b[name]), (i, name)
    for a, b in zip(fresh_on, fresh_off):
        for name in ("flags", "avg", "weight", "stats"):
            assert torch.equal(a[name], b[name]), name
    for s_on, s_off in zip(on, off):
        a, b = binding.rfi_get_state(s_on.ctx), binding.rfi_get_state(s_off.ctx)
        n = 36 * s_on.options["lanes_per_row"] * s_on.R      # the open bins' carry
        assert len(a) == len(b) and a[-n:] == b[-n:]
        binding.rfi_check(s_on.ctx)
    assert "independent" in orders and ("waiting" in orders or "plain" in orders), orders
    for s in on + off:
        s.close()
