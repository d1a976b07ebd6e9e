"""Autotuner for the flagging kernel's launch shape.

For one workload (dtype, M, K, T, rows) it times candidate options of rfi_create_ex
-- lanes per row P, warps per block, register budget, shared-memory staging,
window-parallel lanes, buffered output stores, L2 prefetch group size and distance --
on the
caller's device data with CUDA events, and returns the fastest.  Results are cached
in memory and, when `cache_path` is given, in a JSON file keyed by the workload.

Every candidate computes the same statistics and flags; only the reduction order of
a window (which depends on P) changes, within FP32 rounding.
"""
import json
import os
import statistics

from . import binding as B
from .stream import RfiStream

_MEM = {}


def _key(stations, channels, M, K, T, dtype):
    return f"{B._dtype(dtype)}:{stations}x{channels}:M{M}:K{K}:T{T}"


def candidates_p(M, dtype):
    spu = 2 if (B._dtype(dtype) == B.RFI_C32H and M % 2 == 0) else 1
    ps = [p for p in (1, 2, 4, 8, 16) if M % (p * spu) == 0]
    if B._dtype(dtype) == B.RFI_C32H and spu == 1:
        ps = [1]
    return ps


def time_options(stations, channels, M, K, thr, dtype, vis, reps=30, warmup=5, **opts):
    """Launch period (s) of one option set on `vis` (device tensor): launches back to
    back, as a stream of blocks runs them (consecutive launches may overlap), each into
    the next of four output sets (a ring of output buffers, as a pipeline keeps them;
    one set reused every launch would let the outputs stay in L2), events around each
    of three runs of reps/3 launches, the median run."""
    import torch
    st = RfiStream(stations, channels, M, K, thr, dtype, **opts)
    T = vis.shape[-3]
    outs = [st.alloc_outputs(T, device=vis.device) for _ in range(4)]
    n = max(1, reps // 3)
    try:
        for i in range(warmup):
            st.process(vis, out=outs[i % 4])
        runs = []
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for i in range(n):
                st.process(vis, out=outs[i % 4])
            b.record()
            runs.append((a, b))
        torch.cuda.synchronize()
        return statistics.median(a.elapsed_time(b) for a, b in runs) * 1e-3 / n
    finally:
        st.close()


TUNED_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned.json")


def tune(stations, channels, M, K, thr, dtype, vis, cache_path=None, reps=30, verbose=False,
         fixed=None, write_cache=True):
    """Return (best_options, table) for this workload; coordinate search over the
    launch shape, then the prefetch distance and size.  `fixed` options (for example
    window_F) are part of every candidate."""
    fixed = dict(fixed or {})
    T = vis.shape[-3]
    key = _key(stations, channels, M, K, T, dtype) + "".join(
        f":{k}={v}" for k, v in sorted(fixed.items()))
    if key in _MEM:
        return _MEM[key], []
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            disk = json.load(f)
        if key in disk:
            _MEM[key] = disk[key]
            return disk[key], []
    table = []

    def run(o):
        t = time_options(stations, channels, M, K, thr, dtype, vis, reps=reps, **o, **fixed)
        table.append((dict(o), t))
        if verbose:
            print(f"  {o} {t * 1e6:.1f} us")
        return t

    # stage 1: launch shape without prefetch; stage 2: prefetch for the three best
    shapes = [(4, 0), (8, 0), (16, 0), (4, 96), (2, 96), (4, 80), (8, 80), (4, 64), (8, 64)]
    stage1 = []
    F = fixed.get("window_F", 1)
    for P in [p for p in candidates_p(M, dtype) if p * F <= 32]:
        for wpb, regs in shapes:
            o = dict(lanes_per_row=P, warps_per_block=wpb, max_registers=regs,
                     prefetch_groups=0, prefetch_bytes=1024)
            try:
                stage1.append((run(o), o))
            except B.RfiError:          # no kernel with this register budget
                continue
    # rows staged in shared memory by TMA bulk copies (no register buffers for loads in
    # flight, so tighter register budgets are candidates too)
    for P in [p for p in candidates_p(M, dtype) if p <= 8 and p * F <= 32]:
        for regs in (0, 80, 64):
            for wpb, G, NS in ((4, 2, 2), (4, 1, 2), (8, 1, 2), (4, 1, 3)):
                o = dict(lanes_per_row=P, warps_per_block=wpb, max_registers=regs,
                         prefetch_groups=0, prefetch_bytes=1024, loader=1,
                         tma_stage_windows=G, tma_stages=NS)
                try:
                    stage1.append((run(o), o))
                except B.RfiError:      # no such kernel, or it does not fit the shared memory
                    continue
        # the same staging with one tensor tile per warp and stage (lanes_per_row <= 4)
        for G, NS in ((2, 2), (1, 3)):
            o = dict(lanes_per_row=P, warps_per_block=4, max_registers=0, prefetch_groups=0,
                     prefetch_bytes=1024, loader=2, tma_stage_windows=G, tma_stages=NS)
            try:
                stage1.append((run(o), o))
            except B.RfiError:
                continue
    # window-parallel lanes: the lanes of a row take whole windows in turn (a bin must
    # hold at least lanes_per_row windows)
    for P in (2, 4, 8):
        if P * F > 32 or K // M < P:
            continue
        for wpb, regs in ((4, 0), (8, 0), (4, 96)):     # 96: binary16 odd windows only
            o = dict(lanes_per_row=P, warps_per_block=wpb, max_registers=regs,
                     prefetch_groups=0, prefetch_bytes=1024, lane_split=1)
            try:
                stage1.append((run(o), o))
            except B.RfiError:
                continue
    stage1.sort(key=lambda x: x[0])

    def direct(o):                      # unit-split direct loader: buffered stores, prefetch
        return o.get("loader", 0) == 0 and o.get("lane_split", 0) == 0

    # the best direct-load shapes again with 16-byte buffered output stores (prefetch is
    # tried in stage 2 for the direct loader only)
    for _, base in [x for x in stage1 if direct(x[1])][:3]:
        o = dict(base, buffered_stores=1)
        try:
            stage1.append((run(o), o))
        except B.RfiError:              # no buffered variant of this shape
            continue
    stage1.sort(key=lambda x: x[0])
    best_t, best = stage1[0]
    for _, base in [x for x in stage1 if direct(x[1])][:3]:
        for pg in (1, 2):
            for pb in (512, 1024):
                o = dict(base, prefetch_groups=pg, prefetch_bytes=pb)
                try:
                    t = run(o)
                except B.RfiError:      # a kernel variant without the prefetch code
                    continue
                if t < best_t:
                    best, best_t = o, t
    best = dict(best, seconds=best_t, **fixed)
    _MEM[key] = best
    if cache_path and write_cache:
        disk = {}
        if os.path.exists(cache_path):
            with open(cache_path) as f:
                disk = json.load(f)
        disk[key] = best
        with open(cache_path, "w") as f:
            json.dump(disk, f, indent=1, sort_keys=True)
    return best, table


def options_of(best):
    """Strip the timing from a tuned entry: the keyword options for RfiStream."""
    return {k: v for k, v in best.items() if k != "seconds"}
