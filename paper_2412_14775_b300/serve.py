"""Continuous-batching serving loop over many correlator streams.

Streams (subbands of different station and channel counts) deliver blocks at their
own Poisson rates.  Each stream owns a flagging context whose state (averaging carry,
thresholds, open windows) stays on the device between blocks.  The loop

  * allocates, once, a device block pool sized from the GPU's free memory (minus a
    headroom) and the caller's budget; every admitted block takes one slot of it
    (input block + its outputs, first fit, 256-byte aligned) until it retires;
  * queues every arrived block (blocks of one stream are processed in order, one at a
    time, because each block continues the previous block's averaging bin);
  * admits queued blocks, oldest arrival first, while pool slots and batch slots
    allow;
  * per batch, on one of several CUDA streams: copies each admitted block into its
    slot (from pinned host memory, `source="host"`, or from the producer's device
    buffer, `source="device"`, as a correlator that writes its output on the GPU),
    runs ONE persistent kernel over all of them (rfi_process_batch), and copies each
    block's flags, averages and weights (one contiguous range of its slot) back to
    pinned host memory (the per-window statistics stay on the device); batches
    admitted while others run overlap on the device;
  * retires batches as their CUDA events complete, releasing their slots; a stream's
    next block may be admitted once the kernel of the batch holding its previous block
    is done, while that batch's results are still being copied out.

Block latency = completion of the batch's last copy (device clock) - arrival time
(host clock), the clocks tied by an event recorded at start.  Everything computed runs
in the library's kernels; this module schedules, copies and keeps the books.
"""
import collections
import math
import statistics
import time

import numpy as np

from . import binding as B
from .stream import RfiStream

_ALIGN = 256


class DevicePool:
    """One device allocation carved into slots: first fit over a sorted free list,
    neighbours merged on release, every slot aligned to 256 bytes."""

    def __init__(self, nbytes, device):
        import torch
        self.nbytes = int(nbytes) // _ALIGN * _ALIGN
        self.buf = torch.empty(self.nbytes, dtype=torch.uint8, device=device)
        self.free = [(0, self.nbytes)]           # (offset, size), sorted by offset
        self.used = 0
        self.peak = 0

    @staticmethod
    def rounded(n):
        return (int(n) + _ALIGN - 1) // _ALIGN * _ALIGN

    def alloc(self, n):
        n = self.rounded(n)
        for i, (off, size) in enumerate(self.free):
            if size >= n:
                if size == n:
                    del self.free[i]
                else:
                    self.free[i] = (off + n, size - n)
                self.used += n
                self.peak = max(self.peak, self.used)
                return off
        return None

    def release(self, off, n):
        n = self.rounded(n)
        self.used -= n
        i = 0
        while i < len(self.free) and self.free[i][0] < off:
            i += 1
        self.free.insert(i, (off, n))
        # merge with the right, then the left neighbour
        if i + 1 < len(self.free) and off + n == self.free[i + 1][0]:
            self.free[i] = (off, n + self.free[i + 1][1])
            del self.free[i + 1]
        if i > 0 and self.free[i - 1][0] + self.free[i - 1][1] == off:
            self.free[i - 1] = (self.free[i - 1][0], self.free[i - 1][1] + self.free[i][1])
            del self.free[i]

    def view(self, off, nbytes, dtype, shape):
        return self.buf[off:off + nbytes].view(dtype).view(shape)


class _Stream:
    def __init__(self, idx, cfg, M, K, T, thr, dtype, options, sources, copy_in=True,
                 n_host_buffers=1):
        import torch
        self.idx = idx
        self.T = T
        self.cfg = cfg
        self.st = RfiStream(cfg["stations"], cfg["channels"], M, K, thr, dtype, **options)
        self.sources = sources                    # arriving blocks (host pinned or device)
        self.queue = collections.deque()          # (arrival_time, seq)
        self.busy = False
        self.lat = []                             # latencies of this stream's blocks (s)
        self.done = 0
        R, F = self.st.R, self.st.F
        bits = self.st.bits_per_window
        # a block completes between floor(T/K) and floor(T/K) + 1 averaging bins and,
        # with partial windows, up to ceil(T/M) windows (overlapping windows: T/H, each
        # adding H flag bits); a slot is sized for the larger counts
        n_out_max = T // K + 1
        n_win_max = (T + M - 1) // bits
        words_max = (n_win_max * bits + 31) // 32
        src = sources[0]
        self.in_shape, self.in_dtype = tuple(src.shape), src.dtype
        # slot layout: input, then the outputs returned to the host (flags, averages,
        # weights: one contiguous range), then the statistics
        self.parts = [("vis", src.numel() * src.element_size() if copy_in else 0),
                      ("flags", 4 * R * words_max), ("avg", 4 * R * n_out_max * 8),
                      ("weight", 4 * R * n_out_max), ("stats", 4 * 3 * (R // F) * n_win_max)]
        self.offsets = {}
        o = 0
        for name, n in self.parts:
            self.offsets[name] = o
            o += DevicePool.rounded(n)
        self.slot_bytes = o
        self.ret_lo, self.ret_hi = self.offsets["flags"], self.offsets["stats"]
        # pinned host buffers of the returned outputs, one per CUDA stream of the loop: a
        # stream's blocks may be in several batches' result copies at once (a block is
        # admitted once the previous one's kernel is done), block seq uses seq mod n
        self.out_host = [torch.empty(self.ret_hi - self.ret_lo, dtype=torch.uint8,
                                     pin_memory=True) for _ in range(max(1, n_host_buffers))]

        # contexts whose blocks always complete T/M windows: counts kept here, without a
        # call into the library per block
        o = self.st.options
        self.plain = not o.get("partial_windows") and not o.get("window_hop")
        self.n_seen = 0

    def next_counts(self):
        """(averaging bins, windows) the next block completes; advances the stream."""
        if self.plain:
            K = self.st.K
            n = (self.n_seen + self.T) // K - self.n_seen // K
            nw = self.T // self.st.M
        else:
            n = self.st.outputs_for(self.T)
            nw = self.st.windows_for(self.T)[0]
        self.n_seen += self.T
        return n, nw

    def slot_views(self, pool, off, counts):
        """The block's input and outputs inside its pool slot, shaped for its numbers
        of completed bins and windows."""
        import torch
        R, F = self.st.R, self.st.F
        n, nw = counts
        words = (nw * self.st.bits_per_window + 31) // 32
        shapes = {"vis": (self.in_dtype, self.in_shape), "flags": (torch.int32, (R, words)),
                  "stats": (torch.float32, (3, R // F, nw)),
                  "avg": (torch.float32, (R, n, 4, 2)), "weight": (torch.float32, (R, n))}
        out = {}
        for name, (dt, shape) in shapes.items():
            out[name] = pool.view(off + self.offsets[name], math.prod(shape) * dt.itemsize, dt,
                                  shape)
        return out


class ServingLoop:
    def __init__(self, stream_cfgs, M=16, K=256, T=256, thresholds=None, dtype="f16",
                 options=None, hbm_budget_bytes=8 << 30, max_batch=32, cuda_streams=3,
                 block_seconds=0.128, pool_blocks=2, seed=5, record_outputs=False,
                 blocks=None, source="device", headroom_bytes=2 << 30, results_to_host=True,
                 early_release=True, copy_in=True):
        """source: "device" (blocks arrive in device memory, as from a GPU correlator,
        and are copied into the pool) or "host" (blocks arrive in pinned host memory and
        are copied to the device).  The block pool takes min(hbm_budget_bytes, free
        device memory - headroom_bytes), measured once here.  early_release: a stream's
        next block may be admitted as soon as the kernel of the batch holding its previous
        block is done (its state is final then), before that batch's result copies.
        copy_in=False (device source only): the batch reads each block where it arrived
        (the producer keeps it until the batch's kernel is done) and its slot holds the
        outputs alone, so admission by free memory counts the outputs only."""
        import torch
        from .thresholds import default_thresholds
        import synth
        self.torch = torch
        self.M, self.K, self.T = M, K, T
        self.block_seconds = block_seconds
        self.max_batch = min(int(max_batch), 64)
        self.record = record_outputs
        self.source = source
        self.results_to_host = results_to_host
        self.early_release = early_release
        if source not in ("device", "host"):
            raise ValueError("source is 'device' or 'host'")
        if not copy_in and source != "device":
            raise ValueError("copy_in=False needs blocks in device memory")
        self.copy_in = copy_in
        thr = thresholds or default_thresholds(M)
        opts = dict(options or {})
        self.streams = []
        for i, cfg in enumerate(stream_cfgs):
            if blocks is not None:
                bl = blocks[i]
            else:
                bl = [synth.generate.device_block(cfg["stations"], cfg["channels"], T,
                                                  seed=seed * 1000 + i * 10 + k, dtype=dtype)
                      for k in range(pool_blocks)]
            if source == "host":
                bl = [b.cpu().pin_memory() for b in bl]
            self.streams.append(_Stream(i, cfg, M, K, T, thr, dtype, opts, bl, copy_in,
                                        cuda_streams if early_release else 1))
        torch.cuda.synchronize()
        free, total = torch.cuda.mem_get_info()
        self.free_at_start = int(free)
        self.pool_request = int(hbm_budget_bytes)
        nbytes = max(0, min(int(hbm_budget_bytes), int(free) - int(headroom_bytes)))
        biggest = max(s.slot_bytes for s in self.streams)
        if nbytes < biggest:
            raise MemoryError(f"free device memory ({free / 2**30:.1f} GiB less the headroom) "
                              f"does not hold one block of the largest stream "
                              f"({biggest / 2**20:.0f} MiB)")
        self.pool = DevicePool(nbytes, "cuda")
        self.cuda_streams = [torch.cuda.Stream() for _ in range(cuda_streams)]
        self.outputs = collections.defaultdict(list)     # stream -> [(seq, numpy dict)]

    @property
    def budget(self):
        return self.pool.nbytes

    def _schedule(self, duration, rng):
        arr = []
        for s in self.streams:
            rate = s.cfg.get("rho", 1.0) / self.block_seconds
            t = rng.exponential(1.0 / rate)
            k = 0
            while t < duration:
                arr.append((t, s.idx, k))
                k += 1
                t += rng.exponential(1.0 / rate)
        arr.sort()
        return arr

    def _launch(self, items, cs):
        """Copy the blocks into their slots, run one batch, copy the results out; all on
        CUDA stream cs.  The batch receives addresses inside the pool (no tensor views
        on this path)."""
        torch = self.torch
        buf, base = self.pool.buf, self.pool.buf.data_ptr()
        if self.copy_in:
            with torch.cuda.stream(cs):
                for s, _, k, off, _ in items:
                    src = s.sources[k % len(s.sources)].reshape(-1)
                    n = s.parts[0][1]
                    buf[off:off + n].view(src.dtype).copy_(src, non_blocking=True)
        ptr = {name: [base + off + s.offsets[name] for s, _, _, off, _ in items]
               for name in ("vis", "flags", "avg", "weight", "stats")}
        if not self.copy_in:
            ptr["vis"] = [s.sources[k % len(s.sources)].data_ptr() for s, _, k, _, _ in items]
        has_out = [c[0] > 0 for *_, c in items]
        B.rfi_process_batch([s.st.ctx for s, *_ in items], ptr["vis"], [self.T] * len(items),
                            ptr["flags"], [p if h else None for p, h in zip(ptr["avg"], has_out)],
                            [p if h else None for p, h in zip(ptr["weight"], has_out)],
                            ptr["stats"], stream=cs)
        # the streams' state (carry, thresholds) is final once the kernel is done: their
        # next blocks may be admitted while this batch's results are still being copied
        ev_kernel = torch.cuda.Event()
        ev_kernel.record(cs)
        if self.results_to_host:
            with torch.cuda.stream(cs):
                for s, _, k, off, _ in items:
                    dst = s.out_host[k % len(s.out_host)]
                    dst.copy_(self.pool.buf[off + s.ret_lo:off + s.ret_hi], non_blocking=True)
        ev = torch.cuda.Event(enable_timing=True)
        ev.record(cs)
        return ev_kernel, ev

    def run(self, duration, seed=0, arrivals=None):
        """Serve Poisson arrivals for `duration` seconds of wall time (then drain).
        Returns latency and throughput statistics."""
        torch = self.torch
        rng = np.random.default_rng(seed)
        arrivals = arrivals if arrivals is not None else self._schedule(duration, rng)
        for s in self.streams:
            s.lat = []                # the statistics of this run only
        ai = 0
        inflight = []                 # [kernel event, done event, items, cuda stream, freed]
        free_cs = list(self.cuda_streams)
        lat, samples, nbatches, batch_sizes, waits = [], 0, 0, [], 0
        h2d = d2h = 0
        t_launch = t_retire = 0.0         # host seconds spent launching / retiring batches
        torch.cuda.synchronize()
        ref = torch.cuda.Event(enable_timing=True)
        ref.record()
        ref.synchronize()
        t0 = time.perf_counter()
        while True:
            now = time.perf_counter() - t0
            while ai < len(arrivals) and arrivals[ai][0] <= now:
                ta, si, k = arrivals[ai]
                self.streams[si].queue.append((ta, k))
                ai += 1
            # retire finished batches and release their slots
            tr = time.perf_counter()
            still = []
            for entry in inflight:
                ev_k, ev, items, cs, freed = entry
                if self.early_release and not freed and ev_k.query():
                    for s, *_ in items:
                        s.busy = False         # its next block may be admitted now
                    entry[4] = True
                if ev.query():
                    tdone = ref.elapsed_time(ev) * 1e-3
                    for s, ta, k, off, counts in items:
                        lat.append(tdone - ta)
                        s.lat.append(tdone - ta)
                        samples += s.st.R * self.T
                        s.busy = False
                        s.done += 1
                        if self.record:
                            views = s.slot_views(self.pool, off, counts)
                            self.outputs[s.idx].append(
                                (k, {n: v.cpu().numpy().copy() for n, v in views.items()
                                     if n != "vis"}))
                        self.pool.release(off, s.slot_bytes)
                    free_cs.append(cs)
                else:
                    still.append(entry)
            inflight = still
            t_retire += time.perf_counter() - tr
            # admit: oldest head-of-queue first, while pool slots and batch slots allow
            if free_cs:
                ready = sorted((s.queue[0][0], s.idx) for s in self.streams
                               if s.queue and not s.busy)
                items = []
                for _, si in ready:
                    s = self.streams[si]
                    if len(items) >= self.max_batch:
                        break
                    off = self.pool.alloc(s.slot_bytes)
                    if off is None:           # the pool is full: wait for a retirement
                        waits += 1
                        break
                    ta, k = s.queue.popleft()
                    s.busy = True
                    items.append((s, ta, k, off, s.next_counts()))
                if items:
                    cs = free_cs.pop()
                    tl = time.perf_counter()
                    inflight.append([*self._launch(items, cs), items, cs, False])
                    t_launch += time.perf_counter() - tl
                    nbatches += 1
                    batch_sizes.append(len(items))
                    for s, *_ in items:
                        h2d += s.parts[0][1] if self.source == "host" else 0
                        d2h += (s.ret_hi - s.ret_lo) if self.results_to_host else 0
            if ai >= len(arrivals) and not inflight and all(not s.queue for s in self.streams):
                break
            if not inflight and ai < len(arrivals):
                wait = arrivals[ai][0] - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.002))
            else:
                time.sleep(2e-5)
        wall = time.perf_counter() - t0
        lat_arr = np.array(lat) if lat else np.zeros(1)
        hist = collections.Counter(batch_sizes)
        return {
            "blocks": len(lat), "batches": nbatches,
            "mean_batch": statistics.mean(batch_sizes) if batch_sizes else 0.0,
            "batch_size_hist": {str(k): hist[k] for k in sorted(hist)},
            "p50_latency_s": float(np.percentile(lat_arr, 50)),
            "p99_latency_s": float(np.percentile(lat_arr, 99)),
            "max_latency_s": float(lat_arr.max()),
            "block_seconds": self.block_seconds,
            "p99_over_block": float(np.percentile(lat_arr, 99)) / self.block_seconds,
            "samples_per_s": samples / wall, "wall_s": wall,
            "offered_real_time_streams": sum(s.cfg.get("rho", 1.0) for s in self.streams),
            "source": self.source, "h2d_bytes": h2d, "d2h_bytes": d2h,
            "pool_gb": self.pool.nbytes / 1e9, "pool_peak_gb": self.pool.peak / 1e9,
            "free_gb_at_start": self.free_at_start / 1e9, "admission_waits": waits,
            "host_launch_us_per_batch": 1e6 * t_launch / max(nbatches, 1),
            "host_busy_frac": (t_launch + t_retire) / wall if wall > 0 else 0.0,
            "per_stream_p99_s": [float(np.percentile(s.lat, 99)) if s.lat else None
                                 for s in self.streams],
        }

    def close(self):
        for s in self.streams:
            s.st.close()
        self.pool = None
