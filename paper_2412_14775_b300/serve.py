"""Continuous-batching serving loop over many correlator streams.

Streams (subbands of different station and channel counts) deliver blocks at their
own Poisson rates.  Each stream owns a flagging context whose state (averaging
carry, thresholds) stays on the device between blocks.  The loop

  * queues every arrived block (blocks of one stream are processed in order, one at
    a time, because each block continues the previous block's averaging bin);
  * admits queued blocks while the HBM budget for blocks in flight (input + outputs)
    and the batch slots allow, oldest arrival first;
  * launches each batch of admitted blocks as ONE persistent kernel
    (rfi_process_batch) on one of several CUDA streams, so batches admitted while
    others are still running overlap on the device;
  * retires batches as their CUDA events complete, releasing memory and streams.

Block latency = device completion time - arrival time (both on the loop's clock:
the device clock is tied to the host clock by an event recorded at start).
Everything computed runs in the library's kernels; this module only schedules.
"""
import collections
import statistics
import time

import numpy as np

from . import binding as B
from .stream import RfiStream


class _Stream:
    def __init__(self, idx, cfg, M, K, T, thr, dtype, options, blocks):
        self.idx = idx
        self.T = T
        self.cfg = cfg
        self.st = RfiStream(cfg["stations"], cfg["channels"], M, K, thr, dtype, **options)
        self.blocks = blocks                      # device input blocks, used round robin
        self.queue = collections.deque()          # (arrival_time, seq)
        self.busy = False
        self.done = 0
        # outputs: a block completes between floor(T/K) and floor(T/K) + 1 averaging
        # bins and, with partial windows, between floor(T/M) and floor((T + M - 1)/M)
        # windows (with overlapping windows at most T/H, each adding H flag bits); the
        # storage is sized for the larger counts and viewed at this block's exact ones
        import torch
        R, F = self.st.R, self.st.F
        B = self.st.bits_per_window
        self.n_out_max = T // K + 1
        self.n_win_max = (T + M - 1) // B
        words_max = (self.n_win_max * B + 31) // 32
        dev = blocks[0].device
        self.out_pool = []
        for _ in range(2):
            self.out_pool.append(dict(
                flags_store=torch.empty(R * words_max, dtype=torch.int32, device=dev),
                stats_store=torch.empty(3 * (R // F) * self.n_win_max, device=dev),
                avg_store=torch.empty(R * self.n_out_max * 8, device=dev),
                weight_store=torch.empty(R * self.n_out_max, device=dev)))
        self.out_next = 0
        self.bytes_in = blocks[0].numel() * blocks[0].element_size()
        self.bytes_out = sum(v.numel() * v.element_size() for v in self.out_pool[0].values())

    def outputs(self):
        """Output buffers for the next block, shaped for its numbers of completed
        windows and bins."""
        o = self.out_pool[self.out_next]
        self.out_next = (self.out_next + 1) % len(self.out_pool)
        R, F, M = self.st.R, self.st.F, self.st.M
        n = self.st.outputs_for(self.T)
        nw = self.st.windows_for(self.T)[0]
        words = (nw * self.st.bits_per_window + 31) // 32
        return dict(flags=o["flags_store"][:R * words].view(R, words),
                    stats=o["stats_store"][:3 * (R // F) * nw].view(3, R // F, nw),
                    avg=o["avg_store"][:R * n * 8].view(R, n, 4, 2),
                    weight=o["weight_store"][:R * n].view(R, n))


class ServingLoop:
    def __init__(self, stream_cfgs, M=16, K=256, T=256, thresholds=None, dtype="f16",
                 options=None, hbm_budget_bytes=8 << 30, max_batch=32, cuda_streams=3,
                 block_seconds=0.128, pool_blocks=2, seed=5, record_outputs=False,
                 blocks=None):
        import torch
        from .thresholds import default_thresholds
        import synth
        self.torch = torch
        self.M, self.K, self.T = M, K, T
        self.block_seconds = block_seconds
        self.budget = int(hbm_budget_bytes)
        self.max_batch = min(int(max_batch), 64)
        self.record = record_outputs
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
            self.streams.append(_Stream(i, cfg, M, K, T, thr, dtype, opts, bl))
        self.cuda_streams = [torch.cuda.Stream() for _ in range(cuda_streams)]
        self.outputs = collections.defaultdict(list)     # stream -> [(seq, numpy dict)]

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

    def run(self, duration, seed=0, arrivals=None):
        """Serve Poisson arrivals for `duration` seconds of wall time (then drain).
        Returns latency and throughput statistics."""
        torch = self.torch
        rng = np.random.default_rng(seed)
        arrivals = arrivals if arrivals is not None else self._schedule(duration, rng)
        ai = 0
        free_bytes = self.budget
        inflight = []                 # (event, [(stream, arrival, seq, out)], cuda_stream, bytes)
        free_cs = list(self.cuda_streams)
        lat, samples, nbatches, batch_sizes = [], 0, 0, []
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
            # retire finished batches
            still = []
            for ev, items, cs, nb in inflight:
                if ev.query():
                    tdone = ref.elapsed_time(ev) * 1e-3
                    for s, ta, k, out in items:
                        lat.append(tdone - ta)
                        samples += s.st.R * self.T
                        s.busy = False
                        s.done += 1
                        if self.record:
                            self.outputs[s.idx].append(
                                (k, {n: v.cpu().numpy().copy() for n, v in out.items()}))
                    free_bytes += nb
                    free_cs.append(cs)
                else:
                    still.append((ev, items, cs, nb))
            inflight = still
            # admit: oldest head-of-queue first, while memory and batch slots allow
            if free_cs:
                ready = sorted((s.queue[0][0], s.idx) for s in self.streams
                               if s.queue and not s.busy)
                items, nb = [], 0
                for _, si in ready:
                    s = self.streams[si]
                    need = s.bytes_in + s.bytes_out
                    if len(items) >= self.max_batch or nb + need > free_bytes:
                        break
                    ta, k = s.queue.popleft()
                    out = s.outputs()
                    s.busy = True
                    items.append((s, ta, k, out))
                    nb += need
                if items:
                    cs = free_cs.pop()
                    vis = [s.blocks[k % len(s.blocks)] for s, _, k, _ in items]
                    B.rfi_process_batch([s.st.ctx for s, _, _, _ in items], vis,
                                        [self.T] * len(items),
                                        [o["flags"] for _, _, _, o in items],
                                        [o["avg"] if o["avg"].numel() else None
                                         for _, _, _, o in items],
                                        [o["weight"] if o["weight"].numel() else None
                                         for _, _, _, o in items],
                                        [o["stats"] for _, _, _, o in items], stream=cs)
                    ev = torch.cuda.Event(enable_timing=True)
                    ev.record(cs)
                    inflight.append((ev, items, cs, nb))
                    free_bytes -= nb
                    nbatches += 1
                    batch_sizes.append(len(items))
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
        return {
            "blocks": len(lat), "batches": nbatches,
            "mean_batch": statistics.mean(batch_sizes) if batch_sizes else 0.0,
            "p50_latency_s": float(np.percentile(lat_arr, 50)),
            "p99_latency_s": float(np.percentile(lat_arr, 99)),
            "max_latency_s": float(lat_arr.max()),
            "block_seconds": self.block_seconds,
            "p99_over_block": float(np.percentile(lat_arr, 99)) / self.block_seconds,
            "samples_per_s": samples / wall, "wall_s": wall,
            "offered_real_time_streams": sum(s.cfg.get("rho", 1.0) for s in self.streams),
        }

    def close(self):
        for s in self.streams:
            s.st.close()
