"""Throughput of the sm_103a online RFI flagging path (arXiv 2412.14775).

One step = one rfi_process_block call on a whole LOFAR-scale block: 62 stations
(1953 baselines incl. autocorrelations), 64 channels, 256 samples, 4 correlations
complex64 (1.02 GB), window M = 16, averaging 256 -> 1: Stokes, spectral kurtosis,
directional statistics (Re, Im), flags, flag packing and flagged averaging, all in
one kernel launch.  Inputs are 1 GB, far larger than the 126 MB L2, so no L2 flush
is needed between steps.

Prints ONE JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle on a
bounded sample of the same workload instead.
"""
import argparse
import collections
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("visibility samples/sec and HBM GB/s (% of peak), FP16 vs FP32; "
          "p99 latency vs real time")
WORKLOAD = dict(workload="lofar-scale block", stations=62, baselines=1953, channels=64,
                samples_per_block=256, window_M=16, avg_K=256, correlations=4)
BLOCK_SECONDS = 256 * 0.5e-3       # 2000 samples ~ 1 s in the paper's simulations
# a stricter cadence for sensitivity: one LOFAR subband (195312.5 Hz) split into 64
# channels gives one sample per channel every 64 / 195312.5 s = 327.68 us
NATIVE_BLOCK_SECONDS = 256 * 64 / 195312.5


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


# The main flagging kernel (k_block) and every helper it calls are defined in
# rfi_device.cuh; the instance tables only name template arguments, which the profile
# records in the kernel's name.
KERNEL_SOURCES = ("rfi_device.cuh",)


def kernel_source_hash():
    """Hash of the main kernel's device code; a profile's traffic figure is used only
    while the code it was taken from is unchanged."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2412_14775_b300", "csrc")
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _profile(dtype):
    """Header fields of profiles/k_block_lofar_block_<dtype>.md (dtype f32, f16 or f16_h2),
    or {} when the kernel sources changed after that capture."""
    path = os.path.join(ROOT, "profiles", f"k_block_lofar_block_{dtype}.md")
    try:
        kv = {}
        for line in open(path):
            if ":" in line and not line.startswith(("|", " ", "#")):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        return kv if kv.get("source_sha256_16") == kernel_source_hash() else {}
    except OSError:
        return {}


def profiled_traffic(dtype):
    """DRAM bytes per launch from the ncu capture of the current kernel, or None."""
    v = _profile(dtype).get("traffic_bytes_per_launch")
    return int(v) if v else None


def profiled_dram_gbs(dtype):
    """ncu's DRAM throughput (GB/s) of that capture (cold caches, serialised), or None."""
    v = _profile(dtype).get("ncu_dram_gbs")
    return float(v) if v else None


def algo_bytes(R, T, M, K, n_out, sample_bytes):
    """Bytes the method must move per launch: input, flag words, stats, averages."""
    return R * (T * sample_bytes + 4 * math.ceil(T / 32) + 12 * (T // M) + 36 * n_out)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reference_arm(args):
    """The FP64 CPU oracle on a bounded sample of the workload (rank 0 only)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    import synth
    from paper_2412_14775_b300.thresholds import default_thresholds
    M, K, T = 16, 256, 256
    thr = default_thresholds(M)
    d = synth.lofar_block(seed=2)
    R = d["vis"].shape[0] * d["vis"].shape[1]
    rows = d["vis"].reshape(R, T, 4, 2)
    # size each step's sample so that warm-up plus timed steps take about a minute on
    # all host cores (row ranges on threads)
    cores = host_threads()
    t0 = time.perf_counter()
    oracle.OracleStream(512, M, K, **thr).process(rows[:512])
    per_row = (time.perf_counter() - t0) / 512
    budget = 60.0 / (args.warmup + args.steps)
    n_rows = int(min(R, max(16, cores * budget / max(per_row, 1e-9))))
    if args.ref_rows:
        n_rows = min(n_rows, args.ref_rows)
    times = []
    for step in range(args.warmup + args.steps):
        sel = rows[(step * n_rows) % R:(step * n_rows) % R + n_rows]
        dt = oracle_threads(sel, M, K, thr, cores)
        if step >= args.warmup:
            times.append((len(sel) * T, dt))
    samples = sum(s for s, _ in times)
    secs = sum(t for _, t in times)
    v = samples / secs
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "samples/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(WORKLOAD, dtype="complex64"),
            "cpu_baseline": {"value": v, "unit": "samples/s", "cores": cores, "kind": "oracle",
                             "cpu_model": cpu_model(),
                             "sample": f"{n_rows} of {R} rows x {T} samples per step, "
                                       f"row ranges on {cores} threads"},
            "e2e": {"value": v, "unit": "samples/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_model():
    """The host CPU's model name (Linux), or the platform's processor string."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or "unknown"


def host_threads():
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_threads(rows, M, K, thr, threads):
    """Run the oracle on `rows` split into `threads` contiguous row ranges, one
    OracleStream per range on its own thread (rows are independent streams, so this
    is the same computation; the C oracle releases the GIL while it runs).  Returns
    the wall time in seconds."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    n = len(rows)
    edges = [n * k // threads for k in range(threads + 1)]
    parts = [rows[a:b] for a, b in zip(edges[:-1], edges[1:]) if b > a]
    streams = [oracle.OracleStream(len(p), M, K, **thr) for p in parts]
    with ThreadPoolExecutor(max_workers=len(parts)) as ex:
        t0 = time.perf_counter()
        list(ex.map(lambda sp: sp[0].process(sp[1]), zip(streams, parts)))
        return time.perf_counter() - t0


def cpu_baseline(passes=10, warm=3):
    """The oracle as it stands on the whole LOFAR-scale float32 block, stepped as the
    reference arm steps it: one step = the whole block over row ranges on every host
    core; `warm` untimed steps, then `passes` timed ones (the reported value); and one
    pass single-threaded.  The host's cores are shared with other jobs, so the figure
    moves from run to run."""
    import oracle
    import synth
    from paper_2412_14775_b300.thresholds import default_thresholds
    M, K, T = 16, 256, 256
    thr = default_thresholds(M)
    d = synth.lofar_block(seed=2)
    R = d["vis"].shape[0] * d["vis"].shape[1]
    rows = d["vis"].reshape(R, T, 4, 2)
    cores = host_threads()
    for _ in range(warm):
        oracle_threads(rows, M, K, thr, cores)
    times = [oracle_threads(rows, M, K, thr, cores) for _ in range(passes)]
    dtn = sum(times)
    oracle.OracleStream(256, M, K, **thr).process(rows[:256])
    t0 = time.perf_counter()
    oracle.OracleStream(R, M, K, **thr).process(rows)
    dt1 = time.perf_counter() - t0
    return {"value": passes * R * T / dtn, "unit": "samples/s", "cores": cores, "kind": "oracle",
            "single_thread_value": R * T / dt1, "cpu_model": cpu_model(),
            "best_step_value": R * T / min(times),
            "sample": f"all {R} rows x {T} samples of the float32 block per step, {passes} timed "
                      f"steps after {warm} warm-up steps: {dtn:.2f} s on {cores} threads (row "
                      f"ranges); one pass single-threaded: {dt1:.1f} s"}


def footprint_extras(torch, cs, peak, steps=500, warmup=10, only=None):
    """The paper's time-frequency windows (10 x 2 and 5 x 4, W = 20) on the 62-station,
    64-channel geometry with blocks of T = 250 samples (a multiple of both time
    extents), averaging 250 -> 1, complex64 and binary16; only = (dtype, M, F) times
    that one case."""
    import synth
    from paper_2412_14775_b300 import RfiStream, autotune, default_thresholds
    T, K = 250, 250
    R = 1953 * 64
    res = {}
    v32 = synth.generate.device_block(62, 64, T, seed=400, dtype="f32")
    for dtype in ("f32", "f16"):
        if only and only[0] != dtype:
            continue
        vis = v32 if dtype == "f32" else v32.half()
        sb = 32 if dtype == "f32" else 16
        for M, F in ((10, 2), (5, 4)):
            if only and only[1:] != (M, F):
                continue
            thr = default_thresholds(M * F)
            # binary16 input: float32 arithmetic, and binary16 arithmetic (precision = 2)
            for prec in ((0, 2) if dtype == "f16" else (0,)):
                fixed = {"window_F": F, **({"precision": 2} if prec else {})}
                best, _ = autotune.tune(62, 64, M, K, thr, dtype, vis, fixed=fixed,
                                        cache_path=autotune.TUNED_PATH, write_cache=False)
                opts = dict(autotune.options_of(best), **PIPELINED)
                st = RfiStream(62, 64, M, K, thr, dtype, **opts)
                out = st.alloc_outputs(T)
                k, _, _, _ = time_kernel(st, vis, out, steps, warmup, torch, cs)
                nbytes = R * (T * sb + 4 * math.ceil(T / 32) + 12 * (T // M) // F + 36)
                res[f"{dtype}_{M}x{F}" + ("_h2" if prec else "")] = {
                    "kernel_us": k * 1e6, "samples_per_s": R * T / k,
                    "achieved_gbs": nbytes / k / 1e9, "frac": nbytes / k / 1e9 / peak,
                    "options": opts}
                st.close()
        del vis
    del v32
    torch.cuda.empty_cache()
    return res


def detection_experiment(torch, realizations=8, inrs=(0.01, 0.1, 1.0, 10.0, 100.0), fa=0.05,
                         n_cal=16):
    """False-alarm and missed-detection probabilities against the interference-to-noise
    ratio for SK only, DS only and both, with polarised and with unpolarised
    interference, on blocks simulated as in the paper's Section 4.2 (2000 x 512, one
    baseline), 10 x 2 windows, thresholds calibrated for a 5 % false alarm per test on
    interference-free blocks.  An evaluation, not a speed figure."""
    from synth import paper_sim
    from paper_2412_14775_b300 import RfiStream
    from paper_2412_14775_b300.calibrate import permissive, thresholds_for_false_alarm
    M, F, T, C = 10, 2, 2000, 512
    K = T

    def run(st, vis):
        out = st.process(torch.from_numpy(vis).cuda())
        torch.cuda.synchronize()
        return out

    def sample_flags(out):
        w = out["flags"].to(torch.int64) & 0xFFFFFFFF
        bits = (w[:, :, None] >> torch.arange(32, device=w.device)) & 1
        return bits.reshape(w.shape[0], -1)[:, :T].bool()

    cal = RfiStream(1, C, M, K, permissive(), "f32", window_F=F)
    # the simulated blocks differ in receiver-noise scale, so the clean calibration set
    # spans several blocks
    stats = [run(cal, paper_sim.simulate_block(9000 + k, inr=0.0, n_broadband=0, n_narrow=0)
                 ["vis"])["stats"].clone() for k in range(n_cal)]
    thr = thresholds_for_false_alarm(stats, fa=fa)
    modes = {"SK": dict(thr, gamma=math.inf),
             "DS": dict(thr, s_low=-math.inf, s_high=math.inf),
             "BOTH": thr}
    streams = {m: RfiStream(1, C, M, K, t, "f32", window_F=F) for m, t in modes.items()}
    res = {"thresholds": thr, "window": "10 x 2", "realizations": realizations}
    for pol in (True, False):
        rows = []
        for inr in inrs:
            acc = {m: [0, 0, 0, 0] for m in modes}    # false, clean, missed, rfi
            for k in range(realizations):
                d = paper_sim.simulate_block(100 * k + int(1000 * inr) % 97 + (0 if pol else 50000),
                                             inr=inr, polarised=pol)
                truth = torch.from_numpy(d["truth"]).cuda()
                for m, st in streams.items():
                    st.reset()
                    f = sample_flags(run(st, d["vis"]))
                    a = acc[m]
                    a[0] += int((f & ~truth).sum()); a[1] += int((~truth).sum())
                    a[2] += int((~f & truth).sum()); a[3] += int(truth.sum())
            rows.append({"inr": inr, **{m: {"false_alarm": a[0] / max(a[1], 1),
                                            "missed": a[2] / max(a[3], 1)}
                                        for m, a in acc.items()}})
        res["polarised" if pol else "unpolarised"] = rows
    return res


def _stat_errors(torch, got, ref, M, thr):
    """Worst statistic errors of `got` against `ref` (stats tensors [3, R, n]) with the
    parity floors (1 for tau, M^-1/2 for r) and the fraction of windows whose flag
    differs (the flag rule on each side's own statistics)."""
    g, r = got.double(), ref.double()
    e_tau = ((g[0] - r[0]).abs() / r[0].abs().clamp(min=1.0)).max().item()
    fl = M ** -0.5
    e_r = max(((g[k] - r[k]).abs() / r[k].abs().clamp(min=fl)).max().item() for k in (1, 2))

    def flags(s):
        return (~((s[0] >= thr["s_low"]) & (s[0] <= thr["s_high"])) | ~(s[1] <= thr["gamma"]) |
                ~(s[2] <= thr["gamma"]))
    dis = (flags(got) != flags(ref)).float().mean().item()
    return {"tau_err": e_tau, "r_err": e_r, "flag_disagree": dis}


def fp16_extras(vis32, vis16, tuned, torch, cs, peak, dev, steps, warmup):
    """Binary16 storage of the LOFAR-scale block, windows M = 8, 16, 32, 64 (K = 256), in
    both binary16 modes: float32 arithmetic on exactly widened values (`storage`) and
    binary16 Stokes arithmetic (`h2`, precision = 2).  Per mode: launch time, throughput
    and fraction of the copy bandwidth; statistic error and flag disagreement against the
    float32 kernel run on the same binary16 values widened to float32 (`arith_*`: the
    mode's arithmetic alone; the float32 kernel is within 1e-5 of the FP64 oracle, see the
    parity tests) and on the original float32 block (`total_*`: with the input's
    quantisation)."""
    from paper_2412_14775_b300 import RfiStream, default_thresholds
    R, T = vis32.shape[0], vis32.shape[1]
    vis16w = vis16.float()
    res = {}
    for Mw in (8, 16, 32, 64):
        thr = default_thresholds(Mw)
        refs = {}
        for name, v in (("arith", vis16w), ("total", vis32)):
            f32 = RfiStream(62, 64, Mw, 256, thr, "f32")
            refs[name] = f32.process(v, stream=cs)["stats"]
            torch.cuda.synchronize()
            f32.close()
        b16 = algo_bytes(R, T, Mw, 256, 1, 16)
        entry = {}
        for mode, fixed in (("storage", {}), ("h2", {"precision": 2})):
            o16opts = dict(tuned(Mw, "f16", vis16, fixed), **PIPELINED)
            s16 = RfiStream(62, 64, Mw, 256, thr, "f16", **o16opts)
            o16 = s16.alloc_outputs(T, device=dev)
            k16, _, _, _ = time_kernel(s16, vis16, o16, steps, warmup, torch, cs)
            e = {"kernel_us": k16 * 1e6, "samples_per_s": R * T / k16,
                 "achieved_gbs": b16 / k16 / 1e9, "frac": b16 / k16 / 1e9 / peak,
                 "options": o16opts}
            for name, ref in refs.items():
                for k, val in _stat_errors(torch, o16["stats"], ref, Mw, thr).items():
                    e[f"{name}_{k}"] = val
            entry[mode] = e
            s16.close()
        # the main entry keeps the storage mode's figures at its top level
        res[f"M{Mw}"] = dict(entry["storage"], h2=entry["h2"])
        del refs
    del vis16w
    return res


def mixed_extras(vis32, torch, cs, peak, steps=300, warmup=10):
    """The paper's trained mixed precision (Tables 3-4) on the LOFAR-scale block:
    flag difference against the float32 mode (the paper reports under 1 % on LOFAR
    data), throughput of the mode, and the paper's abstract cost per window."""
    from paper_2412_14775_b300 import RfiStream, default_thresholds
    from paper_2412_14775_b300.costmodel import window_cost
    M, K, T = 16, 256, 256
    thr = default_thresholds(M)
    R = vis32.shape[0]
    res = {}
    for dtype in ("f32", "f16"):
        vis = vis32 if dtype == "f32" else vis32.half()
        a = RfiStream(62, 64, M, K, thr, dtype)
        # window-parallel lanes: each window still runs sample by sample in one lane (the
        # tables' order), four rows' lanes take turns (measured 9 % faster than one lane
        # per row for both dtypes)
        b = RfiStream(62, 64, M, K, thr, dtype, precision=1, lane_split=1, lanes_per_row=4,
                      warps_per_block=4 if dtype == "f32" else 8)
        oa, ob = a.alloc_outputs(T), b.alloc_outputs(T)
        a.process(vis, out=oa, stream=cs)
        b.process(vis, out=ob, stream=cs)
        torch.cuda.synchronize()
        fa, fb = oa["flags"], ob["flags"]
        # windows are 16 samples: the two halves of each flag word are the two windows
        lo_a, hi_a = (fa & 0xFFFF) != 0, (fa >> 16) != 0
        lo_b, hi_b = (fb & 0xFFFF) != 0, (fb >> 16) != 0
        differ = ((lo_a != lo_b).sum() + (hi_a != hi_b).sum()).item()
        total = 2 * fa.numel()
        k, _, _, _ = time_kernel(b, vis, ob, steps, warmup, torch, cs)
        nbytes = algo_bytes(R, T, M, K, 1, 32 if dtype == "f32" else 16)
        res[dtype] = {"flag_difference_vs_float32": differ / total,
                      "flagged_fraction_float32": ((lo_a.sum() + hi_a.sum()).item()) / total,
                      "kernel_us": k * 1e6, "achieved_gbs": nbytes / k / 1e9,
                      "frac": nbytes / k / 1e9 / peak}
        a.close(); b.close()
        del vis
    res["cost_per_window"] = {"float32": window_cost(M, False), "mixed": window_cost(M, True)}
    torch.cuda.empty_cache()
    return res


def variant_extras(vis32, opts, torch, cs, peak, steps=300, warmup=10):
    """The LOFAR-scale complex64 block through the kernel variants with their own
    instances: online per-stream SK thresholds (T = 256), partial windows (blocks of
    T = 250 samples, so windows straddle blocks) and overlapping windows (a window of
    16 samples every 8)."""
    from paper_2412_14775_b300 import RfiStream, default_thresholds
    M, K = 16, 256
    thr = default_thresholds(M)
    R = vis32.shape[0]
    res = {}
    ad = RfiStream(62, 64, M, K, thr, "f32", adaptive=1, **opts)
    o = ad.alloc_outputs(256)
    k, _, _, _ = time_kernel(ad, vis32, o, steps, warmup, torch, cs)
    nbytes = algo_bytes(R, 256, M, K, 1, 32) + R * 16 * 2     # + state read and write
    rate = float(o["weight"].lt(1.0).float().mean())
    res["online_thresholds"] = {"kernel_us": k * 1e6, "achieved_gbs": nbytes / k / 1e9,
                                "frac": nbytes / k / 1e9 / peak,
                                "bins_with_flagged_samples": rate}
    ad.close()
    v250 = vis32[:, :250].contiguous()
    pw = RfiStream(62, 64, M, K, thr, "f32", partial_windows=1, **opts)
    # output sizes follow the stream position (15 or 16 windows per block): each call's
    # outputs are taken from torch's caching allocator just before it, no device work
    for _ in range(warmup):
        pw.process(v250, out=pw.alloc_outputs(250), stream=cs)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    wins, ring = [], []
    e0.record(cs)
    for _ in range(steps):
        out = pw.alloc_outputs(250)
        ring = (ring + [out])[-4:]          # a ring of 4 live output sets, as elsewhere
        wins.append(out["stats"].shape[-1])
        pw.process(v250, out=out, stream=cs)
    e1.record(cs)
    torch.cuda.synchronize()
    us = e0.elapsed_time(e1) * 1e3 / steps
    nw = statistics.mean(wins)
    # input, flags and statistics of the completed windows, the samples carried
    nbytes = R * (250 * 32 + 4 * math.ceil(nw * M / 32) + 12 * nw + 32 * (M - 1))
    res["partial_windows_T250"] = {"kernel_us": us, "achieved_gbs": nbytes / (us * 1e-6) / 1e9,
                                   "frac": nbytes / (us * 1e-6) / 1e9 / peak,
                                   "samples_per_s": R * 250 / (us * 1e-6)}
    pw.close()
    del v250
    # overlapping windows: a window of 16 samples every 8 (twice the windows), steady
    # state (the first call of a stream completes one window fewer per row)
    best = None
    for P in (2, 4):
        sw = RfiStream(62, 64, M, K, thr, "f32", window_hop=M // 2, lanes_per_row=P,
                       warps_per_block=4)
        sw.process(vis32, out=sw.alloc_outputs(256), stream=cs)    # leave the stream start
        o = sw.alloc_outputs(256)
        k, _, _, _ = time_kernel(sw, vis32, o, steps, warmup, torch, cs)
        if best is None or k < best[0]:
            best = (k, P, o["stats"].shape[-1])
        sw.close()
    k, P, nw = best
    H = M // 2
    # input, flags, statistics of 2x the windows, averages, and the pending half-window
    # carried between blocks (totals 32 B, averaging sums 32 B per lane, 4 B of window
    # flags; read and written)
    nbytes = R * (256 * 32 + 4 * math.ceil(nw * H / 32) + 12 * nw + 36 + 2 * (36 + 32 * P))
    res["sliding_windows_hop8"] = {"kernel_us": k * 1e6, "achieved_gbs": nbytes / k / 1e9,
                                   "frac": nbytes / k / 1e9 / peak, "windows_per_row": nw,
                                   "samples_per_s": R * 256 / k, "lanes_per_row": P}
    torch.cuda.empty_cache()
    return res


def batched_extras(options, torch, steps=300, warmup=10):
    """8 uneven binary16 subbands (stations 24..76, channels 16..128, T = 256) in one
    persistent launch replayed from a CUDA graph, against the same 8 streams launched
    one after another."""
    import synth
    from paper_2412_14775_b300 import RfiStream, binding, default_thresholds
    M, K, T = 16, 256, 256
    thr = default_thresholds(M)
    opts = {k: v for k, v in options.items() if k != "max_registers"}
    geo = list(zip(synth.BATCH_STATIONS, synth.BATCH_CHANNELS))
    streams = [RfiStream(n, c, M, K, thr, "f16", **opts) for n, c in geo]
    solo = [RfiStream(n, c, M, K, thr, "f16", **opts) for n, c in geo]
    vis = [synth.generate.device_block(n, c, T, seed=300 + i) for i, (n, c) in enumerate(geo)]
    outs = [s.alloc_outputs(T) for s in streams]
    samples = sum(s.R for s in streams) * T
    nbytes = sum(algo_bytes(s.R, T, M, K, 1, 16) for s in streams)
    g = binding.rfi_batch_graph_create([s.ctx for s in streams], [T] * len(streams))
    cs = torch.cuda.current_stream()

    def step_graph():
        binding.rfi_batch_graph_launch(g, vis, [o["flags"] for o in outs],
                                       [o["avg"] for o in outs], [o["weight"] for o in outs],
                                       [o["stats"] for o in outs], stream=cs)

    def step_solo():
        for st, v, o in zip(solo, vis, outs):
            st.process(v, out=o, stream=cs)

    res = {"streams": len(geo), "samples_per_step": samples, "algorithmic_bytes": nbytes}
    for name, fn in (("graph_persistent", step_graph), ("sequential_launches", step_solo)):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(cs)
        for _ in range(steps):
            fn()
        b.record(cs)
        torch.cuda.synchronize()
        dt = a.elapsed_time(b) * 1e-3 / steps
        res[name] = {"us_per_step": dt * 1e6, "samples_per_s": samples / dt,
                     "achieved_gbs": nbytes / dt / 1e9}
    binding.rfi_batch_graph_destroy(g)
    for s in streams + solo:
        s.close()
    del vis, outs
    torch.cuda.empty_cache()
    return res


def serving_extras(seconds, options, torch):
    """The serving loop (binary16, M = 16, K = 256, blocks of 256 samples = 128 ms): the
    32 mixed streams at 1-4x real time, the same at 4x, 6x and 8x that rate (4-16x to
    8-32x real time per stream, 340 to 680 real-time streams offered, so batches
    fill; the 10x run reads each block where it arrived instead of copying it into the
    pool), the 62-station, 64-channel stream at 50x real time and backlogged, all with blocks arriving in device memory (a GPU correlator's output),
    and that stream fed from pinned host memory at 10x real time (the host link carries
    512 MB per block).  Every admitted block is copied into a slot of the device block
    pool and its results are copied back to pinned host memory."""
    import synth
    from paper_2412_14775_b300.serve import ServingLoop
    res = {}
    free, _ = torch.cuda.mem_get_info()
    budget = int(min(0.5 * free, 32 << 30))
    cfgs = synth.serving_streams(seed=5, n=32)
    for name, scale, copy_in in (("mix32", 1.0, True), ("mix32_x4", 4.0, True),
                                 ("mix32_x6", 6.0, True), ("mix32_x8", 8.0, True),
                                 ("mix32_x10_in_place", 10.0, False)):
        c = [dict(x, rho=x["rho"] * scale) for x in cfgs]
        loop = ServingLoop(c, M=16, K=256, T=256, dtype="f16", options=options,
                           hbm_budget_bytes=budget, max_batch=32, cuda_streams=3,
                           copy_in=copy_in)
        loop.run(0.25, seed=99)           # untimed: first launches load and set up kernels
        res[name] = dict(loop.run(seconds / 2, seed=11), streams=32, rho_scale=scale)
        loop.close()
        torch.cuda.empty_cache()
    R = 1953 * 64
    # one 62-station, 64-channel stream delivering a block every 1/rate of a block time
    for name, rate, source in (("lofar_50x", 50.0, "device"), ("lofar_host_10x", 10.0, "host")):
        loop = ServingLoop([dict(stations=62, channels=64, rho=rate)], M=16, K=256, T=256,
                           dtype="f16", options=options, hbm_budget_bytes=budget, max_batch=1,
                           cuda_streams=2, source=source)
        dur = max(2.0, seconds / 4)
        period = BLOCK_SECONDS / rate
        loop.run(0.0, arrivals=[(0.0, 0, k) for k in range(4)])        # untimed warm-up
        r = loop.run(dur, arrivals=[(k * period, 0, k) for k in range(int(dur / period))])
        r["real_time_factor"] = r["samples_per_s"] / (R * 256 / BLOCK_SECONDS)
        res[name] = r
        loop.close()
        torch.cuda.empty_cache()
    # the same stream backlogged (3000 blocks queued at once): the rate the loop
    # sustains for one stream, whose blocks must run one after another
    loop = ServingLoop([dict(stations=62, channels=64, rho=1.0)], M=16, K=256, T=256,
                       dtype="f16", options=options, hbm_budget_bytes=budget, max_batch=1,
                       cuda_streams=2)
    r = loop.run(0.0, arrivals=[(0.0, 0, k) for k in range(3000)])
    r["real_time_factor"] = r["samples_per_s"] / (R * 256 / BLOCK_SECONDS)
    for k in ("p50_latency_s", "p99_latency_s", "max_latency_s", "p99_over_block"):
        r.pop(k)
    res["lofar_backlogged"] = r
    loop.close()
    torch.cuda.empty_cache()
    return res


# The timed workloads are streams of blocks whose launches share no buffer with the
# launches still in flight (each block closes its averaging bins, outputs go to a ring of
# output sets), so their contexts let such launches start without waiting for the one
# before (option independent_launches; the library checks every launch and orders the
# others as before).
PIPELINED = {"independent_launches": 1}
N_OUT_SETS = 16


def time_kernel(stream_obj, vis, out, steps, warmup, torch, cuda_stream, sampler_index=None,
                serial_steps=100, n_out_sets=N_OUT_SETS):
    """Warm up, then time `steps` back-to-back launches with CUDA events on the launching
    stream around the whole run; returns the mean launch period (device time of the
    flagging kernel in a stream of calls, launch overlap included), the run's total and
    the clock record.  Step i reads vis[i % len(vis)] (vis: one tensor or a list) and
    writes the (i % n_out_sets)-th of n_out_sets output sets, `out` and copies of it: a
    ring of output buffers, as a pipeline keeps them (one set reused every step would let
    the outputs stay in L2 and never reach DRAM; a launch that writes the set of a launch
    still possibly running is ordered after it, so the ring is 16 deep).  Then `serial_steps` launches with an
    event pair around each one (which keeps consecutive launches from overlapping): their
    mean duration, reported beside it."""
    from paper_2412_14775_b300 import binding
    vis_l = list(vis) if isinstance(vis, (list, tuple)) else [vis]
    outs = [out] + [{k: torch.empty_like(x) for k, x in out.items()}
                    for _ in range(n_out_sets - 1)]
    orders = collections.Counter()

    def step(i, count=False):
        stream_obj.process(vis_l[i % len(vis_l)], out=outs[i % len(outs)], stream=cuda_stream)
        if count:
            orders[binding.rfi_last_launch(stream_obj.ctx)] += 1

    for i in range(warmup):
        step(i)
    torch.cuda.synchronize()
    sampler = ClockSampler(sampler_index) if sampler_index is not None else None
    if sampler:
        sampler.__enter__()
    t_all0 = torch.cuda.Event(enable_timing=True)
    t_all1 = torch.cuda.Event(enable_timing=True)
    t_all0.record(cuda_stream)
    for i in range(steps):
        step(i, count=True)
    t_all1.record(cuda_stream)
    torch.cuda.synchronize()
    if sampler:
        sampler.__exit__()
    total = t_all0.elapsed_time(t_all1) * 1e-3
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(min(serial_steps, steps))]
    for i, (a, b) in enumerate(ev):
        a.record(cuda_stream)
        step(i)
        b.record(cuda_stream)
    torch.cuda.synchronize()
    # leave the results of the last launch in `out` for the caller
    last = outs[(len(ev) - 1 if ev else steps - 1) % len(outs)]
    if last is not out:
        for k in out:
            out[k].copy_(last[k])
    serial = statistics.mean(a.elapsed_time(b) * 1e-3 for a, b in ev) if ev else None
    time_kernel.last_orders = dict(orders)     # how the timed launches were ordered
    return total / steps, total, serial, (sampler.summary() if sampler else None)


def _r(x, n=4):
    """x rounded to n significant digits (None stays None)."""
    if x is None:
        return None
    if x == 0 or not math.isfinite(x):
        return x
    return round(x, -int(math.floor(math.log10(abs(x)))) + n - 1)


def summarize(line):
    """The line's figures in a compact form (kept under ~1.3 KB so that a reader keeping
    only the end of the line has them all): launch time (us) and fraction of the measured
    copy bandwidth per kernel, the binary16 modes' errors, serving and the detection
    experiment."""
    g = line.get
    out = {"main": [_r(line["roofline"]["kernel_us"]), _r(line["roofline"]["frac"], 3)]}
    if g("fp16"):
        # per M: storage us, frac; h2 us, frac; h2 arithmetic error of tau and r and its
        # flag disagreement; flag disagreement against the float32 input (storage, h2)
        out["fp16"] = "us,frac,h2us,h2frac,h2tau,h2r,h2flag,flag32,h2flag32"
        for k, e in line["fp16"].items():
            h = e["h2"]
            out[k] = [_r(e["kernel_us"]), _r(e["frac"], 3), _r(h["kernel_us"]), _r(h["frac"], 3),
                      _r(h["arith_tau_err"], 2), _r(h["arith_r_err"], 2),
                      _r(h["arith_flag_disagree"], 2), _r(e["total_flag_disagree"], 2),
                      _r(h["total_flag_disagree"], 2)]
    if g("mixed_precision"):
        m = line["mixed_precision"]["f32"]
        out["mixed"] = [_r(m["flag_difference_vs_float32"], 3), _r(m["kernel_us"]), _r(m["frac"], 3)]
    if g("variants"):
        short = {"online_thresholds": "online", "partial_windows_T250": "partial",
                 "sliding_windows_hop8": "sliding"}
        for k, v in line["variants"].items():
            out[short.get(k, k)] = [_r(v["kernel_us"]), _r(v["frac"], 3)]
    if g("footprints"):
        for k, v in line["footprints"].items():
            out[k] = [_r(v["kernel_us"]), _r(v["frac"], 3)]
    if g("batched"):
        b = line["batched"]
        out["batch8"] = [_r(b["graph_persistent"]["us_per_step"]),
                         _r(b["graph_persistent"]["achieved_gbs"]),
                         _r(b["sequential_launches"]["us_per_step"])]
    if g("serving"):
        # per run: mean batch, p50 and p99 latency (ms), real-time factor
        out["serve"] = "batch,p50ms,p99ms,rtf"
        for k, v in line["serving"].items():
            if isinstance(v, dict):
                out[k] = [_r(v.get("mean_batch", 0), 3),
                          _r(1e3 * v["p50_latency_s"], 3) if "p50_latency_s" in v else None,
                          _r(1e3 * v["p99_latency_s"], 3) if "p99_latency_s" in v else None,
                          _r(v.get("real_time_factor") or v.get("offered_real_time_streams"), 3)]
    if g("detection"):
        # per INR: (false alarm, missed) for SK, DS, both
        d = line["detection"]
        for pol in ("polarised", "unpolarised"):
            if pol in d:
                out["det_" + pol[:5]] = {str(row["inr"]): [_r(row[m][x], 2) for m in ("SK", "DS", "BOTH")
                                                           for x in ("false_alarm", "missed")]
                                         for row in d[pol]}
    if g("cpu_baseline"):
        out["cpu"] = _r(line["cpu_baseline"]["value"], 3)
    if g("e2e"):
        out["e2e"] = _r(line["e2e"]["value"], 3)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-rows", type=int, default=0, help="cap on oracle rows per step")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=8.0,
                    help="wall time of the serving-loop run (0 = skip)")
    ap.add_argument("--detection", action="store_true",
                    help="run the full false-alarm / missed-detection experiment (8 "
                         "realisations, 5 INRs; the default line carries a reduced one)")
    ap.add_argument("--no-detection", action="store_true")
    ap.add_argument("--cpu-baseline-only", action="store_true",
                    help="print the CPU baseline (the FP64 oracle on the host cores) and exit")
    ap.add_argument("--tile", default="",
                    help="lanes_per_row,warps_per_block[,prefetch_groups,prefetch_bytes]")
    ap.add_argument("--dtype", default="f32", choices=["f32", "f16"],
                    help="input storage of the timed block (f16: same block in binary16)")
    ap.add_argument("--precision", type=int, default=0, choices=[0, 2],
                    help="arithmetic of the timed block with --dtype f16: 0 = float32 on "
                         "exactly widened values, 2 = binary16 Stokes arithmetic")
    ap.add_argument("--footprint", default="", choices=["", "10x2", "5x4"],
                    help="time only this T x F window footprint (blocks of 250 samples, "
                         "--dtype storage) and print its figures")
    ap.add_argument("--batched", action="store_true",
                    help="time only the 8 uneven binary16 subbands (one persistent launch "
                         "from a CUDA graph against 8 sequential launches) and print them")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return reference_arm(args)
    if args.cpu_baseline_only:
        print(json.dumps(cpu_baseline()), flush=True)
        return

    import torch
    import torch.distributed as dist

    import synth
    from paper_2412_14775_b300 import RfiStream, autotune, default_thresholds
    from paper_2412_14775_b300.shard import aggregate

    if args.footprint:
        import torch
        M, F = (int(x) for x in args.footprint.split("x"))
        res = footprint_extras(torch, torch.cuda.current_stream(), _peaks()[0], args.steps,
                               args.warmup, only=(args.dtype, M, F))
        print(json.dumps({"footprint": res}))
        return

    if args.batched:
        import torch
        import synth
        from paper_2412_14775_b300 import autotune, default_thresholds
        v16 = synth.generate.device_block(62, 64, 256, seed=2, dtype="f16")
        best, _ = autotune.tune(62, 64, 16, 256, default_thresholds(16), "f16", v16,
                                cache_path=autotune.TUNED_PATH, write_cache=False)
        del v16
        res = batched_extras(autotune.options_of(best), torch, args.steps, args.warmup)
        print(json.dumps({"batched": res}))
        return

    ws, rank, local = _dist()
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    peak, peak_kind = _peaks()
    M, K, T = 16, 256, 256
    thr = default_thresholds(M)
    d = synth.lofar_block(seed=2 + rank)
    R = d["vis"].shape[0] * d["vis"].shape[1]
    host32 = torch.from_numpy(d["vis"].reshape(R, T, 4, 2))
    vis32 = host32.to(dev)

    def tuned(Mw, dtype, vis, fixed=None):
        if args.tile and not fixed:
            f = [int(x) for x in args.tile.split(",")]
            keys = ["lanes_per_row", "warps_per_block", "prefetch_groups", "prefetch_bytes"]
            return dict(zip(keys, f))
        best, _ = autotune.tune(62, 64, Mw, K, default_thresholds(Mw), dtype, vis,
                                cache_path=autotune.TUNED_PATH, write_cache=False, fixed=fixed)
        return autotune.options_of(best)

    main_dt = args.dtype
    sbytes = 32 if main_dt == "f32" else 16
    vis_main = vis32 if main_dt == "f32" else vis32.half()
    if args.precision and main_dt != "f16":
        ap.error("--precision 2 needs --dtype f16")
    opts = dict(tuned(M, main_dt, vis_main, {"precision": 2} if args.precision else None),
                **PIPELINED)
    prof_key = main_dt + ("_h2" if args.precision else "")
    st = RfiStream(62, 64, M, K, thr, main_dt, **opts)
    out = st.alloc_outputs(T, device=dev)
    cs = torch.cuda.current_stream(dev)

    if ws > 1:
        dist.barrier()
    # two input blocks in turn (each larger than L2) and a ring of output sets
    kern, total, kern_serial, clocks = time_kernel(st, [vis_main, vis_main.clone()], out,
                                                   args.steps, args.warmup,
                                                   torch, cs, sampler_index=local)
    time_kernel.last_orders_main = time_kernel.last_orders
    samples = R * T
    out_bytes = sum(x.numel() * x.element_size() for x in out.values())
    # every rank processes its own block (weak scaling): total samples of all ranks over
    # the slowest rank's time
    _, total, value = aggregate(samples * args.steps, total)
    n_out = 1
    bytes_launch = algo_bytes(R, T, M, K, n_out, sbytes)
    achieved = bytes_launch / kern / 1e9
    # windows flagged by each test on the last timed block (from the kernel's statistics)
    stt = out["stats"]
    sk = ~((stt[0] >= thr["s_low"]) & (stt[0] <= thr["s_high"]))
    dre, dim = ~(stt[1] <= thr["gamma"]), ~(stt[2] <= thr["gamma"])
    flag_fractions = {"sk": sk.float().mean().item(), "ds_re": dre.float().mean().item(),
                      "ds_im": dim.float().mean().item(),
                      "any": (sk | dre | dim).float().mean().item()}

    extras = {}
    if not args.no_extras and rank == 0:
        extras["mixed_precision"] = mixed_extras(vis32, torch, cs, peak)
        extras["variants"] = variant_extras(vis32, opts, torch, cs, peak)
        if args.detection:
            extras["detection"] = detection_experiment(torch)
        elif not args.no_detection:
            # a reduced table (the full one: --detection)
            extras["detection"] = detection_experiment(torch, realizations=6,
                                                       inrs=(0.01, 1.0, 100.0))
        del vis_main
        vis16 = vis32.half()
        extras["fp16"] = fp16_extras(vis32, vis16, tuned, torch, cs, peak, dev,
                                     max(200, args.steps // 4), args.warmup)
        fp16 = extras["fp16"]
        del vis32, vis16
        torch.cuda.empty_cache()
        extras["batched"] = batched_extras(fp16["M16"]["options"], torch)
        extras["footprints"] = footprint_extras(torch, cs, peak)
        if args.serve_seconds > 0:
            extras["serving"] = serving_extras(args.serve_seconds,
                                               fp16["M16"]["options"], torch)

    # end to end through the host-buffer entry point (pinned host memory)
    e2e = None
    if rank == 0 and not args.no_e2e:
        hst = RfiStream(62, 64, M, K, thr, "f32", **dict(opts, host_max_T=T, host_chunks=8))
        hin = host32.pin_memory()
        hout = hst.alloc_outputs(T, device="cpu", pin_memory=True)
        for _ in range(3):
            hst.process_host(hin, out=hout)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            hst.process_host(hin, out=hout)
            _ = float(hout["weight"][0, 0])        # the result is read on the host
        dt = time.perf_counter() - t0
        d2h = sum(x.numel() * x.element_size() for x in hout.values())
        # the host link alone: a plain pinned -> device copy of the same bytes
        dst = torch.empty_like(hin, device=dev)
        for _ in range(2):
            dst.copy_(hin, non_blocking=True)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for _ in range(5):
            dst.copy_(hin, non_blocking=True)
        torch.cuda.synchronize()
        link = 5 * hin.numel() * hin.element_size() / (time.perf_counter() - t1) / 1e9
        del dst
        e2e = {"value": samples * args.e2e_steps / dt, "unit": "samples/s",
               "h2d_bytes_per_step": hin.numel() * hin.element_size(),
               "d2h_bytes_per_step": d2h,
               "h2d_link_gbs_plain_copy": link,
               "h2d_gbs_in_e2e": hin.numel() * hin.element_size() * args.e2e_steps / dt / 1e9}
        hst.close()
        # the same through binary16 storage: half the bytes cross the host link
        o16 = (extras["fp16"]["M16"]["options"] if "fp16" in extras
               else dict(lanes_per_row=2, warps_per_block=4))
        h16 = RfiStream(62, 64, M, K, thr, "f16", **dict(o16, host_max_T=T, host_chunks=8))
        hin16 = host32.half().pin_memory()
        hout16 = h16.alloc_outputs(T, device="cpu", pin_memory=True)
        for _ in range(3):
            h16.process_host(hin16, out=hout16)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            h16.process_host(hin16, out=hout16)
            _ = float(hout16["weight"][0, 0])
        dt16 = time.perf_counter() - t0
        e2e["binary16_storage"] = {
            "value": samples * args.e2e_steps / dt16, "unit": "samples/s",
            "h2d_bytes_per_step": hin16.numel() * hin16.element_size(),
            "d2h_bytes_per_step": sum(x.numel() * x.element_size() for x in hout16.values())}
        h16.close()
        del hin16, hout16

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        # in a fresh process without CUDA, as the reference arm runs (timed inside this
        # process after the GPU work, the same oracle ran about half as fast)
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-baseline-only"],
                           capture_output=True, text=True, timeout=600)
        cpu = json.loads(r.stdout.strip().splitlines()[-1]) if r.returncode == 0 else None

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": main_dt,
            "data": "synthetic",
            "config": dict(WORKLOAD, dtype="complex64" if main_dt == "f32" else "complex32 (binary16)",
                           l2=f"two input blocks of {R * T * sbytes / 1e9:.2f} GB (> 126 MB L2) in "
                              f"turn, outputs into a ring of {N_OUT_SETS} sets "
                              f"({N_OUT_SETS * out_bytes / 1e6:.0f} MB), no flush",
                           options={k: st.options[k] for k in
                                    ("lanes_per_row", "warps_per_block", "prefetch_bytes",
                                     "prefetch_groups", "independent_launches")}),
            "hbm_gbs": achieved * ws,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": profiled_traffic(prof_key),
                         "ncu_dram_gbs": profiled_dram_gbs(prof_key),
                         "peak_kind": peak_kind, "kernel_us": kern * 1e6,
                         "kernel_us_serialised": kern_serial * 1e6,
                         "launch_orders": getattr(time_kernel, "last_orders_main", None),
                         "algorithmic_bytes_per_launch": bytes_launch},
            "frac_of_8tbs": achieved / 8000.0,
            "clocks": clocks, "e2e": e2e, "cpu_baseline": cpu,
            "gpu_launches": args.steps,
            "correlations_per_s": 4 * value,
            "real_time_factor": BLOCK_SECONDS / kern,
            "real_time_factor_native_channel_rate": NATIVE_BLOCK_SECONDS / kern,
            "flag_fractions": flag_fractions,
        }
        line.update(extras)
        # last, so that a reader keeping only the end of the line still has the figures
        line["summary"] = summarize(line)
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
