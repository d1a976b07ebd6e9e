"""Seeded synthetic correlator blocks with a ground-truth interference mask.

This module only draws inputs; it contains none of the flagging method's arithmetic.
Both the CUDA path (via the tests and the bench) and the FP64 oracle receive the
arrays it returns.

Layout of every block: float32 (or float16) array [B, C, T, 4, 2]
  B = N(N+1)/2 baselines including autocorrelations, ordered (p, q) with p <= q,
  C channels, T time samples, 4 correlations xx, xy, yx, yy, and (re, im).

Noise model: circular complex Gaussian with E|z|^2 = 1 (re and im each of variance
1/2), independent per correlation; optionally scaled per (baseline (p, q),
correlation (a, b)) by station gains g[p, a] * g[q, b] with g ~ U[0.8, 1.2].

Interference model: bursts of a fully polarised signal c * A * e e^H with a random
phase c, Jones vector e = (cos t, sin t e^{j f}), t ~ U[0, pi), f = 0 (linear) or
f ~ U[0, 2 pi) (elliptical) with probability 1/2 each, and the amplitude A chosen so
that the mean over the four correlations of |A e_a e_b^*|^2 equals the
interference-to-noise ratio times E|noise|^2 = 1, i.e. A = 2 sqrt(INR).
Burst lengths are uniform on {2, ..., 20}; bursts are placed at uniform starts
until the requested fraction of samples is covered.
"""
import math
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_CHUNK_ROWS = 4096          # rows (baseline x channel) per independent noise stream


def n_baselines(stations: int) -> int:
    """N(N+1)/2 baselines including autocorrelations."""
    return stations * (stations + 1) // 2


def baseline_pairs(stations: int):
    """Station pairs (p, q), p <= q, in row-major order (0,0), (0,1), ..., (N-1,N-1)."""
    p, q = np.triu_indices(stations)
    return p.astype(np.int64), q.astype(np.int64)


def _noise(seed: int, rows: int, T: int, threads: int = 8) -> np.ndarray:
    """[rows, T, 4, 2] float32 circular Gaussian, E|z|^2 = 1, reproducible for any
    thread count (each fixed chunk of rows has its own child seed)."""
    out = np.empty((rows, T, 4, 2), np.float32)
    nchunks = (rows + _CHUNK_ROWS - 1) // _CHUNK_ROWS
    seeds = np.random.SeedSequence([seed, rows, T]).spawn(max(nchunks, 1))
    scale = np.float32(math.sqrt(0.5))

    def fill(i):
        a, b = i * _CHUNK_ROWS, min(rows, (i + 1) * _CHUNK_ROWS)
        rng = np.random.default_rng(seeds[i])
        view = out[a:b].reshape(-1)
        rng.standard_normal(out=view, dtype=np.float32)
        view *= scale

    if nchunks <= 1:
        for i in range(nchunks):
            fill(i)
    else:
        with ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(fill, range(nchunks)))
    return out


def _jones(rng):
    t = rng.uniform(0.0, math.pi)
    f = 0.0 if rng.uniform() < 0.5 else rng.uniform(0.0, 2 * math.pi)
    return np.array([math.cos(t), math.sin(t) * complex(math.cos(f), math.sin(f))])


def _coherency(e):
    """e e^H flattened in correlation order xx, xy, yx, yy."""
    return np.array([e[0] * np.conj(e[0]), e[0] * np.conj(e[1]),
                     e[1] * np.conj(e[0]), e[1] * np.conj(e[1])])


def _bursts(rng, T: int, duty: float):
    """Bursts (start, stop) with lengths U{2..20} until >= duty * T samples are covered."""
    covered = np.zeros(T, bool)
    out = []
    target = duty * T
    while covered.sum() < target:
        length = int(rng.integers(2, 21))
        t0 = int(rng.integers(0, T))
        t1 = min(T, t0 + length)
        covered[t0:t1] = True
        out.append((t0, t1))
    return out


def _add(vis, b, c, t0, t1, val):
    """vis[b, c, t0:t1, :] += val (complex [..., 4]) on the float layout."""
    seg = vis[b, c, t0:t1]
    seg[..., 0] += val.real.astype(np.float32)
    seg[..., 1] += val.imag.astype(np.float32)


def tiny_block(seed: int = 1, stations: int = 6, channels: int = 16, T: int = 1024,
               duty: float = 0.05, inr_db: float = 10.0):
    """Tiny FP32 reference block: sigma = 1 noise plus 5%-duty polarised bursts per
    (baseline, channel) at INR 10 dB."""
    B = n_baselines(stations)
    vis = _noise(seed, B * channels, T).reshape(B, channels, T, 4, 2)
    truth = np.zeros((B, channels, T), bool)
    rng = np.random.default_rng([seed, 7])
    A = 2.0 * math.sqrt(10 ** (inr_db / 10))
    for b in range(B):
        for c in range(channels):
            for t0, t1 in _bursts(rng, T, duty):
                ph = rng.uniform(0, 2 * math.pi)
                val = A * complex(math.cos(ph), math.sin(ph)) * _coherency(_jones(rng))
                _add(vis, b, c, t0, t1, np.broadcast_to(val, (t1 - t0, 4)))
                truth[b, c, t0:t1] = True
    return dict(vis=vis, truth=truth, stations=stations, channels=channels, T=T)


def lofar_block(seed: int = 2, stations: int = 62, channels: int = 64, T: int = 256,
                rfi_channel_frac: float = 0.10, inr_db=(-5.0, 15.0), duty=(0.01, 0.10),
                dtype=np.float32):
    """LOFAR-scale block: noise with per-station gain spread U[0.8, 1.2] plus
    intermittent polarised interference on 10% of the channels, INR U[-5, 15] dB per
    burst, duty cycle U[1%, 10%] per interfered channel.  The (channel, time) footprint
    is shared by all baselines, each baseline with its own random phase."""
    B = n_baselines(stations)
    vis = _noise(seed, B * channels, T).reshape(B, channels, T, 4, 2)
    rng = np.random.default_rng([seed, 11])
    g = rng.uniform(0.8, 1.2, size=(stations, 2)).astype(np.float32)
    p, q = baseline_pairs(stations)
    # correlation (a, b) of baseline (p, q) scales by g[p, a] * g[q, b]
    ab = [(0, 0), (0, 1), (1, 0), (1, 1)]
    gain = np.stack([g[p, a] * g[q, b] for a, b in ab], axis=-1)      # [B, 4]
    vis *= gain[:, None, None, :, None]
    truth = np.zeros((B, channels, T), bool)
    n_rfi = max(1, int(round(rfi_channel_frac * channels)))
    rfi_ch = rng.choice(channels, size=n_rfi, replace=False)
    for c in rfi_ch:
        dc = rng.uniform(*duty)
        for t0, t1 in _bursts(rng, T, dc):
            inr = 10 ** (rng.uniform(*inr_db) / 10)
            A = 2.0 * math.sqrt(inr)
            coh = A * _coherency(_jones(rng))                          # [4]
            ph = rng.uniform(0, 2 * math.pi, size=B)
            val = (np.cos(ph) + 1j * np.sin(ph))[:, None] * coh[None, :]   # [B, 4]
            seg = vis[:, c, t0:t1]                                     # [B, L, 4, 2]
            seg[..., 0] += val.real[:, None, :].astype(np.float32)
            seg[..., 1] += val.imag[:, None, :].astype(np.float32)
            truth[:, c, t0:t1] = True
    if dtype == np.float16:
        vis = vis.astype(np.float16)
    return dict(vis=vis, truth=truth, stations=stations, channels=channels, T=T)


# Geometry of the batched uneven-stream workload: 8 subbands.
BATCH_STATIONS = (24, 38, 48, 62, 76, 24, 48, 62)
BATCH_CHANNELS = (16, 32, 64, 128, 64, 32, 16, 64)


def serving_streams(seed: int = 5, n: int = 32):
    """Geometry and arrival rate of the serving-loop streams: stations U{24..76},
    channels in {16, 32, 64, 128}, rate factor rho ~ U[1, 4] (blocks per block time)."""
    rng = np.random.default_rng([seed, 13])
    st = rng.integers(24, 77, size=n)
    ch = rng.choice([16, 32, 64, 128], size=n)
    rho = rng.uniform(1.0, 4.0, size=n)
    return [dict(stations=int(a), channels=int(b), rho=float(r)) for a, b, r in zip(st, ch, rho)]


def device_block(stations: int, channels: int, T: int, seed: int, device="cuda",
                 dtype="f16", rfi_channel_frac: float = 0.10, inr_db=(-5.0, 15.0),
                 duty=(0.01, 0.10)):
    """A block with the LOFAR-scale noise and interference model drawn on the GPU by
    torch's generator (for the serving workload, whose many streams would take minutes
    to draw on the host).  Returns a tensor [B*C, T, 4, 2] of float16 or float32.
    Not bit-identical to lofar_block for the same seed (different generator)."""
    import torch
    B = n_baselines(stations)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    vis = torch.randn((B, channels, T, 4, 2), generator=g, device=device,
                      dtype=torch.float32) * math.sqrt(0.5)
    rng = np.random.default_rng([seed, 17])
    gains = rng.uniform(0.8, 1.2, size=(stations, 2)).astype(np.float32)
    p, q = baseline_pairs(stations)
    ab = [(0, 0), (0, 1), (1, 0), (1, 1)]
    gain = np.stack([gains[p, a] * gains[q, b] for a, b in ab], axis=-1)
    vis *= torch.from_numpy(gain).to(device)[:, None, None, :, None]
    n_rfi = max(1, int(round(rfi_channel_frac * channels)))
    for c in rng.choice(channels, size=n_rfi, replace=False):
        for t0, t1 in _bursts(rng, T, rng.uniform(*duty)):
            A = 2.0 * math.sqrt(10 ** (rng.uniform(*inr_db) / 10))
            coh = A * _coherency(_jones(rng))
            ph = rng.uniform(0, 2 * math.pi, size=B)
            val = (np.cos(ph) + 1j * np.sin(ph))[:, None] * coh[None, :]
            v = torch.from_numpy(np.stack([val.real, val.imag], -1).astype(np.float32)).to(device)
            vis[:, int(c), t0:t1] += v[:, None]
    vis = vis.reshape(B * channels, T, 4, 2)
    return vis.half() if dtype == "f16" else vis
