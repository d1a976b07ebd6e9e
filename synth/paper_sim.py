"""Simulated data in the manner of the paper's Section 4.2 (input generator only).

One baseline, a time x frequency block (the paper uses 2000 x 512, about 1 s x
200 kHz), laid out as rows = channels, columns = time, 4 correlations each:

* receiver noise: the conjugate product of two stations' dual-polarisation complex
  Gaussian voltages, scaled by 100 U(0, 1) (one factor per block), plus sky noise
  (complex circular Gaussian correlations);
* 200 unpolarised point sources: baseline coordinates u, v, w ~ 300 N(0, 1) (metres),
  directions l, m ~ U(-0.5, 0.5), n = sqrt(1 - l^2 - m^2), flux ~ U(1, 10) Jy, coherence
  flux * exp(j 2 pi f (u l + v m + w (n - 1)) / c) at channel frequencies spread over
  120-120.2 MHz, constant in time, on xx and yy;
* interference: broadband footprints (uniformly placed time x frequency rectangles,
  constant amplitude) and narrowband / narrow-duration ones (a single channel carrying
  a complex exponential over a time span, or a single time over a frequency span), each
  with a 2 x 2 polarisation matrix J / ||J|| from complex Gaussian entries whose degree
  of polarisation is at most 0.9 (or exactly unpolarised: J = identity);
* the interference is scaled so that its total power over the block divided by the
  total power of the sky signal (noise plus sources) equals the requested INR.

Returns float32 visibilities [channels, T, 4, 2], the boolean truth mask [channels, T]
and the drawn parameters (receiver-noise scale, baseline u, v, w, source positions and
fluxes, the per-channel source coherence, every interferer's footprint and J, the
interference scale).
"""
import math

import numpy as np

C_LIGHT = 299792458.0


def _cgauss(rng, shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2)


def _degree_of_polarisation(J):
    xx, xy, yx, yy = J[0, 0], J[0, 1], J[1, 0], J[1, 1]
    I, Q, U, V = xx + yy, xx - yy, xy + yx, 1j * (xy - yx)
    return math.sqrt(abs(Q) ** 2 + abs(U) ** 2 + abs(V) ** 2) / max(abs(I), 1e-30)


def _polarisation(rng, polarised):
    if not polarised:
        return np.eye(2, dtype=np.complex128) / math.sqrt(2)
    while True:
        J = _cgauss(rng, (2, 2))
        if _degree_of_polarisation(J) <= 0.9:
            return J / np.linalg.norm(J)


def simulate_block(seed, T=2000, C=512, inr=100.0, polarised=True, n_broadband=5,
                   n_narrow=2, n_sources=200, f0=120e6, f1=120.2e6):
    rng = np.random.default_rng([seed, 2412])
    # receiver noise: x_p x_q^H per sample, two polarisations per station
    xp = _cgauss(rng, (C, T, 2))
    xq = _cgauss(rng, (C, T, 2))
    recv = xp[..., :, None] * np.conj(xq[..., None, :])          # [C, T, 2, 2]
    recv_scale = 100.0 * rng.uniform()
    sky = recv * recv_scale + _cgauss(rng, (C, T, 2, 2))
    # point sources (unpolarised, constant in time)
    u, v, w = 300.0 * rng.standard_normal(3)
    l = rng.uniform(-0.5, 0.5, n_sources)
    m = rng.uniform(-0.5, 0.5, n_sources)
    n = np.sqrt(1.0 - l * l - m * m)
    flux = rng.uniform(1.0, 10.0, n_sources)
    freqs = np.linspace(f0, f1, C)
    phase = 2 * np.pi * freqs[:, None] * (u * l + v * m + w * (n - 1.0))[None, :] / C_LIGHT
    coh = (flux[None, :] * np.exp(1j * phase)).sum(axis=1)          # [C]
    sky[..., 0, 0] += coh[:, None]
    sky[..., 1, 1] += coh[:, None]
    # interference
    rfi = np.zeros_like(sky)
    truth = np.zeros((C, T), bool)
    emitters = []          # (kind, channel span, time span, J) of every interferer
    for _ in range(n_broadband):
        t0 = int(rng.integers(0, T)); t1 = min(T, t0 + int(rng.integers(2, max(3, T // 20))))
        c0 = int(rng.integers(0, C)); c1 = min(C, c0 + int(rng.integers(1, max(2, C // 8))))
        J = _polarisation(rng, polarised)
        rfi[c0:c1, t0:t1] += J
        truth[c0:c1, t0:t1] = True
        emitters.append(("broadband", (c0, c1), (t0, t1), J))
    for k in range(n_narrow):
        J = _polarisation(rng, polarised)
        if k % 2 == 0:     # narrowband: one channel, a complex exponential over a time span
            c = int(rng.integers(0, C))
            t0 = int(rng.integers(0, T)); t1 = min(T, t0 + int(rng.integers(T // 10, T // 2)))
            period = max(2.0, 120.0 * rng.uniform())
            tt = np.arange(t0, t1)
            rfi[c, t0:t1] += np.exp(2j * np.pi * tt / period)[:, None, None] * J
            truth[c, t0:t1] = True
            emitters.append(("narrowband", (c, c + 1), (t0, t1), J))
        else:              # narrow duration: one time, a complex exponential over channels
            t = int(rng.integers(0, T))
            c0 = int(rng.integers(0, C)); c1 = min(C, c0 + int(rng.integers(C // 10, C // 2)))
            period = max(2.0, 1024.0 * rng.uniform())
            cc = np.arange(c0, c1)
            rfi[c0:c1, t] += np.exp(2j * np.pi * cc / period)[:, None, None] * J
            truth[c0:c1, t] = True
            emitters.append(("narrow_duration", (c0, c1), (t, t + 1), J))
    p_rfi = float(np.sum(np.abs(rfi) ** 2))
    p_sky = float(np.sum(np.abs(sky) ** 2))
    if p_rfi > 0:
        rfi *= math.sqrt(inr * p_sky / p_rfi)
    vis = (sky + rfi).reshape(C, T, 4)
    out = np.empty((C, T, 4, 2), np.float32)
    out[..., 0] = vis.real
    out[..., 1] = vis.imag
    return dict(vis=out, truth=truth, inr=inr, rfi_power=float(np.sum(np.abs(rfi) ** 2)),
                sky_power=p_sky, recv_scale=recv_scale, uvw=(u, v, w), l=l, m=m, flux=flux,
                freqs=freqs, source_coherence=coh, emitters=emitters,
                rfi_scale=math.sqrt(inr * p_sky / p_rfi) if p_rfi > 0 else 0.0)
