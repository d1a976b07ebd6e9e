"""The simulator of the paper's detection experiment (synth/paper_sim.py) against the
recipe of Section 4.2, checked on the generated blocks:

  * receiver noise: conjugate product of two unit complex Gaussian voltages, one scale
    factor 100 U(0, 1) per block, plus unit sky noise: mean power per correlation
    scale^2 + 1, the same over the block;
  * 200 point sources, l, m ~ U(-0.5, 0.5), flux U(1, 10) Jy, coherence constant in
    time on xx and yy only (unpolarised), |coherence| <= total flux;
  * interference polarisation J / ||J|| (unit Frobenius norm) at most 90 % polarised,
    or exactly unpolarised, visible as such in the block;
  * footprints as the recipe draws them (broadband rectangles, one-channel narrowband,
    one-sample narrow-duration) and the truth mask their union;
  * INR = total interference power / total sky power, on the block itself.
"""
import math

import numpy as np
import pytest

from synth import paper_sim

T, C = 400, 128          # smaller than the paper's 2000 x 512, same recipe


def _cplx(vis):
    return vis[..., 0].astype(np.float64) + 1j * vis[..., 1].astype(np.float64)


def _dop(J):
    xx, xy, yx, yy = J[0, 0], J[0, 1], J[1, 0], J[1, 1]
    I, Q, U, V = xx + yy, xx - yy, xy + yx, 1j * (xy - yx)
    return math.sqrt(abs(Q) ** 2 + abs(U) ** 2 + abs(V) ** 2) / abs(I)


@pytest.mark.parametrize("inr", [0.01, 1.0, 100.0])
def test_inr_is_total_rfi_power_over_total_sky_power(inr):
    d = paper_sim.simulate_block(3, T=T, C=C, inr=inr)
    sky = paper_sim.simulate_block(3, T=T, C=C, inr=0.0)      # same draws, no interference
    rfi = _cplx(d["vis"]) - _cplx(sky["vis"])
    ratio = np.sum(np.abs(rfi) ** 2) / np.sum(np.abs(_cplx(sky["vis"])) ** 2)
    assert abs(ratio - inr) <= 1e-4 * inr + 1e-9, ratio
    assert abs(d["rfi_power"] / d["sky_power"] - inr) <= 1e-12 * inr
    # interference only where the truth mask says
    assert np.all(np.abs(rfi[~d["truth"]]) < 1e-3 * np.abs(_cplx(sky["vis"])).max())


def test_receiver_noise_scale_and_stationarity():
    for seed in (1, 2, 5):
        d = paper_sim.simulate_block(seed, T=T, C=C, inr=0.0, n_sources=0)
        s = d["recv_scale"]
        assert 0.0 <= s < 100.0
        p = np.abs(_cplx(d["vis"])) ** 2                # [C, T, 4]
        want = s * s + 1.0                               # E|x_p x_q*|^2 = 1, sky noise 1
        assert abs(p.mean() / want - 1) < 0.02, (seed, p.mean(), want)
        a, b = p[:, :T // 2].mean(), p[:, T // 2:].mean()
        assert abs(a / b - 1) < 0.03
    # the factor is drawn per block: different blocks, different scales
    scales = [paper_sim.simulate_block(k, T=8, C=8, inr=0.0)["recv_scale"] for k in range(40)]
    assert 0 < min(scales) < 25 and max(scales) > 75


def test_point_sources():
    d = paper_sim.simulate_block(7, T=T, C=C, inr=0.0)
    assert d["l"].size == d["m"].size == d["flux"].size == 200
    assert np.all(np.abs(d["l"]) < 0.5) and np.all(np.abs(d["m"]) < 0.5)
    assert np.all((d["flux"] >= 1.0) & (d["flux"] <= 10.0))
    assert np.all((d["freqs"] >= 120e6) & (d["freqs"] <= 120.2e6)) and d["freqs"].size == C
    no_src = paper_sim.simulate_block(7, T=T, C=C, inr=0.0, n_sources=0)
    src = _cplx(d["vis"]) - _cplx(no_src["vis"])           # [C, T, 4]
    tol = 1e-5 * (np.abs(_cplx(d["vis"])).max() + 1)
    coh = d["source_coherence"]
    for k in (0, 3):                                         # xx and yy carry it
        assert np.all(np.abs(src[..., k] - coh[:, None]) <= tol)
    for k in (1, 2):                                         # unpolarised: no xy, yx
        assert np.all(np.abs(src[..., k]) <= tol)
    assert np.all(np.abs(coh) <= d["flux"].sum() + 1e-9)


@pytest.mark.parametrize("polarised", [True, False])
def test_interference_polarisation_and_footprints(polarised):
    d = paper_sim.simulate_block(11, T=T, C=C, inr=10.0, polarised=polarised)
    sky = paper_sim.simulate_block(11, T=T, C=C, inr=0.0, polarised=polarised)
    rfi = (_cplx(d["vis"]) - _cplx(sky["vis"])) / d["rfi_scale"]
    mask = np.zeros((C, T), bool)
    cover = np.zeros((C, T), int)
    for kind, (c0, c1), (t0, t1), J in d["emitters"]:
        assert abs(np.linalg.norm(J) - 1) < 1e-12
        if polarised:
            assert _dop(J) <= 0.9 + 1e-12
        else:
            assert _dop(J) < 1e-12
        if kind == "broadband":
            assert 2 <= t1 - t0 < T // 20 or t1 == T
            assert 1 <= c1 - c0 < C // 8 or c1 == C
        elif kind == "narrowband":
            assert c1 - c0 == 1 and (T // 10 <= t1 - t0 < T // 2 or t1 == T)
        else:
            assert t1 - t0 == 1 and (C // 10 <= c1 - c0 < C // 2 or c1 == C)
        mask[c0:c1, t0:t1] = True
        cover[c0:c1, t0:t1] += 1
    assert np.array_equal(mask, d["truth"])
    # a broadband footprint not overlapped by another carries J itself, in every cell
    tol = 1e-4 * np.abs(_cplx(d["vis"])).max() / d["rfi_scale"]
    for kind, (c0, c1), (t0, t1), J in d["emitters"]:
        if kind != "broadband":
            continue
        alone = cover[c0:c1, t0:t1] == 1
        if alone.any():
            cells = rfi[c0:c1, t0:t1][alone]
            assert np.all(np.abs(cells - J.reshape(4)) <= tol)
