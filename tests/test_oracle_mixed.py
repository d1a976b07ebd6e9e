"""The mixed-precision emulation (oracle/mixed.py) against the FP64 oracle: within
error bounds that follow from counting the binary16 roundings of Tables 3 and 4, and
the paper's cost model against the Cost columns of Tables 1 and 2."""
import math

import numpy as np

import oracle
import synth
from oracle import mixed

U16 = 2.0 ** -11          # unit roundoff of binary16


def _data():
    d = synth.tiny_block(seed=12, stations=5, channels=8, T=256)["vis"]
    return d.reshape(-1, 256, 4, 2)


def test_mixed_within_binary16_error_bounds():
    M = 16
    thr = dict(d=1.0, s_low=-1e9, s_high=1e9, gamma=1e9, eps=2.0 ** -23)
    v = _data()
    ref = oracle.OracleStream(v.shape[0], M, M, **thr).process(v)
    got = mixed.process_block_mixed(v.reshape(v.shape[0], 256, 8), M, **thr)
    lead = (M * thr["d"] + 1) / (M - 1)
    # tau: about 9 binary16 roundings act on lead * t, one more on the final subtraction
    bound_tau = 10 * U16 * (np.abs(ref["tau"]) + lead + 1) + 1e-6
    assert np.all(np.abs(got["tau"] - ref["tau"]) <= bound_tau)
    # r: W rounded terms and W-1 rounded partial sums (each partial sum <= its count),
    # then ~5 roundings on r itself
    sum_err = math.sqrt(3) * U16 * (M + M * (M + 1) / 2) / M
    for key in ("r_re", "r_im"):
        assert np.all(np.abs(got[key] - ref[key]) <= sum_err + 5 * U16 * ref[key] + 1e-6), key
    # and the approximation is not trivially exact: binary16 effects are visible
    assert np.any(got["tau"] != ref["tau"])


def test_cost_model():
    from paper_2412_14775_b300.costmodel import window_cost
    for W in (16, 20, 64):
        assert window_cost(W, False) == 30 * W + 21     # Table 1: 6W+5; Table 2: 12W+8 per part
        assert window_cost(W, True) < window_cost(W, False)
