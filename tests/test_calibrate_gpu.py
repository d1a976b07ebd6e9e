"""Thresholds calibrated for a false-alarm probability give that rate on fresh
interference-free data drawn from the same (stationary) noise model: circular Gaussian
correlations, 16 stations x 16 channels."""
import math

import pytest
import torch

import synth
from paper_2412_14775_b300 import RfiStream
from paper_2412_14775_b300.calibrate import permissive, thresholds_for_false_alarm

pytestmark = pytest.mark.gpu


def _clean(seed):
    d = synth.tiny_block(seed=seed, stations=16, channels=16, T=1000, duty=0.0)["vis"]
    return torch.from_numpy(d.reshape(-1, 1000, 4, 2)).cuda()


@pytest.mark.parametrize("fa", [0.05, 0.01])
def test_false_alarm_matches_target(fa):
    M, F, C, T = 10, 2, 16, 1000
    cal = RfiStream(16, C, M, T, permissive(), "f32", window_F=F)
    stats = [cal.process(_clean(100 + k))["stats"].clone() for k in range(4)]
    thr = thresholds_for_false_alarm(stats, fa=fa)
    assert thr["s_low"] < thr["s_high"] and 0 < thr["gamma"] < 1
    for name, t in (("SK", dict(thr, gamma=math.inf)),
                    ("DS", dict(thr, s_low=-math.inf, s_high=math.inf))):
        st = RfiStream(16, C, M, T, t, "f32", window_F=F)
        flagged = total = 0
        for k in range(4):
            w = st.process(_clean(200 + k))["weight"]      # weight = unflagged fraction
            flagged += float((1 - w).sum()) * T
            total += w.numel() * T
        rate = flagged / total
        assert abs(rate - fa) < max(0.3 * fa, 0.004), (name, rate)
