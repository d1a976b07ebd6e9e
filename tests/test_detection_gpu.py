"""The flagging kernel on the paper's simulated data (Section 4.2: one baseline, 2000
time x 512 frequency samples, 10 x 2 windows, INR 100) against the FP64 oracle: the
same statistics, flags and averages within the float32 tolerances of tests/parity.py,
for polarised and unpolarised interference."""
import numpy as np
import pytest

import oracle
from paper_2412_14775_b300 import RfiStream, default_thresholds
from parity import compare, run_gpu, to_device_rows
from synth import paper_sim

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("polarised", [True, False])
def test_simulated_block_flags_match_oracle(polarised):
    M, F, T, C = 10, 2, 2000, 512
    K = 200
    thr = default_thresholds(M * F)
    d = paper_sim.simulate_block(2024, inr=100.0, polarised=polarised)
    st = RfiStream(1, C, M, K, thr, "f32", window_F=F)
    g = run_gpu(st, to_device_rows(d["vis"], "f32"))
    o = oracle.OracleStream(C, M, K, **thr, F=F).process(d["vis"])
    rep = compare(g, o, thr, M, K, F=F)
    # the interference is found: most of its samples lie in flagged windows
    flagged = np.repeat(np.repeat(o["wflag"].astype(bool), F, axis=0), M, axis=1)
    assert flagged[d["truth"]].mean() > 0.5
    print("simulated block", "polarised" if polarised else "unpolarised", rep,
          "detected", flagged[d["truth"]].mean(), "false", flagged[~d["truth"]].mean())
    st.close()
