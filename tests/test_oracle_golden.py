"""The oracle on hand-derived worked examples (tests/golden/worked_examples.json)."""
import json
import os

import numpy as np
import pytest

from oracle import OracleStream

HERE = os.path.dirname(os.path.abspath(__file__))
with open(os.path.join(HERE, "golden", "worked_examples.json")) as f:
    CASES = json.load(f)["cases"]


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_worked_example(case):
    s = np.array(case["samples"], dtype=np.float64)            # [T, 4, 2]
    M = case["M"]
    K = case.get("K", M)
    st = OracleStream(1, M, K, case["d"], case.get("s_low", -1e300), case.get("s_high", 1e300),
                      case.get("gamma", 1e300), case["eps"])
    out = st.process(s[None])
    for key in ("tau", "r_re", "r_im"):
        if key in case:
            assert out[key][0, 0] == pytest.approx(case[key], rel=1e-14, abs=1e-15), key
    if "avg" in case:
        want = np.array(case["avg"], dtype=np.float64).reshape(8)
        assert np.allclose(out["avg"][0, 0], want, rtol=1e-15, atol=1e-15)
        assert out["weight"][0, 0] == case["weight"]
