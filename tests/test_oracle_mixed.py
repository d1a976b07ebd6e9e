"""Pins of the mixed-precision emulation (oracle/mixed.py; paper Tables 3 and 4).

1. The exact route (tests/ieee_exact.py) is itself pinned: binary16 / binary32
   rounding facts that follow from the IEEE 754 definition, and agreement with
   numpy's conversions of random doubles (a library routine).
2. The emulation equals, bit for bit, the exact evaluation (rationals, one IEEE
   rounding per operation, the tables' group-to-format map: tests/mixed_exact.py) on a
   set of windows built so that every single-group change of the map that can change
   a result does change one: each group of Tables 1 and 2 flipped between binary16
   and binary32, and Table 3's groups 5 and 6 swapped (the "0.497" label, reading 13).
   So an emulation that ran any group at the wrong precision fails here.
3. Table 4's group 5 is the exception, proven rather than tested by search: with
   groups 4 and 6 in binary16, the square of a binary16 sum is exact in binary32 and
   group 6 rounds it to binary16 on entry, which is what a binary16 group 5 does; the
   evaluator shows both maps equal on every window.
4. The emulation stays within error bounds counted from its binary16 roundings of the
   FP64 oracle, and the paper's cost model matches the Cost columns of Tables 1-2.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import ieee_exact as X
import mixed_exact as E
import oracle
import synth
from oracle import mixed

U16 = 2.0 ** -11          # unit roundoff of binary16
D_DEFAULT = math.pi / (4.0 - math.pi)
# a d whose binary16 rounding (1 + 2^-10) and binary32 value (1 + 2^-11 + 2^-20) give a
# different binary16 lead (W d + 1)/(W - 1) at W = 16 (1162/1024 against 1161/1024)
D_SPLIT = 1.0 + 2.0 ** -11 + 2.0 ** -20
# a d that rounds to binary16 differently directly (1 + 2^-10) than through binary32
# (1 + 2^-11, a tie, then 1): the library holds parameters as binary32 values
D_DOUBLE = 1.0 + 2.0 ** -11 + 2.0 ** -40
EPS = 2.0 ** -23
WIDE = dict(s_low=-1e30, s_high=1e30, gamma=1e30)


# ---- 1. the exact route --------------------------------------------------------
def test_exact_rounding_facts():
    F = Fraction
    assert X.rnd(2049, X.B16) == 2048                     # tie: to the even 2048
    assert X.rnd(2051, X.B16) == 2052                     # tie: to the even 2052
    assert X.rnd(65519, X.B16) == 65504                   # below the overflow tie
    assert X.rnd(65520, X.B16) == X.INF                   # the tie rounds to 2^16
    assert X.rnd(F(1, 2 ** 25), X.B16) == 0               # half the smallest subnormal
    assert X.rnd(F(3, 2 ** 26), X.B16) == F(1, 2 ** 24)
    assert X.rnd(1 + F(1, 2 ** 24), X.B32) == 1           # tie: to even
    assert X.rnd(1 + F(3, 2 ** 24), X.B32) == 1 + F(1, 2 ** 22)
    assert X.rnd(2 ** 24 + 1, X.B32) == 2 ** 24
    assert X.sqrt(2, X.B16) == F(1448, 1024)               # 1.4140625
    assert X.sqrt(2, X.B32) == F(11863283, 2 ** 23)         # 0x3FB504F3
    assert X.sqrt(F(9, 4), X.B16) == F(3, 2)               # exact square
    assert X.div(1, 3, X.B16) == F(1365, 4096)              # 0x3555


def test_exact_rounding_matches_numpy_conversions():
    rng = np.random.default_rng(5)
    xs = rng.standard_normal(4000) * np.exp2(rng.integers(-30, 20, 4000))
    with np.errstate(over="ignore"):
        for x in xs:
            assert float(X.rnd(Fraction(float(x)), X.B16)) == float(np.float16(x))
            assert float(X.rnd(Fraction(float(x)), X.B32)) == float(np.float32(x))


def test_exact_sqrt_matches_correctly_rounded_float32():
    # numpy's float32 sqrt is IEEE's correctly rounded square root
    rng = np.random.default_rng(6)
    xs = (rng.random(3000) * np.exp2(rng.integers(-40, 40, 3000))).astype(np.float32)
    for x in xs:
        assert float(X.sqrt(Fraction(float(x)), X.B32)) == float(np.sqrt(x))


# ---- 2. the windows --------------------------------------------------------------
def _windows():
    """(vis [n, W, 8] float32, thresholds) cases: noise and polarised bursts over a
    range of scales (including scales where binary16 groups overflow), three window
    lengths, two values of d, and windows whose thresholds sit just below a binary16
    statistic (only the test's own precision decides the flag)."""
    rng = np.random.default_rng(20241477)
    cases = []
    for W in (5, 16, 20):
        for d in (D_DEFAULT, D_SPLIT, D_DOUBLE):
            for e in (-7, -2, 0, 3, 5):
                n = 3
                v = rng.standard_normal((n, W, 8)) * 2.0 ** e
                # a polarised burst on the middle window: c A e e^H plus noise
                th, ph = rng.uniform(0, np.pi), rng.uniform(0, 2 * np.pi)
                jv = np.array([np.cos(th), np.sin(th) * np.exp(1j * ph)])
                c = np.exp(1j * rng.uniform(0, 2 * np.pi)) * 2.0 ** (e + 2)
                cor = c * np.outer(jv, jv.conj()).reshape(4)
                v[1, :, 0::2] += cor.real
                v[1, :, 1::2] += cor.imag
                cases.append((v.astype(np.float32), dict(d=d, eps=EPS, **WIDE)))
    return cases


def _threshold_cases():
    """Windows with s_high (SK) or gamma (DS) set 2^-13 (relative) below the window's
    binary16 statistic: binary16 rounds the threshold back onto the statistic (not
    flagged), binary32 keeps it below (flagged)."""
    rng = np.random.default_rng(11)
    out = []
    for W in (16, 20):
        v = rng.standard_normal((1, W, 8)).astype(np.float32)
        tau, r_re, r_im, _ = E.window_exact(v[0], D_DEFAULT, -1e30, 1e30, 1e30, EPS)
        out.append((v, dict(d=D_DEFAULT, s_low=-1e30, s_high=tau * (1 - 2.0 ** -13),
                            gamma=1e30, eps=EPS)))
        g = max(r_re, r_im)
        out.append((v, dict(d=D_DEFAULT, s_low=-1e30, s_high=1e30,
                            gamma=g * (1 - 2.0 ** -13), eps=EPS)))
    return out


def _order_cases():
    """A window whose binary32 power sum S2 (Table 1 group 4) lands on a binary16 tie
    only when summed in window order: sample 0 has xx = 42 + 17j (|I|^2 = 2053, odd,
    halfway between the binary16 values 2052 and 2054), the 15 others |I|^2 = 2^-14,
    below half a binary32 ulp of 2053.  In order, S2 stays 2053 and group 7's binary16
    conversion takes the even 2052; summed the other way the small terms first add up
    to 15 2^-14 and S2 = 2053 + 2^-10, which converts to 2054."""
    v = np.zeros((1, 16, 8), np.float32)
    v[0, 0, 0:2] = (42.0, 17.0)
    v[0, 1:, 0] = 2.0 ** -7
    return [(v, dict(d=D_DEFAULT, eps=EPS, **WIDE))]


def _exact(v, thr, prec=E.TABLES_3_4):
    return [E.window_exact(w, thr["d"], thr["s_low"], thr["s_high"], thr["gamma"], thr["eps"],
                           prec) for w in v]


def _same(a, b):
    return a == b or (a != a and b != b)


@pytest.fixture(scope="module")
def cases():
    return _windows() + _threshold_cases() + _order_cases()


@pytest.fixture(scope="module")
def exact_tables(cases):
    return [_exact(v, thr) for v, thr in cases]


def pin_emulation_exact(cases, exact_tables, emulation=mixed):
    """Every statistic and flag of the emulation equals the exact evaluation with the
    tables' map (NaN where the exact route gives NaN).  Raises AssertionError."""
    for (v, thr), want in zip(cases, exact_tables):
        W = v.shape[1]
        got = emulation.process_block_mixed(v, W, **thr)
        for i, (tau, rre, rim, f) in enumerate(want):
            assert _same(got["tau"][i, 0], tau), (W, thr, i, "tau", got["tau"][i, 0], tau)
            assert _same(got["r_re"][i, 0], rre), (W, thr, i, "r_re")
            assert _same(got["r_im"][i, 0], rim), (W, thr, i, "r_im")
            assert bool(got["wflag"][i, 0]) == f, (W, thr, i, "flag")


def test_emulation_equals_exact_evaluation(cases, exact_tables):
    pin_emulation_exact(cases, exact_tables)


def _flipped(key):
    p = dict(E.TABLES_3_4)
    p[key] = 48 - p[key]
    return p


FLIPS = [k for k in E.TABLES_3_4 if k != ("ds", 5)]


@pytest.mark.parametrize("key", FLIPS, ids=[f"{a}_g{b}" for a, b in FLIPS])
def test_every_group_flip_changes_a_result(key, cases, exact_tables):
    """The window set discriminates: running this one group at the other precision
    changes some statistic or flag, so the equality above pins the group's format."""
    prec = _flipped(key)
    for (v, thr), base in zip(cases, exact_tables):
        alt = _exact(v, thr, prec)
        if any(not _same(a, b) for x, y in zip(base, alt) for a, b in zip(x, y)):
            return
    pytest.fail(f"no window tells {key} at binary{prec[key]} from the tables' map")


def test_sk_g5_g6_swap_changes_a_result(cases, exact_tables):
    prec = dict(E.TABLES_3_4)
    prec[("sk", 5)], prec[("sk", 6)] = prec[("sk", 6)], prec[("sk", 5)]
    for (v, thr), base in zip(cases, exact_tables):
        alt = _exact(v, thr, prec)
        if any(not _same(a, b) for x, y in zip(base, alt) for a, b in zip(x, y)):
            return
    pytest.fail("swapping Table 3 groups 5 and 6 changes nothing on the window set")


def test_ds_g5_precision_cannot_change_results(cases, exact_tables):
    """Table 4 group 5 between binary16 groups 4 and 6: both formats give the same
    statistics and flags on every window (the argument in the module docstring)."""
    prec = _flipped(("ds", 5))
    for (v, thr), base in zip(cases, exact_tables):
        alt = _exact(v, thr, prec)
        for x, y in zip(base, alt):
            assert all(_same(a, b) for a, b in zip(x, y))


# ---- 4. error bounds and cost --------------------------------------------------
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
