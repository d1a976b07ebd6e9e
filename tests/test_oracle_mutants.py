"""The pins must catch plausible mistakes.

Each case copies the oracle's C source, plants one mistake (a dropped term, a wrong
sign or index, a misread formula), builds it into a separate library on the CPU and
runs every pin against it.  A mutant that passes every pin would mean the pins do
not protect that part of the oracle.
"""
import os

import pytest

import oracle
import oracle.build
import oracle.oracle
import oracle_pins

MUTANTS = {
    # Eq. IQUV
    "U_sign": ("s[4] = xy_re + yx_re;", "s[4] = xy_re - yx_re;"),
    "Q_uses_xy": ("s[2] = xx_re - yy_re;", "s[2] = xy_re - yy_re;"),
    "V_re_from_real_parts": ("s[6] = -(xy_im - yx_im);", "s[6] = -(xy_re - yx_re);"),
    "I_im_dropped_yy": ("s[1] = xx_im + yy_im;", "s[1] = xx_im;"),
    # Section 2.1 / Table 1
    "tau_minus_one_outside": ("return lead * (Wd * s2 / (s12 + eps) - 1.0);",
                              "return lead * (Wd * s2 / (s12 + eps)) - 1.0;"),
    "tau_lead_W_not_W_minus_1": ("(Wd * d + 1.0) / (Wd - 1.0);", "(Wd * d + 1.0) / (Wd);"),
    "S1_sums_power": ("acc_add(&S1, z, compensated);", "acc_add(&S1, y, compensated);"),
    "eps_dropped_from_S1sq": ("/ (s12 + eps) - 1.0", "/ (s12) - 1.0"),
    # Section 2.2 / Table 2
    "r_not_divided_by_W": ("return sqrt(qb + ub + vb) / (double)W;", "return sqrt(qb + ub + vb);"),
    "p_without_sqrt": ("const double p = sqrt(a + b + c) + eps;", "const double p = (a + b + c) + eps;"),
    "v_from_wrong_part": ("const double v = stokes[8 * i + 6 + part];",
                          "const double v = stokes[8 * i + 7 - part];"),
    "eps_dropped_from_p": ("const double p = sqrt(a + b + c) + eps;", "const double p = sqrt(a + b + c);"),
    # flag rule
    "sk_and_ds": ("return f_sk | (f_re | f_im);", "return f_sk & (f_re | f_im);"),
    "im_part_ignored": ("return f_sk | (f_re | f_im);", "return f_sk | f_re;"),
    "flag_bit_shifted": ("fb[ts / 32] |= (uint32_t)1u << (ts % 32)",
                         "fb[ts / 32] |= (uint32_t)1u << ((ts + 1) % 32)"),
    # averaging and carry
    "avg_divides_by_K": ("acc_val(&bin[c]) / bin_n", "acc_val(&bin[c]) / (double)K"),
    # T x F footprints
    "tf_sk_first_channel_only": ("oracle_sk_window(stokes, W, d", "oracle_sk_window(stokes, Mt, d"),
    "tf_ds_im_first_channel_only": ("oracle_ds_window(stokes, W, 1,", "oracle_ds_window(stokes, Mt, 1,"),
    "tf_flag_first_channel_only": ("if (f) fb[ts / 32] |= (uint32_t)1u << (ts % 32);",
                                   "if (f && k == 0) fb[ts / 32] |= (uint32_t)1u << (ts % 32);"),
    "weight_counts_windows": ("weight[(size_t)row * n_out + b] = bin_n / (double)K;",
                              "weight[(size_t)row * n_out + b] = bin_n / (double)W / (double)K;"),
    "flagged_samples_averaged": ("if (!f) {\n                    for (int i = 0; i < Mt; ++i)",
                                 "if (1) {\n                    for (int i = 0; i < Mt; ++i)"),
    "carry_dropped": ("bin[c].s = carry_sum[(size_t)row * 8 + c]; bin[c].c = 0;",
                      "bin[c].s = 0; bin[c].c = 0;"),
}


@pytest.fixture(scope="module")
def src():
    with open(oracle.build.SRC) as f:
        return f.read()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, src, tmp_path):
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mutated = tmp_path / "rfi_oracle_mutant.c"
    mutated.write_text(src.replace(old, new))
    lib = oracle.build.compile_source(str(mutated), str(tmp_path / "libmutant.so"))
    oracle.oracle.use_library(lib)
    try:
        caught = []
        for pin in oracle_pins.ALL_PINS:
            try:
                pin()
            except (AssertionError, ValueError, FloatingPointError):
                caught.append(pin.__name__)
                break
        assert caught, f"no pin detects mutant {name}"
    finally:
        oracle.oracle.use_library(None)
    assert os.path.exists(lib)


# Partial windows live in the Python wrapper (oracle/oracle.py), which buffers the
# samples of a window left open by a block; mistakes there must fail pin P10.
PY_MUTANTS = {
    "partial_pending_dropped": ("v = np.concatenate([self.pending, v], axis=1)", "v = v"),
    "partial_pending_not_kept": ("v[:, whole:].copy()", "v[:, :0].copy()"),
}


@pytest.mark.parametrize("name", sorted(PY_MUTANTS))
def test_partial_window_pin_catches_mutant(name, monkeypatch):
    import types
    old, new = PY_MUTANTS[name]
    with open(oracle.oracle.__file__) as f:
        text = f.read()
    assert text.count(old) == 1, f"mutation site for {name} not found exactly once"
    mod = types.ModuleType("oracle._mutant")
    mod.__dict__["__package__"] = "oracle"
    exec(compile(text.replace(old, new), "oracle_mutant.py", "exec"), mod.__dict__)
    monkeypatch.setattr(oracle_pins, "OracleStream", mod.OracleStream)
    with pytest.raises((AssertionError, ValueError)):
        oracle_pins.pin_p10_partial_windows()


# The online thresholds (oracle/adaptive.py): mistakes there must fail pin P11.
ADAPTIVE_MUTANTS = {
    "adaptive_updates_flagged_windows": ("                if f:\n                    continue\n", ""),
    "adaptive_sd_without_mean": ("np.maximum(m2 - mu * mu, 0.0)", "np.maximum(m2, 0.0)"),
    "adaptive_ignores_alpha": ("w = max(self.alpha, 1.0 / n)", "w = 1.0 / n"),
    "adaptive_weight_alpha_only": ("w = max(self.alpha, 1.0 / n)", "w = self.alpha"),
    "adaptive_warm_never": ("warm = n >= self.n_warm", "warm = n > 1e300"),
}


@pytest.mark.parametrize("name", sorted(ADAPTIVE_MUTANTS))
def test_online_threshold_pin_catches_mutant(name, monkeypatch):
    import types
    import oracle.adaptive
    old, new = ADAPTIVE_MUTANTS[name]
    with open(oracle.adaptive.__file__) as f:
        text = f.read()
    assert text.count(old) == 1, f"mutation site for {name} not found exactly once"
    mod = types.ModuleType("oracle._adaptive_mutant")
    mod.__dict__["__package__"] = "oracle"
    exec(compile(text.replace(old, new), "adaptive_mutant.py", "exec"), mod.__dict__)
    monkeypatch.setattr(oracle, "AdaptiveOracleStream", mod.AdaptiveOracleStream)
    with pytest.raises((AssertionError, ValueError, ZeroDivisionError)):
        oracle_pins.pin_p11_online_thresholds()


# Overlapping windows (oracle/sliding.py): mistakes there must fail pin P13.
SLIDING_MUTANTS = {
    "sliding_or_misses_oldest_window": ("allw[:, i:i + L].any(axis=1)",
                                        "allw[:, i + 1:i + L].any(axis=1)"),
    "sliding_history_not_kept": ("self.history = allw[:, allw.shape[1] - (L - 1):].copy()",
                                 "self.history = self.history"),
    "sliding_pending_dropped": ("self.pending = buf[:, nbits:].copy()",
                                "self.pending = buf[:, :0].copy()"),
    "sliding_counts_flagged_samples": ("self.carry_cnt[keep] += 1.0", "self.carry_cnt += 1.0"),
    "sliding_hop_ignored": ("max(0, (n - self.M) // self.H + 1)",
                            "max(0, (n - self.M) // self.M + 1)"),
}


@pytest.mark.parametrize("name", sorted(SLIDING_MUTANTS))
def test_sliding_window_pin_catches_mutant(name, monkeypatch):
    import types
    import oracle.sliding
    old, new = SLIDING_MUTANTS[name]
    with open(oracle.sliding.__file__) as f:
        text = f.read()
    assert text.count(old) == 1, f"mutation site for {name} not found exactly once"
    mod = types.ModuleType("oracle._sliding_mutant")
    mod.__dict__["__package__"] = "oracle"
    exec(compile(text.replace(old, new), "sliding_mutant.py", "exec"), mod.__dict__)
    monkeypatch.setattr(oracle, "SlidingOracleStream", mod.SlidingOracleStream)
    with pytest.raises((AssertionError, ValueError, IndexError)):
        oracle_pins.pin_p13_sliding_windows()


# The mixed-precision emulation (oracle/mixed.py, Tables 3 and 4): each group run at the
# other precision, Table 3's groups 5 and 6 swapped, and mistakes in its formulas must
# fail the exact-evaluation pin.  (Table 4's group 5 cannot change a result; see
# tests/test_oracle_mixed.py.)
_PREC_SITE = {
    "sk": '"sk": {1: F32, 2: F32, 3: F32, 4: F32, 5: F16, 6: F32, 7: F16},',
    "ds": '"ds": {1: F32, 2: F32, 3: F32, 4: F16, 5: F16, 6: F16, 7: F16},',
}


def _prec_flip(stat, group):
    old = _PREC_SITE[stat]
    fmt = "F16" if f"{group}: F32" in old else "F32"
    other = "F32" if fmt == "F16" else "F16"
    return old, old.replace(f"{group}: {other}", f"{group}: {fmt}")


MIXED_MUTANTS = {f"mixed_{s}_g{g}_flipped": _prec_flip(s, g)
                 for s in ("sk", "ds") for g in range(1, 8) if (s, g) != ("ds", 5)}
MIXED_MUTANTS.update({
    "mixed_sk_g5_g6_swapped": (_PREC_SITE["sk"], _PREC_SITE["sk"].replace(
        "5: F16, 6: F32", "5: F32, 6: F16")),
    "mixed_tau_minus_one_outside": ("tau = f7(lead) * (t - one7)", "tau = f7(lead) * t - one7"),
    "mixed_eps16_is_callers_eps": ("return F16(2.0 ** -10) if fmt is F16 else F32(eps)",
                                   "return fmt(eps)"),
    "mixed_params_not_binary32": ("return fmt(F32(x))", "return fmt(x)"),
    "mixed_sk_sums_reversed": ("for i in range(W):                               # g3, g4",
                               "for i in reversed(range(W)):                    # g3, g4"),
    "mixed_ds_sums_reversed": ("for i in range(W):                                # g4",
                               "for i in reversed(range(W)):                     # g4"),
    "mixed_r_without_sqrt": ("r = np.sqrt((qb.astype(f6) + ub.astype(f6)) + vb.astype(f6))",
                             "r = ((qb.astype(f6) + ub.astype(f6)) + vb.astype(f6))"),
    "mixed_p_eps_dropped": ("p = np.sqrt((a.astype(f2) + b.astype(f2)) + c.astype(f2)) + _eps(f2, eps)",
                            "p = np.sqrt((a.astype(f2) + b.astype(f2)) + c.astype(f2))"),
})


@pytest.fixture(scope="module")
def mixed_cases():
    import test_oracle_mixed as T
    cases = T._windows() + T._threshold_cases() + T._order_cases()
    return cases, [T._exact(v, thr) for v, thr in cases]


@pytest.mark.parametrize("name", sorted(MIXED_MUTANTS))
def test_mixed_precision_pin_catches_mutant(name, mixed_cases):
    import types
    import oracle.mixed
    import test_oracle_mixed as T
    old, new = MIXED_MUTANTS[name]
    with open(oracle.mixed.__file__) as f:
        text = f.read()
    assert text.count(old) == 1, f"mutation site for {name} not found exactly once"
    mod = types.ModuleType("oracle._mixed_mutant")
    mod.__dict__["__package__"] = "oracle"
    exec(compile(text.replace(old, new), "mixed_mutant.py", "exec"), mod.__dict__)
    cases, exact = mixed_cases
    with pytest.raises(AssertionError):
        T.pin_emulation_exact(cases, exact, emulation=mod)
