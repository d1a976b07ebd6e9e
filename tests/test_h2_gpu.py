"""The binary16 Stokes arithmetic mode (precision = 2) against the FP64 oracle.

The oracle runs on the binary16 input values themselves, so every difference is the
mode's arithmetic: one binary16 rounding per Stokes component, then exact products and
float32 sums.  tests/parity.py (compare_h2) derives the bounds each statistic and
average must meet from that; flags must agree wherever the oracle's statistic is
farther from its threshold than its bound, and the flag disagreement must stay within
0.1 % of windows.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2412_14775_b300 import RfiStream, autotune, binding, default_thresholds
from paper_2412_14775_b300.binding import RfiError
from parity import compare, compare_h2, run_gpu, to_device_rows

pytestmark = pytest.mark.gpu

SHAPES = [  # (stations, channels, M, K, T, options)
    (6, 16, 16, 64, 256, {}),
    (6, 16, 16, 64, 256, dict(lanes_per_row=1)),
    (6, 16, 8, 32, 256, dict(lanes_per_row=4)),
    (6, 16, 32, 64, 256, dict(lanes_per_row=4)),
    (6, 16, 64, 128, 256, {}),                                   # Kahan S1, S2
    (6, 16, 15, 45, 225, {}),                                    # odd M: one sample per unit
    (6, 16, 10, 20, 200, dict(window_F=2)),                      # the paper's 10 x 2
    (6, 16, 5, 20, 200, dict(window_F=4, lane_split=1, lanes_per_row=2)),   # 5 x 4
    (6, 16, 8, 64, 256, dict(lane_split=1, lanes_per_row=4)),
    (6, 16, 16, 64, 256, dict(lanes_per_row=2, max_registers=96)),
    (6, 16, 32, 64, 256, dict(lanes_per_row=4, max_registers=96)),
]


@pytest.mark.parametrize("N,C,M,K,T,opts", SHAPES,
                         ids=[f"M{s[2]}-K{s[3]}-{'-'.join(f'{k[:4]}{v}' for k, v in s[5].items())}"
                              for s in SHAPES])
def test_h2_against_oracle(N, C, M, K, T, opts):
    F = opts.get("window_F", 1)
    thr = default_thresholds(M * F)
    data = synth.tiny_block(seed=41 + M, stations=N, channels=C, T=T, duty=0.08)["vis"]
    st = RfiStream(N, C, M, K, thr, "f16", precision=2, **opts)
    assert st.options["precision"] == 2
    assert st.options["max_registers"] == opts.get("max_registers", 128)
    g = run_gpu(st, to_device_rows(data, "f16"))
    R = st.R
    v16 = data.reshape(R, T, 4, 2).astype(np.float16)
    o = oracle.OracleStream(R, M, K, **thr, F=F).process(v16)
    rep = compare_h2(g, o, v16.reshape(R, T, 8).astype(np.float64), thr, M, K, F=F)
    assert rep["flag_disagree_frac"] <= 1e-3, rep
    assert 0 < o["wflag"].mean() < 1
    binding.rfi_check(st.ctx)
    st.close()
    print(f"h2 M={M} F={F} {opts}", rep)


def test_h2_block_split_is_bit_identical():
    """Splits at multiples of M (bins straddling blocks) give the one-block outputs."""
    N, C, M, K = 5, 8, 16, 64
    thr = default_thresholds(M)
    data = synth.tiny_block(seed=44, stations=N, channels=C, T=256, duty=0.08)["vis"]
    one = RfiStream(N, C, M, K, thr, "f16", precision=2)
    whole = one.process(to_device_rows(data, "f16"))
    two = RfiStream(N, C, M, K, thr, "f16", precision=2)
    a = two.process(to_device_rows(data[:, :, :96], "f16"))
    b = two.process(to_device_rows(data[:, :, 96:], "f16"))
    torch.cuda.synchronize()
    st = torch.cat([a["stats"], b["stats"]], dim=2)
    assert torch.equal(st, whole["stats"])
    assert torch.equal(torch.cat([a["avg"], b["avg"]], dim=1), whole["avg"])
    assert torch.equal(torch.cat([a["weight"], b["weight"]], dim=1), whole["weight"])
    one.close(); two.close()


def test_h2_batch_equals_single_launches():
    """Uneven binary16 streams in one persistent launch give the bits of single calls."""
    M, K, T = 16, 64, 128
    thr = default_thresholds(M)
    geo = [(4, 8), (7, 16), (5, 24)]
    vis = [to_device_rows(synth.tiny_block(seed=50 + i, stations=n, channels=c, T=T,
                                           duty=0.08)["vis"], "f16") for i, (n, c) in enumerate(geo)]
    solo = [RfiStream(n, c, M, K, thr, "f16", precision=2) for n, c in geo]
    bs = [RfiStream(n, c, M, K, thr, "f16", precision=2) for n, c in geo]
    want = [s.process(v) for s, v in zip(solo, vis)]
    outs = [s.alloc_outputs(T) for s in bs]
    binding.rfi_process_batch([s.ctx for s in bs], vis, [T] * 3, [o["flags"] for o in outs],
                              [o["avg"] for o in outs], [o["weight"] for o in outs],
                              [o["stats"] for o in outs])
    torch.cuda.synchronize()
    for w, o in zip(want, outs):
        for k in ("flags", "stats", "avg", "weight"):
            assert torch.equal(w[k], o[k]), k
    for s in solo + bs:
        s.close()


@pytest.mark.parametrize("M", [8, 16, 32, 64])
def test_h2_lofar_scale_sampled_rows(M):
    """62 stations, 64 channels, T = K = 256 in the tuned binary16 launch shape; the
    oracle checks 2048 seeded rows: on the binary16 values (the mode's arithmetic,
    bounded) and on the unrounded float32 values (with the input's quantisation;
    flag disagreement within 0.1 %)."""
    K = 256
    thr = default_thresholds(M)
    d = synth.lofar_block(seed=2)
    vis = to_device_rows(d["vis"], "f16")
    best, _ = autotune.tune(62, 64, M, K, thr, "f16", vis, cache_path=autotune.TUNED_PATH,
                            write_cache=False, fixed={"precision": 2})
    st = RfiStream(62, 64, M, K, thr, "f16", **autotune.options_of(best))
    assert st.options["precision"] == 2
    g = run_gpu(st, vis)
    del vis
    rows = np.sort(np.random.default_rng(17).choice(st.R, size=2048, replace=False))
    v = d["vis"].reshape(st.R, 256, 4, 2)[rows]
    v16 = v.astype(np.float16)
    gs = {k: val[rows] for k, val in g.items()}
    o = oracle.OracleStream(len(rows), M, K, **thr).process(v16)
    rep = compare_h2(gs, o, v16.reshape(len(rows), 256, 8).astype(np.float64), thr, M, K)
    o32 = oracle.OracleStream(len(rows), M, K, **thr).process(v)
    rep32 = compare(gs, o32, thr, M, K, stat_rtol=None, avg_rtol=None, check_flags=False)
    assert rep["flag_disagree_frac"] <= 1e-3 and rep32["flag_disagree_frac"] <= 1e-3, (rep, rep32)
    print(f"lofar h2 M={M}", rep, "vs float32 input", rep32)
    st.close()


def test_h2_needs_binary16_input():
    with pytest.raises(RfiError):
        RfiStream(4, 4, 16, 64, default_thresholds(16), "f32", precision=2)
    with pytest.raises(RfiError):
        RfiStream(4, 4, 16, 64, default_thresholds(16), "f16", precision=2, partial_windows=1)
