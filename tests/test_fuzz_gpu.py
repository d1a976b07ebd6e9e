"""Seeded random combinations of geometry, window, footprint, lanes per row, loader,
register budget, prefetch, buffered stores, Kahan summation and partial windows, each
checked against the FP64 oracle block by block (the tolerances of tests/parity.py).

A combination the library has no kernel for is rejected at create (RFI_EUNSUPPORTED or
RFI_EINVAL) and replaced by the next draw; every test draws until it has run its cases."""
import numpy as np
import pytest

from paper_2412_14775_b300 import RfiStream, binding
from paper_2412_14775_b300.binding import RfiError
from test_parity_gpu import _check_stream

pytestmark = pytest.mark.gpu


def _draw(rng):
    dtype = str(rng.choice(["f32", "f16"]))
    M = int(rng.choice([2, 3, 4, 5, 6, 8, 10, 12, 16, 20, 24, 32, 64]))
    F = int(rng.choice([1, 1, 1, 2, 4]))
    channels = F * int(rng.integers(1, 5))
    stations = int(rng.integers(2, 9))
    K = M * int(rng.integers(1, 5))
    opts = {"window_F": F}
    spu = 2 if (dtype == "f16" and M % 2 == 0) else 1
    ps = [p for p in (1, 2, 4, 8, 16, 32) if M % (p * spu) == 0 and p * F <= 32]
    if dtype == "f16" and spu == 1:
        ps = [1]
    opts["lanes_per_row"] = int(rng.choice(ps))
    roll = rng.random(6)
    if roll[0] < 0.25:
        opts["loader"] = 1 if roll[0] < 0.15 else 2      # row copies or tensor tiles
        opts["tma_stage_windows"] = int(rng.integers(1, 3))
        opts["tma_stages"] = int(rng.integers(2, 4))
        opts["warps_per_block"] = int(rng.choice([2, 4]))
    if roll[1] < 0.3:
        opts["max_registers"] = int(rng.choice([80, 64]))
        opts["warps_per_block"] = int(rng.choice([2, 4, 8]))
    if roll[2] < 0.3:
        opts["compensated"] = int(rng.choice([-1, 1]))
    if roll[3] < 0.3:
        opts["prefetch_groups"] = int(rng.integers(1, 3))
        opts["prefetch_bytes"] = int(rng.choice([256, 512, 1024]))
    if roll[4] < 0.2:
        opts["buffered_stores"] = 1
    partial = roll[5] < 0.3
    if partial:
        opts["partial_windows"] = 1
        step = 2 if (dtype == "f16" and M % 2 == 0) else 1
        Ts = [int(rng.integers(1, 3 * M + 1)) * step for _ in range(int(rng.integers(2, 5)))]
    else:
        Ts = [M * int(rng.integers(1, 6)) for _ in range(int(rng.integers(1, 4)))]
    return dtype, stations, channels, M, K, Ts, opts


def _creatable(dtype, stations, channels, M, K, opts):
    try:
        RfiStream(stations, channels, M, K, dict(d=1.0, s_low=0.0, s_high=2.0, gamma=0.5,
                                                eps=2.0 ** -23), dtype, **opts).close()
        return True
    except RfiError as e:
        assert e.status in (1, 6), e          # EINVAL / EUNSUPPORTED, never another error
        return False


@pytest.mark.parametrize("seed", range(12))
def test_random_combinations_match_oracle(seed):
    rng = np.random.default_rng(1000 + seed)
    ran = 0
    while ran < 6:
        dtype, stations, channels, M, K, Ts, opts = _draw(rng)
        if not _creatable(dtype, stations, channels, M, K, opts):
            continue
        _check_stream(stations, channels, M, K, Ts, dtype, seed=int(rng.integers(1, 1 << 30)),
                      **opts)
        ran += 1
