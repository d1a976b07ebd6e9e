"""The serving loop's device block pool, exercised on host memory (its bookkeeping is
the same): first fit, 256-byte alignment, neighbours merged on release, and a random
sequence of allocations and releases never overlapping and always returning every
byte."""
import numpy as np

from paper_2412_14775_b300.serve import DevicePool


def test_pool_first_fit_alignment_and_merge():
    p = DevicePool(4096, "cpu")
    a = p.alloc(100)
    b = p.alloc(300)
    c = p.alloc(256)
    assert (a, b, c) == (0, 256, 768) and p.used == 256 + 512 + 256
    assert p.alloc(4096) is None                    # does not fit any more
    p.release(b, 300)
    assert p.alloc(200) == 256                      # first fit reuses the hole
    p.release(256, 200)
    p.release(a, 100)
    p.release(c, 256)
    assert p.free == [(0, 4096)] and p.used == 0


def test_pool_random_sequence_never_overlaps():
    rng = np.random.default_rng(3)
    p = DevicePool(1 << 20, "cpu")
    live = {}
    for step in range(3000):
        if live and (rng.random() < 0.45 or p.used > (1 << 20) * 0.9):
            off = list(live)[rng.integers(len(live))]
            p.release(off, live.pop(off))
        else:
            n = int(rng.integers(1, 40000))
            off = p.alloc(n)
            if off is None:
                continue
            assert off % 256 == 0
            for o, m in live.items():
                assert off + DevicePool.rounded(n) <= o or o + DevicePool.rounded(m) <= off
            live[off] = n
        assert p.used == sum(DevicePool.rounded(m) for m in live.values())
    for off, n in list(live.items()):
        p.release(off, n)
    assert p.free == [(0, 1 << 20)]
