"""The seeded input generator: published SplitMix64 outputs, ranges, classes."""
import numpy as np

from paper_1806_10113_gb300 import inputs


def test_splitmix64_published_outputs():
    # Reference outputs of SplitMix64 (Steele, Lea and Flood 2014; Vigna's
    # splitmix64.c) for seeds 0 and 1234567.
    r = inputs.SplitMix64(0)
    assert r.next_u64() == 0xE220A8397B1DCDAF
    r = inputs.SplitMix64(1234567)
    assert [r.next_u64() for _ in range(3)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423]


def test_uniform_int_range_and_reproducible():
    r = inputs.SplitMix64(7)
    xs = [r.uniform_int(50_000, 2_000_000) for _ in range(5000)]
    assert min(xs) >= 50_000 and max(xs) <= 2_000_000
    r2 = inputs.SplitMix64(7)
    assert xs[:10] == [r2.uniform_int(50_000, 2_000_000) for _ in range(10)]
    r3 = inputs.SplitMix64(9)
    small = [r3.uniform_int(0, 2) for _ in range(3000)]
    assert set(small) == {0, 1, 2}


def test_single_group_uniform_config():
    b = inputs.single_group_uniform(n=6, seed=0)
    assert b.G == 1 and b.tasks.shape == (6, 3)
    assert b.tasks.min() >= 50_000 and b.tasks.max() <= 2_000_000


def test_dk_dt_groups_classes():
    b = inputs.dk_dt_groups(groups=8, n=10, seed=1)
    assert b.G == 16 and list(b.dma[:8]) == [2] * 8 and list(b.dma[8:]) == [1] * 8
    for g in range(8):
        t = b.group(g).astype(np.int64)
        dk = (t[:, 0] + t[:, 2] <= t[:, 1])
        assert dk.all() if g < 4 else (~dk).all()
        assert (b.group(g) == b.group(g + 8)).all()


def test_ragged_mixed_classes_and_sizes():
    b = inputs.ragged_mixed(groups=64, seed=2)
    sizes = b.sizes()
    assert sizes.min() >= 4 and sizes.max() <= 9
    assert b.tasks.min() >= 10_000 and b.tasks.max() <= 10_000_000
    assert list(b.dma[:4]) == [2, 1, 2, 1]
    t = b.tasks.astype(np.int64)
    dk = t[:, 0] + t[:, 2] <= t[:, 1]
    assert 0.3 < dk.mean() < 0.7


def test_half_dk_half_dt():
    b = inputs.half_dk_half_dt(groups=3, n=12, seed=3)
    for g in range(b.G):
        t = b.group(g).astype(np.int64)
        dk = t[:, 0] + t[:, 2] <= t[:, 1]
        assert dk[:6].all() and (~dk[6:]).all()
