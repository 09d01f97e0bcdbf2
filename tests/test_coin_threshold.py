"""The IC coin as the device evaluates it.  Reading 3 of the paper's IC model:
edge e is live for a Philox word x when a * 2^-24 < p[e] in fp32, a = x >> 8.
Both sides are exact (a < 2^24, and p * 2^24 only shifts p's exponent), so the
coin equals the integer compare a < ceil(p * 2^24) that the library makes with
thresholds computed once per edge at graph upload.  Checked here on the
boundary values of every kind of p, exhaustively around each threshold."""
import numpy as np


def coin_fp32(a, p):
    return (np.float32(a) * np.float32(2.0 ** -24)) < np.float32(p)


def threshold(p):
    return int(np.ceil(np.float64(np.float32(p)) * 16777216.0))


def test_threshold_equals_fp32_coin_on_boundaries():
    rng = np.random.default_rng(5)
    ps = [0.0, 1.0, 2.0 ** -24, 2.0 ** -25, 2.0 ** -149, 0.5, 0.1, 0.05, 1.0 - 2.0 ** -24, 1.0 - 2.0 ** -25]
    ps += [float(np.float32(k) / np.float32(2 ** 24)) for k in (1, 2, 3, 1000, 12345, 2 ** 23, 2 ** 24 - 1)]
    ps += rng.random(300, dtype=np.float32).tolist()
    ps += (rng.random(300, dtype=np.float32) * np.float32(0.1)).tolist()
    for p in ps:
        p32 = np.float32(p)
        t = threshold(p32)
        assert 0 <= t <= 2 ** 24
        for a in {0, 1, max(t - 2, 0), max(t - 1, 0), t, min(t + 1, 2 ** 24 - 1), 2 ** 24 - 1}:
            assert bool(coin_fp32(a, p32)) == (a < t), (p, a, t)


def test_threshold_equals_fp32_coin_random():
    rng = np.random.default_rng(9)
    p = rng.random(20000, dtype=np.float32)
    a = rng.integers(0, 2 ** 24, size=20000, dtype=np.int64)
    t = np.ceil(p.astype(np.float64) * 16777216.0).astype(np.int64)
    got = a < t
    want = (a.astype(np.float32) * np.float32(2.0 ** -24)) < p
    assert np.array_equal(got, want)
