"""The division by an invariant divisor that the mesh kernels use to turn a
word index into (row, x word) and a row into (y, z) (Granlund and
Montgomery, "Division by invariant integers using multiplication", 1994):
multiplier and shifts chosen on the host, one multiply-high, a subtract, an
add and two shifts on the device.  Restated here in 64-bit integers and
checked against exact integer division over every divisor size and the
dividends at the ends of the 32-bit range."""

import numpy as np


def make_div(d):
    l = 0
    while (1 << l) < d:
        l += 1
    m = ((1 << 32) * ((1 << l) - d)) // d + 1
    assert 0 < m < (1 << 32)
    return m, min(l, 1), max(l - 1, 0)


def fast_div(n, m, s1, s2):
    n = np.asarray(n, np.uint64)
    t = (n * np.uint64(m)) >> np.uint64(32)
    return (t + ((n - t) >> np.uint64(s1))) >> np.uint64(s2)


def test_exact_for_every_divisor_size():
    rng = np.random.default_rng(3)
    divisors = set(range(1, 2100)) | {(1 << k) + o for k in range(1, 31) for o in (-1, 0, 1)} | \
        set(rng.integers(1, 1 << 31, 2000).tolist())
    ends = np.array([0, 1, 2, (1 << 31) - 1, 1 << 31, (1 << 32) - 2, (1 << 32) - 1], np.uint64)
    for d in sorted(x for x in divisors if 1 <= x < (1 << 31)):
        m, s1, s2 = make_div(d)
        n = np.concatenate([ends, rng.integers(0, 1 << 32, 256, dtype=np.uint64),
                            np.array([d * k + r for k in (1, 2, 1000) for r in (-1, 0, 1)
                                      if 0 <= d * k + r < (1 << 32)], np.uint64)])
        assert np.array_equal(fast_div(n, m, s1, s2), n // np.uint64(d)), d
