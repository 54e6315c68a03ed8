"""Pins of the scale-ordered codec (Sec. 2.4): bijection and bit positions."""
import numpy as np

from oracle import quantics as q


def test_roundtrip():
    rng = np.random.default_rng(0)
    for n in (1, 2, 3):
        N = 1 << n
        a = rng.standard_normal((N, N, N))
        t = q.encode(a)
        assert t.shape == (2,) * (3 * n)
        np.testing.assert_array_equal(q.decode(t), a)


def test_bit_positions():
    # a single 1 at (x, y, z) must appear at the site bits MSB-first, x-y-z interleaved
    n = 3
    N = 8
    for (x, y, z) in [(5, 2, 7), (1, 0, 4), (7, 7, 0)]:
        a = np.zeros((N, N, N))
        a[x, y, z] = 1.0
        idx = np.argwhere(q.encode(a) == 1.0)
        assert len(idx) == 1
        bits = idx[0]
        for lev in range(n):
            assert bits[3 * lev + 0] == (x >> (n - 1 - lev)) & 1
            assert bits[3 * lev + 1] == (y >> (n - 1 - lev)) & 1
            assert bits[3 * lev + 2] == (z >> (n - 1 - lev)) & 1
        assert q.site_of(2, 1) == 5


def test_site_bits_index_the_encoded_tensor():
    # every cell of a random field is found at its site bits in the encoded tensor
    rng = np.random.default_rng(3)
    n, N = 3, 8
    a = rng.standard_normal((N, N, N))
    t = q.encode(a)
    for x in range(N):
        for y in range(N):
            for z in range(N):
                assert t[tuple(q.site_bits(n, (x, y, z)))] == a[x, y, z]
