"""The FP32 walks' draws in R^3 with N_V = 1: one Philox4x32-10 block per step
gives the directions of Theta (words x, y) and Z (words z, w) by Archimedes'
theorem from the words' low 23 bits, and the radius uniform U from their top
bytes (bits 24..31 of x and y, 24..30 of z).  Pinned here on words drawn from
the oracle's Philox4x32-10 (Random123 known-answer vectors pin that generator):
the directions are uniform on S^2, U is uniform on its 2^23 grid, and U is
independent of the four direction uniforms (its bits are disjoint from theirs)."""
import math

import numpy as np
from scipy import stats

import oracle as O

KEY = (0x5851F42D, 0x4C957F2D)


def u23(word):
    """2 - (1 + m / 2^23): a uniform in (0, 1] from the low 23 bits."""
    return 2.0 - (1.0 + (word & 0x7FFFFF) / 2.0 ** 23)


def radius_bits(x, y, z):
    """The 23 bits of U: byte 3 of x, byte 3 of y, the low 7 bits of byte 3 of z."""
    return ((x >> 24) & 0xFF) | (((y >> 24) & 0xFF) << 8) | (((z >> 24) & 0x7F) << 16)


def direction(uz, uphi):
    s = 2.0 * math.sqrt(uz * (1.0 - uz))
    return (s * math.cos(2.0 * math.pi * uphi), s * math.sin(2.0 * math.pi * uphi), 2.0 * uz - 1.0)


def _draws(n):
    d = np.zeros((2 * n, 3))
    U = np.zeros(n)
    low = np.zeros((n, 4))
    for s in range(n):
        k, i = s % 525, s // 525                      # step of walk i at point 5
        x, y, z, w = O.philox((0, k, i, 5), KEY)
        d[2 * s] = direction(u23(x), u23(y))
        d[2 * s + 1] = direction(u23(z), u23(w))
        U[s] = u23(radius_bits(x, y, z))
        low[s] = (u23(x), u23(y), u23(z), u23(w))
    return d, U, low


def test_directions_uniform_on_the_sphere():
    d, _, _ = _draws(20000)                           # 40,000 directions
    n = len(d)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-12)
    assert np.all(np.abs(d.mean(axis=0)) < 5.0 / math.sqrt(3.0 * n))
    # second moment I/3 (Var(d_j^2) = 4/45 on the sphere, Var(d_i d_j) = 1/15)
    M2 = d.T @ d / n
    for a in range(3):
        assert abs(M2[a, a] - 1.0 / 3.0) < 5.0 * math.sqrt(4.0 / 45.0 / n)
        for b in range(a):
            assert abs(M2[a, b]) < 5.0 * math.sqrt(1.0 / 15.0 / n)
    # each coordinate of a uniform point of S^2 is uniform on [-1, 1] (Archimedes)
    for a in range(3):
        assert stats.kstest(d[:, a], "uniform", args=(-1.0, 2.0)).pvalue > 1e-3


def test_radius_uniform_is_uniform_and_independent():
    _, U, low = _draws(20000)
    n = len(U)
    assert np.all((U > 0.0) & (U <= 1.0))
    assert stats.kstest(U, "uniform").pvalue > 1e-3
    for j in range(4):
        assert abs(np.corrcoef(U, low[:, j])[0, 1]) < 5.0 / math.sqrt(n)
        # coarse joint histogram (8 x 8 bins) against independence
        table = np.histogram2d(U, low[:, j], bins=8, range=[[0, 1], [0, 1]])[0]
        assert stats.chi2_contingency(table)[1] > 1e-3


def test_radius_bits_are_disjoint_from_the_direction_bits():
    rng = np.random.default_rng(3)
    for _ in range(200):
        x, y, z = (int(v) for v in rng.integers(0, 2 ** 32, 3))
        low_mask = 0x00FFFFFF                         # the 23 direction bits and bit 23
        assert radius_bits(x, y, z) == radius_bits(x & ~low_mask & 0xFFFFFFFF, y & ~low_mask & 0xFFFFFFFF,
                                                   z & ~low_mask & 0xFFFFFFFF)
        assert radius_bits(x ^ (1 << 24), y, z) != radius_bits(x, y, z)
        assert radius_bits(x, y ^ (1 << 31), z) != radius_bits(x, y, z)
        assert radius_bits(x, y, z ^ (1 << 30)) != radius_bits(x, y, z)
    # all 23 bits used: U covers its full grid range
    assert radius_bits(0xFFFFFFFF, 0xFFFFFFFF, 0x7FFFFFFF) == 0x7FFFFF
