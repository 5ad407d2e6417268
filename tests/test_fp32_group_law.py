"""The FP32 walks' Gaussian transform in R^n (16-component groups: two Philox blocks of
radial words, one of 16-bit angle halves; the layout of gauss_group16) produces the
normal law, pinned against scipy's normal CDF on words drawn from the oracle's
Philox4x32-10 (Random123 known-answer vectors pin that generator).

A pair is sqrt(-log2 u) (cos 2 pi a, sin 2 pi a): times sqrt(2 ln 2) it is Box-Muller,
so each component must be N(0, 1/(2 ln 2)); the 16-bit angles must be uniform on their
65536 values, and |g|^2 of a group is the sum of its radial halves."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle as O

KEY = (0x2545F491, 0x4F6CDD1D)


def _groups(n_groups, seed_k=7):
    """Components (n_groups x 16) and radial sums of the groups of one step's vectors."""
    comps = np.zeros((n_groups, 16))
    sums = np.zeros(n_groups)
    angles = []
    for gi in range(n_groups):
        G, i = gi % 64, gi // 64          # group of a vector, walk index
        w = [O.philox((seed_k, 4 * G + c, i, 3), KEY) for c in range(3)]
        R = []
        for word in w[0] + w[1]:
            m = word & 0x7FFFFF
            u = 2.0 - (1.0 + m / 2.0 ** 23)          # (0, 1]
            R.append(math.sqrt(-math.log2(u)))
        sums[gi] = sum(r * r for r in R)
        for kw, word in enumerate(w[2]):
            for half, bits in enumerate((word & 0xFFFF, word >> 16)):
                a = bits / 65536.0
                angles.append(bits)
                q = 2 * kw + half                     # pair 2k from the low, 2k + 1 from the high half
                comps[gi, 2 * q] = R[q] * math.cos(2 * math.pi * a)
                comps[gi, 2 * q + 1] = R[q] * math.sin(2 * math.pi * a)
    return comps, sums, np.array(angles)


def test_group_components_are_normal():
    comps, sums, angles = _groups(8000)       # 128,000 components
    x = comps.ravel() * math.sqrt(2.0 * math.log(2.0))
    n = x.size
    assert abs(x.mean()) < 5.0 / math.sqrt(n)
    assert abs(x.var() - 1.0) < 5.0 * math.sqrt(2.0 / n)
    assert abs(stats.kurtosis(x, fisher=False) - 3.0) < 5.0 * math.sqrt(24.0 / n)
    assert stats.kstest(x, "norm").pvalue > 1e-3
    # the two components of a pair are uncorrelated
    assert abs(np.corrcoef(comps[:, 0::2].ravel(), comps[:, 1::2].ravel())[0, 1]) < 5.0 / math.sqrt(n / 2)
    # |g|^2 of a group from its radial halves alone equals the sum of its squared components
    assert np.allclose(sums, (comps ** 2).sum(axis=1), rtol=1e-12, atol=1e-12)
    # 16-bit angles uniform: 256 coarse bins
    counts = np.bincount(angles >> 8, minlength=256)
    assert stats.chisquare(counts).pvalue > 1e-3


def test_angle_grid_moments_match_the_uniform_angle():
    """On 65536 equally spaced angles every trigonometric moment of degree below 65536 equals
    the continuous uniform angle's (zero): the 16-bit angle changes no moment a walk sees."""
    a = np.arange(65536) / 65536.0
    for m in (1, 2, 3, 7, 100, 4095, 65535):
        assert abs(np.mean(np.cos(2 * math.pi * m * a))) < 1e-9
        assert abs(np.mean(np.sin(2 * math.pi * m * a))) < 1e-9
    assert abs(np.mean(np.cos(2 * math.pi * 65536 * a)) - 1.0) < 1e-9
