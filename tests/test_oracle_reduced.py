"""Oracle pins for the dimension-reduced exact sampler.

The reduced sampler replaces the n Gaussians of a direction by the few
coordinates the walk reads, plus an independent chi^2 for the rest of |g|^2
(an exact reformulation of the same walk's law).  It is pinned against
things other than itself:

* the chi^2 draws against scipy's chi^2 distribution (KS test, moments);
* textbook solutions in R^n whose value depends on the whole of |g|^2 (a
  dropped or mis-sized chi^2 term changes the exit distribution);
* the telescoping identity (f = sigma, g = 1 -> S = 1 per walk);
* the full-dimensional oracle on the same problems, statistically.
"""
import numpy as np
import pytest
from scipy import stats

import oracle as O
from paper_2606_21883_b300 import workloads as W


@pytest.mark.parametrize("m", [1, 2, 5, 40, 979])
def test_chi2_draws_follow_chi2(m):
    x = np.array([O.chi2(11, 32, k, 3, 1, m) for k in range(6000)])
    assert stats.kstest(x, stats.chi2(m).cdf).pvalue > 1e-3
    assert abs(x.mean() - m) < 5 * np.sqrt(2 * m / x.size)
    assert abs(x.var() - 2 * m) < 0.15 * 2 * m


def test_chi2_zero_dof_is_zero():
    assert O.chi2(0, 32, 0, 0, 0, 0) == 0.0


def test_tracked_set():
    w = W.hypersphere_half(P=2, walks=1, n=64)
    assert O.tracked_set(w.problem, w.params) == [0, 1, 2]
    w = W.torus_closed(P=2, walks=1)
    assert O.tracked_set(w.problem, w.params) is None   # torus Fourier data


def _reduced(w):
    w.params.sampler = W.SAMPLER_REDUCED
    return w


@pytest.mark.parametrize("n", [12, 40])
def test_reduced_euclid_exponential_solution(n):
    """R^n, x_1 > 0, f = 0, g = 1: u = exp(-sqrt(sigma) x_1); T = {x_1}, chi^2 with n - 1 dof."""
    sigma = 2.0
    w = _reduced(W.euclid_halfspace(P=5, walks=1, n=n, sigma=sigma, seed=4))
    w.params.c_kappa = 1e3   # kappa = 0 in R^n: the ball rule r = theta dist
    m, se, ms, nf = O.solve(w.problem, w.params, w.points, 1500)
    u = np.exp(-np.sqrt(sigma) * w.points[:, 0])
    assert nf == 0
    assert np.all(np.abs(m - u) <= 4 * se + 2e-3)


def test_reduced_telescoping_sphere():
    """f = sigma, g = 1 on the half of S^63: each walk's score is exactly 1."""
    w = _reduced(W.constant_solution(W.hypersphere_half(P=3, walks=1, n=64, seed=5)))
    S, K, F = O.walk_scores(w.problem, w.params, w.points, 40)
    assert np.all(np.abs(S - 1.0) <= 1e-12 * np.maximum(K, 1))
    assert np.all(F == 0)


def test_reduced_closed_embedded_sphere_same_K_as_full():
    """The weights do not depend on the sampler: K = ceil(ln tau / ln c) for both."""
    w = W.embedded_s20(P=2, walks=1, n=64, d=5, sigma=6.0)
    w.params.tau_w = 1e-4
    _, Kf, _ = O.walk_scores(w.problem, w.params, w.points, 3)
    _, Kr, _ = O.walk_scores(w.problem, _reduced(w).params, w.points, 3)
    assert np.all(Kf == Kr) and np.all(Kf == Kf.flat[0])


@pytest.mark.parametrize("case", ["hemisphere", "embedded"])
def test_reduced_matches_full_oracle_statistically(case):
    if case == "hemisphere":
        w = W.hypersphere_half(P=3, walks=1, n=64, seed=3)
        N = 800
    else:
        w = W.embedded_s20(P=3, walks=1, n=64, d=5, sigma=6.0)
        w.params.tau_w = 1e-4
        N = 500
    mf, sf, tf, _ = O.solve(w.problem, w.params, w.points, N)
    mr, sr, tr, _ = O.solve(w.problem, _reduced(w).params, w.points, N)
    assert np.all(np.abs(mf - mr) < 4 * np.sqrt(sf ** 2 + sr ** 2))
    assert np.all(np.abs(tf - tr) < 0.1 * tf + 5)
    assert np.all(np.abs(mr - w.exact) < 4 * sr + 0.03)
