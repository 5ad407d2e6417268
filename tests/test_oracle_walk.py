"""Walk-level pins of the oracle (Algorithm 1, eq. path_score_definition).

Exact identities that a dropped term, a wrong sign, an off-by-one in the weight
update or a mis-drawn interior sample would break:
  * f = sigma, g = 1 has the solution u = 1 and every path score telescopes:
    S = 1 (boundary), S = 1 - W_K (closed);
  * constant radius on the torus makes the stopping index deterministic,
    K = ceil(ln tau_W / ln c) with c = a / sinh a;
  * in M = R^n (cp = identity, so the compensation term vanishes) the
    estimator is unbiased up to the epsilon-layer, checked against closed-form
    solutions, including a non-harmonic one that weighs the Green sample;
  * the manufactured S^2 cap stays within its stated error floor.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2606_21883_b300 import workloads as W


def test_telescoping_boundary_case():
    w = W.constant_solution(W.sphere_cap(P=6, walks=1))
    S, K, fl = O.walk_scores(w.problem, w.params, w.points, 40)
    assert not fl.any()
    assert np.all(np.abs(S - 1.0) <= 1e-13 * np.maximum(K, 1))


def test_telescoping_closed_case_and_deterministic_K():
    w = W.constant_solution(W.torus_closed(P=3, walks=1))
    S, K, fl = O.walk_scores(w.problem, w.params, w.points, 8)
    r = 0.95 * 1.2 / (1.0 + 1.0 / 0.4)
    a = math.sqrt(2.0) * r
    c = a / math.sinh(a)
    Kexp = math.ceil(math.log(1e-8) / math.log(c))
    assert Kexp == 525
    assert np.all(K == Kexp)
    assert np.allclose(S, 1.0 - c ** Kexp, rtol=0, atol=1e-12)
    assert np.all((S > 1 - 1e-8) & (S <= 1.0))


def test_deterministic_K_embedded_sphere_against_bessel():
    """Constant radius on an embedded unit sphere: K = ceil(ln tau_W / ln c),
    c from its Bessel definition (eq. def_c_sigma_r, mpmath)."""
    import mpmath as mp
    n, d, sigma = 40, 5, 2.0
    w = W.embedded_s20(P=2, walks=1, n=n, d=d, sigma=sigma)
    w.params.tau_w = 1e-3
    r = 0.95 * 1.2 / 2.0
    nu = (n - 2) / 2
    a = mp.sqrt(sigma) * r
    c = float(a ** nu / (2 ** nu * mp.gamma(nu + 1) * mp.besseli(nu, a)))
    Kexp = math.ceil(math.log(1e-3) / math.log(c))
    S, K, fl = O.walk_scores(w.problem, w.params, w.points, 2)
    assert np.all(K == Kexp)


def test_max_steps_flags_and_partial_score():
    w = W.torus_closed(P=2, walks=1)
    w.params.max_steps = 7
    S, K, fl = O.walk_scores(w.problem, w.params, w.points, 3)
    assert np.all(K == 7) and np.all(fl == 1)
    w.params.max_steps = 10_000_000
    S2, K2, fl2 = O.walk_scores(w.problem, w.params, w.points, 3)
    assert np.all(fl2 == 0) and not np.allclose(S, S2)


def test_thread_count_invariance_and_stream_independence():
    w = W.sphere_cap(P=4, walks=1)
    S1, K1, _ = O.walk_scores(w.problem, w.params, w.points, 16, n_threads=1)
    S8, K8, _ = O.walk_scores(w.problem, w.params, w.points, 16, n_threads=8)
    assert np.array_equal(S1, S8) and np.array_equal(K1, K8)
    assert len(np.unique(S1)) == S1.size
    w.params.seed = 99
    S3, _, _ = O.walk_scores(w.problem, w.params, w.points, 16)
    assert not np.any(S3 == S1)


def _euclid(f, g, exact, sigma=1.0, P=6, N=1500, seed=0):
    w = W.euclid_halfspace(P=P, walks=N, sigma=sigma, seed=seed)
    w.params.c_kappa = 1e3       # kappa = 0 in R^n: rho_geo = c_kappa, keep the ball rule r = theta dist
    w.problem.f, w.problem.g = f, g
    m, se, ms, nf = O.solve(w.problem, w.params, w.points, N)
    u = exact(w.points)
    return m, se, u, ms


def test_euclid_exponential_solution():
    """-Delta u + sigma u = 0, u = exp(-sqrt(sigma) x_1), g = 1 on x_1 = 0."""
    m, se, u, ms = _euclid(W.Func.const(0.0), W.Func.const(1.0),
                           lambda x: np.exp(-np.sqrt(2.0) * x[:, 0]), sigma=2.0)
    assert np.all(np.abs(m - u) <= 4 * se + 2e-3)


def test_euclid_quadratic_solution_weighs_green_sample():
    """u = |x|^2 in R^3: f = -6 + sigma |x|^2 is not harmonic, so the source term
    sum W_k omega_k f(Z_{k+1}) carries the second moment of the Green sample."""
    sigma = 3.0
    f = W.Func.poly([(-6.0, []), (sigma, [(0, 2)]), (sigma, [(1, 2)]), (sigma, [(2, 2)])])
    g = W.Func.poly([(1.0, [(0, 2)]), (1.0, [(1, 2)]), (1.0, [(2, 2)])])
    m, se, u, ms = _euclid(f, g, lambda x: np.sum(x * x, axis=1), sigma=sigma, P=5, N=1500, seed=3)
    assert np.all(np.abs(m - u) <= 4 * se + 5e-3)


def test_manufactured_cap_error_floor():
    """S^2 cap, u = xy + z: the baseline (m_* = 0) estimator has a bias floor
    (Sec. 4, Example 1); stated floor: |error| <= 4 se + 0.04."""
    w = W.sphere_cap(P=8, walks=600)
    m, se, ms, nf = O.solve(w.problem, w.params, w.points, w.walks)
    assert nf == 0
    assert np.all(np.abs(m - w.exact) <= 4 * se + 0.04)


def test_trace_tiny_case():
    """One walk, step by step: W_{k+1} = W_k c_k, the radius rule, points on M."""
    w = W.sphere_cap(P=1, walks=1)
    rows, S, K = O.trace(w.problem, w.params, w.points[0])
    assert len(rows) == K and K > 0
    Wp = 1.0
    for rec in rows:
        assert rec["W"] == Wp * rec["c"]
        Wp = rec["W"]
        assert rec["r"] == pytest.approx(0.95 * min(rec["delta_gamma"], 0.6))
        assert abs(np.linalg.norm(rec["y"]) - 1) < 1e-14
        assert 0 < rec["t0"] < 1
        assert rec["omega"] == pytest.approx((1 - rec["c"]) / 1.0, rel=1e-9)
