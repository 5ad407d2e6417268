"""Pins of the oracle's hypersurface of revolution (Example 2's dumbbell), each against
something other than the oracle:

* the profile's derivatives against central differences of R(t);
* the Newton closest point against brute force over a dense profile grid, and its
  residual x - cp(x) normal to M (orthogonal to the profile tangent in the meridian plane);
* the curvature indicator against the curvature of the profile curve by finite differences
  and the parallel curvature 1 / (R sqrt(1 + R'^2));
* f = (-Delta_M + sigma) u against the ambient finite-difference Laplacian of u o cp at
  points of M (on M the Laplacian of the closest-point extension is Delta_M u);
* a walk on a small dumbbell against the exact solution.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2606_21883_b300 import workloads as W


def _op(n=7, seed=0):
    w = W.dumbbell(P=4, walks=1, n=n, seed=seed)
    return w, O.OracleProblem(w.problem, w.params)


def test_profile_derivatives():
    w, op = _op()
    for t in (-1.0, -0.5, 0.0, 0.3, 0.9, 1.1):
        R, R1, R2 = O.profile(op, t)
        assert R == pytest.approx(W.dumbbell_profile(t), rel=1e-14)
        h = 1e-5
        assert R1 == pytest.approx((W.dumbbell_profile(t + h) - W.dumbbell_profile(t - h)) / (2 * h), rel=1e-7, abs=1e-8)
        assert R2 == pytest.approx((W.dumbbell_profile(t + h) - 2 * R + W.dumbbell_profile(t - h)) / h ** 2,
                                   rel=1e-4, abs=1e-4)


@pytest.mark.parametrize("n", [5, 1001])
def test_newton_cp_against_brute_force(n):
    w, op = _op(n)
    rng = np.random.default_rng(n)
    tg = np.linspace(-1.2 * (1 - 1e-9), 1.2 * (1 - 1e-9), 400001)
    Rg = W.dumbbell_profile(tg)
    for _ in range(12):
        y = w.points[rng.integers(len(w.points))]
        x = y + 0.3 * rng.standard_normal(n) / math.sqrt(n) * rng.uniform(0.2, 1.5)
        c = O.cp(op, x)
        rho0 = np.linalg.norm(x[:-1])
        j = int(np.argmin((Rg - rho0) ** 2 + (tg - x[-1]) ** 2))
        assert c[-1] == pytest.approx(tg[j], abs=2e-5)
        assert np.linalg.norm(c[:-1]) == pytest.approx(W.dumbbell_profile(c[-1]), rel=1e-12)
        # residual normal to M: orthogonal to the meridian tangent (R' w, 1)
        _, R1, _ = O.profile(op, c[-1])
        wv = c[:-1] / np.linalg.norm(c[:-1])
        tangent = np.concatenate([R1 * wv, [1.0]])
        assert abs(np.dot(x - c, tangent)) < 1e-10 * (1 + np.linalg.norm(x - c))
        assert np.allclose(O.cp(op, c), c, atol=1e-13)


def test_curvature_indicator():
    w, op = _op()
    for t in (-0.9, -0.2, 0.0, 0.5, 0.95):
        y = np.zeros(7)
        y[0] = W.dumbbell_profile(t)
        y[-1] = t
        h = 1e-4
        r = W.dumbbell_profile(np.array([t - h, t, t + h]))
        d1 = (r[2] - r[0]) / (2 * h)
        d2 = (r[2] - 2 * r[1] + r[0]) / h ** 2
        k_mer = abs(d2) / (1 + d1 * d1) ** 1.5      # curvature of the plane curve (R(t), t)
        k_par = 1.0 / (r[1] * math.sqrt(1 + d1 * d1))
        assert O.kappa_at(op, y) == pytest.approx(max(k_mer, k_par), rel=1e-5)


def _stencil_neg_lap(op, x, h=1e-4):
    def F(z):
        return O.func_eval(op, "u_star", O.cp(op, z))
    c = F(x)
    acc = 0.0
    for i in range(len(x)):
        d = np.zeros(len(x))
        d[i] = h
        acc += F(x + d) - 2 * c + F(x - d)
    return -acc / h ** 2


@pytest.mark.parametrize("n", [5, 12])
def test_source_is_the_screened_laplace_beltrami(n):
    w, _ = _op(n, seed=3)
    f = w.problem.f
    prob = w.problem
    prob.comp = W.COMP_NORMAL2          # only to marshal u (apply_op = 0) as the oracle's u_star
    prob.u_star = W.Func.revolution_quad(f.coef[0], f.coef[1], f.v, f.A, apply_op=False)
    op = O.OracleProblem(prob, w.params)
    for y in w.points:
        want = _stencil_neg_lap(op, y) + prob.sigma * O.func_eval(op, "u_star", y)
        assert O.func_eval(op, "f", y) == pytest.approx(want, rel=2e-5, abs=2e-4)


def test_u_matches_the_workload_solution():
    w, op = _op(1001)
    prob = w.problem
    f = prob.f
    prob.comp = W.COMP_NORMAL2
    prob.u_star = W.Func.revolution_quad(f.coef[0], f.coef[1], f.v, f.A, apply_op=False)
    op = O.OracleProblem(prob, w.params)
    for y, u in zip(w.points, w.exact):
        assert O.func_eval(op, "u_star", y) == pytest.approx(u, rel=1e-12, abs=1e-14)


def test_small_dumbbell_walk_mean():
    """R^5 dumbbell (sigma = 8): the walk's mean against u within 4 standard errors plus the
    baseline method's bias (m_* = 0), 0.03 at this radius."""
    w, _ = _op(5, seed=1)
    m, se, ms, nf = O.solve(w.problem, w.params, w.points, 1500)
    assert nf == 0 and np.all(ms > 5)
    assert np.all(np.abs(m - w.exact) < 4 * se + 0.03), (m, w.exact, se)


def test_constant_solution_telescopes():
    """u = 1 (c0 = 1, f = sigma): S = 1 - W_K exactly, W_K < tau_W."""
    w, _ = _op(1001, seed=5)
    f = w.problem.f
    w.problem.f = W.Func.revolution_quad(0.0, 0.0, np.zeros_like(f.v), np.zeros_like(f.A), apply_op=True, c0=1.0)
    S, K, F = O.walk_scores(w.problem, w.params, w.points[:2], 6)
    assert not F.any()
    assert np.all((S > 1 - w.params.tau_w - 1e-12 * K) & (S <= 1 + 1e-12 * K))
