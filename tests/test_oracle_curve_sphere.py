"""Pins of the oracle's Fourier curve x S^2(a) in R^9 (Example 3), each against something
other than the oracle:

* the Newton closest point on the curve against brute force over a dense phi grid, the
  sphere factor against normalisation, the residual normal to M, idempotence;
* the curvature indicator against the curvature of the curve by finite differences;
* f = (-Delta_M + sigma) u against the ambient finite-difference Laplacian of u o cp at
  points of M (on M the Laplacian of the closest-point extension is Delta_M u);
* the constant solution's telescoping, and a walk against u.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2606_21883_b300 import workloads as W


def _op(P=4, seed=0):
    w = W.curve_sphere(P=P, walks=1, seed=seed)
    return w, O.OracleProblem(w.problem, w.params)


def test_cp_against_brute_force():
    w, op = _op()
    rng = np.random.default_rng(1)
    phs = np.linspace(0.0, 2 * math.pi, 2000001)
    Cg = W.fourier_curve(phs)
    for _ in range(10):
        y = w.points[rng.integers(len(w.points))]
        x = y + 0.25 * rng.standard_normal(9) / 3.0
        c = O.cp(op, x)
        j = int(np.argmin(np.sum((Cg - x[:6]) ** 2, axis=1)))
        assert np.linalg.norm(c[:6] - Cg[j]) < 1e-5
        assert np.allclose(c[6:], 0.65 * x[6:] / np.linalg.norm(x[6:]), atol=1e-15)
        ph = O.curve_cp_phi(op, x)
        C1 = np.array([-math.sin(ph), math.cos(ph), -math.sin(2 * ph), math.cos(2 * ph), -math.sin(3 * ph),
                       math.cos(3 * ph)])
        assert abs(np.dot(x[:6] - c[:6], C1)) < 1e-10        # residual normal to the curve
        assert np.allclose(O.cp(op, c), c, atol=1e-13)


def test_curvature_indicator():
    w, op = _op()
    h = 1e-4
    for ph in (0.0, 0.7, 2.0, 4.1):
        C = W.fourier_curve(np.array([ph - h, ph, ph + h]))
        d1 = (C[2] - C[0]) / (2 * h)
        d2 = (C[2] - 2 * C[1] + C[0]) / h ** 2
        kc = math.sqrt(np.dot(d1, d1) * np.dot(d2, d2) - np.dot(d1, d2) ** 2) / np.dot(d1, d1) ** 1.5
        assert O.kappa_at(op, w.points[0]) == pytest.approx(max(kc, 1 / 0.65), rel=1e-6)


def _stencil_neg_lap(op, x, h=1e-4):
    def F(z):
        return O.func_eval(op, "u_star", O.cp(op, z))
    c = F(x)
    acc = 0.0
    for i in range(9):
        d = np.zeros(9)
        d[i] = h
        acc += F(x + d) - 2 * c + F(x - d)
    return -acc / h ** 2


def test_source_is_the_screened_laplace_beltrami():
    w, _ = _op(P=6, seed=3)
    prob = w.problem
    f = prob.f
    prob.comp = W.COMP_NORMAL2        # only to marshal u (apply_op = 0) as the oracle's u_star
    prob.u_star = W.Func(kind=f.kind, apply_op=0, coef=f.coef, modes=f.modes, v=f.v, A=f.A)
    op = O.OracleProblem(prob, w.params)
    for y, u in zip(w.points, w.exact):
        assert O.func_eval(op, "u_star", y) == pytest.approx(u, rel=1e-12, abs=1e-14)
        want = _stencil_neg_lap(op, y) + prob.sigma * u
        assert O.func_eval(op, "f", y) == pytest.approx(want, rel=2e-5, abs=2e-4)


def test_constant_solution_telescopes():
    w, _ = _op(P=2)
    w.problem.f = W.Func.curve_sphere([(0, W.TRIG_COS, 1.0, np.zeros(3), np.zeros((3, 3)))], apply_op=True)
    S, K, F = O.walk_scores(w.problem, w.params, w.points, 4)
    assert not F.any()
    assert np.all((S > 1 - w.params.tau_w - 1e-12 * K) & (S <= 1 + 1e-12 * K))


def test_walk_mean_matches_u():
    """Example 3 at 500 walks per point: within 4 standard errors (+0.03 for the baseline
    method's bias, m_* = 0)."""
    w, _ = _op(P=3, seed=2)
    m, se, ms, nf = O.solve(w.problem, w.params, w.points, 500)
    assert nf == 0
    assert np.all(np.abs(m - w.exact) < 4 * se + 0.03), (m, w.exact, se)
