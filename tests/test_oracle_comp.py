"""Pins of the oracle's torus boundary (a plane through the axis, Example 1's cut) and of
the compensation term m_* (Sec. 2.3.3), each against something other than the oracle:

* delta_Gamma on the cut torus against brute force: the nearest point of Gamma by dense
  sampling of both meridian circles, then the distance to the normal segment of
  eq. extended_boundary_disk by dense sampling of the segment;
* R_*(s; y) against an ambient 7-point finite-difference Laplacian of u_* o cp at y + s n(y)
  (the oracle's closed forms in toroidal / spherical coordinates are not used there);
* R_*(0; y) = 0 when u_* = u (m vanishes on M, since f = (-Delta_M + sigma) u);
* the second-order expansion's error against the exact m falls like eta^3;
* a constant predictor gives m_* = 0 and walks identical to the baseline method.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2606_21883_b300 import workloads as W


def _e1(comp=W.COMP_NORMAL2, u_star=None):
    w = W.torus_cut(P=4, walks=1, comp=comp, u_star=u_star)
    return w, O.OracleProblem(w.problem, w.params)


def _torus_point(th, ph, R=1.0, a=0.45):
    return W.torus_points(np.array([th]), np.array([ph]), R, a)[0]


def _brute_delta(y, e, R, a, ell, n=200001):
    t = np.linspace(0.0, 2 * math.pi, n)
    best = (np.inf, None, None)
    for sgn in (1.0, -1.0):
        u = sgn * np.array([-e[1], e[0], 0.0])
        c = R * u
        nb = np.cos(t)[:, None] * u[None, :] + np.sin(t)[:, None] * np.array([0.0, 0.0, 1.0])[None, :]
        q = c[None, :] + a * nb
        d2 = np.sum((q - y) ** 2, axis=1)
        j = int(np.argmin(d2))
        if d2[j] < best[0]:
            best = (d2[j], q[j], nb[j])
    _, yg, nrm = best
    tau = np.linspace(-ell, ell, n)
    seg = yg[None, :] + tau[:, None] * nrm[None, :]
    return float(np.min(np.linalg.norm(seg - y, axis=1))), yg


def test_torus_cut_delta_gamma_brute_force():
    w, op = _e1(W.COMP_NONE)
    e = w.problem.bnd_normal
    ell = w.params.c_kappa / (1.0 + 1.0 / 0.45)
    rng = np.random.default_rng(2)
    phc = W.E1_PHI_C
    cases = [(rng.uniform(0, 2 * math.pi), phc + rng.uniform(0.01, math.pi - 0.01)) for _ in range(12)]
    cases += [(rng.uniform(0, 2 * math.pi), phc + s) for s in (1e-3, 0.05, math.pi - 0.02, math.pi - 1e-3)]
    for th, ph in cases:
        y = _torus_point(th, ph)
        d, yg = O.delta_gamma(op, y)
        db, ygb = _brute_delta(y, e, 1.0, 0.45, ell)
        assert d == pytest.approx(db, abs=1e-5), (th, ph)
        assert np.linalg.norm(yg - ygb) < 1e-4
    # outside Omega (phi - phi_c in (pi, 2 pi)): inside the boundary layer
    for s in (math.pi + 0.3, 1.5 * math.pi):
        d, _ = O.delta_gamma(op, _torus_point(0.7, phc + s))
        assert d == 0.0


def _stencil_neg_lap(op, x, h=1e-4):
    def F(z):
        return O.func_eval(op, "u_star", O.cp(op, z))
    c = F(x)
    acc = 0.0
    for i in range(3):
        d = np.zeros(3)
        d[i] = h
        acc += F(x + d) - 2 * c + F(x - d)
    return -acc / h ** 2


def _normal(kind, y, R=1.0):
    if kind == "torus":
        c = R * np.array([y[0], y[1], 0.0]) / math.hypot(y[0], y[1])
        v = y - c
        return v / np.linalg.norm(v)
    return y / np.linalg.norm(y)


def _cap_comp(comp=W.COMP_NORMAL2):
    w = W.sphere_cap(P=4, walks=1)
    A = np.zeros((3, 3))
    A[0, 1] = A[1, 0] = 0.5
    w.problem.comp = comp
    w.problem.u_star = W.Func.sphere_quad(0.0, np.array([0.0, 0.0, 1.0]), A, apply_op=False)   # u = xy + z
    return w, O.OracleProblem(w.problem, w.params)


@pytest.mark.parametrize("kind", ["torus", "sphere"])
def test_comp_R_matches_ambient_stencil(kind):
    """R_*(s; y) = -Delta(E u_*)(y + s n) + sigma u_*(y) - f(y), the Laplacian by finite differences."""
    w, op = _e1() if kind == "torus" else _cap_comp()
    rng = np.random.default_rng(5)
    for _ in range(6):
        if kind == "torus":
            y = _torus_point(rng.uniform(0, 2 * math.pi), W.E1_PHI_C + rng.uniform(0.1, 3.0))
        else:
            y = W.sphere_cap_points(1, int(rng.integers(1000)))[0]
        n = _normal(kind, y)
        fy = O.func_eval(op, "f", y)
        uy = O.func_eval(op, "u_star", y)
        for s in (-0.2, -0.05, 0.0, 0.1, 0.25):
            want = _stencil_neg_lap(op, y + s * n) + w.problem.sigma * uy - fy
            assert O.comp_R(op, y, s) == pytest.approx(want, rel=1e-5, abs=1e-4), (y, s)
            assert O.normal_coord(op, y + s * n) == pytest.approx(s, abs=1e-12)


@pytest.mark.parametrize("kind", ["torus", "sphere"])
def test_mismatch_vanishes_on_M_for_the_exact_predictor(kind):
    w, op = _e1() if kind == "torus" else _cap_comp()
    rng = np.random.default_rng(7)
    for _ in range(10):
        if kind == "torus":
            y = _torus_point(rng.uniform(0, 2 * math.pi), rng.uniform(0, 2 * math.pi))
        else:
            y = W.sphere_cap_points(1, int(rng.integers(1000)))[0]
        assert abs(O.comp_R(op, y, 0.0)) < 1e-11


@pytest.mark.parametrize("kind", ["torus", "sphere"])
def test_second_order_expansion_error_is_third_order(kind):
    """|m_*(y + eta n) - m(y + eta n)| = O(eta^3), m from the stencil: halving eta divides the
    error by about 8."""
    w, op = _e1() if kind == "torus" else _cap_comp()
    rng = np.random.default_rng(11)
    ratios = []
    for _ in range(4):
        if kind == "torus":
            y = _torus_point(rng.uniform(0, 2 * math.pi), W.E1_PHI_C + rng.uniform(0.3, 2.8))
        else:
            y = W.sphere_cap_points(1, int(rng.integers(1000)))[0]
        n = _normal(kind, y)
        fy = O.func_eval(op, "f", y)
        uy = O.func_eval(op, "u_star", y)
        errs = []
        for eta in (0.08, 0.04):
            x = y + eta * n
            m_exact = _stencil_neg_lap(op, x) + w.problem.sigma * uy - fy
            errs.append(abs(O.comp_m(op, x) - m_exact))
        assert errs[1] < 0.05 * abs(m_exact) + 1e-6
        ratios.append(errs[0] / errs[1])
    assert 5.0 < np.median(ratios) < 11.0, ratios


def test_exact_mode_is_the_mismatch():
    w, op = _e1(W.COMP_EXACT)
    y = _torus_point(0.4, W.E1_PHI_C + 1.0)
    x = y + 0.2 * _normal("torus", y)
    want = _stencil_neg_lap(op, x) + w.problem.sigma * O.func_eval(op, "u_star", y) - O.func_eval(op, "f", y)
    assert O.comp_m(op, x) == pytest.approx(want, rel=1e-5, abs=1e-4)


def test_constant_predictor_gives_the_baseline_walk():
    """u_* = 0.7: -Delta(E u_*) = 0, so R_* is the same at every s and m_* = 0 (the
    sigma u_* - f part cancels in both differences); walks equal the baseline method's."""
    const = W.Func.torus([(0.7, 0, 0, W.TRIG_COS, W.TRIG_COS)], apply_op=False)
    w, op = _e1(W.COMP_NORMAL2, const)
    y = _torus_point(1.0, W.E1_PHI_C + 0.5)
    assert abs(O.comp_m(op, y + 0.2 * _normal("torus", y))) < 1e-9
    w.params.max_steps = 200
    S1, K1, F1 = O.walk_scores(w.problem, w.params, w.points, 16)
    base = W.torus_cut(P=4, walks=1)
    base.params.max_steps = 200
    S0, K0, F0 = O.walk_scores(base.problem, base.params, base.points, 16)
    assert np.array_equal(K1, K0) and np.array_equal(F1, F0)
    assert np.all(np.abs(S1 - S0) <= 1e-9)


def test_torus_cut_dirichlet_zero_on_gamma():
    """u = 0 on both cut circles (the example's homogeneous Dirichlet data)."""
    th = np.linspace(0, 2 * math.pi, 7)
    for ph in (W.E1_PHI_C, W.E1_PHI_C + math.pi):
        assert np.all(np.abs(W.torus_series_value(W.torus_cut_terms(), th, np.full_like(th, ph))) < 1e-12)


def test_rejected_forms():
    w = W.torus_cut(P=2, walks=1)
    w.problem.bnd_normal = np.array([0.0, 0.6, 0.8])   # not a plane through the axis
    with pytest.raises(ValueError):
        O.walk_scores(w.problem, w.params, w.points, 2)
    w = W.hypersphere_half(P=2, walks=1, n=8)
    w.problem.comp = W.COMP_NORMAL2
    w.problem.u_star = W.Func.const(1.0)
    with pytest.raises(ValueError):
        O.walk_scores(w.problem, w.params, w.points, 2)


def test_compensation_reduces_e1_bias():
    """Example 1 at 6000 walks per point on 3 points (common random numbers in both runs):
    the exact mismatch leaves the estimate unbiased (within 4 standard errors) where the
    baseline is off by many; the second-order m_* lies in between."""
    errs = {}
    for comp in (W.COMP_NONE, W.COMP_NORMAL2, W.COMP_EXACT):
        w = W.torus_cut(P=3, walks=1, comp=comp, seed=1)
        m, se, _, nf = O.solve(w.problem, w.params, w.points, 6000)
        assert nf == 0
        errs[comp] = (m - w.exact, se)
    e0, se0 = errs[W.COMP_NONE]
    e2, se2 = errs[W.COMP_EXACT]
    e1, _ = errs[W.COMP_NORMAL2]
    assert np.all(np.abs(e2) < 4 * se2 + 1e-3)
    assert np.sqrt(np.mean(e0 ** 2)) > 3 * np.sqrt(np.mean(e2 ** 2)) + 0.01
    assert np.sqrt(np.mean(e1 ** 2)) < 0.7 * np.sqrt(np.mean(e0 ** 2))

