"""Pins of the oracle's point-cloud closest point (Sec. 2.1 representation
(iii), eq. rho_geo_spacing): neighbours against a k-d tree, the fitted
projection against the analytic surface the cloud samples, and the exact
telescoping identity of f = sigma on the cloud manifold."""
import numpy as np
import pytest
from scipy.optimize import minimize
from scipy.spatial import cKDTree

import oracle as O
from paper_2606_21883_b300 import workloads as W


@pytest.fixture(scope="module")
def cloud():
    w = W.point_cloud(P=4, walks=1, N_cloud=30000)
    return w, O.OracleProblem(w.problem, w.params)


def test_knn_matches_kdtree(cloud):
    w, op = cloud
    cl = w.problem.manifold.cloud
    tree = cKDTree(cl)
    rng = np.random.default_rng(0)
    for _ in range(20):
        x = cl[rng.integers(len(cl))] + 0.02 * rng.standard_normal(3)
        idx, d2, h = O.cloud_knn(op, x)
        dd, ii = tree.query(x, k=16)
        assert ii.tolist() == idx.tolist()
        assert np.allclose(np.sqrt(d2), dd, rtol=1e-12)
        assert h == pytest.approx(dd.mean(), rel=1e-12)


def _analytic_cp(x, alpha):
    def f(th):
        w = np.array([np.sin(th[0]) * np.cos(th[1]), np.sin(th[0]) * np.sin(th[1]), np.cos(th[0])])
        return np.sum((W.perturbed_sphere_radius(w[None], alpha)[0] * w - x) ** 2)
    wx = x / np.linalg.norm(x)
    res = minimize(f, [np.arccos(wx[2]), np.arctan2(wx[1], wx[0])], method="Nelder-Mead",
                   options=dict(xatol=1e-12, fatol=1e-22, maxiter=8000))
    th = res.x
    w = np.array([np.sin(th[0]) * np.cos(th[1]), np.sin(th[0]) * np.sin(th[1]), np.cos(th[0])])
    return W.perturbed_sphere_radius(w[None], alpha)[0] * w


def test_fit_projection_close_to_analytic_surface(cloud):
    w, op = cloud
    cl = w.problem.manifold.cloud
    alpha = W.perturbed_sphere_coeffs(0)
    rng = np.random.default_rng(1)
    fit_err, nn_err = [], []
    for _ in range(8):
        x = cl[rng.integers(len(cl))] + 0.01 * rng.standard_normal(3)
        ya = _analytic_cp(x, alpha)
        fit_err.append(np.linalg.norm(O.cp(op, x) - ya))
        idx, _, _ = O.cloud_knn(op, x)
        nn_err.append(np.linalg.norm(cl[idx[0]] - ya))
    assert max(fit_err) < 1e-4 and max(fit_err) < 0.05 * np.mean(nn_err)


def test_cloud_telescoping(cloud):
    w, op = cloud
    w.params.max_steps = 100000
    w.params.tau_w = 1e-3
    S, K, fl = O.walk_scores(w.problem, w.params, w.points[:2], 2)
    assert not fl.any()
    # closed case, f = sigma: S = 1 - W_K with W_K < tau_W <= W_{K-1}
    assert np.all((S > 1 - 1e-3) & (S <= 1 + 1e-12))


# ---------------------------------------------------------------- Example 4
@pytest.fixture(scope="module")
def e4():
    w = W.sphere_cloud_legendre(P=6, walks=1)
    return w, O.OracleProblem(w.problem, w.params)


def test_e4_source_is_the_screened_laplacian_of_u():
    """f = (-Delta_S + sigma) u on S^2, checked by finite differences of u in the polar angle
    (u depends on x_3 = cos t only: Delta_S u = u'' + cot t u')."""
    w = W.sphere_cloud_legendre(P=1, walks=1, N_cloud=100)
    cu = [0.0, 1.0, 0.0, 0.2, 0.0, 0.1]
    u = lambda t: np.polynomial.legendre.legval(np.cos(t), cu)
    op = O.OracleProblem(w.problem, w.params)
    for t in [0.3, 1.1, 1.9, 2.7]:
        h = 1e-4
        d1 = (u(t + h) - u(t - h)) / (2 * h)
        d2 = (u(t + h) - 2 * u(t) + u(t - h)) / h ** 2
        x = np.array([np.sin(t), 0.0, np.cos(t)])
        want = -(d2 + d1 / np.tan(t)) + w.problem.sigma * u(t)
        assert O.func_eval(op, "f", x) == pytest.approx(want, rel=1e-6, abs=1e-6)


def test_e4_nearest_cp_is_the_nearest_cloud_point(e4):
    w, op = e4
    cl = w.problem.manifold.cloud
    tree = cKDTree(cl)
    rng = np.random.default_rng(3)
    for _ in range(30):
        x = cl[rng.integers(len(cl))] + 0.05 * rng.standard_normal(3)
        _, j = tree.query(x, k=1)
        assert np.array_equal(O.cp(op, x), cl[j])


def test_e4_walk_mean_matches_legendre_solution(e4):
    """Example 4 at 300 walks per point: mean within 4 standard errors (+0.02 for the bias of the
    nearest-point projection) of u = P_1 + 0.2 P_3 + 0.1 P_5."""
    w, _ = e4
    m, se, ms, nf = O.solve(w.problem, w.params, w.points, 300)
    assert nf == 0 and np.all(ms > 500)
    assert np.all(np.abs(m - w.exact) <= 4 * se + 0.02), (m, w.exact, se)
