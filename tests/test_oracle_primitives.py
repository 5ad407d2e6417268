"""Pins of the oracle's primitives against what the paper and the mathematics fix.

None of these compare the oracle with itself: Philox against the published
known-answer vectors, c_{sigma,r} / omega / the radial CDF against mpmath
quadrature of the paper's Green function (golden file), closed forms, limits
and brute force.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2606_21883_b300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLD, name)) as fh:
        return [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]


# --------------------------------------------------------------------- Philox
def test_philox_known_answers():
    for r in _rows("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in r]
        assert O.philox(v[0:4], v[4:6]) == v[6:10]


def test_u53_range_and_exactness():
    assert O.u53(0, 0) == 2.0 ** -53
    assert O.u53(0xFFFFFFFF, 0xFFFFFFFF) == 1.0
    # 2^53 distinct values: the low 11 bits of lo are dropped
    assert O.u53(0, 0x7FF) == O.u53(0, 0)
    assert O.u53(0, 0x800) == 2 * 2.0 ** -53


def test_box_muller_moments():
    g = np.concatenate([O.gaussians(7, 0, k, 0, 0, 2000) for k in range(100)])  # 2e5 draws
    n = g.size
    assert abs(g.mean()) < 5 / math.sqrt(n)
    assert abs(g.var() - 1) < 5 * math.sqrt(2 / n)
    assert abs(np.mean(g ** 4) - 3) < 5 * math.sqrt(96 / n)
    # distribution function at a few quantiles (Kolmogorov-type bound)
    for q in (-1.5, -0.5, 0.0, 0.7, 2.0):
        emp = np.mean(g <= q)
        ref = 0.5 * (1 + math.erf(q / math.sqrt(2)))
        assert abs(emp - ref) < 5 * math.sqrt(ref * (1 - ref) / n)


def test_direction_isotropy():
    """E[zeta zeta^T] = I/n for zeta = g/|g| (uniform on S^{n-1}, Sec. 2.3.2)."""
    n = 3
    Z = np.array([O.gaussians(3, 0, k, i, 0, n) for k in range(200) for i in range(100)])
    Z /= np.linalg.norm(Z, axis=1, keepdims=True)
    M = Z.T @ Z / len(Z)
    assert np.allclose(M, np.eye(n) / n, atol=5 * math.sqrt(2 / len(Z)) / n + 2e-3)


# ----------------------------------------------------------- c, omega, CDF
def test_c_sigma_r_n3_closed_form():
    """n = 3: I_{1/2} is elementary and c = a / sinh a (eq. def_c_sigma_r)."""
    for a in (1e-3, 0.05, 0.4606, 1.0, 3.0, 10.0):
        assert O.c_sigma_r(3, a) == pytest.approx(a / math.sinh(a), rel=1e-14)


def test_c_sigma_r_bound_lemma_3_1():
    """c <= (1 + sigma r^2 / (2n))^{-1} (eq. uniform_screened_weight)."""
    for n in (3, 4, 21, 1000):
        for a in (0.01, 0.3, 1.0, 5.0):
            assert O.c_sigma_r(n, a) <= 1.0 / (1.0 + a * a / (2 * n)) * (1 + 1e-15)


def test_green_quantities_against_quadrature():
    rows = _rows("green_quadrature.txt")
    assert len(rows) >= 60
    for r in rows:
        n, sigma, rad, t, c, omega, F = int(r[0]), *map(float, r[1:])
        a = math.sqrt(sigma) * rad
        assert O.c_sigma_r(n, a) == pytest.approx(c, rel=1e-13)
        em1 = O.em1(n, a)
        om = (em1 / (1 + em1)) / sigma          # omega = (1 - c)/sigma (Thm 2.2)
        assert om == pytest.approx(omega, rel=1e-10)
        assert O.green_cdf(n, a, t) == pytest.approx(F, rel=1e-12, abs=1e-15)


def test_green_cdf_endpoints_and_laplace_limit():
    for n in (3, 4, 7, 1000):
        nu = (n - 2) / 2
        for a in (1e-4, 0.2, 1.0):
            assert O.green_cdf(n, a, 1 - 1e-13) == pytest.approx(1.0, abs=1e-11)
            # F is increasing
            ts = np.linspace(0.01, 0.99, 40)
            Fs = [O.green_cdf(n, a, t) for t in ts]
            assert np.all(np.diff(Fs) > 0)
        # sigma -> 0: F -> (n t^2 - 2 t^n)/(n - 2), the Laplace Green density
        for t in (0.1, 0.5, 0.9):
            lim = (n * t * t - 2 * t ** n) / (n - 2)
            assert O.green_cdf(n, 1e-5, t) == pytest.approx(lim, rel=1e-8)


def test_green_cdf_n3_remark_closed_form():
    """n = 3: G = sinh(lam (r - rho)) / (4 pi rho sinh(lam r)) (Remark, n = 3);
    F(t) by Simpson quadrature of rho^2 G, independent of the oracle's series."""
    lam, r = math.sqrt(2.0), 0.3257142857142857
    G = lambda rho: math.sinh(lam * (r - rho)) / (4 * math.pi * rho * math.sinh(lam * r))
    s = np.linspace(1e-12, r, 200001)
    dens = s * s * np.array([G(x) for x in s])
    cum = np.concatenate([[0], np.cumsum((dens[1:] + dens[:-1]) / 2 * np.diff(s))])
    for t in (0.2, 0.5, 0.8):
        idx = int(round(t * (len(s) - 1)))
        assert O.green_cdf(3, lam * r, t) == pytest.approx(cum[idx] / cum[-1], rel=1e-8)


def test_green_cdf_inverse_roundtrip():
    for n, a in ((3, 0.46), (3, 4.0), (1000, 0.4), (1001, 13.4), (6, 0.8)):
        for U in (1e-9, 0.01, 0.3, 0.77, 0.999999):
            t = O.green_cdf_inv(n, a, U)
            assert O.green_cdf(n, a, t) == pytest.approx(U, rel=1e-13, abs=1e-16)


def test_kt_against_mpmath():
    """K~_mu(x) = 2 (x/2)^mu K_mu(x) / Gamma(mu) for integer and half-integer order."""
    import mpmath as mp
    mp.mp.dps = 30
    for mu in (0.5, 1.0, 1.5, 2.0, 3.5, 11.0, 500.0, 500.5):
        for x in (0.01, 0.3, 1.0, 3.0):
            if x * x / 4 > max(mu, 1.0):
                continue
            ref = 2 * (mp.mpf(x) / 2) ** mu * mp.besselk(mu, x) / mp.gamma(mu) - 1
            assert O.kt_minus_one(mu, x) == pytest.approx(float(ref), rel=1e-12, abs=1e-16)


# ------------------------------------------------------------------ geometry
def _op(work):
    return O.OracleProblem(work.problem, work.params)


def test_cp_idempotent_and_nearest_sphere_torus():
    rng = np.random.default_rng(1)
    for work, n in ((W.sphere_cap(4, 1), 3), (W.torus_closed(4, 1), 3)):
        op = _op(work)
        # dense sample of M from the seeded inputs
        if work.problem.manifold.kind == W.MANIFOLD_SPHERE:
            cloud = W.sphere_cap_points(200000, seed=5)
            cloud[::2, 2] *= -1
        else:
            th, ph = W.torus_angles(200000, seed=5)
            cloud = W.torus_points(th, ph, 1.0, 0.4)
        for _ in range(20):
            x = cloud[rng.integers(len(cloud))] + 0.15 * rng.standard_normal(n)
            y = O.cp(op, x)
            assert np.allclose(O.cp(op, y), y, atol=1e-14)
            brute = np.min(np.linalg.norm(cloud - x, axis=1))
            assert np.linalg.norm(x - y) <= brute + 1e-12
            assert np.linalg.norm(x - y) >= brute - 0.02


def test_cp_embedded_sphere():
    work = W.embedded_s20(P=8, walks=1, n=60, d=5)
    op = _op(work)
    Q, b = work.problem.manifold.Q, work.problem.manifold.b
    assert np.allclose(Q.T @ Q, np.eye(6), atol=1e-14)
    rng = np.random.default_rng(2)
    for _ in range(10):
        x = work.points[rng.integers(8)] + 0.1 * rng.standard_normal(60)
        y = O.cp(op, x)
        assert np.allclose(O.cp(op, y), y, atol=1e-13)
        s = Q.T @ (y - b)
        assert abs(np.linalg.norm(s) - 1) < 1e-13 and np.allclose(Q @ s + b, y, atol=1e-13)
        # the residual's component in span(Q) is normal to S^d at s (parallel to s)
        w = Q.T @ (x - y)
        assert np.allclose(w - (w @ s) * s, 0.0, atol=1e-12)
        s_rand = rng.standard_normal(6)
        s_rand /= np.linalg.norm(s_rand)
        assert np.linalg.norm(x - y) <= np.linalg.norm(x - (Q @ s_rand + b)) + 1e-12


def test_delta_gamma_is_distance_to_normal_disk():
    """eq. delta_Gamma_general = dist(y, E_Gamma(y_Gamma)), the normal disk of
    radius ell = rho_geo(y_Gamma) (eq. extended_boundary_disk): brute force."""
    work = W.sphere_cap(4, 1)
    op = _op(work)
    ell = 1.2 / 2.0
    rng = np.random.default_rng(3)
    for z in (1e-4, 0.01, 0.3, 0.9, 0.97, 0.999):
        phi = rng.uniform(0, 2 * math.pi)
        rho = math.sqrt(1 - z * z)
        y = np.array([rho * math.cos(phi), rho * math.sin(phi), z])
        d, yg = O.delta_gamma(op, y)
        assert np.allclose(yg, [math.cos(phi), math.sin(phi), 0.0], atol=1e-14)
        # normal space of S^2 at y_Gamma is span(y_Gamma): the disk is a segment
        s = np.linspace(-ell, ell, 400001)
        pts = yg[None, :] + s[:, None] * yg[None, :]
        brute = np.min(np.linalg.norm(pts - y, axis=1))
        assert d == pytest.approx(brute, rel=1e-6, abs=1e-9)


def test_delta_gamma_pole_tie_break():
    work = W.sphere_cap(4, 1)
    d, yg = O.delta_gamma(_op(work), np.array([0.0, 0.0, 1.0]))
    assert np.allclose(yg, [1.0, 0.0, 0.0])
    assert d == pytest.approx(math.sqrt(1 + (1 - 0.6) ** 2))


# ------------------------------------------------------------- f and g data
def test_torus_source_is_laplace_beltrami():
    """(-Delta_M + sigma) u from the torus metric, symbolically (sympy), against
    the oracle's closed form of the Fourier-mode operator."""
    import sympy as sp
    th, ph = sp.symbols("theta phi", real=True)
    R, a, sig = 1, sp.Rational(2, 5), 2
    u = sp.sin(th) * sp.cos(2 * ph)
    rr = R + a * sp.cos(th)
    # metric diag(a^2, rr^2), sqrt(det g) = a rr
    lap = (sp.diff(a * rr / a ** 2 * sp.diff(u, th), th) + sp.diff(a * rr / rr ** 2 * sp.diff(u, ph), ph)) / (a * rr)
    fexpr = sp.lambdify((th, ph), -lap + sig * u)
    work = W.torus_closed(8, 1)
    op = _op(work)
    ths, phs = W.torus_angles(8, seed=9)
    for t_, p_ in zip(ths, phs):
        x = W.torus_points(np.array([t_]), np.array([p_]), 1.0, 0.4)[0]
        assert O.func_eval(op, "f", x) == pytest.approx(fexpr(t_, p_), rel=1e-12, abs=1e-12)


def test_sphere_quad_source_is_laplace_beltrami():
    """On S^d the Laplace-Beltrami operator equals the ambient Laplacian of the
    cp-extension on M (eq. LB_cp_identity): finite differences in R^{d+1}."""
    d = 4
    Q = np.eye(d + 1)
    v, A = W.quadratic_coeffs(d + 1, seed=4)
    A = A + 0.3 * np.eye(d + 1)     # exercise the trace part too
    sigma = 0.7
    man = W.Manifold(W.MANIFOLD_EMBEDDED_SPHERE, n=d + 1, d=d, Q=Q, b=np.zeros(d + 1))
    prob = W.Problem(man, sigma, True, W.Func.sphere_quad(0.25, v, A, True), W.Func.const(0.0))
    op = O.OracleProblem(prob, W.Params())
    u = lambda x: (lambda s: 0.25 + v @ s + s @ A @ s)(x / np.linalg.norm(x))
    rng = np.random.default_rng(0)
    h = 1e-4
    for _ in range(5):
        y = rng.standard_normal(d + 1)
        y /= np.linalg.norm(y)
        lap = sum((u(y + h * e) - 2 * u(y) + u(y - h * e)) / h ** 2 for e in np.eye(d + 1))
        assert O.func_eval(op, "f", y) == pytest.approx(-lap + sigma * u(y), rel=1e-5, abs=1e-5)


def test_poly_eval():
    work = W.sphere_cap(4, 1)
    op = _op(work)
    x = np.array([0.3, -0.4, math.sqrt(1 - 0.25)])
    assert O.func_eval(op, "f", x) == pytest.approx(7 * 0.3 * -0.4 + 3 * x[2], rel=1e-15)
    assert O.func_eval(op, "g", x) == pytest.approx(0.3 * -0.4, rel=1e-15)
