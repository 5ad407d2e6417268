"""Seeded synthetic inputs for the MPWoS workloads.

This module only draws query points, embeddings and coefficient sets from
seeded NumPy generators and writes the problem data (manifold, source f,
boundary data g, screening sigma) as plain descriptors.  It holds none of the
walk's arithmetic: both the CUDA library binding and the CPU oracle consume
what it produces, and neither is imported here.

Problem data conventions (the screened Poisson problem of Sec. 2.1, eqs.
surface_pde / surface_bc):

* a *function* (f or g) is one of
    - ``poly``: sparse polynomial in the ambient coordinates of a point on M,
      ``sum_t coef_t * prod_j x[var_tj] ** pow_tj``;
    - ``torus_fourier``: ``sum_t coef_t * T_t(m_t theta) * P_t(q_t phi)`` in
      the torus angles, T/P in {cos, sin}; with ``apply_op`` the function is
      replaced by ``(-Delta_M + sigma)`` applied to that series (closed form);
    - ``sphere_quad``: ``c0 + v.s + s^T A s`` in the intrinsic unit vector s
      of a (possibly embedded) round sphere; with ``apply_op`` likewise.
* manufactured solutions follow the workloads' definitions: the source is
  ``(-Delta_M + sigma) u`` written out with the sphere/torus spectra.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

# ----------------------------------------------------------------------------
# function descriptors
# ----------------------------------------------------------------------------

FUNC_POLY = 0
FUNC_TORUS_FOURIER = 1
FUNC_SPHERE_QUAD = 2
FUNC_REVOLUTION_QUAD = 3   # c0 + c1 t + c2 t^2 + v.xh + sum_j A_j xh_j^2 on a hypersurface of revolution
FUNC_CURVE_SPHERE = 4      # sum_t T_t(q_t phi) (c_t + v_t.w + w^T A_t w) on the Fourier curve x sphere

MANIFOLD_EUCLID = 0
MANIFOLD_SPHERE = 1
MANIFOLD_TORUS = 2
MANIFOLD_EMBEDDED_SPHERE = 3
MANIFOLD_POINT_CLOUD = 4
MANIFOLD_REVOLUTION = 5    # {(xh, t): |xh| = R(t)} about the last axis, dumbbell profile (Example 2)
MANIFOLD_CURVE_SPHERE = 6  # Fourier-embedded circle x S^2(a) in R^9 (Example 3)

SAMPLER_FULL = 0      # n Gaussians per direction
SAMPLER_REDUCED = 1   # dimension-reduced exact sampler (tracked coordinates + chi^2 remainder)

COMP_NONE = 0      # compensation term m_* = 0 (the baseline method)
COMP_NORMAL2 = 1   # second-order normal expansion of m from a predictor u_* (Sec. 2.3.3)
COMP_EXACT = 2     # m from its definition with u_* in place of u (exact when u_* = u)

CLOUD_CP_FIT = 0       # kNN + PCA plane + quadratic height fit + projection
CLOUD_CP_NEAREST = 1   # nearest cloud point

TRIG_COS = 0
TRIG_SIN = 1


@dataclass
class Func:
    kind: int
    apply_op: int = 0
    coef: List[float] = field(default_factory=list)
    # poly: per term list of (var, pow)
    terms: List[List[Tuple[int, int]]] = field(default_factory=list)
    # torus: per term (m, q, theta_trig, phi_trig)
    modes: List[Tuple[int, int, int, int]] = field(default_factory=list)
    # sphere quad
    c0: float = 0.0
    v: Optional[np.ndarray] = None
    A: Optional[np.ndarray] = None

    @staticmethod
    def poly(terms: Sequence[Tuple[float, Sequence[Tuple[int, int]]]]) -> "Func":
        return Func(kind=FUNC_POLY, coef=[float(c) for c, _ in terms],
                    terms=[[(int(v), int(p)) for v, p in vp] for _, vp in terms])

    @staticmethod
    def const(value: float) -> "Func":
        return Func.poly([(value, [])])

    @staticmethod
    def torus(terms: Sequence[Tuple[float, int, int, int, int]], apply_op: bool) -> "Func":
        return Func(kind=FUNC_TORUS_FOURIER, apply_op=int(apply_op),
                    coef=[float(t[0]) for t in terms],
                    modes=[(int(t[1]), int(t[2]), int(t[3]), int(t[4])) for t in terms])

    @staticmethod
    def revolution_quad(c1: float, c2: float, v: np.ndarray, a_diag: np.ndarray, apply_op: bool,
                        c0: float = 0.0) -> "Func":
        return Func(kind=FUNC_REVOLUTION_QUAD, apply_op=int(apply_op), coef=[float(c1), float(c2)], c0=float(c0),
                    v=np.ascontiguousarray(v, dtype=np.float64), A=np.ascontiguousarray(a_diag, dtype=np.float64))

    @staticmethod
    def curve_sphere(terms, apply_op: bool) -> "Func":
        """terms: (q, trig, c, v (3), A (3 x 3)) for T(q phi) (c + v.w + w^T A w)."""
        return Func(kind=FUNC_CURVE_SPHERE, apply_op=int(apply_op), coef=[float(t[2]) for t in terms],
                    modes=[(int(t[0]), int(t[1]), 0, 0) for t in terms],
                    v=np.ascontiguousarray(np.concatenate([np.asarray(t[3], float).reshape(3) for t in terms])),
                    A=np.ascontiguousarray(np.concatenate([np.asarray(t[4], float).reshape(9) for t in terms])))

    @staticmethod
    def sphere_quad(c0: float, v: np.ndarray, A: np.ndarray, apply_op: bool) -> "Func":
        return Func(kind=FUNC_SPHERE_QUAD, apply_op=int(apply_op), c0=float(c0),
                    v=np.ascontiguousarray(v, dtype=np.float64),
                    A=np.ascontiguousarray(A, dtype=np.float64))

    # flattened arrays shared by both bindings -------------------------------
    def flat_poly(self):
        off = [0]
        var: List[int] = []
        pw: List[int] = []
        for t in self.terms:
            for v, p in t:
                var.append(v)
                pw.append(p)
            off.append(len(var))
        return (np.asarray(self.coef, dtype=np.float64), np.asarray(off, dtype=np.int32),
                np.asarray(var if var else [0], dtype=np.int32),
                np.asarray(pw if pw else [0], dtype=np.int32))

    def flat_modes(self):
        m = np.asarray(self.modes, dtype=np.int32).reshape(-1)
        return np.asarray(self.coef, dtype=np.float64), (m if m.size else np.zeros(4, np.int32))


@dataclass
class Manifold:
    kind: int
    n: int
    d: int
    R: float = 0.0
    a: float = 0.0
    Q: Optional[np.ndarray] = None   # n x (d+1), row-major float64
    b: Optional[np.ndarray] = None   # n
    cloud: Optional[np.ndarray] = None   # N_c x 3 float64 (point cloud)
    k_nn: int = 16
    c_h: float = 2.4
    cp_mode: int = CLOUD_CP_FIT
    prof_alpha: float = 0.0   # hypersurface of revolution: R(t) = sqrt(1 - (t/k)^2) (1 - al + 2 al (t/k)^2)
    prof_kappa: float = 0.0


@dataclass
class Problem:
    manifold: Manifold
    sigma: float
    closed: bool
    f: Func
    g: Func
    bnd_normal: Optional[np.ndarray] = None
    bnd_offset: float = 0.0
    comp: int = COMP_NONE           # COMP_NORMAL2: source f + m_* with predictor u_star
    u_star: Optional[Func] = None   # torus Fourier (torus) or sphere quad (unit S^2), apply_op = 0
    h_eta: float = 1e-2             # normal finite-difference step of m_*


@dataclass
class Params:
    eps: float = 1e-3
    tau_w: float = 1e-8
    theta: float = 0.95
    c_kappa: float = 1.2
    n_v: int = 1
    max_steps: int = 10_000_000
    seed: int = 0
    sampler: int = 0   # SAMPLER_FULL or SAMPLER_REDUCED (dimension-reduced exact sampler)


# ----------------------------------------------------------------------------
# seeded geometry
# ----------------------------------------------------------------------------

def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def sphere_cap_points(P: int, seed: int = 0) -> np.ndarray:
    """Uniform (area) points on the cap z>0 of the unit sphere S^2."""
    x = _rng(seed).standard_normal((P, 3))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    x[:, 2] = np.abs(x[:, 2])
    return x


def hemisphere_points(P: int, n: int, seed: int = 0) -> np.ndarray:
    """Uniform points on the half {x_1 > 0} of the unit sphere S^{n-1}."""
    x = _rng(seed).standard_normal((P, n))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    x[:, 0] = np.abs(x[:, 0])
    return x


def torus_angles(P: int, seed: int = 0) -> Tuple[np.ndarray, np.ndarray]:
    """(theta, phi) uniform in [0, 2pi)^2 (parameter-uniform)."""
    g = _rng(seed)
    return g.uniform(0.0, 2 * math.pi, P), g.uniform(0.0, 2 * math.pi, P)


def torus_points(theta: np.ndarray, phi: np.ndarray, R: float, a: float) -> np.ndarray:
    """X(theta, phi) = ((R + a cos t) cos p, (R + a cos t) sin p, a sin t) (Example 1's parametrisation)."""
    rr = R + a * np.cos(theta)
    return np.stack([rr * np.cos(phi), rr * np.sin(phi), a * np.sin(theta)], axis=1)


def torus_domain_points(problem: "Problem", P: int, seed: int = 12345) -> np.ndarray:
    """P points of a torus problem's Omega, (theta, phi) uniform, rejecting e.x <= h
    on a boundary problem (P x 3)."""
    man = problem.manifold
    g = _rng(seed)
    out, have = [], 0
    while have < P:
        x = torus_points(g.uniform(0.0, 2 * math.pi, 4 * P), g.uniform(0.0, 2 * math.pi, 4 * P), man.R, man.a)
        if not problem.closed:
            x = x[x @ problem.bnd_normal > problem.bnd_offset]
        out.append(x)
        have += len(x)
    return np.concatenate(out)[:P]


def embedding(n: int, d: int, seed: int = 0) -> Tuple[np.ndarray, np.ndarray]:
    """Seeded orthonormal Q (n x (d+1), from a Gaussian QR, sign-fixed) and shift b ~ N(0, I)."""
    g = _rng(seed)
    G = g.standard_normal((n, d + 1))
    Q, Rm = np.linalg.qr(G)
    Q = Q * np.sign(np.diag(Rm))[None, :]
    b = g.standard_normal(n)
    return np.ascontiguousarray(Q), np.ascontiguousarray(b)


def embedded_sphere_points(P: int, Q: np.ndarray, b: np.ndarray, seed: int = 0) -> Tuple[np.ndarray, np.ndarray]:
    """Uniform intrinsic s on S^d and the ambient points Q s + b."""
    s = _rng(seed).standard_normal((P, Q.shape[1]))
    s /= np.linalg.norm(s, axis=1, keepdims=True)
    return s @ Q.T + b[None, :], s


def quadratic_coeffs(dim: int, seed: int = 0) -> Tuple[np.ndarray, np.ndarray]:
    """v ~ N(0, I)/sqrt(dim); A symmetric, trace-free, ||A||_F = 1."""
    g = _rng(seed)
    v = g.standard_normal(dim) / math.sqrt(dim)
    M = g.standard_normal((dim, dim))
    A = 0.5 * (M + M.T)
    A -= np.trace(A) / dim * np.eye(dim)
    A /= np.linalg.norm(A)
    return v, A


# ----------------------------------------------------------------------------
# the workloads
# ----------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    problem: Problem
    points: np.ndarray          # P x n float64
    walks: int
    params: Params
    exact: np.ndarray           # manufactured solution at the points
    precision: str              # "f64" or "f32"


def sphere_cap(P: int = 64, walks: int = 1000, seed: int = 0) -> Workload:
    """Unit S^2, domain z>0, sigma=1, u = xy + z  =>  f = 7xy + 3z, g = xy on z=0.

    xy and z are spherical harmonics of degree 2 and 1 (-Delta eigenvalues 6, 2)."""
    man = Manifold(MANIFOLD_SPHERE, n=3, d=2)
    f = Func.poly([(7.0, [(0, 1), (1, 1)]), (3.0, [(2, 1)])])
    g = Func.poly([(1.0, [(0, 1), (1, 1)])])
    prob = Problem(man, sigma=1.0, closed=False, f=f, g=g,
                   bnd_normal=np.array([0.0, 0.0, 1.0]), bnd_offset=0.0)
    pts = sphere_cap_points(P, seed)
    exact = pts[:, 0] * pts[:, 1] + pts[:, 2]
    return Workload("s2_cap", prob, pts, walks, Params(eps=1e-3), exact, "f64")


def torus_closed(P: int = 4096, walks: int = 10_000, seed: int = 0, R: float = 1.0, a: float = 0.4,
                 sigma: float = 2.0) -> Workload:
    """Closed torus R=1, tube radius 0.4, sigma=2, u = sin(theta) cos(2 phi)."""
    man = Manifold(MANIFOLD_TORUS, n=3, d=2, R=R, a=a)
    term = [(1.0, 1, 2, TRIG_SIN, TRIG_COS)]
    f = Func.torus(term, apply_op=True)
    g = Func.const(0.0)
    prob = Problem(man, sigma=sigma, closed=True, f=f, g=g)
    th, ph = torus_angles(P, seed)
    pts = torus_points(th, ph, R, a)
    exact = np.sin(th) * np.cos(2 * ph)
    return Workload("torus_closed", prob, pts, walks, Params(), exact, "f32")


def hypersphere_half(P: int = 16384, walks: int = 4096, n: int = 1000, seed: int = 0) -> Workload:
    """S^{n-1} in R^n, domain x_1>0, sigma=1, u = x_1 + x_2 x_3.

    On S^{n-1}: x_1 has eigenvalue n-1, x_2 x_3 has 2n; f = n x_1 + (2n+1) x_2 x_3, g = x_2 x_3."""
    man = Manifold(MANIFOLD_SPHERE, n=n, d=n - 1)
    f = Func.poly([(float(n), [(0, 1)]), (float(2 * n + 1), [(1, 1), (2, 1)])])
    g = Func.poly([(1.0, [(1, 1), (2, 1)])])
    e = np.zeros(n)
    e[0] = 1.0
    prob = Problem(man, sigma=1.0, closed=False, f=f, g=g, bnd_normal=e, bnd_offset=0.0)
    pts = hemisphere_points(P, n, seed)
    exact = pts[:, 0] + pts[:, 1] * pts[:, 2]
    return Workload("s999_half", prob, pts, walks, Params(eps=1e-3), exact, "f32")


def embedded_s20(P: int = 32768, walks: int = 2048, n: int = 1000, d: int = 20, sigma: float = 0.5,
                 seed: int = 0) -> Workload:
    """S^d embedded in R^n by a seeded orthonormal Q plus shift b; u = v.s + s^T A s (A trace-free)."""
    Q, b = embedding(n, d, seed)
    v, A = quadratic_coeffs(d + 1, seed + 1)
    man = Manifold(MANIFOLD_EMBEDDED_SPHERE, n=n, d=d, Q=Q, b=b)
    f = Func.sphere_quad(0.0, v, A, apply_op=True)
    g = Func.const(0.0)
    prob = Problem(man, sigma=sigma, closed=True, f=f, g=g)
    pts, s = embedded_sphere_points(P, Q, b, seed + 2)
    exact = s @ v + np.einsum("pi,ij,pj->p", s, A, s)
    return Workload("s20_in_r1000", prob, pts, walks, Params(), exact, "f32")


def constant_solution(base: Workload) -> Workload:
    """Same geometry with f = sigma, g = 1: u = 1 exactly (each walk telescopes)."""
    p = base.problem
    prob = Problem(p.manifold, p.sigma, p.closed, Func.const(p.sigma), Func.const(1.0),
                   p.bnd_normal, p.bnd_offset)
    return Workload(base.name + "_const", prob, base.points, base.walks, base.params,
                    np.ones(len(base.points)), base.precision)


def euclid_halfspace(P: int = 16, walks: int = 2000, n: int = 3, sigma: float = 1.0, seed: int = 0) -> Workload:
    """M = R^n (cp = identity), domain x_1 > 0, f = 0, g = 1: u = exp(-sqrt(sigma) x_1)."""
    man = Manifold(MANIFOLD_EUCLID, n=n, d=n)
    e = np.zeros(n)
    e[0] = 1.0
    prob = Problem(man, sigma=sigma, closed=False, f=Func.const(0.0), g=Func.const(1.0),
                   bnd_normal=e, bnd_offset=0.0)
    g = _rng(seed)
    pts = g.standard_normal((P, n))
    pts[:, 0] = g.uniform(0.05, 1.5, P)
    exact = np.exp(-math.sqrt(sigma) * pts[:, 0])
    return Workload("euclid_half", prob, pts, walks, Params(eps=1e-3), exact, "f64")


# ----------------------------------------------------------------------------
# point cloud on a radius-perturbed sphere
# ----------------------------------------------------------------------------

def _harmonics_l123(w: np.ndarray) -> np.ndarray:
    """The 15 real spherical harmonics of degrees 1-3 (unnormalised polynomial
    forms) at unit vectors w (M x 3)."""
    x, y, z = w[:, 0], w[:, 1], w[:, 2]
    return np.stack([x, y, z,
                     x * y, y * z, 3 * z * z - 1, x * z, x * x - y * y,
                     y * (3 * x * x - y * y), x * y * z, y * (5 * z * z - 1), z * (5 * z * z - 3),
                     x * (5 * z * z - 1), z * (x * x - y * y), x * (x * x - 3 * y * y)], axis=1)


def perturbed_sphere_coeffs(seed: int = 0) -> np.ndarray:
    """alpha for r(w) = 1 + 0.2 sum alpha_i Y_i(w), scaled so max |sum| <= 1."""
    a = _rng(seed).standard_normal(15)
    probe = _rng(seed + 100).standard_normal((200000, 3))
    probe /= np.linalg.norm(probe, axis=1, keepdims=True)
    m = np.max(np.abs(_harmonics_l123(probe) @ a))
    return a / (1.02 * m)


def perturbed_sphere_radius(w: np.ndarray, alpha: np.ndarray) -> np.ndarray:
    return 1.0 + 0.2 * (_harmonics_l123(w) @ alpha)


def perturbed_sphere_cloud(N: int = 200_000, seed: int = 0) -> Tuple[np.ndarray, np.ndarray]:
    """N points r(w) w with w area-uniform on S^2 (seed), and the coefficients alpha."""
    alpha = perturbed_sphere_coeffs(seed)
    w = _rng(seed + 1).standard_normal((N, 3))
    w /= np.linalg.norm(w, axis=1, keepdims=True)
    return np.ascontiguousarray(perturbed_sphere_radius(w, alpha)[:, None] * w), alpha


def point_cloud(P: int = 256, walks: int = 1000, N_cloud: int = 200_000, k_nn: int = 16, c_h: float = 2.4,
                sigma: float = 100.0, seed: int = 0, cp_mode: int = CLOUD_CP_FIT) -> Workload:
    """Closed point-cloud surface (radius-perturbed sphere), f = sigma: u = 1.

    Query points are cloud points (on the sampled surface), chosen by seed."""
    cloud, alpha = perturbed_sphere_cloud(N_cloud, seed)
    man = Manifold(MANIFOLD_POINT_CLOUD, n=3, d=2, cloud=cloud, k_nn=k_nn, c_h=c_h, cp_mode=cp_mode)
    prob = Problem(man, sigma=sigma, closed=True, f=Func.const(sigma), g=Func.const(0.0))
    idx = _rng(seed + 7).choice(N_cloud, size=P, replace=False)
    return Workload("point_cloud", prob, cloud[idx].copy(), walks, Params(), np.ones(P), "f32")


# ----------------------------------------------------------------------------
# Example 4: the unit sphere given only by a point cloud
# ----------------------------------------------------------------------------

def _legendre_poly_in_z(coef_by_degree: Sequence[float]) -> List[Tuple[float, List[Tuple[int, int]]]]:
    """sum_l c_l P_l(x_3) as monomial terms in x_3 (index 2)."""
    mono = np.polynomial.legendre.leg2poly(np.asarray(coef_by_degree, dtype=np.float64))
    return [(float(c), [(2, p)] if p else []) for p, c in enumerate(mono) if c != 0.0]


def sphere_cloud_legendre(P: int = 100, walks: int = 2000, N_cloud: int = 8000, k_nn: int = 6, c_h: float = 2.4,
                          sigma: float = 10.0, seed: int = 0) -> Workload:
    """Example 4: closed S^2 known only through N_cloud area-uniform points, k_nn = 6, c_h = 2.4,
    closest point = nearest cloud point, m_* = 0;
    u = P_1(x_3) + 0.2 P_3(x_3) + 0.1 P_5(x_3), f = sum_l c_l (l(l+1) + sigma) P_l(x_3).

    sigma is not given for this example; 10 keeps a walk near 10^3 steps at tau_W = 1e-8.
    Query points are P cloud points chosen by seed (the walk only visits cloud points)."""
    g = _rng(seed)
    cloud = g.standard_normal((N_cloud, 3))
    cloud /= np.linalg.norm(cloud, axis=1, keepdims=True)
    cloud = np.ascontiguousarray(cloud)
    cu = [0.0, 1.0, 0.0, 0.2, 0.0, 0.1]
    cf = [c * (l * (l + 1) + sigma) for l, c in enumerate(cu)]
    man = Manifold(MANIFOLD_POINT_CLOUD, n=3, d=2, cloud=cloud, k_nn=k_nn, c_h=c_h, cp_mode=CLOUD_CP_NEAREST)
    prob = Problem(man, sigma=sigma, closed=True, f=Func.poly(_legendre_poly_in_z(cf)), g=Func.const(0.0))
    idx = _rng(seed + 7).choice(N_cloud, size=P, replace=False)
    pts = cloud[idx].copy()
    exact = np.polynomial.legendre.legval(pts[:, 2], cu)
    return Workload("sphere_cloud_e4", prob, pts, walks, Params(), exact, "f32")


# ----------------------------------------------------------------------------
# Example 1: the torus with a planar cut (effect of the compensation term)
# ----------------------------------------------------------------------------

E1_PHI_C = 0.35 * math.pi


def torus_cut_terms(phi_c: float = E1_PHI_C) -> List[Tuple[float, int, int, int, int]]:
    """u = sin(s) A(theta) + sin(2s) B(theta) + sin(3s) C(theta), s = phi - phi_c, as torus
    Fourier terms (coef, m, q, theta trig, phi trig); sin(q s) = sin(q phi) cos(q phi_c) -
    cos(q phi) sin(q phi_c).
    A = 1 + 0.9 cos t + 0.6 sin 2t + 0.35 cos 3t, B = 0.45 cos 2t, C = 0.3 (0.5 + sin t)."""
    theta_parts = {1: [(1.0, 0, TRIG_COS), (0.9, 1, TRIG_COS), (0.6, 2, TRIG_SIN), (0.35, 3, TRIG_COS)],
                   2: [(0.45, 2, TRIG_COS)],
                   3: [(0.15, 0, TRIG_COS), (0.3, 1, TRIG_SIN)]}
    terms = []
    for q, parts in theta_parts.items():
        for c, m, tk in parts:
            terms.append((c * math.cos(q * phi_c), m, q, tk, TRIG_SIN))
            terms.append((-c * math.sin(q * phi_c), m, q, tk, TRIG_COS))
    return terms


def torus_series_value(terms, theta: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """sum_t coef_t T_t(m_t theta) P_t(q_t phi) at parameter values."""
    trig = (np.cos, np.sin)
    out = np.zeros(np.broadcast(theta, phi).shape)
    for c, m, q, tk, pk in terms:
        out = out + c * trig[tk](m * theta) * trig[pk](q * phi)
    return out


def torus_cut(P: int = 100, walks: int = 2000, seed: int = 0, R: float = 1.0, a: float = 0.45,
              sigma: float = 4.0, comp: int = COMP_NONE, u_star: Optional[Func] = None) -> Workload:
    """Example 1: torus R = 1, a = 0.45 cut by the plane -sin(phi_c) x + cos(phi_c) y = 0,
    Omega = {phi - phi_c in (0, pi)}, sigma = 4, the three-mode u above (u = 0 on Gamma), eps = 1e-5.
    comp: COMP_NORMAL2 / COMP_EXACT with predictor u_star (the exact u when None)."""
    man = Manifold(MANIFOLD_TORUS, n=3, d=2, R=R, a=a)
    terms = torus_cut_terms()
    e = np.array([-math.sin(E1_PHI_C), math.cos(E1_PHI_C), 0.0])
    prob = Problem(man, sigma=sigma, closed=False, f=Func.torus(terms, apply_op=True), g=Func.const(0.0),
                   bnd_normal=e, bnd_offset=0.0)
    if comp:
        prob.comp = int(comp)
        prob.u_star = u_star if u_star is not None else Func.torus(terms, apply_op=False)
    g = _rng(seed)
    th = g.uniform(0.0, 2 * math.pi, P)
    ph = E1_PHI_C + g.uniform(0.0, math.pi, P)
    pts = torus_points(th, ph, R, a)
    exact = torus_series_value(terms, th, ph)
    return Workload("torus_cut_e1", prob, pts, walks, Params(eps=1e-5), exact, "f32")


# ----------------------------------------------------------------------------
# Example 2: the dumbbell hypersurface of revolution in R^1001
# ----------------------------------------------------------------------------

def dumbbell_profile(t: np.ndarray, alpha: float = 0.35, kappa: float = 1.2) -> np.ndarray:
    """R(t) = sqrt(1 - (t/kappa)^2) (1 - alpha + 2 alpha (t/kappa)^2) (Example 2's profile)."""
    s = np.asarray(t) / kappa
    return np.sqrt(1.0 - s * s) * (1.0 - alpha + 2.0 * alpha * s * s)


def dumbbell(P: int = 100, walks: int = 1000, n: int = 1001, seed: int = 0, alpha: float = 0.35,
             kappa: float = 1.2) -> Workload:
    """Example 2: M = {x = (xh, t) in R^n : |xh| = R(t)}, closed, d = n - 1, sigma = 2d,
    u = 0.15 t + 0.05 t^2 + v1.xh + 0.2 xh^T diag(a) xh, v1 = (1, ..., 1)/sqrt(n-1),
    sum_j a_j = 0 (a seeded: centred normal draws); theta = 0.95, c_kappa = 1.2.

    Query points: t = kappa s with s uniform in [-0.9, 0.9] (away from the two tips),
    xh = R(t) w with w uniform on S^{n-2}."""
    g = _rng(seed)
    m = n - 1
    a = g.standard_normal(m)
    a -= a.mean()
    v = np.full(m, 1.0 / math.sqrt(m))
    A = 0.2 * a
    man = Manifold(MANIFOLD_REVOLUTION, n=n, d=n - 1, prof_alpha=alpha, prof_kappa=kappa)
    sigma = 2.0 * (n - 1)
    prob = Problem(man, sigma=sigma, closed=True, f=Func.revolution_quad(0.15, 0.05, v, A, apply_op=True),
                   g=Func.const(0.0))
    t = kappa * g.uniform(-0.9, 0.9, P)
    w = g.standard_normal((P, m))
    w /= np.linalg.norm(w, axis=1, keepdims=True)
    xh = dumbbell_profile(t, alpha, kappa)[:, None] * w
    pts = np.ascontiguousarray(np.concatenate([xh, t[:, None]], axis=1))
    exact = 0.15 * t + 0.05 * t * t + xh @ v + (xh * xh) @ A
    return Workload("dumbbell_e2", prob, pts, walks, Params(theta=0.95, c_kappa=1.2), exact, "f32")


# ----------------------------------------------------------------------------
# Example 3: the Fourier-embedded circle times S^2(a) in R^9
# ----------------------------------------------------------------------------

def fourier_curve(phi: np.ndarray, R: float = 1.0) -> np.ndarray:
    """C(phi) = R (cos phi, sin phi, cos 2phi / 2, sin 2phi / 2, cos 3phi / 3, sin 3phi / 3)."""
    phi = np.asarray(phi)
    return R * np.stack([np.cos(phi), np.sin(phi), np.cos(2 * phi) / 2, np.sin(2 * phi) / 2,
                         np.cos(3 * phi) / 3, np.sin(3 * phi) / 3], axis=-1)


def curve_sphere(P: int = 100, walks: int = 1000, R: float = 1.0, a: float = 0.65, sigma: float = 2.0,
                 seed: int = 0) -> Workload:
    """Example 3: M = C(S^1) x S^2(a) in R^9, closed, d = 3,
    u = cos(phi) w_1 + 0.3 sin(2 phi) w_2 + 0.2 cos(3 phi) (w_1^2 - w_2^2).

    sigma is not given for this example; 2 keeps a walk near 800 steps at tau_W = 1e-8.
    Query points: phi uniform in [0, 2 pi), w uniform on S^2 (seed)."""
    man = Manifold(MANIFOLD_CURVE_SPHERE, n=9, d=3, R=R, a=a)
    z3 = np.zeros(3)
    z33 = np.zeros((3, 3))
    terms = [(1, TRIG_COS, 0.0, np.array([1.0, 0.0, 0.0]), z33),
             (2, TRIG_SIN, 0.0, np.array([0.0, 0.3, 0.0]), z33),
             (3, TRIG_COS, 0.0, z3, np.diag([0.2, -0.2, 0.0]))]
    prob = Problem(man, sigma=sigma, closed=True, f=Func.curve_sphere(terms, apply_op=True), g=Func.const(0.0))
    g = _rng(seed)
    phi = g.uniform(0.0, 2 * math.pi, P)
    w = g.standard_normal((P, 3))
    w /= np.linalg.norm(w, axis=1, keepdims=True)
    pts = np.ascontiguousarray(np.concatenate([fourier_curve(phi, R), a * w], axis=1))
    exact = (np.cos(phi) * w[:, 0] + 0.3 * np.sin(2 * phi) * w[:, 1]
             + 0.2 * np.cos(3 * phi) * (w[:, 0] ** 2 - w[:, 1] ** 2))
    return Workload("curve_sphere_e3", prob, pts, walks, Params(), exact, "f32")
