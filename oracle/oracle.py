"""ctypes binding of the C oracle (test infrastructure only)."""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from .build import build

__all__ = ["lib", "philox", "u53", "gaussians", "chi2", "tracked_set", "em1", "c_sigma_r", "green_cdf", "green_cdf_inv",
           "kt_minus_one", "cp", "delta_gamma", "func_eval", "profile", "kappa_at", "curve_cp_phi", "normal_coord", "comp_R", "comp_m", "walk_scores", "solve", "trace",
           "OracleProblem", "cloud_knn"]

_lib: Optional[C.CDLL] = None

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class _Manifold(C.Structure):
    _fields_ = [("kind", C.c_int), ("n", C.c_int), ("d", C.c_int), ("R", C.c_double),
                ("a", C.c_double), ("Q", _dp), ("b", _dp), ("cloud", _dp), ("n_cloud", C.c_int64),
                ("k_nn", C.c_int), ("c_h", C.c_double), ("cp_mode", C.c_int),
                ("prof_alpha", C.c_double), ("prof_kappa", C.c_double)]


class _Func(C.Structure):
    _fields_ = [("kind", C.c_int), ("apply_op", C.c_int), ("n_terms", C.c_int), ("coef", _dp),
                ("term_off", _ip), ("var", _ip), ("pw", _ip), ("modes", _ip), ("c0", C.c_double),
                ("v", _dp), ("A", _dp)]


class _Problem(C.Structure):
    _fields_ = [("sigma", C.c_double), ("closed", C.c_int), ("bnd_normal", _dp),
                ("bnd_offset", C.c_double), ("f", _Func), ("g", _Func),
                ("comp", C.c_int), ("u_star", _Func), ("h_eta", C.c_double)]


class _Params(C.Structure):
    _fields_ = [("eps", C.c_double), ("tau_w", C.c_double), ("theta", C.c_double),
                ("c_kappa", C.c_double), ("n_v", C.c_int), ("max_steps", C.c_int64),
                ("seed", C.c_uint64), ("sampler", C.c_int)]


class _Trace(C.Structure):
    _fields_ = [("k", C.c_int64), ("r", C.c_double), ("c", C.c_double), ("omega", C.c_double),
                ("delta_gamma", C.c_double), ("W", C.c_double), ("S", C.c_double),
                ("F", C.c_double), ("U0", C.c_double), ("t0", C.c_double),
                ("theta_norm", C.c_double), ("y", C.c_double * 3)]


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        L.orc_u53.restype = C.c_double
        L.orc_u53.argtypes = [C.c_uint32, C.c_uint32]
        L.orc_em1.restype = C.c_double
        L.orc_em1.argtypes = [C.c_int, C.c_double]
        L.orc_c_sigma_r.restype = C.c_double
        L.orc_c_sigma_r.argtypes = [C.c_int, C.c_double]
        L.orc_green_cdf.restype = C.c_double
        L.orc_green_cdf.argtypes = [C.c_int, C.c_double, C.c_double]
        L.orc_green_cdf_inv.restype = C.c_double
        L.orc_green_cdf_inv.argtypes = [C.c_int, C.c_double, C.c_double]
        L.orc_kt_minus_one.restype = C.c_double
        L.orc_kt_minus_one.argtypes = [C.c_double, C.c_double]
        L.orc_delta_gamma.restype = C.c_double
        L.orc_func_eval.restype = C.c_double
        L.orc_trace.restype = C.c_int64
        L.orc_cloud_knn.restype = C.c_double
        L.orc_normal_coord.restype = C.c_double
        L.orc_kappa_at.restype = C.c_double
        L.orc_curve_cp_phi.restype = C.c_double
        L.orc_comp_R.restype = C.c_double
        L.orc_comp_R.argtypes = [C.c_void_p, C.c_void_p, _dp, C.c_double]
        L.orc_comp_m.restype = C.c_double
        L.orc_chi2.restype = C.c_double
        L.orc_chi2.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, C.c_int]
        _lib = L
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _iptr(a: np.ndarray):
    return a.ctypes.data_as(_ip)


class OracleProblem:
    """Marshals a workloads.Problem into the oracle's structs (keeps arrays alive)."""

    def __init__(self, problem, params):
        self._keep = []
        m = problem.manifold
        self.man = _Manifold(kind=m.kind, n=m.n, d=m.d, R=m.R, a=m.a,
                             prof_alpha=getattr(m, "prof_alpha", 0.0), prof_kappa=getattr(m, "prof_kappa", 0.0))
        if m.Q is not None:
            Q = self._arr(m.Q)
            b = self._arr(m.b)
            self.man.Q = _dptr(Q)
            self.man.b = _dptr(b)
        if m.cloud is not None:
            cl = self._arr(m.cloud)
            self.man.cloud = _dptr(cl)
            self.man.n_cloud = cl.shape[0]
            self.man.k_nn = m.k_nn
            self.man.c_h = m.c_h
            self.man.cp_mode = m.cp_mode
        self.prob = _Problem(sigma=problem.sigma, closed=int(problem.closed),
                             bnd_offset=problem.bnd_offset)
        if problem.bnd_normal is not None:
            self.prob.bnd_normal = _dptr(self._arr(problem.bnd_normal))
        self.prob.f = self._func(problem.f)
        self.prob.g = self._func(problem.g)
        if getattr(problem, "comp", 0):
            self.prob.comp = problem.comp
            self.prob.u_star = self._func(problem.u_star)
            self.prob.h_eta = problem.h_eta
        self.n = m.n
        self.set_params(params)

    def set_params(self, params):
        self.params = _Params(eps=params.eps, tau_w=params.tau_w, theta=params.theta,
                              c_kappa=params.c_kappa, n_v=params.n_v,
                              max_steps=params.max_steps, seed=params.seed,
                              sampler=getattr(params, "sampler", 0))

    def _arr(self, a, dtype=np.float64):
        a = np.ascontiguousarray(a, dtype=dtype)
        self._keep.append(a)
        return a

    def _func(self, f) -> _Func:
        from paper_2606_21883_b300 import workloads as W
        cf = _Func(kind=f.kind, apply_op=f.apply_op, n_terms=len(f.coef), c0=f.c0)
        if f.kind == W.FUNC_POLY:
            coef, off, var, pw = f.flat_poly()
            cf.coef = _dptr(self._arr(coef))
            cf.term_off = _iptr(self._arr(off, np.int32))
            cf.var = _iptr(self._arr(var, np.int32))
            cf.pw = _iptr(self._arr(pw, np.int32))
        elif f.kind in (W.FUNC_TORUS_FOURIER, W.FUNC_CURVE_SPHERE):
            coef, modes = f.flat_modes()
            cf.coef = _dptr(self._arr(coef))
            cf.modes = _iptr(self._arr(modes, np.int32))
            if f.kind == W.FUNC_CURVE_SPHERE:
                cf.v = _dptr(self._arr(f.v))
                cf.A = _dptr(self._arr(f.A))
        else:
            if f.kind == W.FUNC_REVOLUTION_QUAD:
                cf.coef = _dptr(self._arr(np.asarray(f.coef, dtype=np.float64)))
            cf.v = _dptr(self._arr(f.v))
            cf.A = _dptr(self._arr(f.A))
        return cf


# ---------------------------------------------------------------------------
def philox(ctr, key):
    L = lib()
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    L.orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def u53(hi, lo):
    return lib().orc_u53(hi, lo)


def gaussians(seed, j0, k, i, p, n):
    g = np.zeros(n)
    lib().orc_gaussians(C.c_uint64(seed), C.c_uint32(j0), C.c_uint32(k), C.c_uint32(i),
                        C.c_uint32(p), C.c_int(n), _dptr(g))
    return g


def chi2(seed, j0, k, i, p, m):
    """chi^2_m from the reduced sampler's counter stream at block j0 of step k."""
    return lib().orc_chi2(seed, j0, k, i, p, m)


def tracked_set(problem, params):
    op = OracleProblem(problem, params)
    T = (C.c_int * 32)()
    nT = lib().orc_tracked_set(C.byref(op.man), C.byref(op.prob), T)
    return list(T[:nT]) if nT >= 0 else None


def em1(n, a):
    return lib().orc_em1(n, a)


def c_sigma_r(n, a):
    return lib().orc_c_sigma_r(n, a)


def green_cdf(n, a, t):
    return lib().orc_green_cdf(n, a, t)


def green_cdf_inv(n, a, U):
    return lib().orc_green_cdf_inv(n, a, U)


def kt_minus_one(mu, x):
    return lib().orc_kt_minus_one(mu, x)


def cp(op: OracleProblem, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    lib().orc_cp(C.byref(op.man), _dptr(x), _dptr(out))
    return out


def delta_gamma(op: OracleProblem, y):
    y = np.ascontiguousarray(y, dtype=np.float64)
    yg = np.zeros_like(y)
    d = lib().orc_delta_gamma(C.byref(op.man), C.byref(op.prob), C.byref(op.params), _dptr(y), _dptr(yg))
    return d, yg


def cloud_knn(op: OracleProblem, x):
    """k nearest cloud points of x (indices ordered by distance^2, then index) and h(x)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    k = op.man.k_nn
    idx = np.zeros(k, dtype=np.int64)
    d2 = np.zeros(k)
    h = lib().orc_cloud_knn(C.byref(op.man), _dptr(x), idx.ctypes.data_as(C.POINTER(C.c_int64)), _dptr(d2))
    return idx, d2, h


def func_eval(op: OracleProblem, which: str, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    f = {"f": op.prob.f, "g": op.prob.g, "u_star": op.prob.u_star}[which]
    return lib().orc_func_eval(C.byref(op.man), C.byref(f), C.c_double(op.prob.sigma), _dptr(x))


def profile(op: OracleProblem, t):
    """R(t), R'(t), R''(t) of a hypersurface of revolution's profile."""
    R, R1, R2 = C.c_double(), C.c_double(), C.c_double()
    lib().orc_profile(C.byref(op.man), C.c_double(t), C.byref(R), C.byref(R1), C.byref(R2))
    return R.value, R1.value, R2.value


def curve_cp_phi(op: OracleProblem, x):
    """phi of the nearest point of the Fourier curve to x's first six coordinates."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    return lib().orc_curve_cp_phi(C.byref(op.man), _dptr(x))


def kappa_at(op: OracleProblem, y):
    """The curvature indicator (largest absolute principal curvature) at y on M."""
    y = np.ascontiguousarray(y, dtype=np.float64)
    return lib().orc_kappa_at(C.byref(op.man), _dptr(y))


def normal_coord(op: OracleProblem, x):
    """Signed normal distance eta of x from M (torus, unit sphere of R^3)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    return lib().orc_normal_coord(C.byref(op.man), _dptr(x))


def comp_R(op: OracleProblem, y, s):
    """R_*(s; y) of the compensation term at y on M."""
    y = np.ascontiguousarray(y, dtype=np.float64)
    return lib().orc_comp_R(C.byref(op.man), C.byref(op.prob), _dptr(y), s)


def comp_m(op: OracleProblem, x):
    """m_*(x), the second-order normal expansion of the compensation term."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    return lib().orc_comp_m(C.byref(op.man), C.byref(op.prob), _dptr(x))


def walk_scores(problem, params, pts, N, n_threads=0):
    op = OracleProblem(problem, params)
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    P = pts.shape[0]
    S = np.zeros(P * N)
    K = np.zeros(P * N, dtype=np.int64)
    fl = np.zeros(P * N, dtype=np.int32)
    rc = lib().orc_walk_scores(C.byref(op.man), C.byref(op.prob), C.byref(op.params), _dptr(pts),
                               C.c_int64(P), C.c_int64(N), _dptr(S), K.ctypes.data_as(C.POINTER(C.c_int64)),
                               fl.ctypes.data_as(C.POINTER(C.c_int32)), C.c_int(n_threads))
    if rc != 0:
        raise ValueError("the oracle does not implement this problem form")
    return S.reshape(P, N), K.reshape(P, N), fl.reshape(P, N)


def solve(problem, params, pts, N, n_threads=0):
    op = OracleProblem(problem, params)
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    P = pts.shape[0]
    mean = np.zeros(P)
    se = np.zeros(P)
    ms = np.zeros(P)
    nf = C.c_int64(0)
    rc = lib().orc_solve(C.byref(op.man), C.byref(op.prob), C.byref(op.params), _dptr(pts),
                         C.c_int64(P), C.c_int64(N), _dptr(mean), _dptr(se), _dptr(ms), C.byref(nf),
                         C.c_int(n_threads))
    if rc != 0:
        raise ValueError("the oracle does not implement this problem form")
    return mean, se, ms, int(nf.value)


def trace(problem, params, y0, p=0, i=0, cap=100000):
    op = OracleProblem(problem, params)
    y0 = np.ascontiguousarray(y0, dtype=np.float64)
    rec = (_Trace * cap)()
    S = C.c_double(0)
    K = C.c_int64(0)
    nrec = lib().orc_trace(C.byref(op.man), C.byref(op.prob), C.byref(op.params), _dptr(y0),
                           C.c_int64(p), C.c_int64(i), rec, C.c_int64(cap), C.byref(S), C.byref(K))
    rows = [dict(k=r.k, r=r.r, c=r.c, omega=r.omega, delta_gamma=r.delta_gamma, W=r.W, S=r.S,
                 F=r.F, U0=r.U0, t0=r.t0, theta_norm=r.theta_norm, y=list(r.y)) for r in rec[:nrec]]
    return rows, S.value, K.value
