"""B300 MPWoS: the modified projected Walk on Spheres hot path in CUDA (sm_103a).

This module is the thin Python binding of the C ABI in ``include/mpwos.h``
(``libmpwos.so``, built in-tree by ``build.py``).  It only marshals arguments:
every step of the walk runs in the library's kernels.  Importing the package
does not load the library; the first call does, and raises if the library or
a CUDA device is missing — there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

__all__ = ["lib", "Context", "MPWOS_OK", "MPWOS_EMAXSTEPS", "FP64", "FP32", "MpwosError"]

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmpwos.so")

MPWOS_OK, MPWOS_EINVAL, MPWOS_ENOMEM, MPWOS_ECUDA = 0, 1, 2, 3
MPWOS_ETIMEDOUT, MPWOS_ECANCELED, MPWOS_EMAXSTEPS, MPWOS_ENOTFOUND, MPWOS_EBUSY = 4, 5, 6, 7, 8
FP64, FP32 = 0, 1
PROJ_AUTO, PROJ_TENSOR, PROJ_CUDA = 0, 1, 2
SAMPLER_FULL, SAMPLER_REDUCED = 0, 1
KNN_GRID, KNN_GRID_WARP, KNN_SCAN = 0, 1, 2
COMP_NONE, COMP_NORMAL2, COMP_EXACT = 0, 1, 2

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class MpwosError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"mpwos error {code}: {msg}")
        self.code = code


class ManifoldDesc(C.Structure):
    _fields_ = [("kind", C.c_int), ("n", C.c_int), ("d", C.c_int), ("R", C.c_double), ("a", C.c_double),
                ("Q", _dp), ("b", _dp), ("cloud", _dp), ("n_cloud", C.c_int64), ("k_nn", C.c_int),
                ("c_h", C.c_double), ("cp_mode", C.c_int), ("prof_alpha", C.c_double),
                ("prof_kappa", C.c_double)]


class Func(C.Structure):
    _fields_ = [("kind", C.c_int), ("apply_op", C.c_int), ("n_terms", C.c_int), ("coef", _dp),
                ("term_off", _ip), ("var", _ip), ("pw", _ip), ("modes", _ip), ("c0", C.c_double),
                ("v", _dp), ("A", _dp)]


class ProblemDesc(C.Structure):
    _fields_ = [("sigma", C.c_double), ("closed", C.c_int), ("bnd_normal", _dp), ("bnd_offset", C.c_double),
                ("f", Func), ("g", Func), ("comp", C.c_int), ("u_star", Func), ("h_eta", C.c_double)]


class Params(C.Structure):
    _fields_ = [("eps", C.c_double), ("tau_w", C.c_double), ("theta", C.c_double), ("c_kappa", C.c_double),
                ("n_v", C.c_int), ("max_steps", C.c_int64), ("seed", C.c_uint64), ("precision", C.c_int),
                ("projection", C.c_int), ("sampler", C.c_int)]


class TuneEntry(C.Structure):
    _fields_ = [("kernel", C.c_char_p), ("n", C.c_int), ("block", C.c_int), ("n_candidates", C.c_int),
                ("candidates", C.c_int * 4), ("ns_per_walk_step", C.c_double * 4)]


_lib: Optional[C.CDLL] = None


def lib() -> C.CDLL:
    """Load libmpwos.so (built in-tree); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2606_21883_b300/build.py (no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        L.mpwos_last_error.restype = C.c_char_p
        L.mpwos_launch_count.restype = C.c_int64
        L.mpwos_create.argtypes = [C.c_int, C.c_void_p, C.POINTER(C.c_void_p)]
        L.mpwos_manifold_create.argtypes = [C.c_void_p, C.POINTER(ManifoldDesc), C.POINTER(C.c_void_p)]
        L.mpwos_manifold_destroy.argtypes = [C.c_void_p]
        for name in ("mpwos_destroy", "mpwos_last_error", "mpwos_launch_count"):
            getattr(L, name).argtypes = [C.c_void_p]
        L.mpwos_set_stream.argtypes = [C.c_void_p, C.c_void_p]
        L.mpwos_solve.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(ProblemDesc), C.POINTER(Params),
                                  C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]
        L.mpwos_walk_scores.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(ProblemDesc),
                                        C.POINTER(Params), C.c_void_p, C.c_int64, C.c_int64, C.c_void_p,
                                        C.c_void_p, C.c_void_p]
        L.mpwos_philox.argtypes = [C.c_void_p, C.c_void_p, C.c_uint32, C.c_uint32, C.c_void_p, C.c_int64]
        L.mpwos_green_radius.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.c_int64, C.c_int]
        L.mpwos_c_sigma_r.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int64]
        L.mpwos_tc_project.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int64,
                                       C.c_void_p, C.c_void_p]
        L.mpwos_serve_config.argtypes = [C.c_void_p, C.c_int, C.c_size_t, C.c_int64]
        L.mpwos_submit.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(ProblemDesc), C.POINTER(Params),
                                   C.c_void_p, C.c_int64, C.c_int64, C.c_double, C.POINTER(C.c_uint64)]
        L.mpwos_poll.argtypes = [C.c_void_p, C.c_uint64, C.POINTER(C.c_int)]
        L.mpwos_wait.argtypes = [C.c_void_p, C.c_uint64, C.c_double]
        L.mpwos_cancel.argtypes = [C.c_void_p, C.c_uint64]
        L.mpwos_fetch.argtypes = [C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.POINTER(C.c_double)]
        L.mpwos_set_autotune.argtypes = [C.c_void_p, C.c_int]
        L.mpwos_cloud_knn.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_int,
                                      C.c_void_p, C.c_void_p, C.c_void_p]
        L.mpwos_autotune_entries.argtypes = [C.c_void_p, C.POINTER(TuneEntry), C.c_int, C.POINTER(C.c_int)]
        L.mpwos_solve_partial.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(ProblemDesc),
                                          C.POINTER(Params), C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_int64,
                                          C.c_void_p]
        L.mpwos_block_partials_host.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_void_p]
        L.mpwos_merge_partials.argtypes = [C.POINTER(C.c_void_p), C.c_void_p, C.c_int, C.c_int64, C.c_void_p,
                                           C.c_void_p, C.c_void_p, C.POINTER(C.c_int64)]
        L.mpwos_fit_torus_series.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_double, C.c_int, C.c_int,
                                             C.c_void_p, C.c_void_p, C.POINTER(C.c_int)]
        _lib = L
    return _lib


EST_BLOCK, EST_FIELDS = 1024, 5   # walks per estimator block; fields of a block record


def n_blocks(walks: int) -> int:
    """Estimator blocks of a walk range of the given length."""
    return (int(walks) + EST_BLOCK - 1) // EST_BLOCK


def block_partials_host(S, K, flags):
    """mpwos_block_partials_host: the block records (P x nblk x 5) of per-walk
    outputs (P x N host arrays), in the device's summation order; no GPU."""
    S = np.ascontiguousarray(S, dtype=np.float64)
    K = np.ascontiguousarray(K, dtype=np.int32)
    flags = np.ascontiguousarray(flags, dtype=np.int32)
    P, N = S.shape
    part = np.zeros((P, n_blocks(N), EST_FIELDS))
    rc = lib().mpwos_block_partials_host(_ptr(S), _ptr(K), _ptr(flags), int(P), int(N), _ptr(part))
    if rc != MPWOS_OK:
        raise MpwosError(rc, "mpwos_block_partials_host")
    return part


def merge_partials(parts):
    """mpwos_merge_partials: merge the block records of consecutive walk ranges
    (a list of P x nblk_r x 5 host arrays, in range order) into (mean, stderr,
    mean_steps, n_flagged); no GPU."""
    parts = [np.ascontiguousarray(p, dtype=np.float64) for p in parts]
    P = int(parts[0].shape[0]) if parts else 0
    ptrs = (C.c_void_p * max(len(parts), 1))(*[C.c_void_p(p.ctypes.data) for p in parts])
    nblk = np.array([p.shape[1] for p in parts] or [0], dtype=np.int64)
    mean, se, ms = np.zeros(P), np.zeros(P), np.zeros(P)
    nf = C.c_int64(0)
    rc = lib().mpwos_merge_partials(ptrs, _ptr(nblk), len(parts), P, _ptr(mean), _ptr(se), _ptr(ms), C.byref(nf))
    if rc not in (MPWOS_OK, MPWOS_EMAXSTEPS):
        raise MpwosError(rc, "mpwos_merge_partials")
    return mean, se, ms, int(nf.value)


def fit_torus_series(pts, u, R: float, max_m: int = 3, max_q: int = 3):
    """mpwos_fit_torus_series: the least-squares torus Fourier series (modes m <=
    max_m, q <= max_q) through estimates u at points pts (P x 3) of a torus of
    centre-circle radius R, as a u_star closed form; no GPU."""
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    coef = np.zeros(64)
    modes = np.zeros((64, 4), dtype=np.int32)
    nt = C.c_int(0)
    rc = lib().mpwos_fit_torus_series(_ptr(pts), _ptr(u), int(len(u)), float(R), int(max_m), int(max_q),
                                      _ptr(coef), _ptr(modes), C.byref(nt))
    if rc != MPWOS_OK:
        raise MpwosError(rc, "mpwos_fit_torus_series")
    from . import workloads as W
    n = nt.value
    return W.Func.torus([(float(coef[t]), *map(int, modes[t])) for t in range(n)], apply_op=False)


def _ptr(x):
    """Address of a host numpy array or a device torch tensor."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return C.c_void_p(x.data_ptr())
    return C.c_void_p(x.ctypes.data)


class _Marshal:
    """Keeps the arrays behind a ProblemDesc alive for the duration of a call."""

    def __init__(self):
        self.keep = []

    def arr(self, a, dtype=np.float64):
        a = np.ascontiguousarray(a, dtype=dtype)
        self.keep.append(a)
        return a

    def func(self, f) -> Func:
        from . import workloads as W
        cf = Func(kind=f.kind, apply_op=f.apply_op, n_terms=len(f.coef), c0=f.c0)
        if f.kind == W.FUNC_POLY:
            coef, off, var, pw = f.flat_poly()
            cf.coef = self.arr(coef).ctypes.data_as(_dp)
            cf.term_off = self.arr(off, np.int32).ctypes.data_as(_ip)
            cf.var = self.arr(var, np.int32).ctypes.data_as(_ip)
            cf.pw = self.arr(pw, np.int32).ctypes.data_as(_ip)
        elif f.kind in (W.FUNC_TORUS_FOURIER, W.FUNC_CURVE_SPHERE):
            coef, modes = f.flat_modes()
            cf.coef = self.arr(coef).ctypes.data_as(_dp)
            cf.modes = self.arr(modes, np.int32).ctypes.data_as(_ip)
            if f.kind == W.FUNC_CURVE_SPHERE:
                cf.v = self.arr(f.v).ctypes.data_as(_dp)
                cf.A = self.arr(f.A).ctypes.data_as(_dp)
        else:
            if f.kind == W.FUNC_REVOLUTION_QUAD:
                cf.coef = self.arr(np.asarray(f.coef, dtype=np.float64)).ctypes.data_as(_dp)
            cf.v = self.arr(f.v).ctypes.data_as(_dp)
            cf.A = self.arr(f.A).ctypes.data_as(_dp)
        return cf

    def manifold(self, m) -> ManifoldDesc:
        md = ManifoldDesc(kind=m.kind, n=m.n, d=m.d, R=m.R, a=m.a, prof_alpha=getattr(m, "prof_alpha", 0.0),
                          prof_kappa=getattr(m, "prof_kappa", 0.0))
        if m.Q is not None:
            md.Q = self.arr(m.Q).ctypes.data_as(_dp)
            md.b = self.arr(m.b).ctypes.data_as(_dp)
        if m.cloud is not None:
            # the same host array on every call, so the context's grid cache hits
            if not (m.cloud.flags.c_contiguous and m.cloud.dtype == np.float64):
                m.cloud = np.ascontiguousarray(m.cloud, dtype=np.float64)
            md.cloud = m.cloud.ctypes.data_as(_dp)
            md.n_cloud = m.cloud.shape[0]
            md.k_nn = m.k_nn
            md.c_h = m.c_h
            md.cp_mode = m.cp_mode
        return md

    def problem(self, problem):
        pd = ProblemDesc(sigma=problem.sigma, closed=int(problem.closed), bnd_offset=problem.bnd_offset)
        if problem.bnd_normal is not None:
            pd.bnd_normal = self.arr(problem.bnd_normal).ctypes.data_as(_dp)
        pd.f = self.func(problem.f)
        pd.g = self.func(problem.g)
        if getattr(problem, "comp", COMP_NONE) != COMP_NONE:
            pd.comp = problem.comp
            pd.u_star = self.func(problem.u_star)
            pd.h_eta = problem.h_eta
        return pd


def make_params(params, precision, projection=PROJ_AUTO) -> Params:
    return Params(eps=params.eps, tau_w=params.tau_w, theta=params.theta, c_kappa=params.c_kappa,
                  n_v=params.n_v, max_steps=params.max_steps, seed=params.seed, precision=precision,
                  projection=projection, sampler=getattr(params, "sampler", SAMPLER_FULL))


class Context:
    """One library context (mpwos_create) on a CUDA device."""

    def __init__(self, device: int = 0, stream_handle: Optional[int] = None):
        self.L = lib()
        h = C.c_void_p()
        rc = self.L.mpwos_create(device, C.c_void_p(stream_handle) if stream_handle else None, C.byref(h))
        if rc != MPWOS_OK:
            raise MpwosError(rc, f"mpwos_create(device={device}) failed")
        self.h = h
        self.device = device
        self._manifolds = {}   # id(manifold) -> (manifold, signature, handle)

    def close(self):
        if getattr(self, "h", None):
            for _, _, mh in self._manifolds.values():
                self.L.mpwos_manifold_destroy(mh)
            self._manifolds = {}
            self.L.mpwos_destroy(self.h)
            self.h = None

    @staticmethod
    def _signature(m):
        arrs = tuple((id(a), a.ctypes.data, a.shape) if a is not None else None
                     for a in (getattr(m, "Q", None), getattr(m, "b", None), getattr(m, "cloud", None)))
        return (m.kind, m.n, m.d, m.R, m.a, getattr(m, "prof_alpha", 0.0), getattr(m, "prof_kappa", 0.0),
                getattr(m, "k_nn", 0), getattr(m, "c_h", 0.0), getattr(m, "cp_mode", 0), arrs)

    def manifold_handle(self, m) -> C.c_void_p:
        """The mpwos_manifold handle of a workloads.Manifold on this context
        (mpwos_manifold_create once per manifold object; made again if the
        object's fields or arrays are replaced)."""
        sig = self._signature(m)
        hit = self._manifolds.get(id(m))
        if hit is not None and hit[0] is m and hit[1] == sig:
            return hit[2]
        if hit is not None:
            self.L.mpwos_manifold_destroy(hit[2])
            del self._manifolds[id(m)]
        mar = _Marshal()
        md = mar.manifold(m)
        mh = C.c_void_p()
        self._check(self.L.mpwos_manifold_create(self.h, md, C.byref(mh)))
        self._manifolds[id(m)] = (m, sig, mh)
        return mh

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self) -> str:
        return self.L.mpwos_last_error(self.h).decode()

    def launch_count(self) -> int:
        return int(self.L.mpwos_launch_count(self.h))

    def _check(self, rc, allow=(MPWOS_OK,)):
        if rc not in allow:
            raise MpwosError(rc, self.last_error())
        return rc

    def set_stream(self, stream_handle: int):
        return self._check(self.L.mpwos_set_stream(self.h, C.c_void_p(stream_handle)))

    def cloud_knn(self, problem, x, precision=FP32, method=KNN_GRID, out=None):
        """mpwos_cloud_knn: the k nearest cloud points of the queries x (nq x 3) as the
        walk finds them: (idx nq x k, d2 nq x k, h nq).  x host or device; out, if given,
        is a tuple of device tensors (idx int32, d2, h) written in place."""
        mar = _Marshal()
        md = self.manifold_handle(problem.manifold)
        nq = int(x.shape[0])
        if not hasattr(x, "data_ptr"):
            x = mar.arr(x)
        k = int(problem.manifold.k_nn)
        if out is None:
            idx = np.zeros((nq, k), dtype=np.int32)
            d2 = np.zeros((nq, k))
            h = np.zeros(nq)
        else:
            idx, d2, h = out
        rc = self.L.mpwos_cloud_knn(self.h, md, _ptr(x), nq, int(precision), int(method), _ptr(idx),
                                    _ptr(d2), _ptr(h))
        self._check(rc)
        return idx, d2, h

    def set_autotune(self, enable: bool = True):
        """Turn the launch-shape autotuner on or off (mpwos_set_autotune)."""
        return self._check(self.L.mpwos_set_autotune(self.h, 1 if enable else 0))

    def autotune_entries(self) -> list:
        """The autotuner's picks: one dict per (kernel, n) with the pick and the
        measured GPU ns per walk-step of each candidate block size."""
        count = C.c_int(0)
        self._check(self.L.mpwos_autotune_entries(self.h, None, 0, C.byref(count)))
        arr = (TuneEntry * max(count.value, 1))()
        self._check(self.L.mpwos_autotune_entries(self.h, arr, count.value, C.byref(count)))
        out = []
        for e in arr[:count.value]:
            nc = e.n_candidates
            out.append({"kernel": e.kernel.decode() if e.kernel else None, "n": e.n, "block": e.block,
                        "ns_per_walk_step": {int(e.candidates[c]): float(e.ns_per_walk_step[c])
                                             for c in range(nc)}})
        return out

    # -- the walk ---------------------------------------------------------------
    def solve(self, problem, params, pts, N, precision=FP64, out=None, projection=PROJ_AUTO):
        """mpwos_solve: returns (mean, stderr, mean_steps, status); pts host or device."""
        mar = _Marshal()
        pd = mar.problem(problem)
        md = self.manifold_handle(problem.manifold)
        prm = make_params(params, precision, projection)
        P = int(pts.shape[0])
        if out is None:
            out = (np.zeros(P), np.zeros(P), np.zeros(P))
        if not hasattr(pts, "data_ptr"):
            pts = mar.arr(pts)
        rc = self.L.mpwos_solve(self.h, md, C.byref(pd), C.byref(prm), _ptr(pts), P, int(N),
                                _ptr(out[0]), _ptr(out[1]), _ptr(out[2]))
        self._check(rc, (MPWOS_OK, MPWOS_EMAXSTEPS))
        return out[0], out[1], out[2], rc

    def solve_partial(self, problem, params, pts, N, i0, i1, precision=FP64, projection=PROJ_AUTO, out=None):
        """mpwos_solve_partial: block records (P x nblk x 5) of walks [i0, i1) of a
        request of N walks per point; pts host or device; out a host array or a
        device tensor of that shape."""
        mar = _Marshal()
        pd = mar.problem(problem)
        md = self.manifold_handle(problem.manifold)
        prm = make_params(params, precision, projection)
        P = int(pts.shape[0])
        if out is None:
            out = np.zeros((P, n_blocks(int(i1) - int(i0)), EST_FIELDS))
        if not hasattr(pts, "data_ptr"):
            pts = mar.arr(pts)
        rc = self.L.mpwos_solve_partial(self.h, md, C.byref(pd), C.byref(prm), _ptr(pts), P, int(N),
                                        int(i0), int(i1), _ptr(out))
        self._check(rc)
        return out

    def fit_torus_predictor(self, problem, params, P=400, walks=2000, max_m=3, max_q=3, seed=12345,
                            precision=FP32):
        """u_* of Sec. 2.3.3 for a torus problem: the baseline solve (m_* = 0) at P
        points of Omega, then mpwos_fit_torus_series through its estimates."""
        from . import workloads as W
        if problem.manifold.kind != W.MANIFOLD_TORUS:
            raise ValueError("fit_torus_predictor needs a torus problem")
        base = W.Problem(problem.manifold, problem.sigma, problem.closed, problem.f, problem.g,
                         problem.bnd_normal, problem.bnd_offset)
        pts = W.torus_domain_points(problem, P, seed)
        u = self.solve(base, params, pts, walks, precision=precision)[0]
        return fit_torus_series(pts, u, problem.manifold.R, max_m, max_q)

    def walk_scores(self, problem, params, pts, N, precision=FP64, projection=PROJ_AUTO):
        """mpwos_walk_scores: per-walk S (P x N), K, flags."""
        mar = _Marshal()
        pd = mar.problem(problem)
        md = self.manifold_handle(problem.manifold)
        prm = make_params(params, precision, projection)
        P = int(pts.shape[0])
        if not hasattr(pts, "data_ptr"):
            pts = mar.arr(pts)
        S = np.zeros((P, int(N)))
        K = np.zeros((P, int(N)), dtype=np.int32)
        fl = np.zeros((P, int(N)), dtype=np.int32)
        rc = self.L.mpwos_walk_scores(self.h, md, C.byref(pd), C.byref(prm), _ptr(pts), P, int(N),
                                      _ptr(S), _ptr(K), _ptr(fl))
        self._check(rc)
        return S, K, fl

    def walk_scores_device(self, problem, params, pts, N, precision, S, K, flags, projection=PROJ_AUTO):
        """mpwos_walk_scores into caller-owned device tensors (no host copies)."""
        mar = _Marshal()
        pd = mar.problem(problem)
        md = self.manifold_handle(problem.manifold)
        prm = make_params(params, precision, projection)
        rc = self.L.mpwos_walk_scores(self.h, md, C.byref(pd), C.byref(prm), _ptr(pts),
                                      int(pts.shape[0]), int(N), _ptr(S), _ptr(K), _ptr(flags))
        return self._check(rc)

    # -- serving ------------------------------------------------------------------
    def serve_config(self, max_active=0, mem_bytes=0, chunk_walks=0):
        return self._check(self.L.mpwos_serve_config(self.h, int(max_active), int(mem_bytes), int(chunk_walks)))

    def submit(self, problem, params, pts, walk_budget, target_stderr=0.0, precision=FP32, projection=PROJ_AUTO):
        """mpwos_submit: returns the request id (query points copied at submit)."""
        mar = _Marshal()
        pd = mar.problem(problem)
        md = self.manifold_handle(problem.manifold)
        prm = make_params(params, precision, projection)
        pts = mar.arr(pts)
        rid = C.c_uint64(0)
        self._check(self.L.mpwos_submit(self.h, md, C.byref(pd), C.byref(prm), _ptr(pts),
                                        int(pts.shape[0]), int(walk_budget), float(target_stderr), C.byref(rid)))
        return int(rid.value)

    def poll(self, rid):
        st = C.c_int(0)
        self._check(self.L.mpwos_poll(self.h, C.c_uint64(rid), C.byref(st)))
        return int(st.value)

    def wait(self, rid, timeout_s=-1.0):
        return self._check(self.L.mpwos_wait(self.h, C.c_uint64(rid), float(timeout_s)), (MPWOS_OK, MPWOS_ETIMEDOUT))

    def cancel(self, rid):
        return self._check(self.L.mpwos_cancel(self.h, C.c_uint64(rid)))

    def fetch(self, rid, P):
        """mpwos_fetch: (mean, stderr, mean_steps, walks, latency_s, status)."""
        mean, se, ms = np.zeros(P), np.zeros(P), np.zeros(P)
        walks = np.zeros(P, dtype=np.int64)
        lat = C.c_double(0.0)
        rc = self.L.mpwos_fetch(self.h, C.c_uint64(rid), _ptr(mean), _ptr(se), _ptr(ms), _ptr(walks), C.byref(lat))
        self._check(rc, (MPWOS_OK, MPWOS_EMAXSTEPS, MPWOS_ECANCELED))
        return mean, se, ms, walks, float(lat.value), rc

    # -- primitives -------------------------------------------------------------
    def philox(self, ctr, key0, key1):
        ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
        out = np.zeros_like(ctr)
        self._check(self.L.mpwos_philox(self.h, _ptr(ctr), key0, key1, _ptr(out), ctr.shape[0]))
        return out

    def tc_project(self, Q, G):
        """mpwos_tc_project: (G Q, |G_r|^2) through the tensor-core contraction (FP32)."""
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        G = np.ascontiguousarray(G, dtype=np.float32)
        n, D = Q.shape
        rows = G.shape[0]
        assert G.shape[1] == n
        out = np.zeros((rows, D), dtype=np.float32)
        gg = np.zeros(rows, dtype=np.float32)
        self._check(self.L.mpwos_tc_project(self.h, _ptr(Q), int(n), int(D), _ptr(G), int(rows), _ptr(out),
                                            _ptr(gg)))
        return out, gg

    def green_radius(self, n, a_max, a, U, precision=FP64):
        a = np.ascontiguousarray(a, dtype=np.float64)
        U = np.ascontiguousarray(U, dtype=np.float64)
        t = np.zeros_like(a)
        self._check(self.L.mpwos_green_radius(self.h, n, a_max, _ptr(a), _ptr(U), _ptr(t), a.size, precision))
        return t

    def c_sigma_r(self, n, a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        c = np.zeros_like(a)
        self._check(self.L.mpwos_c_sigma_r(self.h, n, _ptr(a), _ptr(c), a.size))
        return c
