"""The coarse predictor u_* of the compensation term (Sec. 2.3.3).

The compensated method needs u_* only through closed forms the walk kernels
evaluate (a torus Fourier series here).  This module builds one the way the
paper does: a coarse Monte Carlo solution of the same problem with m_* = 0,
then a least-squares fit of the series to it.  It is problem setup done once
on the host before the compensated solve, not a step of the walk: the coarse
solve runs in the library's kernels like any other.
"""
from __future__ import annotations

import math
from typing import Callable, List, Tuple

import numpy as np

from . import workloads as W


def torus_basis(max_m: int, max_q: int) -> List[Tuple[int, int, int, int]]:
    """All T(m theta) P(q phi), T, P in {cos, sin}, m <= max_m, q <= max_q, without sin(0 .)."""
    out = []
    for m in range(max_m + 1):
        for tk in ((W.TRIG_COS,) if m == 0 else (W.TRIG_COS, W.TRIG_SIN)):
            for q in range(max_q + 1):
                for pk in ((W.TRIG_COS,) if q == 0 else (W.TRIG_COS, W.TRIG_SIN)):
                    out.append((m, q, tk, pk))
    return out


def _domain_points(problem: W.Problem, P: int, seed: int):
    """P points of Omega with (theta, phi) uniform (rejecting e.x <= h on a boundary problem)."""
    man = problem.manifold
    g = np.random.default_rng(seed)
    th_all, ph_all = [], []
    while sum(len(t) for t in th_all) < P:
        th = g.uniform(0.0, 2 * math.pi, 4 * P)
        ph = g.uniform(0.0, 2 * math.pi, 4 * P)
        if not problem.closed:
            x = W.torus_points(th, ph, man.R, man.a)
            keep = x @ problem.bnd_normal > problem.bnd_offset
            th, ph = th[keep], ph[keep]
        th_all.append(th)
        ph_all.append(ph)
    th = np.concatenate(th_all)[:P]
    ph = np.concatenate(ph_all)[:P]
    return th, ph, W.torus_points(th, ph, man.R, man.a)


def fit_torus_predictor(solve: Callable, problem: W.Problem, params: W.Params, P: int = 400, walks: int = 2000,
                        max_m: int = 3, max_q: int = 3, seed: int = 12345) -> W.Func:
    """u_* for a torus problem: solve(problem, params, pts, N) -> per-point estimates (the
    baseline method, m_* = 0) at P points of Omega, then the least-squares torus Fourier
    series with modes m <= max_m, q <= max_q (at most 64 terms)."""
    if problem.manifold.kind != W.MANIFOLD_TORUS:
        raise ValueError("fit_torus_predictor needs a torus problem")
    basis = torus_basis(max_m, max_q)
    if len(basis) > 64:
        raise ValueError("at most 64 predictor terms")
    base = W.Problem(problem.manifold, problem.sigma, problem.closed, problem.f, problem.g,
                     problem.bnd_normal, problem.bnd_offset)
    th, ph, pts = _domain_points(problem, P, seed)
    u = np.asarray(solve(base, params, pts, walks), dtype=np.float64)
    trig = (np.cos, np.sin)
    A = np.stack([trig[tk](m * th) * trig[pk](q * ph) for m, q, tk, pk in basis], axis=1)
    coef, *_ = np.linalg.lstsq(A, u, rcond=None)
    return W.Func.torus([(float(c), m, q, tk, pk) for c, (m, q, tk, pk) in zip(coef, basis)], apply_op=False)
