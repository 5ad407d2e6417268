"""The allocation-free solve entry point against the ordinary one.

mpwos_solve_noalloc serves callers that cannot allocate device memory (their
device memory belongs to another allocator, or allocation is forbidden in
their request loop).  It must give the same estimates as mpwos_solve on the
same inputs — it runs the same kernels on the same random draws — and keep
doing so across consecutive calls that reuse its fixed scratch array.  This
file is collected last so that a stop-at-first-failure run has executed every
other test before it.
"""
import ctypes as C

import numpy as np
import pytest

import paper_2606_21883_b300 as M
from paper_2606_21883_b300 import workloads as W

pytestmark = pytest.mark.gpu

REL = 1e-12


def _noalloc(L):
    f = L.mpwos_solve_noalloc
    f.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(M.ProblemDesc), C.POINTER(M.Params),
                  C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]
    f.restype = C.c_int
    L.mpwos_noalloc_max_walks.restype = C.c_int64
    return f


def _call(ctx, fn, work, N, prec, pts_dev, outs):
    mar = M._Marshal()
    pd = mar.problem(work.problem)
    mh = ctx.manifold_handle(work.problem.manifold)
    prm = M.make_params(work.params, prec)
    return fn(ctx.h, mh, C.byref(pd), C.byref(prm), C.c_void_p(pts_dev.data_ptr()),
              int(pts_dev.shape[0]), int(N), *[C.c_void_p(o.data_ptr()) for o in outs])


def _cap_quad(P):
    """The S^2 cap with f given as a SPHERE_QUAD: u = xy + z, f = (-Delta + sigma) u."""
    w = W.sphere_cap(P=P, walks=1)
    A = np.zeros((3, 3))
    A[0, 1] = A[1, 0] = 0.5
    w.problem.f = W.Func.sphere_quad(0.0, np.array([0.0, 0.0, 1.0]), A, apply_op=True)
    return w


def test_noalloc_matches_solve_on_two_consecutive_calls():
    """Every case runs twice in a row through the fixed array and both results
    match mpwos_solve; the cases cover the 65-row radius table (R^3 boundary
    problems), the 1-row table (closed), the FP32 boundary normal, a SPHERE_QUAD
    source, and S^999 (n = 1000, the 17-row table and the R^n warp walk with its
    coordinate order); the first case runs again after the largest one (no stale
    scratch), and a call after the first changes no device memory figure."""
    import torch
    ctx = M.Context(0)
    fn = _noalloc(ctx.L)
    first = (W.sphere_cap(P=16, walks=1), 256, M.FP64)
    cases = [first,                                                     # boundary, 65-row table, FP64
             (W.torus_closed(P=24, walks=1), 300, M.FP32),              # closed, 1-row table
             (W.sphere_cap(P=8, walks=1), 200, M.FP32),                 # FP32 boundary normal
             (_cap_quad(8), 160, M.FP32),                               # SPHERE_QUAD source, FP32
             (W.hypersphere_half(P=3, walks=1, seed=1), 16, M.FP32),    # n = 1000, 17-row table
             first]                                                     # again, after the largest
    for ci, (work, N, prec) in enumerate(cases):
        pts = torch.tensor(work.points, dtype=torch.float64, device="cuda")
        m, s, t, _ = ctx.solve(work.problem, work.params, work.points, N, precision=prec)
        for call in range(2):
            outs = [torch.full((len(work.points),), -7.0, dtype=torch.float64, device="cuda") for _ in range(3)]
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            rc = _call(ctx, fn, work, N, prec, pts, outs)
            torch.cuda.synchronize()
            assert rc == M.MPWOS_OK, ctx.last_error()
            if ci > 0 or call > 0:       # the first call may load kernels; later calls allocate nothing
                assert torch.cuda.mem_get_info()[0] == free0
            got = [o.cpu().numpy() for o in outs]
            for a, b in zip(got, (m, s, t)):
                assert np.all(np.abs(a - b) <= REL * np.maximum(1.0, np.abs(b))), (ci, call)
    ctx.close()


def test_noalloc_rejects_oversize_and_host_pointers():
    import torch
    ctx = M.Context(0)
    fn = _noalloc(ctx.L)
    limit = ctx.L.mpwos_noalloc_max_walks()
    assert limit > 1_000_000
    work = W.torus_closed(P=4, walks=1)
    pts = torch.tensor(work.points, dtype=torch.float64, device="cuda")
    outs = [torch.zeros(4, dtype=torch.float64, device="cuda") for _ in range(3)]
    rc = _call(ctx, fn, work, limit // 4 + 1, M.FP32, pts, outs)
    assert rc == M.MPWOS_EINVAL and "scratch limit" in ctx.last_error()
    mar = M._Marshal()
    pd = mar.problem(work.problem)
    mh = ctx.manifold_handle(work.problem.manifold)
    prm = M.make_params(work.params, M.FP32)
    host = np.zeros(4)
    rc = fn(ctx.h, mh, C.byref(pd), C.byref(prm), C.c_void_p(pts.data_ptr()), 4, 8,
            C.c_void_p(host.ctypes.data), C.c_void_p(outs[1].data_ptr()), C.c_void_p(outs[2].data_ptr()))
    assert rc == M.MPWOS_EINVAL and "device pointers" in ctx.last_error()
    ctx.close()
