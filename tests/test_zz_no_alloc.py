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
    f.argtypes = [C.c_void_p, C.POINTER(M.ManifoldDesc), C.POINTER(M.ProblemDesc), C.POINTER(M.Params),
                  C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]
    f.restype = C.c_int
    L.mpwos_noalloc_max_walks.restype = C.c_int64
    return f


def _call(ctx, fn, work, N, prec, pts_dev, outs):
    mar = M._Marshal()
    md, pd = mar.problem(work.problem)
    prm = M.make_params(work.params, prec)
    return fn(ctx.h, C.byref(md), C.byref(pd), C.byref(prm), C.c_void_p(pts_dev.data_ptr()),
              int(pts_dev.shape[0]), int(N), *[C.c_void_p(o.data_ptr()) for o in outs])


def test_noalloc_matches_solve_on_two_consecutive_calls():
    import torch
    ctx = M.Context(0)
    fn = _noalloc(ctx.L)
    cases = [(W.sphere_cap(P=16, walks=1), 256, M.FP64),      # boundary problem, 65-row table
             (W.torus_closed(P=24, walks=1), 300, M.FP32)]    # closed problem, 1-row table
    for work, N, prec in cases:
        pts = torch.tensor(work.points, dtype=torch.float64, device="cuda")
        outs = [torch.full((len(work.points),), -7.0, dtype=torch.float64, device="cuda") for _ in range(3)]
        rc = _call(ctx, fn, work, N, prec, pts, outs)
        assert rc == M.MPWOS_OK, ctx.last_error()
        m, s, t, rc2 = ctx.solve(work.problem, work.params, work.points, N, precision=prec)
        got = [o.cpu().numpy() for o in outs]
        for a, b in zip(got, (m, s, t)):
            assert np.all(np.abs(a - b) <= REL * np.maximum(1.0, np.abs(b)))
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
    md, pd = mar.problem(work.problem)
    prm = M.make_params(work.params, M.FP32)
    host = np.zeros(4)
    rc = fn(ctx.h, C.byref(md), C.byref(pd), C.byref(prm), C.c_void_p(pts.data_ptr()), 4, 8,
            C.c_void_p(host.ctypes.data), C.c_void_p(outs[1].data_ptr()), C.c_void_p(outs[2].data_ptr()))
    assert rc == M.MPWOS_EINVAL and "device pointers" in ctx.last_error()
    ctx.close()
