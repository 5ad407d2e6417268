"""Request serving (continuous batching) on the GPU.

Each walk draws from (seed, point, walk index) only, so a request's results
cannot depend on the other requests in flight: a request served inside a mixed
batch equals the same request served alone, bit for bit, and a request with
no target standard error equals mpwos_solve with the same walk count."""
import time

import numpy as np
import pytest

import paper_2606_21883_b300 as M
from paper_2606_21883_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = M.Context(0)
    yield c
    c.close()


def _serve(ctx, work, budget, target, prec):
    rid = ctx.submit(work.problem, work.params, work.points, budget, target, precision=prec)
    assert ctx.wait(rid, 120.0) == M.MPWOS_OK
    return ctx.fetch(rid, len(work.points))


def test_served_request_equals_solve(ctx):
    for work, N, prec in [(W.sphere_cap(P=12, walks=1), 300, M.FP64), (W.torus_closed(P=40, walks=1), 500, M.FP32)]:
        mean, se, ms, walks, lat, rc = _serve(ctx, work, N, 0.0, prec)
        m2, s2, t2, rc2 = ctx.solve(work.problem, work.params, work.points, N, precision=prec)
        assert np.array_equal(mean, m2) and np.array_equal(se, s2) and np.array_equal(ms, t2)
        assert np.all(walks == N) and lat > 0


def _mix():
    cap = W.sphere_cap(P=20, walks=1)
    tor = W.torus_closed(P=300, walks=1, seed=3)
    hyp = W.hypersphere_half(P=3, walks=1, seed=4)
    hyp.points[:, 0] = 0.01
    hyp.points[:, 1:] *= np.sqrt(1 - 1e-4) / np.linalg.norm(hyp.points[:, 1:], axis=1, keepdims=True)
    cld = W.point_cloud(P=6, walks=1, N_cloud=20000)
    cld.params.tau_w = 1e-3
    emb = W.embedded_s20(P=2, walks=1, n=64, d=5, sigma=6.0)
    emb.params.tau_w = 1e-4
    cut = W.torus_cut(P=10, walks=1, comp=W.COMP_NORMAL2)   # Example 1, compensated
    dmb = W.dumbbell(P=3, walks=1)                           # Example 2, R^1001
    crv = W.curve_sphere(P=4, walks=1)                       # Example 3, R^9
    return [(cap, 4096, 5e-3, M.FP32), (tor, 8192, 2e-2, M.FP32), (hyp, 256, 0.0, M.FP32),
            (cld, 1024, 2e-2, M.FP32), (emb, 512, 0.0, M.FP64), (cap, 2048, 0.0, M.FP64),
            (cut, 2048, 0.0, M.FP32), (cut, 256, 0.0, M.FP64), (dmb, 512, 0.0, M.FP32),
            (crv, 1024, 1e-2, M.FP32)]


def test_same_alone_and_in_mix(ctx):
    cases = _mix()
    alone = [_serve(ctx, w, b, t, p) for w, b, t, p in cases]
    ids = [ctx.submit(w.problem, w.params, w.points, b, t, precision=p) for w, b, t, p in cases]
    # a second copy of every request, interleaved, so requests overlap on the device
    ids2 = [ctx.submit(w.problem, w.params, w.points, b, t, precision=p) for w, b, t, p in reversed(cases)]
    for rid in ids + ids2:
        assert ctx.wait(rid, 300.0) == M.MPWOS_OK
    mixed = [ctx.fetch(rid, len(w.points)) for rid, (w, _, _, _) in zip(ids, cases)]
    mixed2 = [ctx.fetch(rid, len(w.points)) for rid, (w, _, _, _) in zip(ids2, list(reversed(cases)))]
    mixed2 = list(reversed(mixed2))
    for a, b, c in zip(alone, mixed, mixed2):
        for q in range(4):
            assert np.array_equal(a[q], b[q]) and np.array_equal(a[q], c[q])


def test_target_stderr_rounds(ctx):
    w = W.torus_closed(P=16, walks=1)
    target = 2e-2
    mean, se, ms, walks, lat, rc = _serve(ctx, w, 65536, target, M.FP32)
    assert np.all((se <= target) | (walks == 65536))
    assert np.all(np.isin(walks, 256 * 2 ** np.arange(9)))
    assert np.all(np.abs(mean - w.exact) < 5 * se + 0.05)


def test_cancel_timeout_and_queueing(ctx):
    w = W.torus_closed(P=2048, walks=1)
    ctx.serve_config(mem_bytes=int(2048 * 20000 * 16 * 1.5))       # room for one big request at a time
    big = [ctx.submit(w.problem, w.params, w.points, 20000, 0.0) for _ in range(3)]
    assert ctx.poll(big[2]) == 0                                   # queued behind memory
    assert ctx.wait(big[2], 0.0) == M.MPWOS_ETIMEDOUT
    ctx.cancel(big[2])
    assert ctx.wait(big[2], 10.0) == M.MPWOS_OK
    *_, rc = ctx.fetch(big[2], 2048)
    assert rc == M.MPWOS_ECANCELED
    for rid in big[:2]:
        assert ctx.wait(rid, 120.0) == M.MPWOS_OK
        assert ctx.fetch(rid, 2048)[-1] == M.MPWOS_OK
    ctx.serve_config(mem_bytes=64 << 30)


def test_submit_validation(ctx):
    w = W.sphere_cap(P=2, walks=1)
    w.problem.sigma = 0.0
    with pytest.raises(M.MpwosError) as ei:
        ctx.submit(w.problem, w.params, w.points, 16)
    assert ei.value.code == M.MPWOS_EINVAL
    with pytest.raises(M.MpwosError) as ei:
        ctx.fetch(987654321, 1)
    assert ei.value.code == M.MPWOS_ENOTFOUND


def test_small_request_runs_its_budget_in_one_round(ctx):
    """A request whose P x budget walks fill a small part of one resident wave (not on a
    point cloud) runs the whole budget at once: walks == budget for every point, even where
    the target was met earlier, and the results equal mpwos_solve's with that budget."""
    w = W.embedded_s20(P=2, walks=1, n=64, d=5, sigma=6.0)
    w.params.sampler = W.SAMPLER_REDUCED
    mean, se, ms, walks, lat, rc = _serve(ctx, w, 1024, 0.5, M.FP32)
    assert np.all(walks == 1024)
    m2, s2, t2, rc2 = ctx.solve(w.problem, w.params, w.points, 1024, precision=M.FP32)
    assert np.array_equal(mean, m2) and np.array_equal(se, s2)
