"""The point cloud's k-nearest search (the first step of its closest point, Sec. 2.1
representation (iii); h(x) of eq. rho_geo_spacing is the mean neighbour distance) on the
GPU against the oracle's brute force, and the three device methods against each other.

* FP64: the grid search equals the oracle's brute force bit for bit (indices, distances,
  h): the same differences and products without contraction, the same order by
  (distance^2, index).
* Each precision: the grid search, its warp-cooperative form (FP32) and the all-pairs
  scan agree bit for bit.
* FP32 against the oracle: every chosen neighbour lies within FP32 rounding of the true k
  nearest, and the distances agree to FP32 rounding.

Queries: near the surface (cloud points moved by up to 0.02), exactly on cloud points,
far outside the cloud's box and near its centre; one cloud holds exact duplicates, so
ties are decided by index."""
import numpy as np
import pytest

import oracle as O
import paper_2606_21883_b300 as M
from paper_2606_21883_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = M.Context(0)
    yield c
    c.close()


def _queries(cloud, nq, seed):
    rng = np.random.default_rng(seed)
    pick = rng.choice(cloud.shape[0], size=nq, replace=False)
    near = cloud[pick] + rng.uniform(-0.02, 0.02, size=(nq, 3))
    exact = cloud[pick[: nq // 8]]
    far = rng.normal(size=(16, 3))
    far = 3.0 * far / np.linalg.norm(far, axis=1, keepdims=True)
    centre = rng.uniform(-0.1, 0.1, size=(8, 3))
    return np.ascontiguousarray(np.vstack([near, exact, far, centre]))


def _cloud_workload(N, k, dup=0, seed=0):
    w = W.point_cloud(P=4, walks=1, N_cloud=N, k_nn=k, seed=seed)
    if dup:
        c = w.problem.manifold.cloud
        w.problem.manifold.cloud = np.ascontiguousarray(np.vstack([c, c[:dup]]))
    return w


@pytest.mark.parametrize("N,k,dup", [(20_000, 16, 0), (5_000, 6, 200), (5_000, 32, 200)])
def test_knn_fp64_grid_equals_oracle(ctx, N, k, dup):
    w = _cloud_workload(N, k, dup)
    cloud = w.problem.manifold.cloud
    x = _queries(cloud, 256, seed=N + k)
    if dup:   # queries on duplicated points: two neighbours at distance 0
        x = np.ascontiguousarray(np.vstack([x, cloud[:20], cloud[N:N + 20]]))
    idx, d2, h = ctx.cloud_knn(w.problem, x, precision=M.FP64, method=M.KNN_GRID)
    op = O.OracleProblem(w.problem, w.params)
    for q in range(x.shape[0]):
        oi, od, oh = O.cloud_knn(op, x[q])
        assert np.array_equal(idx[q], oi), (q, idx[q], oi)
        assert np.array_equal(d2[q], od), q
        assert h[q] == oh, q
    if dup:   # duplicates tie: the lower index comes first
        on_dup = np.flatnonzero(np.isin(idx[:, 0], np.arange(dup)) & (d2[:, 0] == 0.0))
        assert on_dup.size >= 40
        assert np.all(idx[on_dup, 1] == idx[on_dup, 0] + N)


@pytest.mark.parametrize("k", [6, 16, 32])
def test_knn_methods_identical(ctx, k):
    w = _cloud_workload(200_000, k)
    x = _queries(w.problem.manifold.cloud, 2048, seed=k)
    g64 = ctx.cloud_knn(w.problem, x, precision=M.FP64, method=M.KNN_GRID)
    s64 = ctx.cloud_knn(w.problem, x, precision=M.FP64, method=M.KNN_SCAN)
    for a, b in zip(g64, s64):
        assert np.array_equal(a, b)
    g32 = ctx.cloud_knn(w.problem, x, precision=M.FP32, method=M.KNN_GRID)
    for meth in (M.KNN_GRID_WARP, M.KNN_SCAN):
        o = ctx.cloud_knn(w.problem, x, precision=M.FP32, method=meth)
        for a, b in zip(g32, o):
            assert np.array_equal(a, b), meth


def test_knn_fp32_within_rounding_of_oracle(ctx):
    w = _cloud_workload(200_000, 16)
    cloud = w.problem.manifold.cloud
    x = _queries(cloud, 192, seed=5)
    idx, d2, h = ctx.cloud_knn(w.problem, x, precision=M.FP32, method=M.KNN_GRID)
    op = O.OracleProblem(w.problem, w.params)
    for q in range(x.shape[0]):
        oi, od, oh = O.cloud_knn(op, x[q])
        true_d2 = np.sum((cloud[idx[q]] - x[q]) ** 2, axis=1)
        scale = np.sum(x[q] ** 2) + 1.0
        tol = 4 * 2.0 ** -23 * scale
        assert np.all(true_d2 <= od[-1] + tol), q            # every pick is among the k nearest up to rounding
        assert np.all(np.abs(d2[q] - true_d2) <= tol), q
        assert abs(h[q] - oh) <= 1e-3 * max(oh, 1e-3), q


def test_knn_device_buffers_and_empty(ctx):
    import torch
    w = _cloud_workload(5_000, 16)
    x = _queries(w.problem.manifold.cloud, 300, seed=9)
    host = ctx.cloud_knn(w.problem, x, precision=M.FP32)
    xd = torch.tensor(x, device="cuda")
    out = (torch.empty((x.shape[0], 16), dtype=torch.int32, device="cuda"),
           torch.empty((x.shape[0], 16), dtype=torch.float64, device="cuda"),
           torch.empty(x.shape[0], dtype=torch.float64, device="cuda"))
    ctx.cloud_knn(w.problem, xd, precision=M.FP32, out=out)
    for a, b in zip(host, out):
        assert np.array_equal(a, b.cpu().numpy())
    e = ctx.cloud_knn(w.problem, np.zeros((0, 3)), precision=M.FP32)
    assert e[0].shape == (0, 16)


def test_knn_rejects_bad_arguments(ctx):
    w = _cloud_workload(5_000, 16)
    x = _queries(w.problem.manifold.cloud, 8, seed=1)
    with pytest.raises(M.MpwosError):
        ctx.cloud_knn(w.problem, x, precision=M.FP64, method=M.KNN_GRID_WARP)
    with pytest.raises(M.MpwosError):
        ctx.cloud_knn(w.problem, x, precision=M.FP32, method=7)
    sph = W.sphere_cap(P=2, walks=1)
    sph.problem.manifold.k_nn = 16
    with pytest.raises(M.MpwosError):
        ctx.cloud_knn(sph.problem, x, precision=M.FP32)
