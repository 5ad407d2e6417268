"""The FP32 embedded-sphere walk with the projection Q^T g on the tensor cores.

Both FP32 embedded walks draw identical Philox numbers; they differ only in how
Q^T g is formed.  The tensor-core product (BF16 hi/lo split, three products,
FP32 accumulation) has, per component, |error| <= ~2^-15.5 |g| (each term
q g loses at most the lo x lo product and the two BF16 residual roundings,
2^-18 + 2 * 2^-17 of |q g|, and sum_i |Q_ij g_i| <= |g| for an orthonormal
column); the CUDA-core walk has FP32 accumulation error of the same order.
The stopping index is exact arithmetic on the weights (constant radius), so K
and the flags must match bit for bit; S is compared with a tolerance that
covers the per-step error accumulated over K steps (see the test).
Against the FP64 oracle the FP32 walk is compared statistically:
|mean32 - mean64| < 4 sqrt(se32^2 + se64^2).
"""
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


def _both(ctx, w, N):
    a = ctx.walk_scores(w.problem, w.params, w.points, N, precision=M.FP32, projection=M.PROJ_TENSOR)
    b = ctx.walk_scores(w.problem, w.params, w.points, N, precision=M.FP32, projection=M.PROJ_CUDA)
    return a, b


def _per_walk_close(a, b, K):
    (St, Kt, Ft), (Sc, Kc, Fc) = a, b
    assert np.array_equal(Kt, Kc)
    assert np.array_equal(Ft, Fc)
    # per-step perturbation of s ~ r 2^-15 |g|/|g| per component, accumulated as
    # a random walk over K steps and weighted by sum W omega <= 1/sigma times the
    # Lipschitz constant of f (O(10) here): |dS| <= 1e-4 sqrt(K) max(1, |S|) is
    # > 10x the expected size and far below the Monte Carlo spread of S.
    tol = 1e-4 * np.sqrt(np.maximum(K, 1)) * np.maximum(1.0, np.abs(Sc))
    d = np.abs(St - Sc)
    assert np.all(d <= tol), f"max |dS| {d.max():.3e}, tol {tol.min():.3e}"
    assert np.median(d) <= 1e-5 * np.sqrt(max(int(K.max()), 1)) * max(1.0, float(np.median(np.abs(Sc))))


@pytest.mark.parametrize("n,d,P,N", [(1000, 20, 5, 61),    # 16 K-chunks (last 40 wide), 3 tiles, ragged
                                     (1024, 30, 3, 128),   # n = 1024 exactly, D = 31 (DQ 32)
                                     (200, 7, 4, 50),      # 4 chunks (last 8 wide), DQ 8
                                     (64, 12, 3, 100)])    # one chunk, forced tensor path below n = 128
def test_tc_matches_cuda_cores_per_walk(ctx, n, d, P, N):
    w = W.embedded_s20(P=P, walks=1, n=n, d=d)
    w.params.max_steps = 40
    a, b = _both(ctx, w, N)
    assert np.all(a[2] == 1) and np.all(a[1] == 40)
    _per_walk_close(a, b, a[1])


def test_tc_complete_walks_match_cuda_cores(ctx):
    """Walks that end by W < tau_W (every walk of the tile at the same index)."""
    w = W.embedded_s20(P=6, walks=1, n=128, d=5, sigma=6.0)
    w.params.tau_w = 1e-4
    a, b = _both(ctx, w, 40)
    assert np.all(a[2] == 0) and np.all(a[1] == a[1].flat[0])
    _per_walk_close(a, b, a[1])


def test_tc_walk_independent_of_batch(ctx):
    """A walk's score depends on (point, walk index) only, not on the tile it shares."""
    w = W.embedded_s20(P=7, walks=1)
    w.params.max_steps = 12
    S7, K7, _ = ctx.walk_scores(w.problem, w.params, w.points, 45, precision=M.FP32, projection=M.PROJ_TENSOR)
    S3, K3, _ = ctx.walk_scores(w.problem, w.params, w.points[:3], 45, precision=M.FP32,
                                projection=M.PROJ_TENSOR)
    assert np.array_equal(S7[:3], S3) and np.array_equal(K7[:3], K3)
    S7b, _, _ = ctx.walk_scores(w.problem, w.params, w.points, 45, precision=M.FP32, projection=M.PROJ_TENSOR)
    assert np.array_equal(S7, S7b)


def test_tc_vs_oracle_statistical_complete(ctx):
    """S^5 in R^128, sigma = 6: complete walks, FP32 tensor-core mean vs the FP64 oracle."""
    w = W.embedded_s20(P=4, walks=1, n=128, d=5, sigma=6.0)
    w.params.tau_w = 1e-4
    N = 600
    m32, s32, t32, rc = ctx.solve(w.problem, w.params, w.points, N, precision=M.FP32, projection=M.PROJ_TENSOR)
    mo, so, to, nf = O.solve(w.problem, w.params, w.points, N)
    assert rc == M.MPWOS_OK and nf == 0
    assert np.all(np.abs(m32 - mo) < 4 * np.sqrt(s32 ** 2 + so ** 2))
    assert np.all(np.abs(t32 - to) <= 1)


def test_tc_vs_oracle_statistical_n1000(ctx):
    """S^20 in R^1000 (the 1000-dimensional embedding), walks capped at 30 steps."""
    w = W.embedded_s20(P=3, walks=1)
    w.params.max_steps = 30
    N = 400
    m32, s32, t32, rc = ctx.solve(w.problem, w.params, w.points, N, precision=M.FP32, projection=M.PROJ_TENSOR)
    mo, so, to, nf = O.solve(w.problem, w.params, w.points, N)
    assert rc == M.MPWOS_EMAXSTEPS and nf == 3 * N
    assert np.all(np.abs(m32 - mo) < 4 * np.sqrt(s32 ** 2 + so ** 2))


def test_tc_auto_selects_tensor_path_for_large_n(ctx):
    w = W.embedded_s20(P=2, walks=1)
    w.params.max_steps = 5
    auto = ctx.walk_scores(w.problem, w.params, w.points, 20, precision=M.FP32)
    tcr = ctx.walk_scores(w.problem, w.params, w.points, 20, precision=M.FP32, projection=M.PROJ_TENSOR)
    assert np.array_equal(auto[0], tcr[0])


def test_tc_rejected_outside_fp32_embedded(ctx):
    w = W.embedded_s20(P=2, walks=1)
    w.params.max_steps = 5
    with pytest.raises(M.MpwosError) as e:
        ctx.walk_scores(w.problem, w.params, w.points, 4, precision=M.FP64, projection=M.PROJ_TENSOR)
    assert e.value.code == M.MPWOS_EINVAL
    t = W.torus_closed(P=2, walks=1)
    with pytest.raises(M.MpwosError) as e:
        ctx.walk_scores(t.problem, t.params, t.points, 4, precision=M.FP32, projection=M.PROJ_TENSOR)
    assert e.value.code == M.MPWOS_EINVAL


def test_tc_empty(ctx):
    w = W.embedded_s20(P=2, walks=1)
    S, K, F = ctx.walk_scores(w.problem, w.params, w.points[:0], 5, precision=M.FP32, projection=M.PROJ_TENSOR)
    assert S.size == 0


# ------------------------------------------------- the contraction on its own
def _embedding(n, D, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, D)))
    return Q


@pytest.mark.parametrize("n,D,rows", [(1000, 21, 300), (1024, 31, 129), (200, 6, 128), (64, 12, 1), (37, 3, 77)])
def test_tc_project_vs_fp64_product(ctx, n, D, rows):
    """out = G Q through the tensor cores: per component |out - G Q| <= 2^-15.5 |g| (derivation in the module
    docstring), |G_r|^2 to FP32 summation accuracy; tiles of 128 rows with a ragged tail."""
    Q = _embedding(n, D, n + D)
    G = np.random.default_rng(rows).standard_normal((rows, n)).astype(np.float32)
    out, gg = ctx.tc_project(Q, G)
    ref = G.astype(np.float64) @ Q
    gn = np.linalg.norm(G.astype(np.float64), axis=1)
    assert np.all(np.abs(out - ref) <= 2 ** -15.5 * gn[:, None])
    assert np.allclose(gg, gn ** 2, rtol=n * 2 ** -24, atol=0)


def test_tc_project_unit_rows(ctx):
    """G = unit rows e_k: out row = Q[k, :] to the hi + lo split's accuracy (the row and column maps)."""
    n, D = 1000, 21
    Q = _embedding(n, D, 5)
    ks = np.arange(0, n, 3)
    G = np.zeros((ks.size, n), dtype=np.float32)
    G[np.arange(ks.size), ks] = 1.0
    out, gg = ctx.tc_project(Q, G)
    assert np.all(np.abs(out - Q[ks]) <= 2 ** -16 * np.abs(Q[ks]) + 1e-30)
    assert np.all(gg == 1.0)
