"""The S^999 and S^20-in-R^1000 workloads at their full sizes, in the launch
configurations the benchmark times (FP32, device buffers), where the oracle cannot
follow every walk:

* S^999 half (16384 points x 4096 walks to completion, dimension-reduced sampler):
  with f = sigma and g = 1 (u = 1) every walk's score telescopes to exactly 1 and no
  walk reaches max_steps; on the real data the per-point means stay within the
  standard error plus the method's bias of u = x_1 + x_2 x_3 (the bench's RMSE);
* S^20 in R^1000 (32768 points x 2048 walks, a fixed window of steps): on the closed
  sphere with f = sigma every walk's score after k steps is 1 - c^k, c the oracle's
  c_{sigma,r} in R^1000, for the tensor-core walk (16 steps) and the reduced sampler
  (256 steps); every walk is flagged at the window and none earlier."""
import math

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


def _device_walks(ctx, w, N, **kw):
    import torch
    P = len(w.points)
    pts = torch.tensor(w.points, dtype=torch.float64, device="cuda")
    S = torch.empty((P, N), dtype=torch.float64, device="cuda")
    K = torch.empty((P, N), dtype=torch.int32, device="cuda")
    F = torch.empty((P, N), dtype=torch.int32, device="cuda")
    ctx.walk_scores_device(w.problem, w.params, pts, N, M.FP32, S, K, F, **kw)
    return S, K, F


def test_s999_half_full_size_telescoping(ctx):
    w = W.constant_solution(W.hypersphere_half(P=16384, walks=1))
    w.params.sampler = W.SAMPLER_REDUCED
    S, K, F = _device_walks(ctx, w, 4096)
    assert not bool(F.any())
    assert int(K.min()) >= 0 and float(K.double().mean()) > 1000.0
    assert float((S - 1.0).abs().max()) < 1e-5


def test_s999_half_full_size_means(ctx):
    w = W.hypersphere_half(P=16384, walks=1)
    w.params.sampler = W.SAMPLER_REDUCED
    mean, se, ms, rc = ctx.solve(w.problem, w.params, w.points, 4096, precision=M.FP32)
    assert rc == M.MPWOS_OK
    err = mean - w.exact
    # the baseline method's bias (m_* = 0) is ~1e-3 here: RMSE 1.1e-3 against a mean
    # standard error of 5.3e-4
    assert float(np.sqrt(np.mean(err ** 2))) < 2e-3
    assert np.all(np.abs(err) < 6.0 * se + 4e-3)


def _s20_const(P):
    w = W.embedded_s20(P=P, walks=1)
    D = w.problem.manifold.d + 1
    f = W.Func.sphere_quad(w.problem.sigma, np.zeros(D), np.zeros((D, D)), apply_op=False)
    prob = W.Problem(w.problem.manifold, w.problem.sigma, True, f, W.Func.const(0.0))
    return W.Workload("s20_const", prob, w.points, 1, w.params, np.ones(P), "f32")


def _c_s20(w):
    r = w.params.theta * w.params.c_kappa / 2.0        # rho_geo = c_kappa / (1 + 1) on the unit sphere
    return O.c_sigma_r(w.problem.manifold.n, math.sqrt(w.problem.sigma) * r)


@pytest.mark.parametrize("window,kw", [(16, {"projection": M.PROJ_TENSOR}), (256, {"sampler": True})])
def test_s20_full_size_window_telescoping(ctx, window, kw):
    w = _s20_const(32768)
    w.params.max_steps = window
    if kw.pop("sampler", False):
        w.params.sampler = W.SAMPLER_REDUCED
    S, K, F = _device_walks(ctx, w, 2048, **kw)
    assert bool((K == window).all()) and bool((F == 1).all())
    want = 1.0 - _c_s20(w) ** window
    assert float((S - want).abs().max()) < 2e-6 * window
