"""The benchmark's workload at full size, in the launch configuration the benchmark times:
the closed torus (R = 1, a = 0.4, sigma = 2), 4096 points x 10^4 walks, FP32 walk into
device buffers (4.1e7 walks, 2.15e10 walk-steps per launch).

Checked where the oracle cannot follow every walk:
* properties of every walk: the common stopping index K = 525 (the oracle's
  ceil(ln tau_W / ln c)) and no flags; with f = sigma (u = 1) every score telescopes to
  1 - c^525;
* sampled outputs: per-point means at 8 of the 4096 points against the FP64 oracle's
  (|mean32 - mean64| < 4 combined standard errors)."""
import math

import numpy as np
import pytest

import oracle as O
import paper_2606_21883_b300 as M
from paper_2606_21883_b300 import workloads as W

pytestmark = pytest.mark.gpu
P, N = 4096, 10000


@pytest.fixture(scope="module")
def ctx():
    c = M.Context(0)
    yield c
    c.close()


def _device_walks(ctx, w):
    import torch
    pts = torch.tensor(w.points, dtype=torch.float64, device="cuda")
    S = torch.empty((P, N), dtype=torch.float64, device="cuda")
    K = torch.empty((P, N), dtype=torch.int32, device="cuda")
    F = torch.empty((P, N), dtype=torch.int32, device="cuda")
    ctx.walk_scores_device(w.problem, w.params, pts, N, M.FP32, S, K, F)
    return S, K, F


def _c_of(w):
    r = w.params.theta * w.params.c_kappa / (1.0 + 1.0 / w.problem.manifold.a)
    return O.c_sigma_r(3, math.sqrt(w.problem.sigma) * r)


def test_bench_size_stopping_index_and_means(ctx):
    w = W.torus_closed(P=P, walks=1)
    S, K, F = _device_walks(ctx, w)
    c = _c_of(w)
    k_stop = math.ceil(math.log(w.params.tau_w) / math.log(c))
    assert k_stop == 525
    assert bool((K == k_stop).all()) and not bool(F.any())
    mean32 = S.mean(dim=1).cpu().numpy()
    se32 = (S.std(dim=1) / math.sqrt(N)).cpu().numpy()
    idx = np.random.default_rng(11).choice(P, size=8, replace=False)
    mo, so, to, nf = O.solve(w.problem, w.params, w.points[idx], 1500)
    assert nf == 0 and np.all(to == k_stop)
    assert np.all(np.abs(mean32[idx] - mo) < 4 * np.sqrt(se32[idx] ** 2 + so ** 2))


def test_bench_size_telescoping(ctx):
    w = W.constant_solution(W.torus_closed(P=P, walks=1))
    S, K, F = _device_walks(ctx, w)
    want = 1.0 - _c_of(w) ** 525
    assert bool((K == 525).all()) and not bool(F.any())
    assert float((S - want).abs().max()) < 1e-6
