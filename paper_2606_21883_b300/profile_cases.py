"""Small seeded cases that launch one walk kernel each, for profiler captures.

    python -m paper_2606_21883_b300.profile_cases torus     # walk3_f32_kernel<torus>
    python -m paper_2606_21883_b300.profile_cases s20_tc    # embed_tc_kernel (tensor cores)
    python -m paper_2606_21883_b300.profile_cases s20_cuda  # walkn_f32_kernel<embedded> (CUDA cores)
    python -m paper_2606_21883_b300.profile_cases s999      # walkn_f32_kernel<sphere>
    python -m paper_2606_21883_b300.profile_cases s999_red  # walkr_kernel<float, sphere> (reduced sampler)
    python -m paper_2606_21883_b300.profile_cases s20_red   # walkr_kernel<float, embedded> (reduced sampler)
    python -m paper_2606_21883_b300.profile_cases dumbbell  # walkn_f32_kernel<revolution> (Example 2, n = 1001)
    python -m paper_2606_21883_b300.profile_cases cloud     # walk3_f32_cloud_coop_kernel (the 200k-point cloud, k = 16)
    python -m paper_2606_21883_b300.profile_cases e1_comp   # walk3_f32_kernel<torus, general, m_*> (Example 1)
    python -m paper_2606_21883_b300.profile_cases knn       # cloud_knn_query_kernel and cloud_knn_scan_kernel (200k cloud, k = 16)

Each case runs `--reps` walk launches into device buffers (the first one
warms tables and caches) and prints one line with the walk-steps and the
wall time of the last launch.  Inputs are the same seeded workloads the
tests and the benchmark use, at sizes a profiler replays in seconds.
"""
from __future__ import annotations

import argparse
import time

import numpy as np

from . import FP32, PROJ_CUDA, PROJ_TENSOR, Context
from . import workloads as W


def _case(name):
    if name == "torus":   # 64 points x 2048 walks x 525 steps = 6.9e7 walk-steps
        w = W.torus_closed(P=64, walks=2048)
        return w, 2048, {}
    if name in ("s20_tc", "s20_cuda"):   # S^20 in R^1000, 4 tiles per SM, walks capped at 16 steps
        w = W.embedded_s20(P=148, walks=1)
        w.params.max_steps = 16
        return w, 512, {"projection": PROJ_TENSOR if name == "s20_tc" else PROJ_CUDA}
    if name == "s999":   # S^999 in R^1000, walks capped at 16 steps
        w = W.hypersphere_half(P=148, walks=1)
        w.params.max_steps = 16
        return w, 128, {}
    if name == "s999_red":   # S^999 half to completion (~4900 steps per walk), reduced sampler, ~7 walks per thread
        w = W.hypersphere_half(P=4096, walks=1)
        w.params.sampler = W.SAMPLER_REDUCED
        return w, 256, {}
    if name == "s20_red":   # S^20 in R^1000, reduced sampler, walks capped at 20000 steps
        w = W.embedded_s20(P=1184, walks=1)
        w.params.sampler = W.SAMPLER_REDUCED
        w.params.max_steps = 20000
        return w, 16, {}
    if name == "cloud":   # the serving mix's 200k-point cloud, 64 points x 1024 walks (~720 steps each)
        w = W.point_cloud(P=64, walks=1)
        w.params.tau_w = 1e-4
        return w, 1024, {}
    if name == "e1_comp":   # Example 1's cut torus with the second-order m_*, 100 points x 16384 walks (~73 steps)
        w = W.torus_cut(P=100, walks=1, comp=W.COMP_NORMAL2)
        return w, 16384, {}
    if name == "dumbbell":   # Example 2 in R^1001, walks to completion (~85 steps), 4 walks per warp slot
        w = W.dumbbell(P=2368, walks=1)
        return w, 64, {}
    raise SystemExit(f"unknown case {name}")


def _knn(reps, nq=262144):
    """The 200k cloud's k = 16 nearest of nq queries near the surface: per rep, the
    FP32 grid search (cloud_knn_query_kernel) and then the all-pairs scan
    (cloud_knn_scan_kernel), each timed by wall clock around synchronisation."""
    import torch
    from . import KNN_GRID, KNN_SCAN
    w = W.point_cloud(P=1, walks=1)
    cloud = w.problem.manifold.cloud
    rng = np.random.default_rng(3)
    x = cloud[rng.choice(cloud.shape[0], nq)] + rng.uniform(-0.02, 0.02, (nq, 3))   # the benchmark's queries
    xd = torch.tensor(x, device="cuda")
    k = w.problem.manifold.k_nn
    out = (torch.empty((nq, k), dtype=torch.int32, device="cuda"), torch.empty((nq, k), dtype=torch.float64, device="cuda"),
           torch.empty(nq, dtype=torch.float64, device="cuda"))
    ctx = Context(0)
    for _ in range(max(1, reps)):
        for name, meth in (("grid", KNN_GRID), ("scan", KNN_SCAN)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.cloud_knn(w.problem, xd, precision=FP32, method=meth, out=out)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            print(f"knn {name}: {nq} queries x {cloud.shape[0]} points, {dt * 1e3:.2f} ms wall, {nq / dt:.3e} queries/s")
    ctx.close()


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["torus", "s20_tc", "s20_cuda", "s999", "s999_red", "s20_red", "dumbbell", "cloud",
                                         "e1_comp", "knn"])
    ap.add_argument("--reps", type=int, default=2)
    args = ap.parse_args(argv)
    import torch
    if args.case == "knn":
        return _knn(args.reps)

    w, N, kw = _case(args.case)
    ctx = Context(0)
    P = w.points.shape[0]
    pts = torch.from_numpy(np.ascontiguousarray(w.points)).cuda()
    S = torch.empty((P, N), dtype=torch.float64, device="cuda")
    K = torch.empty((P, N), dtype=torch.int32, device="cuda")
    F = torch.empty((P, N), dtype=torch.int32, device="cuda")
    dt = 0.0
    for _ in range(max(1, args.reps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.walk_scores_device(w.problem, w.params, pts, N, FP32, S, K, F, **kw)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    steps = int(K.sum().item())
    print(f"{args.case}: {P} points x {N} walks, {steps} walk-steps, last launch {dt * 1e3:.2f} ms wall, "
          f"{steps / dt:.3e} walk-steps/s")
    ctx.close()


if __name__ == "__main__":
    main()
