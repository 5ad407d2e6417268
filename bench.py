"""Benchmark of the MPWoS hot path on B300.

Workload (the metric's configuration): the closed torus R = 1, tube radius
0.4, sigma = 2, manufactured u = sin(theta) cos(2 phi), 4096 query points
uniform in (theta, phi), 10^4 walks each (every walk takes exactly 525
steps: 2.15e10 walk-steps per step of the benchmark), FP32 walks with FP64
weights and estimator sums.  A benchmark "step" is one mpwos_solve of that
whole batch (walk kernel + per-point reduction).

Output: one JSON line (rank 0).  ``value`` is whole-job walk-steps/s with the
query points already on the device; ``e2e`` is the same metric through the C
ABI with pinned host buffers (host<->device copies inside the timed region);
``roofline`` is the walk kernel's algorithmic ALU work per launch over its
CUDA-event duration against the SM issue peak; ``cpu_baseline`` times the CPU
oracle on a bounded sample of the same workload.

``--impl reference`` times the CPU oracle (the reference arm of this build).
"""
from __future__ import annotations

import argparse
import copy
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2606_21883_b300 import workloads as W  # noqa: E402

METRIC = "walk-steps/s at fixed RMSE (torus, FP32 walk + FP64 accumulation)"
UNIT = "walk-steps/s"
# Algorithmic lane-operations per walk-step of the FP32 torus walk (N_V = 1):
# the minimal operation count of one step, one wide multiply, three-input XOR
# or MUFU op counting as one: 1 Philox4x32-10 block whose rounds 0..2 have
# their per-walk and per-step work hoisted 34, 5 uniforms (4 from low bits, 1
# from high bits) 14, 2 uniform directions on S^2 (Archimedes: height,
# sqrt(1 - z^2), sincos of the azimuth, 2 products) 18, radius table (side,
# sqrt, index, one 16-byte load, 3 FMA, clamp) 17, Theta and Z 7, torus angles
# of cp(Z) 11, torus source (-Delta_M + sigma) u for one mode 16, closest point
# of Theta 13, weight and score in float pairs (S += V F by TwoSum, V *= c) 15,
# loop 3.
OPS_PER_STEP = 148
# DRAM bytes (read + write) of one bench launch of the walk kernel, measured
# by ncu (dram__bytes_read.sum + dram__bytes_write.sum, one pass) on the
# kernel as built now; the profile summary gives the command.
TRAFFIC_BYTES = 15.51e6 + 600.60e6


# Algorithmic lane-operations per walk-step of the other walk kernels (N_V = 1),
# counted the same way (warp-uniform scalar work once per walker).
def ops_full_sampler(n, revolution=False):
    """The R^n warp walk with the full sampler (n Gaussians per direction), per
    16-component group of a direction: 3 Philox blocks with rounds 0..2 hoisted
    (3 x 34 = 102), 8 radial halves (mask, 2 - m, log2, sqrt, sum: 40), 8 angle
    halves (16-bit fraction: 2, 2 pi scale, sin, cos, 2 products: 56); then Z:
    Yh.g with Yh from shared memory (16 FMA + 4 loads), Theta: radii to and
    from shared memory (4), Yh += s g and |Yh|^2 (32 FMA + 8 loads/stores).
    The hypersurface of revolution's Z adds (Yh + s g), v and A terms per
    component (5.5, with v and A loads).  Scalar part of a step: 200."""
    groups = n / 16.0
    z = 102 + 40 + 56 + (16 * 5.5 + 10 if revolution else 20)
    theta = 102 + 40 + 56 + 4 + 40
    return groups * (z + theta) + 200


def ops_tc_embedded(n):
    """The tensor-core embedded-sphere walk: per component of each of the two
    directions, its share of a 16-component group (3 hoisted Philox blocks
    102 / 16, 8 radial halves 40 / 16, 8 angle halves 56 / 16), the BF16 hi/lo
    split (3), the shared-memory store (0.25); the Q^T g products run on the
    tensor pipe.  Scalar part: 300."""
    return 2 * n * ((102 + 40 + 56) / 16 + 3 + 0.25) + 300


# The dimension-reduced sampler on S^999 (walkr_kernel): per direction one
# Philox block of 4 normals (40 + 2 Box-Muller pairs 23.5) and one chi^2 by
# Marsaglia-Tsang (its block 40 + a pair 11.75 + the acceptance test 17), and
# per step the radius, weights, stop test and source (~80).
OPS_REDUCED_S999 = 2 * (40 + 23.5 + 40 + 11.75 + 17) + 80
MUFU_PER_PAIR = 4   # log2, sqrt, sin, cos of one Box-Muller pair


def ops_reduced_embedded(d):
    """The dimension-reduced sampler on S^d embedded in R^1000 (walkr_kernel), per
    direction: d + 1 intrinsic normals (ceil((d + 1) / 4) Philox blocks at 40,
    ceil((d + 1) / 2) Box-Muller pairs at 11.75) and one chi^2 by Marsaglia-Tsang
    (68.75); per step: the Theta and Z updates with their normalisations
    (2 x (3 (d + 1) + 2)), the source v.z + z^T A z ((d + 1)^2 + 2 (d + 1)) and the
    radius, weights and stop test (80)."""
    D = d + 1
    direction = 40 * math.ceil(D / 4) + 11.75 * math.ceil(D / 2) + 68.75
    return 2 * direction + 2 * (3 * D + 2) + D * D + 2 * D + 80


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for ln in fh:
                parts = [p.strip() for p in ln.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        loaded = sorted(sm)[len(sm) // 4:] if sm else []
        return {"sm_mhz": float(np.median(loaded)) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def _serving_mix(rng, n_req, cloud_w):
    """Seeded request mix: (workload, points, walk budget, target stderr).

    Points log-uniform in [1, P_max], budget log-uniform in [256, 65536], target
    standard error log-uniform in [1e-3, 1e-2].  P_max: 4096 on the torus, 64
    on the S^2 cap, the point cloud and S^999 (thousands of steps per walk;
    budget <= 4096), 4 on S^20 in R^1000 (226,786 steps per walk; budget
    <= 1024); S^999 and S^20 use the dimension-reduced sampler."""
    import math as _m
    out = []
    kinds = ["torus", "cap", "cloud", "s999", "s20"]
    for q in range(n_req):
        kind = kinds[int(rng.integers(len(kinds)))]
        lo = lambda a, b: int(round(_m.exp(rng.uniform(_m.log(a), _m.log(b)))))
        target = _m.exp(rng.uniform(_m.log(1e-3), _m.log(1e-2)))
        budget = lo(256, 65536)
        seed = int(rng.integers(1 << 30))
        if kind == "torus":
            w = W.torus_closed(P=lo(1, 4096), walks=1, seed=seed)
        elif kind == "cap":
            w = W.sphere_cap(P=lo(1, 64), walks=1, seed=seed)
        elif kind == "cloud":
            P = lo(1, 64)
            idx = rng.choice(len(cloud_w.problem.manifold.cloud), size=P, replace=False)
            w = W.Workload("cloud", cloud_w.problem, cloud_w.problem.manifold.cloud[idx].copy(), 1,
                           cloud_w.params, np.ones(P), "f32")
        elif kind == "s999":
            w = W.hypersphere_half(P=lo(1, 64), walks=1, seed=seed)
            w.params.sampler = W.SAMPLER_REDUCED
            budget = min(budget, 4096)
        else:
            w = W.embedded_s20(P=lo(1, 4), walks=1, seed=seed % 7)
            w.params.sampler = W.SAMPLER_REDUCED
            budget = min(budget, 1024)
        out.append((kind, w, budget, target))
    return out


def _lat_summary(lat, by_kind):
    lat = np.asarray(lat)
    rest = np.concatenate([np.asarray(v) for k, v in by_kind.items() if k != "s20"] or [np.zeros(0)])
    pct = lambda a, q: 1e3 * float(np.percentile(a, q)) if len(a) else None
    return {"p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99), "mean_ms": 1e3 * float(lat.mean()),
            "p99_ms_without_s20": pct(rest, 99),
            "by_kind_ms": {k: {"p50": pct(v, 50), "max": 1e3 * float(np.max(v))} for k, v in sorted(by_kind.items())}}


def _fifo(arrivals, service):
    """Latencies of one FIFO server: request q starts at max(its arrival, the end of q - 1)."""
    fin, out = 0.0, []
    for a, d in zip(arrivals, service):
        fin = max(fin, a) + d
        out.append(fin - a)
    return out


def serving_leg(M, ctx, n_req=48, seed=7, baseline=True):
    """p50/p99 latency of Poisson arrivals at ~70% of the measured capacity, and the
    same arrivals served one request at a time (the latency baselines)."""
    import time as _t
    rng = np.random.default_rng(seed)
    cloud_w = W.point_cloud(P=1, walks=1)
    cloud_w.params.tau_w = 1e-4

    def log(msg):
        print(f"[serving {_t.perf_counter() - T0:8.2f} s] {msg}", file=sys.stderr, flush=True)

    T0 = _t.perf_counter()

    def run(c, reqs, arrivals, prec):
        lat, steps, pending, q = [None] * len(reqs), [0.0] * len(reqs), {}, 0
        t0 = _t.perf_counter()
        t_log = t0
        while q < len(reqs) or pending:
            if _t.perf_counter() - t_log > 10.0:
                t_log = _t.perf_counter()
                log(f"{q} of {len(reqs)} submitted, {len(pending)} pending: "
                    + ", ".join(f"{reqs[qq][0]}/{len(reqs[qq][1].points)}/{c.poll(rid)}" for rid, qq in pending.items()))
            now = _t.perf_counter() - t0
            while q < len(reqs) and arrivals[q] <= now:
                kind, w, budget, target = reqs[q]
                rid = c.submit(w.problem, w.params, w.points, budget, target, precision=prec)
                pending[rid] = q
                q += 1
            for rid in list(pending):
                if c.poll(rid) >= 2:
                    qq = pending.pop(rid)
                    mean, se, ms, walks, lt, rc = c.fetch(rid, len(reqs[qq][1].points))
                    lat[qq] = lt
                    steps[qq] = float(np.sum(ms * walks))
            _t.sleep(0.0005)
        return np.array(lat), np.array(steps), _t.perf_counter() - t0

    def by_kind(reqs, lat):
        out = {}
        for (kind, *_), lt in zip(reqs, lat):
            out.setdefault(kind, []).append(lt)
        return out

    # capacity of this very stream: its requests submitted at once (16 in flight),
    # then the same requests again with Poisson arrivals at 0.7 x that rate
    reqs = _serving_mix(rng, n_req, cloud_w)
    _, _, T_c = run(ctx, reqs, np.zeros(n_req), M.FP32)
    cap_rate = n_req / T_c
    rate = 0.7 * cap_rate
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
    log(f"capacity {cap_rate:.2f} requests/s")
    lat, steps, T = run(ctx, reqs, arrivals, M.FP32)
    log(f"stream served in {T:.1f} s")
    kinds = {k: sum(1 for r in reqs if r[0] == k) for k in ["torus", "cap", "cloud", "s999", "s20"]}
    out = {**_lat_summary(lat, by_kind(reqs, lat)), "requests": int(len(lat)), "arrival_rate_hz": rate,
           "capacity_hz": cap_rate, "walk_steps_per_s": float(steps.sum()) / T, "mix": kinds,
           "recipe": "Poisson arrivals at 0.7 x capacity (capacity: the same 48 requests submitted at once, served 16 at a time); points log-uniform "
                     "(torus <=4096, cap/cloud/S^999 <=64, S^20 <=4), budget log-uniform 256-65536 (S^999 <=4096, "
                     "S^20 <=1024), target stderr log-uniform 1e-3-1e-2, FP32 walks, reduced sampler on S^999/S^20; "
                     "chunks sized to ~10 ms of GPU time"}
    if baseline:
        # one request at a time: each request's service time alone on a context with
        # one slot, then the FIFO queue the same arrivals form in front of it
        base = M.Context(ctx.device)
        base.serve_config(max_active=1)
        svc32, svc64 = [], []
        for (kind, w, budget, target), st in zip(reqs, steps):
            rid = base.submit(w.problem, w.params, w.points, budget, target, precision=M.FP32)
            base.wait(rid)
            svc32.append(base.fetch(rid, len(w.points))[4])          # submit to done, measured by the library
            # FP64: the FP64 walk is ~10^3 x slower on B300 (the whole stream in FP64
            # would hold the GPU for hours), so the request's FP64 service time is its
            # FP32 one times the FP64 / FP32 time ratio of one sample of it: its points,
            # min(budget, 64) walks each, at most 2048 steps per walk, in both precisions
            smp = copy.deepcopy(w.params)
            smp.max_steps = min(int(smp.max_steps), 2048)
            t_smp = []
            for prec in (M.FP32, M.FP64):
                rid = base.submit(w.problem, smp, w.points, min(budget, 64), 0.0, precision=prec)
                base.wait(rid)
                t_smp.append(base.fetch(rid, len(w.points))[4])
            svc64.append(svc32[-1] * t_smp[1] / max(t_smp[0], 1e-9))
            log(f"one at a time: {kind} {len(w.points)} pts: FP32 {svc32[-1]:.3f} s, sample FP32 {t_smp[0]:.3f} s "
                f"FP64 {t_smp[1]:.3f} s -> FP64 {svc64[-1]:.3f} s")
        base.close()
        l32, l64 = _fifo(arrivals, svc32), _fifo(arrivals, svc64)
        out["fp32_one_at_a_time"] = {**_lat_summary(l32, by_kind(reqs, l32)),
                                     "service_s_total": float(np.sum(svc32)),
                                     "recipe": "the same requests and arrival times, FP32 walks, one request in flight "
                                               "(max_active = 1): each service time measured alone, latency = FIFO "
                                               "finish - arrival"}
        out["fp64_one_at_a_time"] = {**_lat_summary(l64, by_kind(reqs, l64)),
                                     "service_s_total": float(np.sum(svc64)),
                                     "recipe": "estimated: the same requests and arrival times, FP64 walks, one request "
                                               "in flight; each service time = its measured FP32 one-at-a-time time x "
                                               "the FP64 / FP32 time ratio of a sample of the request (its points, "
                                               "min(budget, 64) walks, <= 2048 steps per walk) run in both "
                                               "precisions; latency = FIFO finish - arrival"}
    return out


def _serving_cloud(P):
    w = W.point_cloud(P=P, walks=1)
    w.params.tau_w = 1e-4
    return w


def device_sm_count():
    import torch
    return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)


def issue_peak(sm, mhz):
    """Lane-operations per second: one warp instruction per SM sub-partition per clock."""
    return sm * 4 * 32 * mhz * 1e6


def mufu_peak(sm, mhz):
    """MUFU results per second: 16 per SM per clock (log2, sqrt, sin, cos, ...)."""
    return sm * 16 * mhz * 1e6


def roofline_block(kernel, ops_per_step, walk_steps, seconds, sm, mhz, src, mufu_per_step=None):
    peak = issue_peak(sm, mhz)
    achieved = ops_per_step * walk_steps / seconds
    out = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "Tops/s",
           "frac": achieved / peak, "kernel": kernel, "kernel_ms": 1e3 * seconds,
           "ops_per_walk_step": ops_per_step, "traffic": None,
           "peak_source": f"{sm} SM x 4 SMSP x 32 lanes x {mhz:.0f} MHz ({src} max clock)"}
    if mufu_per_step:
        mp = mufu_peak(sm, mhz)
        out["mufu"] = {"per_walk_step": mufu_per_step, "achieved": mufu_per_step * walk_steps / seconds / 1e12,
                       "peak": mp / 1e12, "frac": mufu_per_step * walk_steps / seconds / mp,
                       "peak_source": f"{sm} SM x 16 per clock x {mhz:.0f} MHz"}
    return out


def kernel_run(M, ctx, w, N, prec, projection=None, reps=1):
    """The walk kernel alone on device buffers (mpwos_walk_scores), timed by CUDA
    events on the library's stream after a small warm call (tables, handles);
    returns (seconds, per-walk S and K as host arrays)."""
    import torch
    kw = {} if projection is None else {"projection": projection}
    P = len(w.points)
    pts = torch.tensor(w.points, dtype=torch.float64, device="cuda")
    S = torch.empty((P, N), dtype=torch.float64, device="cuda")
    K = torch.empty((P, N), dtype=torch.int32, device="cuda")
    F = torch.empty((P, N), dtype=torch.int32, device="cuda")
    pw = min(P, 8)
    ctx.walk_scores_device(w.problem, w.params, pts[:pw], 4, prec, S[:pw, :4].contiguous(), K[:pw, :4].contiguous(),
                           F[:pw, :4].contiguous(), **kw)
    stream = torch.cuda.current_stream()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        ctx.walk_scores_device(w.problem, w.params, pts, N, prec, S, K, F, **kw)
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b) / 1e3)
    return float(min(ts)), S.cpu().numpy(), K.cpu().numpy()


def solve_run(M, ctx, w, N, prec):
    """One mpwos_solve into device buffers, timed by CUDA events after a small warm call."""
    import torch
    P = len(w.points)
    pts = torch.tensor(w.points, dtype=torch.float64, device="cuda")
    outs = tuple(torch.zeros(P, dtype=torch.float64, device="cuda") for _ in range(3))
    ctx.solve(w.problem, w.params, pts[:min(P, 8)], 4, precision=prec)
    stream = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    ctx.solve(w.problem, w.params, pts, N, precision=prec, out=outs)
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / 1e3, tuple(o.cpu().numpy() for o in outs)


def torus_generic(P, walks=1):
    """The closed torus with a two-mode source u = sin(theta) cos(2 phi) + 0.5 cos(2 theta) sin(phi):
    the walk evaluates the generic Fourier series instead of a one-mode kernel instance."""
    w = W.torus_closed(P=P, walks=walks)
    w.problem.f = W.Func.torus([(1.0, 1, 2, W.TRIG_SIN, W.TRIG_COS), (0.5, 2, 1, W.TRIG_COS, W.TRIG_SIN)],
                               apply_op=True)
    th, ph = W.torus_angles(P, 0)
    w.exact = np.sin(th) * np.cos(2 * ph) + 0.5 * np.cos(2 * th) * np.sin(ph)
    return w


def s999_half_reduced_leg(M, ctx, sm, mhz, src):
    """S^999 half at its stated size (16384 points x 4096 walks) with the
    dimension-reduced sampler in FP32: walk-steps/s, RMSE, FP32-vs-FP64 agreement
    on 8 sampled points, roofline of the reduced walk, and the oracle on a subset."""
    import oracle as O
    w = W.hypersphere_half(P=16384, walks=1)
    w.params.sampler = W.SAMPLER_REDUCED
    N = 4096
    dt, (mean, se, ms) = solve_run(M, ctx, w, N, M.FP32)
    steps = float(ms.sum() * N)
    idx = np.random.default_rng(11).choice(len(w.points), 8, replace=False)
    sub = W.Workload("s999_sub", w.problem, w.points[idx].copy(), 1, w.params, w.exact[idx], "f64")
    m64, s64, _, _ = ctx.solve(sub.problem, sub.params, sub.points, N, precision=M.FP64)
    agree = np.abs(mean[idx] - m64) < 4.0 * np.sqrt(se[idx] ** 2 + s64 ** 2)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    mo, so, to, _ = O.solve(w.problem, w.params, w.points[:16], 64, n_threads=cores)
    t_orc = time.perf_counter() - t0
    return {"workload": "S^999 in R^1000, x_1 > 0, sigma = 1, eps = 1e-3, 16384 pts x 4096 walks to completion, "
                        "dimension-reduced sampler, FP32",
            "walk_steps_per_s": steps / dt, "query_pts_per_s": len(w.points) / dt, "seconds": dt,
            "walk_steps": steps, "mean_steps_per_walk": float(ms.mean()),
            "rmse": float(np.sqrt(np.mean((mean - w.exact) ** 2))), "mean_stderr": float(se.mean()),
            "fp32_vs_fp64": {"points": 8, "walks": N, "within_4_combined_se": int(agree.sum()),
                             "max_abs_diff": float(np.max(np.abs(mean[idx] - m64)))},
            "roofline": roofline_block("walkr_kernel<float, sphere>", OPS_REDUCED_S999, steps, dt, sm, mhz, src),
            "cpu_baseline": {"value": float(to.sum() * 64) / t_orc, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"16 points x 64 walks, reduced sampler, FP64, {t_orc:.1f} s"}}


def s20_in_r1000_leg(M, ctx, sm, mhz, src):
    """S^20 in R^1000 (32768 points x 2048 walks of 226,786 steps): a fixed window
    of steps for every walk (the full sampler with Q^T g on the tensor cores, and
    the reduced sampler), and the RMSE of complete walks on a 256-point subset."""
    w = W.embedded_s20(P=32768, walks=1)
    N = 2048
    out = {"workload": "S^20 randomly embedded in R^1000 (seeded orthonormal Q, shift b), sigma = 0.5, "
                       "32768 pts x 2048 walks; every walk runs a fixed window of steps (flagged at the window; "
                       "a complete walk is 226,786 steps), FP32"}
    w.params.max_steps = 16
    dt, S, K = kernel_run(M, ctx, w, N, M.FP32, projection=M.PROJ_TENSOR)
    steps = float(K.sum(dtype=np.int64))
    out["tensor_core_window_16"] = {
        "walk_steps_per_s": steps / dt, "seconds": dt, "walk_steps": steps,
        "roofline": roofline_block("embed_tc_kernel<24>", ops_tc_embedded(1000), steps, dt, sm, mhz, src,
                                   mufu_per_step=MUFU_PER_PAIR * 1000)}
    del S, K
    w.params.sampler = W.SAMPLER_REDUCED
    w.params.max_steps = 256
    dt, S, K = kernel_run(M, ctx, w, N, M.FP32)
    steps = float(K.sum(dtype=np.int64))
    out["reduced_window_256"] = {
        "walk_steps_per_s": steps / dt, "seconds": dt, "walk_steps": steps,
        "roofline": roofline_block("walkr_kernel<float, embedded>", ops_reduced_embedded(20), steps, dt, sm, mhz,
                                   src)}
    del S, K
    import oracle as O
    cores = os.cpu_count() or 1
    cs = W.embedded_s20(P=2, walks=1)
    cs.params.sampler = W.SAMPLER_REDUCED
    cs.params.max_steps = 20000
    t0 = time.perf_counter()
    _, _, to, _ = O.solve(cs.problem, cs.params, cs.points, 8, n_threads=cores)
    t_orc = time.perf_counter() - t0
    out["cpu_baseline"] = {"value": float(to.sum() * 8) / t_orc, "unit": UNIT, "cores": cores, "kind": "oracle",
                           "sample": f"2 points x 8 walks, a window of 20,000 steps each, reduced sampler, FP64, "
                                     f"{t_orc:.1f} s"}
    sub = W.embedded_s20(P=256, walks=1)
    sub.params.sampler = W.SAMPLER_REDUCED
    dt, (mean, se, ms) = solve_run(M, ctx, sub, 16, M.FP32)
    out["rmse_256_points_16_complete_walks_reduced"] = {
        "rmse": float(np.sqrt(np.mean((mean - sub.exact) ** 2))), "mean_stderr": float(se.mean()),
        "mean_steps_per_walk": float(ms.mean()), "seconds": dt}
    return out


def secondary_leg(M, ctx, sm, mhz, src):
    """The other configurations (not the headline metric): short runs, each with
    walk-steps/s and RMSE; the n = 1000 walks and the tensor-core walk also with
    their roofline (kernel alone, CUDA events)."""
    out = {}
    # S^2 cap, 64 points x 1000 walks, FP64 (the per-walk parity mode)
    w = W.sphere_cap(P=64, walks=1)
    dt, (mean, se, ms) = solve_run(M, ctx, w, 1000, M.FP64)
    out["s2_cap_fp64"] = {"workload": "S^2 cap z > 0, 64 pts x 1000 walks, FP64",
                          "walk_steps_per_s": float(ms.sum() * 1000) / dt, "query_pts_per_s": 64 / dt,
                          "latency_ms": 1e3 * dt, "rmse": float(np.sqrt(np.mean((mean - w.exact) ** 2))),
                          "mean_steps_per_walk": float(ms.mean())}
    # the torus with a two-mode source: the generic Fourier-series walk beside the headline's one-mode instance
    w = torus_generic(4096)
    dt, S, K = kernel_run(M, ctx, w, 10_000, M.FP32)
    steps = float(K.sum(dtype=np.int64))
    out["torus_generic_series_fp32"] = {
        "workload": "closed torus, 4096 pts x 1e4 walks, two-mode source (generic series), FP32 walk kernel",
        "walk_steps_per_s": steps / dt, "seconds": dt,
        "rmse": float(np.sqrt(np.mean((S.mean(axis=1) - w.exact) ** 2)))}
    del S, K
    out["s999_half_reduced_16384x4096"] = s999_half_reduced_leg(M, ctx, sm, mhz, src)
    # S^999 with the full sampler (the paper's form of the step: n Gaussians per direction)
    w = W.hypersphere_half(P=4096, walks=1)
    dt, S, K = kernel_run(M, ctx, w, 16, M.FP32)
    steps = float(K.sum(dtype=np.int64))
    out["s999_half_full_sampler_fp32"] = {
        "workload": "S^999 half, 4096 pts x 16 walks to completion, full sampler (2000 Gaussians per step), FP32",
        "walk_steps_per_s": steps / dt, "seconds": dt, "mean_steps_per_walk": float(K.mean()),
        "rmse": float(np.sqrt(np.mean((S.mean(axis=1) - w.exact) ** 2))),
        "roofline": roofline_block("walkn32s_kernel<sphere, 16, 4>", ops_full_sampler(1000), steps, dt, sm, mhz, src,
                                   mufu_per_step=MUFU_PER_PAIR * 1000)}
    del S, K
    out["s20_in_r1000_32768x2048"] = s20_in_r1000_leg(M, ctx, sm, mhz, src)
    # Example 2's dumbbell (full sampler, Newton closest point)
    w = W.dumbbell(P=2368, walks=1)
    dt, S, K = kernel_run(M, ctx, w, 64, M.FP32)
    steps = float(K.sum(dtype=np.int64))
    wr = W.dumbbell(P=100, walks=1)
    _, (mean, se, ms) = solve_run(M, ctx, wr, 1000, M.FP32)
    out["dumbbell_e2_fp32"] = {
        "workload": "Example 2 dumbbell in R^1001 (sigma = 2000, Newton cp), full sampler, FP32; rate on "
                    "2368 pts x 64 walks, RMSE on 100 pts x 1000 walks",
        "walk_steps_per_s": steps / dt, "seconds": dt, "mean_steps_per_walk": float(K.mean()),
        "rmse": float(np.sqrt(np.mean((mean - wr.exact) ** 2))),
        "roofline": roofline_block("walkn32s_kernel<revolution, 16, 4>", ops_full_sampler(1001, True), steps, dt,
                                   sm, mhz, src, mufu_per_step=MUFU_PER_PAIR * 1001)}
    del S, K
    # the rest (solve, wall clock around synchronisation)
    import torch
    cases = [
        ("torus_fp64", lambda: W.torus_closed(P=4096, walks=1), 50, M.FP64, W.SAMPLER_FULL,
         "torus, 4096 pts x 50 walks, FP64 walk (per-walk parity mode)"),
        ("torus_fp32", lambda: W.torus_closed(P=4096, walks=1), 50, M.FP32, W.SAMPLER_FULL,
         "torus, 4096 pts x 50 walks, FP32 walk (same walks and RMSE scale as torus_fp64)"),
        ("torus_cut_e1_baseline_fp32", lambda: W.torus_cut(P=100, walks=1), 100000, M.FP32, W.SAMPLER_FULL,
         "Example 1 cut torus, 100 pts x 1e5 walks, m_* = 0, FP32"),
        ("torus_cut_e1_comp2_fp32", lambda: W.torus_cut(P=100, walks=1, comp=W.COMP_NORMAL2), 100000, M.FP32,
         W.SAMPLER_FULL, "Example 1 cut torus, 100 pts x 1e5 walks, second-order m_* (predictor u), FP32"),
        ("torus_cut_e1_exact_fp32", lambda: W.torus_cut(P=100, walks=1, comp=W.COMP_EXACT), 100000, M.FP32,
         W.SAMPLER_FULL, "Example 1 cut torus, 100 pts x 1e5 walks, exact mismatch m (predictor u), FP32"),
        ("point_cloud_200k_fp32", lambda: _serving_cloud(64), 4096, M.FP32, W.SAMPLER_FULL,
         "the serving mix's 200k-point cloud (k_nn = 16, quadratic-fit cp, tau_W = 1e-4), 64 pts x 4096 walks, FP32"),
        ("sphere_cloud_e4_fp32", lambda: W.sphere_cloud_legendre(P=100, walks=1), 8000, M.FP32, W.SAMPLER_FULL,
         "Example 4 S^2 as 8000 points, k_nn = 6, nearest-point cp, 100 pts x 8000 walks, FP32"),
        ("curve_sphere_e3_fp32", lambda: W.curve_sphere(P=100, walks=1), 10000, M.FP32, W.SAMPLER_FULL,
         "Example 3 Fourier curve x S^2(0.65) in R^9 (Newton cp on the curve), 100 pts x 1e4 walks, FP32"),
    ]
    for name, make, N, prec, sampler, desc in cases:
        w = make()
        w.params.sampler = sampler
        P = len(w.points)
        pts = torch.tensor(w.points, dtype=torch.float64, device="cuda")
        outs = tuple(torch.zeros(P, dtype=torch.float64, device="cuda") for _ in range(3))
        ctx.solve(w.problem, w.params, pts[:8], 4, precision=prec)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.solve(w.problem, w.params, pts, N, precision=prec, out=outs)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        mean, ms = outs[0].cpu().numpy(), outs[2].cpu().numpy()
        out[name] = {"workload": desc, "walk_steps_per_s": float(ms.sum() * N) / dt, "query_pts_per_s": P / dt,
                     "rmse": float(np.sqrt(np.mean((mean - w.exact) ** 2))), "seconds": dt,
                     "mean_steps_per_walk": float(ms.mean())}
    out["torus_fp32_over_fp64"] = out["torus_fp32"]["walk_steps_per_s"] / out["torus_fp64"]["walk_steps_per_s"]
    out["cloud_knn_200k"] = knn_leg(M, ctx)
    return out


def knn_leg(M, ctx, nq=262144):
    """The 200k cloud's k = 16 nearest search on its own: the walk's grid search (per
    thread and warp-cooperative) against the all-pairs scan, queries/s by CUDA events
    on device-resident queries near the surface."""
    import torch
    w = W.point_cloud(P=1, walks=1)
    cloud = w.problem.manifold.cloud
    rng = np.random.default_rng(3)
    x = cloud[rng.choice(cloud.shape[0], nq)] + rng.uniform(-0.02, 0.02, (nq, 3))
    xd = torch.tensor(x, device="cuda")
    k = w.problem.manifold.k_nn
    out = (torch.empty((nq, k), dtype=torch.int32, device="cuda"),
           torch.empty((nq, k), dtype=torch.float64, device="cuda"),
           torch.empty(nq, dtype=torch.float64, device="cuda"))
    res = {"queries": nq, "k": k, "cloud_points": int(cloud.shape[0])}
    for name, prec, meth in (("grid_fp32", M.FP32, M.KNN_GRID), ("grid_warp_fp32", M.FP32, M.KNN_GRID_WARP),
                             ("scan_fp32", M.FP32, M.KNN_SCAN), ("grid_fp64", M.FP64, M.KNN_GRID)):
        ctx.cloud_knn(w.problem, xd, precision=prec, method=meth, out=out)     # warm (grid built once)
        ts = []
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            ctx.cloud_knn(w.problem, xd, precision=prec, method=meth, out=out)
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b) / 1e3)
        res[name + "_queries_per_s"] = nq / float(np.median(ts))
    return res


def cpu_baseline(target_s: float = 25.0):
    """The CPU oracle, as it stands, on a bounded sample of the torus workload."""
    import oracle as O
    w = W.torus_closed(P=64, walks=1)
    cores = os.cpu_count() or 1
    # load and warm the oracle, calibrate on 64 x 16 walks, then size the sample
    # for ~target_s of wall time on all cores
    O.solve(w.problem, w.params, w.points[:2], 2, n_threads=cores)
    t0 = time.perf_counter()
    O.solve(w.problem, w.params, w.points, 16, n_threads=cores)
    per_walk = max(time.perf_counter() - t0, 1e-3) / (64 * 16)
    walks = int(max(16, min(8000, target_s / per_walk / 64)))
    t0 = time.perf_counter()
    m, se, ms, nf = O.solve(w.problem, w.params, w.points, walks, n_threads=cores)
    dt = time.perf_counter() - t0
    steps = float(ms.sum() * walks)
    return {"value": steps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"torus 64 points x {walks} walks x 525 steps ({steps:.3g} walk-steps, FP64, "
                      f"OpenMP over walks), {dt:.1f} s"}


def run_reference(args):
    """The reference arm: the CPU oracle as it stands, W untimed and K timed steps,
    each step a bounded sample of the torus workload (64 points, walks sized so that
    the whole run takes about two minutes), on all host cores; rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle as O
    w = W.torus_closed(P=64, walks=1)
    cores = os.cpu_count() or 1
    O.solve(w.problem, w.params, w.points[:2], 2, n_threads=cores)          # load the oracle
    t0 = time.perf_counter()
    O.solve(w.problem, w.params, w.points, 16, n_threads=cores)
    per_walk = max(time.perf_counter() - t0, 1e-3) / (64 * 16)
    steps_total = max(args.steps, 1) + max(args.warmup, 0)
    walks = int(max(16, min(8000, 120.0 / steps_total / per_walk / 64)))
    for _ in range(max(args.warmup, 0)):
        O.solve(w.problem, w.params, w.points, walks, n_threads=cores)
    t_steps, work = [], 0.0
    for _ in range(max(args.steps, 1)):
        t0 = time.perf_counter()
        m, se, ms, nf = O.solve(w.problem, w.params, w.points, walks, n_threads=cores)
        t_steps.append(time.perf_counter() - t0)
        work += float(ms.sum() * walks)
    T = sum(t_steps)
    value = work / T
    sample = (f"each step: torus 64 points x {walks} walks x 525 steps ({work / len(t_steps):.3g} walk-steps, "
              f"FP64, OpenMP over walks); {len(t_steps)} timed steps, {T:.1f} s")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * T / len(t_steps), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "torus_closed R=1 a=0.4 sigma=2 u=sin(th)cos(2ph)", "points": 4096,
                       "walks_per_point": 10000, "steps_per_walk": 525,
                       "sampled": "each step is a bounded sample of the workload on the host cores "
                                  "(cpu_baseline.sample), the oracle as it stands"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def rank_walk_range(N, rank, world, block=1024):
    """Walk range [i0, i1) of `rank` when a request of N walks per point is split
    over `world` ranks at estimator-block boundaries (block walks each), so that
    the ranks' block records merge to the bits of the whole request."""
    nb = (N + block - 1) // block
    b0, b1 = nb * rank // world, nb * (rank + 1) // world
    return min(N, b0 * block), min(N, b1 * block)


def gather_partials(dist, part, world):
    """Every rank's block records (a P x nblk x 5 FP64 tensor, nblk per rank) in
    rank order: one all_gather of the counts, one of the records padded to the
    largest range; returned as host arrays."""
    import torch
    P, nb, F = part.shape
    cnt = torch.tensor([nb], dtype=torch.int64, device=part.device)
    counts = [torch.zeros_like(cnt) for _ in range(world)]
    dist.all_gather(counts, cnt)
    counts = [int(c.item()) for c in counts]
    pad = torch.zeros((P, max(counts), F), dtype=torch.float64, device=part.device)
    pad[:, :nb] = part
    bufs = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(bufs, pad)
    return [b[:, :c].cpu().numpy() for b, c in zip(bufs, counts)]


def max_over_ranks(dist, device, *values):
    """The max of each value over all ranks (the timed region's slowest rank)."""
    if dist is None:
        return tuple(float(v) for v in values)
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return tuple(float(v) for v in t.tolist())


def aggregate_rate(steps_per_rank_step, steps, world, tmax):
    """Whole-job walk-steps/s: the units all ranks processed over the slowest rank's time."""
    return steps_per_rank_step * steps * world / tmax


# One kernel on a small seeded case, for profiler captures (--leg NAME).
def _leg_case(M, name, P, N, max_steps):
    kw = {}
    if name == "torus":
        w = W.torus_closed(P=P or 64, walks=1)
    elif name in ("s20_tc", "s20_cuda"):
        w = W.embedded_s20(P=P or 148, walks=1)
        kw["projection"] = M.PROJ_TENSOR if name == "s20_tc" else M.PROJ_CUDA
    elif name == "s20_red":
        w = W.embedded_s20(P=P or 1184, walks=1)
        w.params.sampler = W.SAMPLER_REDUCED
    elif name == "s999_full":
        w = W.hypersphere_half(P=P or 148, walks=1)
    elif name == "s999_red":
        w = W.hypersphere_half(P=P or 4096, walks=1)
        w.params.sampler = W.SAMPLER_REDUCED
    elif name == "dumbbell":
        w = W.dumbbell(P=P or 2368, walks=1)
    elif name == "cloud":
        w = _serving_cloud(P or 64)
    elif name == "e1_comp":
        w = W.torus_cut(P=P or 100, walks=1, comp=W.COMP_NORMAL2)
    else:
        raise SystemExit(f"unknown leg {name}")
    if max_steps:
        w.params.max_steps = max_steps
    return w, kw


def run_knn_leg(args, nq=262144):
    """The 200k cloud's k = 16 nearest of nq queries near the surface: per rep the
    FP32 grid search (cloud_knn_query_kernel), then the all-pairs scan
    (cloud_knn_scan_kernel), each timed by wall clock around synchronisation."""
    import torch
    import paper_2606_21883_b300 as M
    w = W.point_cloud(P=1, walks=1)
    cloud = w.problem.manifold.cloud
    rng = np.random.default_rng(3)
    x = cloud[rng.choice(cloud.shape[0], nq)] + rng.uniform(-0.02, 0.02, (nq, 3))
    xd = torch.tensor(x, device="cuda")
    k = w.problem.manifold.k_nn
    out = (torch.empty((nq, k), dtype=torch.int32, device="cuda"), torch.empty((nq, k), dtype=torch.float64, device="cuda"),
           torch.empty(nq, dtype=torch.float64, device="cuda"))
    ctx = M.Context(0)
    for _ in range(max(1, args.reps)):
        for name, meth in (("grid", M.KNN_GRID), ("scan", M.KNN_SCAN)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.cloud_knn(w.problem, xd, precision=M.FP32, method=meth, out=out)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            print(json.dumps({"leg": f"knn_{name}", "queries": nq, "cloud": int(cloud.shape[0]),
                              "wall_ms": 1e3 * dt, "queries_per_s": nq / dt}), flush=True)
    ctx.close()
    return 0


def run_leg(args):
    """One walk kernel on a small case (device buffers), --reps launches; prints
    the walk-steps and the last launch's time.  For profiler captures."""
    import torch
    import paper_2606_21883_b300 as M
    if args.leg == "knn":
        return run_knn_leg(args)
    if args.leg == "serving":
        ctx = M.Context(0)
        for r in range(max(1, args.reps)):
            out = serving_leg(M, ctx, seed=7 + r, baseline=not args.no_baseline)
            print(json.dumps({"leg": "serving", "seed": 7 + r, **out}), flush=True)
        ctx.close()
        return 0
    ctx = M.Context(0)
    w, kw = _leg_case(M, args.leg, args.points, args.walks, args.max_steps)
    P, N = len(w.points), args.walks
    pts = torch.tensor(w.points, dtype=torch.float64, device="cuda")
    S = torch.empty((P, N), dtype=torch.float64, device="cuda")
    K = torch.empty((P, N), dtype=torch.int32, device="cuda")
    F = torch.empty((P, N), dtype=torch.int32, device="cuda")
    dt = 0.0
    for _ in range(max(1, args.reps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.walk_scores_device(w.problem, w.params, pts, N, M.FP32, S, K, F, **kw)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    steps = int(K.sum().item())
    print(json.dumps({"leg": args.leg, "points": P, "walks": N, "max_steps": args.max_steps, "walk_steps": steps,
                      "last_launch_ms": 1e3 * dt, "walk_steps_per_s": steps / dt}), flush=True)
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--points", type=int, default=4096)
    ap.add_argument("--walks", type=int, default=10_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-baseline", action="store_true", help="serving leg without the FP64 one-at-a-time baseline")
    ap.add_argument("--leg", default=None, help="run one kernel case (torus, s999_full, s999_red, s20_tc, s20_cuda, "
                                                 "s20_red, dumbbell, cloud, e1_comp, knn) and exit")
    ap.add_argument("--max-steps", type=int, default=0)
    ap.add_argument("--reps", type=int, default=2)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.leg:
        if args.points == 4096:
            args.points = 0
        return run_leg(args)

    import torch
    import paper_2606_21883_b300 as M

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    # one request (the torus batch, seed 0) on every rank; N = 1: its 10^4 walks per
    # point on one GPU (mpwos_solve); N > 1: 10,240 walks per point and rank, the
    # request's walk range split at estimator blocks, merged on the host
    w = W.torus_closed(P=args.points, walks=1)
    ctx = M.Context(local)
    stream = torch.cuda.current_stream()
    ctx.set_stream(stream.cuda_stream)
    ctx.set_autotune(True)                  # the first warm-up solve picks the walk kernel's block size
    P = args.points
    N_total = args.walks if world == 1 else M.EST_BLOCK * ((args.walks + M.EST_BLOCK - 1) // M.EST_BLOCK) * world
    i0, i1 = rank_walk_range(N_total, rank, world)
    N = i1 - i0
    pts_dev = torch.tensor(w.points, dtype=torch.float64, device="cuda")
    outs = tuple(torch.zeros(P, dtype=torch.float64, device="cuda") for _ in range(3))
    part = torch.zeros((P, M.n_blocks(N), M.EST_FIELDS), dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # 256 MB > L2
    merged = {}

    def step():
        if world == 1:
            return ctx.solve(w.problem, w.params, pts_dev, N, precision=M.FP32, out=outs)
        ctx.solve_partial(w.problem, w.params, pts_dev, N_total, i0, i1, precision=M.FP32, out=part)
        parts = gather_partials(dist, part, world)           # the one exchange: every rank's block records
        merged["r"] = M.merge_partials(parts)                  # same bits as one GPU running all N_total walks

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()

    sampler = ClockSampler(local)
    sampler.start()
    launches0 = ctx.launch_count()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    torch.cuda.synchronize()
    for s in range(args.steps):
        flush.zero_()                       # L2 flushed between timed steps (outside the events)
        starts[s].record(stream)
        step()
        ends[s].record(stream)
    torch.cuda.synchronize()
    launches = ctx.launch_count() - launches0
    t_dev = sum(a.elapsed_time(b) for a, b in zip(starts, ends)) / 1e3
    if world == 1:
        mean = outs[0].cpu().numpy()
        msteps = outs[2].cpu().numpy()
    else:
        mean, _, msteps, _ = merged["r"]

    # the walk kernel alone (device-resident per-walk outputs): its launch duration
    S_dev = torch.empty(P * N, dtype=torch.float64, device="cuda")
    K_dev = torch.empty(P * N, dtype=torch.int32, device="cuda")
    F_dev = torch.empty(P * N, dtype=torch.int32, device="cuda")
    kt = []
    for s in range(3):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.walk_scores_device(w.problem, w.params, pts_dev, N, M.FP32, S_dev, K_dev, F_dev)
        b.record(stream)
        torch.cuda.synchronize()
        kt.append(a.elapsed_time(b) / 1e3)
    t_kernel = float(np.median(kt))

    # end to end through the C ABI with pinned host buffers (copies inside the timed region)
    pts_host = torch.tensor(w.points, dtype=torch.float64).pin_memory()
    host_out = tuple(torch.zeros(P, dtype=torch.float64).pin_memory() for _ in range(3))
    host_part = torch.zeros((P, M.n_blocks(N), M.EST_FIELDS), dtype=torch.float64).pin_memory()
    e2e_t = []
    for s in range(max(2, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if world == 1:
            ctx.solve(w.problem, w.params, pts_host, N, precision=M.FP32, out=host_out)
        else:
            ctx.solve_partial(w.problem, w.params, pts_host, N_total, i0, i1, precision=M.FP32, out=host_part)
            M.merge_partials(gather_partials(dist, host_part.cuda(), world))
        e2e_t.append(time.perf_counter() - t0)
    clocks = sampler.stop()
    tuned = ctx.autotune_entries()
    ctx.set_autotune(False)                 # the serving and secondary legs launch the default shapes

    steps_rank = float(np.sum(msteps) * N) if world == 1 else float(np.sum(msteps) * N_total) / world
    tmax, e2e_mean = max_over_ranks(dist, "cuda", t_dev, float(np.mean(e2e_t)))
    value = aggregate_rate(steps_rank, args.steps, world, tmax)
    rmse = float(np.sqrt(np.mean((mean - w.exact) ** 2)))

    if rank == 0:
        peaks, src = _peaks()
        sm_mhz = float(peaks.get("sm_max_mhz", 2032.0))
        sm = device_sm_count()
        peak_ops = issue_peak(sm, sm_mhz)
        achieved = OPS_PER_STEP * P * N * 525 / t_kernel
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tmax / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "torus_closed R=1 a=0.4 sigma=2 u=sin(th)cos(2ph)", "points": P,
                       "walks_per_point": N_total, "walks_per_point_per_gpu": N, "steps_per_walk": 525,
                       "walk_steps_per_step": steps_rank * world,
                       "precision": "FP32 walk; per-walk weight and score in float pairs (~2^-46 relative per "
                                    "operation, below FP64's 2^-53); per-point FP64 estimator sums",
                       "parallelism": "dp1" if world == 1 else
                                      f"dp{world} (one request split by walk range; block records all-gathered, "
                                      "merged on the host)",
                       "l2": "flushed between timed steps (256 MB write)", "rmse": rmse,
                       "query_pts_per_s": P * args.steps / tmax},
            "rmse": rmse,
            "query_pts_per_s": P * args.steps / tmax,
            "e2e": {"value": steps_rank * world / e2e_mean, "unit": UNIT,
                    "h2d_bytes_per_step": int(P * 3 * 8),
                    "d2h_bytes_per_step": int(3 * P * 8) if world == 1 else int(host_part.numel() * 8)},
            "gpu_launches": int(launches),
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12, "unit": "Tops/s",
                         "frac": achieved / peak_ops, "traffic": TRAFFIC_BYTES, "traffic_unit": "bytes per launch",
                         "traffic_source": "profiles/walk3_f32_torus_bench_traffic.md",
                         "kernel": "walk3_f32_kernel<torus>", "kernel_ms": 1e3 * t_kernel,
                         "ops_per_walk_step": OPS_PER_STEP,
                         "peak_source": f"{sm} SM (device attribute) x 4 SMSP x 32 lanes x {sm_mhz:.0f} MHz "
                                        f"({src} max SM clock): one warp instruction per SM sub-partition per clock"},
            "clocks": clocks,
            "autotune": tuned,
        }
        if not args.no_serving and world == 1:
            line["serving"] = serving_leg(M, ctx)
            line["secondary"] = secondary_leg(M, ctx, sm, sm_mhz, src)
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline()
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
