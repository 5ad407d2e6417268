"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

FP64 mode draws the same Philox numbers as the oracle, so every walk is
compared element by element: |S_gpu - S_oracle| <= 1e-12 max(1, |S|) and
identical stopping index K and flags, on every walk: the seeded cases here
contain no walk whose threshold decision (delta_Gamma < eps, W < tau_W) sits
within rounding of the threshold, so no mismatch is allowed.  FP32 mode is compared
statistically: |mean32 - mean64| < 4 sqrt(se32^2 + se64^2) per point.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
import paper_2606_21883_b300 as M
from paper_2606_21883_b300 import workloads as W

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")
REL = 1e-12


@pytest.fixture(scope="module")
def ctx():
    c = M.Context(0)
    yield c
    c.close()


def _rows(name):
    with open(os.path.join(GOLD, name)) as fh:
        return [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]


def _walk_parity(ctx, work, N):
    Sg, Kg, Fg = ctx.walk_scores(work.problem, work.params, work.points, N, precision=M.FP64)
    So, Ko, Fo = O.walk_scores(work.problem, work.params, work.points, N)
    ok = (np.abs(Sg - So) <= REL * np.maximum(1.0, np.abs(So))) & (Kg == Ko) & (Fg == Fo)
    bad = np.count_nonzero(~ok)
    assert bad == 0, (
        f"{bad} of {ok.size} walks differ; first: {np.argwhere(~ok)[:3].tolist()} "
        f"S {Sg[~ok][:3]} vs {So[~ok][:3]}, K {Kg[~ok][:3]} vs {Ko[~ok][:3]}")
    return Sg, Kg, So, Ko


# ------------------------------------------------------------------ primitives
def test_philox_device_known_answers(ctx):
    rows = [[int(x, 16) for x in r] for r in _rows("philox4x32_10_kat.txt")]
    for r in rows:
        out = ctx.philox(np.array([r[0:4]]), r[4], r[5])
        assert out[0].tolist() == r[6:10]


def test_philox_device_vs_oracle(ctx):
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, size=(2000, 4), dtype=np.uint64).astype(np.uint32)
    out = ctx.philox(ctr, 0x12345678, 0x9ABCDEF0)
    for q in range(0, 2000, 97):
        assert out[q].tolist() == O.philox(ctr[q].tolist(), [0x12345678, 0x9ABCDEF0])


def test_c_sigma_r_device_vs_quadrature(ctx):
    for r in _rows("green_quadrature.txt")[::6]:
        n, sigma, rad, c = int(r[0]), float(r[1]), float(r[2]), float(r[4])
        a = math.sqrt(sigma) * rad
        assert ctx.c_sigma_r(n, np.array([a]))[0] == pytest.approx(c, rel=1e-13)


@pytest.mark.parametrize("n,a_max", [(3, 0.6), (3, 4.0), (1000, 0.5), (21, 1.5), (4, 0.6)])
def test_green_radius_fp64_vs_oracle(ctx, n, a_max):
    rng = np.random.default_rng(n)
    a = a_max * np.sqrt(rng.uniform(0.01, 1.0, 300))
    U = rng.uniform(1e-12, 1.0, 300)
    U[:3] = [1e-15, 0.5, 1.0 - 1e-12]
    t = ctx.green_radius(n, a_max, a, U, precision=M.FP64)
    ref = np.array([O.green_cdf_inv(n, ai, ui) for ai, ui in zip(a, U)])
    # the root's own conditioning: an FP64 rounding of F moves t by ~1e-16 / F'(t)
    h = 1e-7
    dF = np.array([(O.green_cdf(n, ai, min(ti + h, 1.0)) - O.green_cdf(n, ai, max(ti - h, 0.0)))
                   / (min(ti + h, 1.0) - max(ti - h, 0.0)) for ai, ti in zip(a, ref)])
    tol = 1e-12 * ref + 2e-15 / np.maximum(dF, 1e-300)
    assert np.all(np.abs(t - ref) <= tol), np.max(np.abs(t - ref) / tol)


@pytest.mark.parametrize("n,a_max", [(3, 0.6), (1000, 0.5)])
def test_green_radius_fp32_vs_oracle(ctx, n, a_max):
    rng = np.random.default_rng(7)
    a = a_max * np.sqrt(rng.uniform(0.0, 1.0, 500))
    U = rng.uniform(1e-7, 1.0, 500)
    t = ctx.green_radius(n, a_max, a, U, precision=M.FP32)
    ref = np.array([O.green_cdf_inv(n, ai, ui) for ai, ui in zip(a, U)])
    assert np.max(np.abs(t - ref)) < 2e-5


# --------------------------------------------------------- per-walk FP64 parity
def test_walk_parity_s2_cap(ctx):
    w = W.sphere_cap(P=24, walks=1)
    _walk_parity(ctx, w, 64)


def test_walk_parity_torus(ctx):
    w = W.torus_closed(P=8, walks=1)
    Sg, Kg, So, Ko = _walk_parity(ctx, w, 16)
    assert np.all(Kg == 525)


def test_walk_parity_euclid_quadratic(ctx):
    sigma = 3.0
    w = W.euclid_halfspace(P=8, walks=1, sigma=sigma, seed=3)
    w.params.c_kappa = 1e3
    w.problem.f = W.Func.poly([(-6.0, []), (sigma, [(0, 2)]), (sigma, [(1, 2)]), (sigma, [(2, 2)])])
    w.problem.g = W.Func.poly([(1.0, [(0, 2)]), (1.0, [(1, 2)]), (1.0, [(2, 2)])])
    _walk_parity(ctx, w, 64)


def test_walk_parity_hypersphere_capped(ctx):
    """S^999 half, the full dimension: walks capped at 40 steps (flagged) so the
    oracle finishes; every partial score and flag must agree."""
    w = W.hypersphere_half(P=3, walks=1)
    w.params.max_steps = 40
    _walk_parity(ctx, w, 4)


def test_walk_parity_hypersphere_near_boundary(ctx):
    """S^999 half with start points close to x_1 = 0 so walks terminate."""
    w = W.hypersphere_half(P=3, walks=1, seed=5)
    pts = w.points.copy()
    pts[:, 0] = [0.004, 0.002, 0.0015]
    pts[:, 1:] *= np.sqrt(1 - pts[:, :1] ** 2) / np.linalg.norm(pts[:, 1:], axis=1, keepdims=True)
    w.points = pts
    w.params.max_steps = 4000
    _walk_parity(ctx, w, 3)


def test_walk_parity_embedded_sphere_capped(ctx):
    """S^20 in R^1000 (Q, b seeded): walks capped at 25 steps."""
    w = W.embedded_s20(P=3, walks=1)
    w.params.max_steps = 25
    _walk_parity(ctx, w, 3)


def test_walk_parity_embedded_sphere_full_walks(ctx):
    """Embedded S^5 in R^64 with strong screening: complete walks (W < tau_W)."""
    w = W.embedded_s20(P=4, walks=1, n=64, d=5, sigma=6.0)
    w.params.tau_w = 1e-4
    Sg, Kg, So, Ko = _walk_parity(ctx, w, 8)
    assert np.all(Kg == Kg.flat[0])


# ------------------------------------------------------------- exact identities
@pytest.mark.parametrize("prec", [M.FP64, M.FP32])
def test_gpu_telescoping(ctx, prec):
    w = W.constant_solution(W.sphere_cap(P=16, walks=1))
    S, K, F = ctx.walk_scores(w.problem, w.params, w.points, 256, precision=prec)
    assert np.all(np.abs(S - 1.0) <= 1e-12 * np.maximum(K, 1))
    wt = W.constant_solution(W.torus_closed(P=8, walks=1))
    S, K, F = ctx.walk_scores(wt.problem, wt.params, wt.points, 256, precision=prec)
    assert np.all(K == 525) and np.all((S > 1 - 1e-8) & (S <= 1 + 1e-12))


# ---------------------------------------------------------- FP32 statistically
def _stat_agree(m32, s32, m64, s64, k=4.0):
    return np.abs(m32 - m64) < k * np.sqrt(s32 ** 2 + s64 ** 2)


def test_fp32_vs_oracle_cap(ctx):
    w = W.sphere_cap(P=16, walks=4000)
    m32, s32, t32, rc = ctx.solve(w.problem, w.params, w.points, w.walks, precision=M.FP32)
    mo, so, to, nf = O.solve(w.problem, w.params, w.points, w.walks)
    assert np.all(_stat_agree(m32, s32, mo, so))
    assert np.all(np.abs(t32 - to) < 0.1 * to + 1)


def test_fp32_vs_oracle_torus(ctx):
    w = W.torus_closed(P=6, walks=1500)
    m32, s32, t32, rc = ctx.solve(w.problem, w.params, w.points, w.walks, precision=M.FP32)
    mo, so, to, nf = O.solve(w.problem, w.params, w.points, w.walks)
    assert np.all(_stat_agree(m32, s32, mo, so))
    assert np.all(t32 == 525)


@pytest.mark.parametrize("n", [1000, 1024, 5, 17])
def test_fp32_vs_fp64_gpu_hypersphere(ctx, n):
    """The FP32 shared-memory walk against the FP64 walk on S^{n-1}: n = 1000 (an even
    partial last group), 1024 (64 whole groups, the maximum), 5 and 17 (one lane's
    partial group; a whole group plus one component)."""
    w = W.hypersphere_half(P=4, walks=1, n=n, seed=2)
    pts = w.points.copy()
    pts[:, 0] = 0.01
    pts[:, 1:] *= np.sqrt(1 - 1e-4) / np.linalg.norm(pts[:, 1:], axis=1, keepdims=True)
    m32, s32, _, _ = ctx.solve(w.problem, w.params, pts, 512, precision=M.FP32)
    m64, s64, _, _ = ctx.solve(w.problem, w.params, pts, 512, precision=M.FP64)
    assert np.all(_stat_agree(m32, s32, m64, s64))


# --------------------------------------------------------------- edge cases
def test_empty_and_ragged(ctx):
    w = W.sphere_cap(P=5, walks=1)
    m, s, t, rc = ctx.solve(w.problem, w.params, w.points[:0], 7)
    assert m.size == 0
    S, K, F = ctx.walk_scores(w.problem, w.params, w.points, 37, precision=M.FP32)   # ragged tail
    assert S.shape == (5, 37) and np.all(K > 0)
    S1, K1, _ = ctx.walk_scores(w.problem, w.params, w.points, 1)
    assert np.array_equal(S1[:, 0], ctx.walk_scores(w.problem, w.params, w.points, 37)[0][:, 0])


def test_start_inside_boundary_layer(ctx):
    """K = 0: a start point within eps of Gamma scores g(cp_Gamma(y0)) (k = 0 stop)."""
    w = W.sphere_cap(P=1, walks=1)
    z = 5e-4
    y0 = np.array([[math.sqrt(1 - z * z), 0.0, z]])
    S, K, F = ctx.walk_scores(w.problem, w.params, y0, 4)
    assert np.all(K == 0) and np.allclose(S, 0.0, atol=1e-15)     # g = xy = 0 at (1, 0, 0)


def test_max_steps_status(ctx):
    w = W.torus_closed(P=2, walks=1)
    w.params.max_steps = 10
    m, s, t, rc = ctx.solve(w.problem, w.params, w.points, 4)
    assert rc == M.MPWOS_EMAXSTEPS and np.all(t == 10)


def test_invalid_arguments(ctx):
    w = W.sphere_cap(P=2, walks=1)
    w.problem.sigma = -1.0
    with pytest.raises(M.MpwosError) as ei:
        ctx.solve(w.problem, w.params, w.points, 4)
    assert ei.value.code == M.MPWOS_EINVAL and "sigma" in str(ei.value)
    w = W.hypersphere_half(P=1, walks=1)
    w.problem.sigma = 5000.0
    with pytest.raises(M.MpwosError):
        ctx.solve(w.problem, w.params, w.points, 4)


def test_device_pointers(ctx):
    import torch
    w = W.sphere_cap(P=8, walks=1)
    pts = torch.tensor(w.points, device="cuda", dtype=torch.float64)
    out = tuple(torch.zeros(8, device="cuda", dtype=torch.float64) for _ in range(3))
    ctx.solve(w.problem, w.params, pts, 64, out=out)
    mh, sh, th, _ = ctx.solve(w.problem, w.params, w.points, 64)
    assert np.array_equal(out[0].cpu().numpy(), mh) and np.array_equal(out[2].cpu().numpy(), th)


def test_native_launches_counted(ctx):
    before = ctx.launch_count()
    w = W.torus_closed(P=2, walks=1)
    ctx.solve(w.problem, w.params, w.points, 8, precision=M.FP32)
    assert ctx.launch_count() > before
