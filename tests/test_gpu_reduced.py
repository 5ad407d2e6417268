"""GPU walks with the dimension-reduced exact sampler against the CPU oracle.

FP64 mode draws the oracle's reduced stream (same blocks, Box-Muller and
Marsaglia-Tsang attempts), so walks are compared one by one:
|S_gpu - S_orc| <= 1e-12 max(1, |S|) with identical K and flags (a threshold
decision within rounding of eps or tau_W may flip in at most 1e-3 of walks).
FP32 mode is compared statistically: |mean32 - mean64| < 4 sqrt(se32^2 + se64^2).
"""
import numpy as np
import pytest

import oracle as O
import paper_2606_21883_b300 as M
from paper_2606_21883_b300 import workloads as W

pytestmark = pytest.mark.gpu
REL = 1e-12


@pytest.fixture(scope="module")
def ctx():
    c = M.Context(0)
    yield c
    c.close()


def _reduced(w):
    w.params.sampler = W.SAMPLER_REDUCED
    return w


def _walk_parity(ctx, w, N, ):
    Sg, Kg, Fg = ctx.walk_scores(w.problem, w.params, w.points, N, precision=M.FP64)
    So, Ko, Fo = O.walk_scores(w.problem, w.params, w.points, N)
    ok = (np.abs(Sg - So) <= REL * np.maximum(1.0, np.abs(So))) & (Kg == Ko) & (Fg == Fo)
    bad = np.count_nonzero(~ok)
    assert bad == 0, (
        f"{bad} of {ok.size} walks differ; S {Sg[~ok][:3]} vs {So[~ok][:3]}, K {Kg[~ok][:3]} vs {Ko[~ok][:3]}")
    return Sg, Kg


def test_reduced_parity_hemisphere_s63(ctx):
    w = _reduced(W.hypersphere_half(P=6, walks=1, n=64, seed=3))
    _walk_parity(ctx, w, 40)


def test_reduced_parity_hemisphere_s999_capped(ctx):
    """S^999 in R^1000 (T = {x_1, x_2, x_3}, chi^2 with 996 dof), walks capped at 30 steps."""
    w = _reduced(W.hypersphere_half(P=4, walks=1, n=1000, seed=1))
    w.params.max_steps = 30
    _walk_parity(ctx, w, 16)


def test_reduced_parity_embedded_s20_capped(ctx):
    """S^20 in R^1000 (21 intrinsic normals, chi^2 with 979 dof), walks capped at 25 steps."""
    w = _reduced(W.embedded_s20(P=3, walks=1))
    w.params.max_steps = 25
    _walk_parity(ctx, w, 8)


def test_reduced_parity_embedded_complete_walks(ctx):
    w = _reduced(W.embedded_s20(P=4, walks=1, n=64, d=5, sigma=6.0))
    w.params.tau_w = 1e-4
    Sg, Kg = _walk_parity(ctx, w, 8)
    assert np.all(Kg == Kg.flat[0])


def test_reduced_parity_euclid(ctx):
    w = _reduced(W.euclid_halfspace(P=5, walks=1, n=12, sigma=2.0, seed=4))
    w.params.c_kappa = 2.0   # kappa = 0 in R^n: rho_geo = 2 caps the ball radius (inside the table range)
    _walk_parity(ctx, w, 40)


@pytest.mark.parametrize("prec", [M.FP64, M.FP32])
def test_reduced_telescoping(ctx, prec):
    w = _reduced(W.constant_solution(W.hypersphere_half(P=4, walks=1, n=1000, seed=5)))
    w.params.max_steps = 100000
    S, K, F = ctx.walk_scores(w.problem, w.params, w.points, 64, precision=prec)
    tol = 1e-12 if prec == M.FP64 else 1e-9
    assert np.all(F == 0) and np.all(np.abs(S - 1.0) <= tol * np.maximum(K, 1))


def test_reduced_fp32_vs_oracle_hemisphere(ctx):
    w = _reduced(W.hypersphere_half(P=4, walks=1, n=64, seed=3))
    N = 1500
    m32, s32, t32, rc = ctx.solve(w.problem, w.params, w.points, N, precision=M.FP32)
    mo, so, to, nf = O.solve(w.problem, w.params, w.points, N)
    assert rc == M.MPWOS_OK and nf == 0
    assert np.all(np.abs(m32 - mo) < 4 * np.sqrt(s32 ** 2 + so ** 2))
    assert np.all(np.abs(t32 - to) < 0.05 * to + 5)


def test_reduced_fp32_vs_full_fp32_embedded(ctx):
    """Same problem, full and reduced directions: the walk's law is the same."""
    w = W.embedded_s20(P=4, walks=1, n=64, d=5, sigma=6.0)
    w.params.tau_w = 1e-4
    N = 4000
    mf, sf, tf, _ = ctx.solve(w.problem, w.params, w.points, N, precision=M.FP32)
    mr, sr, tr, _ = ctx.solve(w.problem, _reduced(w).params, w.points, N, precision=M.FP32)
    assert np.all(np.abs(mf - mr) < 4 * np.sqrt(sf ** 2 + sr ** 2))
    assert np.all(tf == tr)


def test_reduced_fp32_s999_manufactured(ctx):
    """The 1000-dimensional hemisphere to completion: mean vs u = x_1 + x_2 x_3."""
    w = _reduced(W.hypersphere_half(P=8, walks=1, n=1000, seed=0))
    m, s, t, rc = ctx.solve(w.problem, w.params, w.points, 4096, precision=M.FP32)
    assert rc == M.MPWOS_OK
    assert np.all(np.abs(m - w.exact) < 4 * s + 0.02)


def test_reduced_rejected_where_unsupported(ctx):
    t = _reduced(W.torus_closed(P=2, walks=1))
    with pytest.raises(M.MpwosError) as e:
        ctx.walk_scores(t.problem, t.params, t.points, 4, precision=M.FP32)
    assert e.value.code == M.MPWOS_EINVAL
    c = _reduced(W.sphere_cap(P=2, walks=1))   # n = 3
    with pytest.raises(M.MpwosError) as e:
        ctx.walk_scores(c.problem, c.params, c.points, 4, precision=M.FP32)
    assert e.value.code == M.MPWOS_EINVAL


@pytest.mark.parametrize("case", ["s20_r1000", "s5_r64"])
def test_embedded_reduced_walks_do_not_depend_on_the_launch(ctx, case):
    """A launch of few walks on an embedded sphere runs one warp per walker (FP32);
    walk (p, i) must come out the same bit for bit as in a launch of many walks
    (one thread per walker)."""
    if case == "s20_r1000":
        w = W.embedded_s20(P=4, walks=1)
        w.params.max_steps = 3000
    else:
        w = W.embedded_s20(P=4, walks=1, n=64, d=5, sigma=6.0)
    w.params.sampler = W.SAMPLER_REDUCED
    small = ctx.walk_scores(w.problem, w.params, w.points, 64, precision=M.FP32)      # 256 walks
    large = ctx.walk_scores(w.problem, w.params, w.points, 4096, precision=M.FP32)    # 16,384 walks
    for a, b in zip(small, large):
        assert np.array_equal(np.asarray(a), np.asarray(b)[:, :64])
