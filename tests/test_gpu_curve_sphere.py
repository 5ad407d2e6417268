"""GPU walks on Example 3's Fourier curve x S^2(a) in R^9 against the CPU oracle.

FP64: per-walk parity, |S_gpu - S_orc| <= 1e-12 max(1, |S|) with identical K and flags
(complete walks, 824 steps each).  FP32 (fast sine and cosine in the curve's Newton
iteration, stopped at 1e-6): statistical agreement with the oracle; the example's RMSE."""
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


def test_curve_sphere_parity_fp64(ctx):
    w = W.curve_sphere(P=3, walks=1, seed=1)
    Sg, Kg, Fg = ctx.walk_scores(w.problem, w.params, w.points, 8, precision=M.FP64)
    So, Ko, Fo = O.walk_scores(w.problem, w.params, w.points, 8)
    ok = (np.abs(Sg - So) <= REL * np.maximum(1.0, np.abs(So))) & (Kg == Ko) & (Fg == Fo)
    assert np.count_nonzero(~ok) <= 0, (np.argwhere(~ok)[:3].tolist(), Sg[~ok][:3], So[~ok][:3])
    assert np.all(Kg > 100)


def test_curve_sphere_telescoping(ctx):
    w = W.curve_sphere(P=3, walks=1, seed=2)
    w.problem.f = W.Func.curve_sphere([(0, W.TRIG_COS, 1.0, np.zeros(3), np.zeros((3, 3)))], apply_op=True)
    for prec, tol in ((M.FP64, 1e-12), (M.FP32, 1e-9)):
        S, K, F = ctx.walk_scores(w.problem, w.params, w.points, 16, precision=prec)
        assert not F.any()
        assert np.all((S > 1 - w.params.tau_w - tol * K) & (S <= 1 + tol * K))


def test_curve_sphere_fp32_vs_oracle(ctx):
    w = W.curve_sphere(P=4, walks=1, seed=4)
    m32, s32, t32, rc = ctx.solve(w.problem, w.params, w.points, 40000, precision=M.FP32)
    mo, so, to, nf = O.solve(w.problem, w.params, w.points, 500)
    assert rc == M.MPWOS_OK and nf == 0
    assert np.all(np.abs(m32 - mo) < 4 * np.sqrt(s32 ** 2 + so ** 2))
    assert np.all(t32 == to)


def test_curve_sphere_e3_rmse(ctx):
    """Example 3 (100 points, FP32): RMSE against u falls with the walk count."""
    w = W.curve_sphere(P=100, walks=1)
    rm = []
    for N in (100, 1000, 10000):
        m, s, t, rc = ctx.solve(w.problem, w.params, w.points, N, precision=M.FP32)
        assert rc == M.MPWOS_OK
        rm.append(float(np.sqrt(np.mean((m - w.exact) ** 2))))
    print("E3 RMSE", rm)
    assert rm[0] > rm[1] > rm[2]
