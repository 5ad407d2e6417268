"""FP32 torus walks whose source is one Fourier mode (m, q <= 3) run a kernel
instance with the modes built in; every other source runs the generic series.

Both draw identical numbers and differ only in how cos(m theta), sin(m theta),
cos(q phi), sin(q phi) are formed (closed forms vs repeated rotation, FP32
rounding), so per walk |dS| <= 1e-5 max(1, |S|) and identical K.  A second,
zero-weight term forces the generic path on the same data."""
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


def _with_source(w, terms, apply_op):
    w.problem.f = W.Func.torus(terms, apply_op=apply_op)
    return w


@pytest.mark.parametrize("m,q,ts,ps,op", [(1, 2, W.TRIG_SIN, W.TRIG_COS, True), (0, 0, W.TRIG_COS, W.TRIG_COS, True),
                                          (3, 3, W.TRIG_COS, W.TRIG_SIN, True), (2, 1, W.TRIG_SIN, W.TRIG_SIN, False),
                                          (3, 0, W.TRIG_SIN, W.TRIG_COS, True), (0, 2, W.TRIG_COS, W.TRIG_SIN, False)])
def test_single_mode_instance_matches_generic_series(ctx, m, q, ts, ps, op):
    w = W.torus_closed(P=8, walks=1, seed=m * 4 + q)
    one = _with_source(W.torus_closed(P=8, walks=1, seed=m * 4 + q), [(1.3, m, q, ts, ps)], op)
    two = _with_source(w, [(1.3, m, q, ts, ps), (0.0, 1, 1, W.TRIG_COS, W.TRIG_COS)], op)
    Sa, Ka, Fa = ctx.walk_scores(one.problem, one.params, one.points, 64, precision=M.FP32)
    Sb, Kb, Fb = ctx.walk_scores(two.problem, two.params, two.points, 64, precision=M.FP32)
    assert np.array_equal(Ka, Kb) and np.array_equal(Fa, Fb)
    assert np.all(np.abs(Sa - Sb) <= 1e-5 * np.maximum(1.0, np.abs(Sb)))


def test_single_mode_instance_vs_oracle(ctx):
    """A mode other than the benchmark's, (m, q) = (2, 3), statistically against the FP64 oracle."""
    w = _with_source(W.torus_closed(P=5, walks=1, seed=9), [(1.0, 2, 3, W.TRIG_COS, W.TRIG_SIN)], True)
    m32, s32, t32, rc = ctx.solve(w.problem, w.params, w.points, 1500, precision=M.FP32)
    mo, so, to, nf = O.solve(w.problem, w.params, w.points, 1500)
    assert np.all(np.abs(m32 - mo) < 4 * np.sqrt(s32 ** 2 + so ** 2))
    assert np.all(t32 == 525)
