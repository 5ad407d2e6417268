"""The launch-shape autotuner: picks a block size per walk kernel from timed chunks
of a real call, and changes no result.

Each walk's random numbers depend only on (point, walk, step) and the per-point sums
run in a fixed order, so every per-walk score, stopping index and flag, and every
per-point mean, must be bit-identical with the tuner on or off, in the tuning call
itself (whose first walks run under each candidate shape) and in later calls (which
launch the pick), request serving included."""
import numpy as np
import pytest

import paper_2606_21883_b300 as M
from paper_2606_21883_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _check_entry(e, limit):
    cands = sorted(e["ns_per_walk_step"])
    assert cands == [b for b in (32, 64, 128, 256) if b <= limit]
    assert e["block"] in cands
    times = e["ns_per_walk_step"]
    assert all(t > 0 for t in times.values())
    assert times[e["block"]] == min(times.values())


def test_autotune_torus_thread_walk_identical():
    """The fixed-radius torus walk (one thread per walk, up to 256 threads per block)."""
    w = W.torus_closed(P=256, walks=1)
    N = 10_000   # 2.56e6 walks: five parts of at least two waves each
    plain = M.Context(0)
    S0, K0, F0 = plain.walk_scores(w.problem, w.params, w.points, N, precision=M.FP32)
    plain.close()
    ctx = M.Context(0)
    ctx.set_autotune(True)
    S1, K1, F1 = ctx.walk_scores(w.problem, w.params, w.points, N, precision=M.FP32)
    ents = ctx.autotune_entries()
    assert len(ents) == 1 and ents[0]["n"] == 3
    _check_entry(ents[0], 256)
    assert np.array_equal(S0, S1) and np.array_equal(K0, K1) and np.array_equal(F0, F1)
    # a later call launches the pick and records nothing new
    S2, K2, F2 = ctx.walk_scores(w.problem, w.params, w.points, N, precision=M.FP32)
    assert len(ctx.autotune_entries()) == 1
    assert np.array_equal(S0, S2) and np.array_equal(K0, K2) and np.array_equal(F0, F2)
    ctx.close()


def test_autotune_warp_walk_and_solve_identical():
    """The warp walk (Example 3's curve x sphere in R^9, walks of uneven length, up to
    128 threads per block) through mpwos_solve: same per-point means as untuned."""
    w = W.curve_sphere(P=128, walks=1, seed=3)
    N = 1024
    plain = M.Context(0)
    m0, s0, t0, rc0 = plain.solve(w.problem, w.params, w.points, N, precision=M.FP32)
    plain.close()
    ctx = M.Context(0)
    ctx.set_autotune(True)
    m1, s1, t1, rc1 = ctx.solve(w.problem, w.params, w.points, N, precision=M.FP32)
    ents = ctx.autotune_entries()
    assert len(ents) == 1 and ents[0]["n"] == 9
    _check_entry(ents[0], 128)
    assert rc0 == rc1
    assert np.array_equal(m0, m1) and np.array_equal(s0, s1) and np.array_equal(t0, t1)
    ctx.close()


def test_autotune_small_call_records_nothing():
    w = W.torus_closed(P=4, walks=1)
    ctx = M.Context(0)
    ctx.set_autotune(True)
    S1, K1, F1 = ctx.walk_scores(w.problem, w.params, w.points, 64, precision=M.FP32)
    assert ctx.autotune_entries() == []
    ctx.set_autotune(False)
    S0, K0, F0 = ctx.walk_scores(w.problem, w.params, w.points, 64, precision=M.FP32)
    assert np.array_equal(S0, S1) and np.array_equal(K0, K1)
    ctx.close()
