"""One request split by walk range and merged on the host (mpwos_solve_partial,
mpwos_merge_partials) reproduces mpwos_solve bit for bit; the device's block
records equal the host implementation of the same summation order on the same
per-walk scores.  On one GPU, each range stands for one rank's share."""
import numpy as np
import pytest

import paper_2606_21883_b300 as M
from paper_2606_21883_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = M.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("make,N,prec,cuts", [
    (lambda: W.sphere_cap(P=5, walks=1), 3000, M.FP64, [1024, 2048]),
    (lambda: W.torus_closed(P=33, walks=1), 5000, M.FP32, [2048]),
    (lambda: W.hypersphere_half(P=3, walks=1, seed=4), 1500, M.FP32, [1024]),
])
def test_split_merges_to_solve_bits(ctx, make, N, prec, cuts):
    w = make()
    whole = ctx.solve(w.problem, w.params, w.points, N, precision=prec)
    edges = [0] + cuts + [N]
    parts = [ctx.solve_partial(w.problem, w.params, w.points, N, a, b, precision=prec)
             for a, b in zip(edges, edges[1:])]
    got = M.merge_partials(parts)
    for x, y in zip(got[:3], whole[:3]):
        assert np.array_equal(x, y)


def test_device_records_equal_host_records(ctx):
    w = W.sphere_cap(P=4, walks=1)
    N = 2500
    S, K, F = ctx.walk_scores(w.problem, w.params, w.points, N, precision=M.FP64)
    dev = ctx.solve_partial(w.problem, w.params, w.points, N, 0, N, precision=M.FP64)
    host = M.block_partials_host(S, K, F)
    assert dev.shape == host.shape == (4, 3, M.EST_FIELDS)
    assert np.array_equal(dev, host)
    # a later range's records are those of its own walks
    dev2 = ctx.solve_partial(w.problem, w.params, w.points, N, 1024, N, precision=M.FP64)
    assert np.array_equal(dev2, M.block_partials_host(S[:, 1024:], K[:, 1024:], F[:, 1024:]))


def test_misaligned_range_is_rejected(ctx):
    w = W.sphere_cap(P=2, walks=1)
    with pytest.raises(M.MpwosError) as e:
        ctx.solve_partial(w.problem, w.params, w.points, 3000, 100, 2048, precision=M.FP64)
    assert e.value.code == M.MPWOS_EINVAL
    with pytest.raises(M.MpwosError):
        ctx.solve_partial(w.problem, w.params, w.points, 3000, 1024, 2000, precision=M.FP64)
