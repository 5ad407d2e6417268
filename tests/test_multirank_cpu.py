"""The multi-rank path on CPU: gloo ranks, no GPU.

One request is split over the ranks by walk range at estimator-block
boundaries (bench.rank_walk_range); each rank forms the block records of its
walks (here from the oracle's per-walk scores through the library's host
implementation of the device's summation order); the records of all ranks are
gathered in rank order (bench.gather_partials, one all_gather) and merged on the
host (mpwos_merge_partials).  The merged estimate must equal the single-rank
merge bit for bit and agree with the oracle's own estimator.  The benchmark's
timing helpers (max over ranks, whole-job rate) are checked too."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N_WALKS = 2600


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _scores():
    import oracle as O
    from paper_2606_21883_b300 import workloads as W
    w = W.sphere_cap(P=3, walks=1)
    S, K, F = O.walk_scores(w.problem, w.params, w.points, N_WALKS, n_threads=1)
    return w, S, K.astype(np.int32), F.astype(np.int32)


def _rank(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    import paper_2606_21883_b300 as M
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    _, S, K, F = _scores()
    i0, i1 = bench.rank_walk_range(N_WALKS, rank, world)
    part = torch.from_numpy(M.block_partials_host(S[:, i0:i1], K[:, i0:i1], F[:, i0:i1]))
    parts = bench.gather_partials(dist, part, world)
    mean, se, ms, nf = M.merge_partials(parts)
    t_dev, t_e2e = 1.0 + 0.5 * rank, 2.0 - 0.25 * rank
    tmax, emax = bench.max_over_ranks(dist, "cpu", t_dev, t_e2e)
    rate = bench.aggregate_rate(1000.0, 3, world, tmax)
    np.savez(os.path.join(out_dir, f"r{rank}.npz"), mean=mean, se=se, ms=ms, nf=nf, rng=[i0, i1],
             times=[tmax, emax, rate])
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_walk_range_split_merges_exactly_gloo(world, tmp_path):
    import sys
    sys.path.insert(0, ROOT)
    import oracle as O
    import paper_2606_21883_b300 as M
    port = _free_port()
    mp.start_processes(_rank, args=(world, port, str(tmp_path)), nprocs=world, start_method="spawn")
    res = [np.load(tmp_path / f"r{r}.npz") for r in range(world)]
    rngs = [tuple(r["rng"]) for r in res]
    assert rngs[0][0] == 0 and rngs[-1][1] == N_WALKS
    assert all(a[1] == b[0] for a, b in zip(rngs, rngs[1:]))          # consecutive ranges
    assert all(a % 1024 == 0 for a, _ in rngs)                         # block-aligned starts
    w, S, K, F = _scores()
    whole = M.merge_partials([M.block_partials_host(S, K, F)])
    for r in res:                                                      # every rank merged the same bits
        assert np.array_equal(r["mean"], whole[0]) and np.array_equal(r["se"], whole[1])
        assert np.array_equal(r["ms"], whole[2]) and int(r["nf"]) == whole[3]
        tmax, emax, rate = r["times"]
        assert tmax == 0.5 * world + 0.5 and emax == 2.0               # the slowest rank's times
        assert rate == pytest.approx(1000.0 * 3 * world / tmax)
    mo, so, to, _ = O.solve(w.problem, w.params, w.points, N_WALKS, n_threads=1)
    assert np.allclose(whole[0], mo, rtol=1e-13, atol=1e-15)
    assert np.allclose(whole[1], so, rtol=1e-11)
    assert np.array_equal(whole[2], to)


def test_block_records_merge_like_the_definition():
    """Any split at block boundaries merges to the same bits; the merged mean and
    standard error equal the definitions (two-pass, float128 reference) also where
    the one-pass formula cancels (a large common offset)."""
    import sys
    sys.path.insert(0, ROOT)
    import paper_2606_21883_b300 as M
    rng = np.random.default_rng(5)
    P, N = 4, 5000
    S = 1e6 + rng.standard_normal((P, N)) * 1e-3
    K = rng.integers(1, 600, size=(P, N)).astype(np.int32)
    F = np.zeros((P, N), dtype=np.int32)
    F[1, 77] = 1
    whole = M.merge_partials([M.block_partials_host(S, K, F)])
    for cuts in ([1024], [2048, 3072], [1024, 2048, 3072, 4096]):
        edges = [0] + cuts + [N]
        parts = [M.block_partials_host(S[:, a:b], K[:, a:b], F[:, a:b]) for a, b in zip(edges, edges[1:])]
        got = M.merge_partials(parts)
        assert all(np.array_equal(x, y) for x, y in zip(got[:3], whole[:3])) and got[3] == whole[3] == 1
    Sl = S.astype(np.longdouble)
    mu = Sl.mean(axis=1)
    se = np.sqrt(((Sl - mu[:, None]) ** 2).sum(axis=1) / (N - 1) / N)
    assert np.allclose(whole[0], mu.astype(float), rtol=1e-14)
    assert np.allclose(whole[1], se.astype(float), rtol=1e-6)
    assert np.array_equal(whole[2], K.mean(axis=1))


def test_rank_walk_range_blocks():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    for N in (1, 1023, 1024, 10000, 40960):
        for world in (1, 2, 3, 8):
            rs = [bench.rank_walk_range(N, r, world) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == N
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
            assert all(i0 % 1024 == 0 and (i1 % 1024 == 0 or i1 == N) for i0, i1 in rs)


def test_single_rank_is_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(None, "cpu", 1.25, 3.0) == (1.25, 3.0)
    assert bench.aggregate_rate(10.0, 2, 1, 4.0) == 5.0
