"""The benchmark's multi-rank host logic on CPU: two gloo ranks (no GPU).

Weak scaling shards by query points with no data-path collective: each rank
draws its own batch (seed = rank), the timed region's slowest rank sets the
time (max over ranks), and the whole-job rate counts every rank's units."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = bench.rank_workload(16, 10, rank)
    # every rank sees the others' point checksums: the batches are disjoint draws
    chk = torch.tensor([float(np.sum(w.points * np.arange(1, 4)))], dtype=torch.float64)
    allc = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(allc, chk)
    t_dev, t_e2e = 1.0 + 0.5 * rank, 2.0 - 0.25 * rank
    tmax, emax = bench.max_over_ranks(dist, "cpu", t_dev, t_e2e)
    rate = bench.aggregate_rate(1000.0, 3, world, tmax)
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as fh:
        fh.write(" ".join(str(float(c)) for c in allc) + f"\n{tmax} {emax} {rate}\n")
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_weak_scaling_host_logic_gloo(world, tmp_path):
    port = _free_port()
    mp.start_processes(_rank, args=(world, port, str(tmp_path)), nprocs=world, start_method="spawn")
    lines = [open(tmp_path / f"r{r}.txt").read().split("\n") for r in range(world)]
    chks = [tuple(map(float, l[0].split())) for l in lines]
    assert all(c == chks[0] for c in chks)                     # all ranks agree on the gathered values
    assert len(set(chks[0])) == world                          # disjoint per-rank batches
    for l in lines:
        tmax, emax, rate = map(float, l[1].split())
        assert tmax == 1.5 and emax == 2.0                     # the slowest rank's times
        assert rate == pytest.approx(1000.0 * 3 * world / 1.5)
    assert bool(len(lines) == world)


def test_single_rank_is_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(None, "cpu", 1.25, 3.0) == (1.25, 3.0)
    assert bench.aggregate_rate(10.0, 2, 1, 4.0) == 5.0
