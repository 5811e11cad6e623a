"""The N > 1 path of bench.py on CPU with the gloo backend (world size 2):
every rank gets its own clusters (weak scaling), the job time is the slowest
rank's, and the job value counts every rank's units.  No GPU is used."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    t = 100.0 + 50.0 * rank
    t_max = bench.max_over_ranks(t, dist, "cpu")
    off, adj, clusters, d = bench.workload(10, 8, rank)
    first = [int(c[0]) for c in clusters]
    dist.barrier()
    out[rank] = (t_max, bench.job_value(1000, world, t_max), first, bench.rank_seed(rank))
    dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling_host_logic():
    world = 2
    mgr = tmp.get_context("spawn").Manager()
    out = mgr.dict()
    tmp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    assert out[0][0] == out[1][0] == 150.0  # the slowest rank's time for both
    assert abs(out[0][1] - 1000 * 2 / 0.150 / 1e9) < 1e-12
    assert out[0][3] != out[1][3]  # each rank draws its own clusters
    assert out[0][2] != out[1][2]


def test_single_rank_is_identity():
    import bench

    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert bench.job_value(2_000_000_000, 1, 1000.0) == 2.0
