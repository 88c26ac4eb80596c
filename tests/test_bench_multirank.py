"""Host logic of bench.py for N > 1 replicas, on CPU with world_size 2 over gloo: the job time is
the maximum over ranks, and the rate counts every rank's roundings (weak scaling)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as mp       # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    job = bench.max_over_ranks(100.0 + 50.0 * rank, world, "cpu")
    out[rank] = (job, bench.job_rate(10, world, job))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_count_all_work():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        job, rate = out[r]
        assert job == 150.0                              # max over ranks, seen by every rank
        assert abs(rate - world * 10 / 0.150) < 1e-9     # 20 roundings in 150 ms


def test_single_rank_is_its_own_job():
    import bench
    assert bench.max_over_ranks(42.0, 1, "cpu") == 42.0
    assert bench.job_rate(5, 1, 500.0) == 10.0
