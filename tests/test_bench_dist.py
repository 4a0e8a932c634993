"""Host logic of the multi-rank bench on CPU: two gloo ranks on 127.0.0.1 (no GPU)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, local = bench.dist_env()
    t = bench.max_over_ranks(1.0 + rank)          # rank 1 is the slowest
    v = bench.job_throughput(10.0, ws, t)
    out[rank] = (ws, r, local, t, v)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time_and_sum_the_work():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn",
                       join=True)
    for rank in range(world):
        ws, r, local, t, v = out[rank]
        assert (ws, r, local) == (2, rank, rank)
        assert t == 2.0                                # max over ranks
        assert v == pytest.approx(10.0 * 2 / 2.0)      # all ranks' units / max time


def test_single_process_helpers_without_distributed():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_throughput(5.0, 1, 2.0) == 2.5
