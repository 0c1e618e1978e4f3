"""The N>1 path of bench.py (replicas, one per GPU) on CPU with 2 gloo ranks:
the step time is the maximum over ranks and the job rate counts every rank's
rows."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank 1 is the slow replica
    ms, rate = bench.job_rate(1000.0, 2.0 if rank == 0 else 5.0, world, "cpu")
    out[rank] = (ms, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_job_rate_takes_the_slowest_rank_and_all_rows():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    for r in range(2):
        ms, rate = out[r]
        assert ms == 5.0
        assert rate == pytest.approx(2 * 1000.0 / 0.005)


def test_job_rate_single_rank():
    import bench
    ms, rate = bench.job_rate(60.0, 4.0, 1, "cpu")
    assert ms == 4.0 and rate == pytest.approx(15000.0)
