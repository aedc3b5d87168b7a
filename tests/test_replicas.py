"""Replica runs across ranks, on CPU with gloo (world size 2): the whole-job
rate is the units of all ranks over the slowest rank's time, and every rank
sees the same figure (the benchmark's N-GPU path uses the same function)."""
import os
import socket

import torch.multiprocessing as mp


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1907_02900_gb300.replicas import whole_job_rate
    units = [1000.0, 3000.0][rank]
    ms = [10.0, 40.0][rank]
    out[rank] = whole_job_rate(units, ms)
    dist.barrier()
    dist.destroy_process_group()


def test_whole_job_rate_two_ranks():
    port = _free_port()
    # spawn, not fork: earlier tests may have left threads (OpenMP, CUDA) in this process
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        for r in range(2):
            rate, mx = out[r]
            assert mx == 40.0
            assert abs(rate - 4000.0 / 0.040) < 1e-6


def test_whole_job_rate_without_process_group():
    from paper_1907_02900_gb300.replicas import whole_job_rate
    rate, mx = whole_job_rate(500.0, 20.0)
    assert mx == 20.0 and abs(rate - 25_000.0) < 1e-9
