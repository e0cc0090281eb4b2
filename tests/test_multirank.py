"""Multi-rank timing logic of bench.py on CPU (gloo, world size 2).

bench.py --gpus N runs one replica per GPU (the streams are independent, no
exchange step); rank 0 reports the whole-job rate from the slowest rank.
"""

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


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = [100.0 + 50.0 * rank, 7.0 * (rank + 1)]
    got = bench.max_over_ranks(mine)
    out[rank] = got
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    assert out[0] == [150.0, 14.0] and out[1] == [150.0, 14.0]


def test_whole_job_rate_weak_and_sharded():
    import bench
    block_s = 65536 * 1024 / 200e6
    assert bench.whole_job_rate(1, block_s, 100.0) == pytest.approx(3.3554432)
    # two replicas, slowest rank 110 ms per block
    assert bench.whole_job_rate(2, block_s, 110.0) == pytest.approx(2 * block_s / 0.110)
    # two ranks sharing the beams of one block, slowest rank 60 ms
    assert bench.whole_job_rate(2, block_s, 60.0, sharded=True) == pytest.approx(block_s / 0.060)
