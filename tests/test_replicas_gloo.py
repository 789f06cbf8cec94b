"""Multi-GPU runs are independent replicas (no data-path collective): the
only cross-rank step is bench.py's timing, max over ranks, and the whole-job
throughput.  Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [120.0, 80.0][rank]
    ms = bench.max_over_ranks(local_ms, "cpu")
    out[rank] = (ms, bench.job_throughput(256, world, ms))
    dist.destroy_process_group()


def test_two_replicas_time_is_the_slowest_and_throughput_adds_up():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        ms, value = res[r]
        assert ms == 120.0
        assert value == pytest.approx(2 * 256 / 0.120)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(42.0) == 42.0
    assert bench.job_throughput(256, 1, 64.0) == pytest.approx(4000.0)
