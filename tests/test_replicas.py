"""The multi-GPU path runs independent replicas (one process per GPU, no
data-path collective).  Its host logic, checked here with two gloo ranks on
the CPU: the timed region is the max over the ranks, the value is the
whole-job throughput, and the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        mine = 10.0 * (rank + 1) + 0.25
        got = bench.reduce_max_ms(mine, ws, "cpu")
        # the reference arm does no work off rank 0 (it returns before
        # building or running anything)
        ran_reference = bench.reference_arm(None) is not None if rank != 0 else None
        dist.barrier()
        with open(os.path.join(out_dir, "rank%d.txt" % rank), "w") as f:
            f.write("%r %r\n" % (got, ran_reference))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    ws, port = 2, _free_port()
    mp.spawn(_rank, args=(ws, port, str(tmp_path)), nprocs=ws, join=True)
    for rank in range(ws):
        got, ran_reference = open(tmp_path / ("rank%d.txt" % rank)).read().split()
        assert float(got) == 10.0 * ws + 0.25  # the slowest rank's time, seen by every rank
        if rank != 0:
            assert ran_reference == "False"


def test_job_throughput_counts_every_replica():
    sys.path.insert(0, ROOT)
    import bench
    one = bench.job_throughput(1, 10, 3, 1 << 26, 80.0)
    assert bench.job_throughput(4, 10, 3, 1 << 26, 80.0) == 4 * one
    assert bench.job_throughput(2, 10, 3, 1 << 26, 160.0) == one  # twice the replicas in twice the time
    assert bench.reduce_max_ms(7.5, 1, "cpu") == 7.5  # one rank: no collective
