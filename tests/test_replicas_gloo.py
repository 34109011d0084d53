"""The multi-GPU mode is replicas only (independent systems, no collective
on the data path): the job's rate is all ranks' solves over the slowest
rank's time.  Checked with two gloo ranks on the CPU."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
        dist.barrier()
        ms, value = bench.job_throughput(local_ms, 3, dist, "cpu")
        q.put((rank, ms, value))
    finally:
        dist.destroy_process_group()


def test_replica_rate_is_max_over_ranks():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in out:
        assert ms == 150.0                     # every rank sees the slowest time
        assert value == pytest.approx(2 * 3 / 0.150)


def test_single_process_rate():
    import bench
    ms, value = bench.job_throughput(200.0, 4)
    assert ms == 200.0 and value == pytest.approx(20.0)
