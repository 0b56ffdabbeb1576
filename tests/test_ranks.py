"""The multi-GPU path of bench.py is replicas only (every rank evaluates its own
link, no data exchange): its host logic -- max-over-ranks step time and the sum
of channel evaluations -- checked with two gloo ranks on the CPU."""
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


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = 10.0 + 5.0 * rank      # rank 1 is the slow one
    res = bench.aggregate_ranks(ms_local, 120)
    q.put((rank, res))
    dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        ms, value, world = out[r]
        assert world == 2
        assert ms == pytest.approx(15.0)             # the slowest rank sets the time
        assert value == pytest.approx(240 / 15e-3)   # channel-evals of both ranks


def test_single_process_aggregation():
    import bench
    ms, value, world = bench.aggregate_ranks(20.0, 120)
    assert (ms, world) == (20.0, 1) and value == pytest.approx(6000.0)
