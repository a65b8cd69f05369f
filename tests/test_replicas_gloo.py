"""bench.py's multi-GPU contract (replicas only): every rank solves its own
problems and the job's rate is all ranks' solves over the slowest rank's
time.  Checked with two gloo ranks on the CPU."""
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


def _rank(rank, world, port, local_ms, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    value, max_ms = bench.aggregate_replicas(local_ms[rank], steps=4, world=world)
    out[rank] = (value, max_ms)
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    port = _free_port()
    local_ms = [1000.0, 1600.0]
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, local_ms, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(2):
        value, max_ms = res[r]
        assert max_ms == 1600.0
        assert value == pytest.approx(2 * 4 / 1.6)


def test_single_replica_needs_no_process_group():
    import bench
    value, max_ms = bench.aggregate_replicas(500.0, steps=5, world=1)
    assert max_ms == 500.0 and value == pytest.approx(10.0)
