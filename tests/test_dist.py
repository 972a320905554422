"""Multi-process (gloo, CPU) checks of the replica aggregation used by bench.py."""
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


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r "took" 1 + r seconds and converged 100 eigenpairs per step over 3 steps
    value, t_max, units = bench.aggregate(1.0 + rank, 300.0, "cpu")
    q.put((rank, value, t_max, units))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_replica_aggregation_gloo(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, t_max, units in out:
        assert t_max == float(world)             # max over ranks
        assert units == 300.0 * world            # sum over ranks
        assert value == units / t_max


def test_single_process_aggregation():
    import bench
    assert bench.aggregate(2.0, 10.0)[0] == 5.0
