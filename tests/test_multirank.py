"""The multi-GPU path of bench.py on CPU: world-size-2 gloo ranks simulate
disjoint trajectory ranges and the job time is the max over ranks (the only
exchange; the simulation itself needs no collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t_local = 1.0 + rank                      # rank 1 is the slow one
    value, t = bench.world_throughput(t_local, steps=3, ntraj=1000, dist=dist)
    q.put((rank, value, t, bench.trajectory_base(rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_aggregation():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, value, t, base in out:
        assert t == 2.0                          # max over ranks
        assert value == pytest.approx(2 * 3 * 1000 / 2.0)
    b0, b1 = out[0][3], out[1][3]
    assert b1 - b0 >= 100_000 * 1000             # disjoint trajectory ranges
