"""The benchmark's multi-replica timing logic (max over ranks, whole-job throughput) on two
gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank), GRTX_BENCH_BACKEND="gloo")
    import bench
    d = bench.Dist()
    d.barrier()
    seconds = 1.0 + rank          # rank 1 is the slowest
    value, t = bench.aggregate_throughput(1000.0, seconds, d.world, d.max)
    q.put((rank, value, t))
    d.close()


def test_two_rank_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, value, t in res:
        assert t == 2.0
        assert value == pytest.approx(2 * 1000.0 / 2.0)
