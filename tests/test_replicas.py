"""Multi-GPU runs of bench.py are replicas (no collective on the data path):
the host-side aggregation -- barrier, max over ranks, whole-job rate -- is
checked here with two gloo ranks on the CPU."""
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


def _rank(rank, ws, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    bench.barrier(ws)
    value, ms = bench.weak_scaling_value(1000, 10.0 * (rank + 1), ws)
    env = bench.dist_env()
    dist.destroy_process_group()
    q.put((rank, value, ms, env))


def test_weak_scaling_aggregation_two_gloo_ranks():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(60)
        assert p.exitcode == 0
    for rank, value, ms, env in out:
        assert ms == 20.0  # the slower rank
        assert value == pytest.approx(2 * 1000 / 0.020)
        assert env == (2, rank, 0)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.weak_scaling_value(500, 4.0, 1) == (500 / 0.004, 4.0)
