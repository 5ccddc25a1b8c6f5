"""The multi-GPU path runs independent replicas (one instance per rank, no
collective in the data path); the only exchange is the final aggregation of
the benchmark numbers: max of the ranks' times, sum of their particle pushes.
Checked with two gloo ranks on the CPU."""
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


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r = {"ms": 10.0 + rank, "pushes": 1000 * (rank + 1), "e2e_s": 0.5 * (rank + 1), "e2e_pushes": 7 * (rank + 1)}
    out = bench.reduce_over_ranks(r, dist, "cpu")
    q.put((rank, out))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        assert res[r]["ms"] == 11.0
        assert res[r]["pushes"] == 3000.0
        assert res[r]["e2e_s"] == 1.0
        assert res[r]["e2e_pushes"] == 21.0


def test_single_rank_passthrough():
    import bench
    r = {"ms": 3.0, "pushes": 5, "e2e_s": 1.0, "e2e_pushes": 2}
    out = bench.reduce_over_ranks(r, None, "cpu")
    assert out == {"ms": 3.0, "pushes": 5.0, "e2e_s": 1.0, "e2e_pushes": 2.0}
