"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2): replicas only, the job time is the max over
ranks and the job's work the sum; no other cross-rank communication exists."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, work = bench.reduce_over_ranks(10.0 + rank, 100.0 * (rank + 1), world, "cpu")
    q.put((rank, ms, work))
    dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
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
    for _, ms, work in res:
        assert ms == pytest.approx(11.0)
        assert work == pytest.approx(300.0)


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_over_ranks(3.5, 7.0, 1, "cpu") == (3.5, 7.0)
