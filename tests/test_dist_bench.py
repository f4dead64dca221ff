"""The multi-rank logic of bench.py on CPU (gloo, world size 2): every rank
simulates its own problem with its own seed, the job time is the slowest rank's
and the job's shots are the sum over ranks (weak scaling, no data-path collective)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    d, w, r, local = bench.dist_setup()
    assert (w, r, local) == (world, rank, rank) and d is not None
    t = bench.max_over_ranks(d, 10.0 + rank)
    s = bench.sum_over_ranks(d, 32000)
    q.put((rank, t, s))
    d.destroy_process_group()


def test_two_rank_reductions():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert got == [(0, 11.0, 64000.0), (1, 11.0, 64000.0)]


def test_single_rank_is_identity(monkeypatch):
    import bench

    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    d, w, r, local = bench.dist_setup()
    assert d is None and (w, r, local) == (1, 0, 0)
    assert bench.max_over_ranks(None, 3.5) == 3.5 and bench.sum_over_ranks(None, 7) == 7
