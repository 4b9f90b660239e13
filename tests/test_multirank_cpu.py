"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2): every
rank gets its own set of realisations and the timed region's duration is the
maximum over ranks.  No GPU is involved."""
import os
import socket

import numpy as np
import pytest


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
    t = bench.reduce_max(1.0 + rank, world)
    wl = bench.make_workload("crossing_batch", "2,1", rank)
    q.put((rank, t, float(wl.members[0].eta[0, 0]), len(wl.members)))
    dist.destroy_process_group()


def test_two_ranks_gloo():
    torch = pytest.importorskip("torch")
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(r[1] == 2.0 for r in res)          # max over ranks on every rank
    assert res[0][3] == res[1][3] == 3            # same batch shape
    assert res[0][2] != res[1][2]                 # different realisations per rank


def test_single_rank_reduce_is_identity():
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5
