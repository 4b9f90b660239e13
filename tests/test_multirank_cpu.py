"""Multi-rank host logic on CPU (gloo, world size 2), no GPU involved:

* replicas: every rank gets its own set of realisations and the timed
  region's duration is the maximum over ranks;
* split: one batch is divided over the ranks by cost (largest first into the
  lightest rank), every member lands on exactly one rank, the ranks' loads
  differ by at most one member's cost, and the per-member invariants gathered
  by one all-reduce equal those of a single-rank run (computed here with the
  oracle on small members).
"""
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


def test_partition_of_the_bench_batch():
    from paper_2310_19840_gb300 import shard as S
    shapes = [(256, 256)] * 64 + [(512, 512)] * 32
    for world in (1, 2, 3, 4, 5, 8):
        parts = S.partition(shapes, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(shapes)))            # each member exactly once
        loads = S.rank_loads(shapes, parts)
        biggest = max(S.member_cost(*sh) for sh in shapes)
        assert max(loads) - min(loads) <= biggest + 1e-6, (world, loads)
    # power-of-two rank counts give every rank the same mix
    for world in (2, 4, 8):
        for p in S.partition(shapes, world):
            assert sum(1 for i in p if i >= 64) == 32 // world and len(p) == 96 // world


def test_partition_uneven_shapes_and_edge_cases():
    from paper_2310_19840_gb300 import shard as S
    shapes = [(4096, 2048), (256, 256), (512, 512), (64, 32), (1024, 1), (512, 512), (128, 128)]
    parts = S.partition(shapes, 3)
    assert sorted(i for p in parts for i in p) == list(range(len(shapes)))
    loads = S.rank_loads(shapes, parts)
    assert max(loads) - min(loads) <= max(S.member_cost(*sh) for sh in shapes)
    assert parts[0] == [0]                                 # the largest alone on the first rank
    assert S.partition([], 2) == [[], []]
    assert S.partition([(64, 64)], 4)[0] == [0]
    with pytest.raises(ValueError):
        S.partition(shapes, 0)


def _split_worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from oracle import sbi_oracle as O
    from paper_2310_19840_gb300 import shard as S
    wl = bench.make_workload("crossing_batch", "3,2", rank, world, "split")
    local = {}
    for li, gi in enumerate(wl.notes["global_members"]):
        m = wl.members[li]
        pb = O.Problem(O.Grid(m.nx, m.ny, m.Lx, m.Ly), wl.gravity, m.h0)
        local[gi] = O.invariants(pb, m.eta, m.phi)
    table = S.gather_invariants(wl.notes["global_count"], local, world)
    cfg = bench.workload_config(wl)
    q.put((rank, list(wl.notes["global_members"]), table.tolist(), cfg["points"]))
    dist.destroy_process_group()


def test_split_batch_gathers_invariants_gloo():
    pytest.importorskip("torch")
    import multiprocessing as mp
    import bench
    from oracle import sbi_oracle as O
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_split_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    whole = bench.make_workload("crossing_batch", "3,2")
    # every member on exactly one rank; both ranks report the whole batch's points
    assert sorted(res[0][1] + res[1][1]) == list(range(len(whole.members)))
    assert res[0][3] == res[1][3] == whole.points
    # the gathered table equals the single-rank invariants on every rank
    ref = []
    for m in whole.members:
        pb = O.Problem(O.Grid(m.nx, m.ny, m.Lx, m.Ly), whole.gravity, m.h0)
        ref.append(O.invariants(pb, m.eta, m.phi))
    for r in res:
        assert np.allclose(np.array(r[2]), np.array(ref), rtol=1e-14, atol=0)
