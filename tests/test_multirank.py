"""Host logic of the multi-rank benchmark path, on CPU with the gloo backend
and two ranks. By default the one 256-domain batch is split over the ranks by
cell count (whole domains, longest first to the least-loaded rank): the union
of the shards is the batch, the shards are disjoint, their cell counts differ
by less than the largest domain, and rank 0 reports the cells of all ranks. In
the weak mode every rank advances its own independently seeded batch. Only the
timing (max) and the cell count (sum) are reduced over ranks: there is no
data-path collective."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, scaling, q):
    import torch
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = bench.rank_workload(rank, world, scaling)
        total = bench.over_ranks(wl.cells, world, torch, "sum", device="cpu")
        tmax = bench.over_ranks(0.25 + rank, world, torch, "max", device="cpu")
        sides = [(d.nx, d.ny) for d in wl.domains]
        q.put((rank, wl.cells, total, tmax, sides, wl.meta.get("domains")))
    finally:
        dist.destroy_process_group()


def _run(world, scaling):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, scaling, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


def test_two_ranks_split_one_batch_by_cell_count():
    pytest.importorskip("torch")
    from paper_1709_09073_gb300 import workloads as W
    batch = W.batched_taylor_green(seed=20260101)
    res = _run(2, "strong")
    cells = [r[1] for r in res]
    assert all(r[2] == batch.cells for r in res)          # every rank reports the whole batch
    assert all(r[3] == 1.25 for r in res)                 # time = max over ranks
    owned = [r[5] for r in res]
    assert sorted(owned[0] + owned[1]) == list(range(len(batch.domains)))   # union, disjoint
    for r in res:                                         # each shard is those domains, in order
        assert r[4] == [(batch.domains[i].nx, batch.domains[i].ny) for i in r[5]]
    largest = max(d.nx * d.ny for d in batch.domains)
    assert abs(cells[0] - cells[1]) <= largest            # balanced within one domain


def test_two_ranks_weak_mode_runs_independent_batches():
    pytest.importorskip("torch")
    import bench
    res = _run(2, "weak")
    cells = [r[1] for r in res]
    assert all(r[2] == sum(cells) for r in res)
    assert res[0][4] != res[1][4]                         # independent batches per rank
    assert res[0][4] == [(d.nx, d.ny) for d in bench.rank_workload(0, 2, "weak").domains]


def test_split_by_cells_properties():
    from paper_1709_09073_gb300 import partition
    cells = [5, 9, 1, 1, 7, 3, 3, 8, 2]
    for n in (1, 2, 3, 4, 9, 12):
        parts = partition.split_by_cells(cells, n)
        assert len(parts) == n
        assert sorted(i for p in parts for i in p) == list(range(len(cells)))
        loads = [sum(cells[i] for i in p) for p in parts]
        assert max(loads) - sum(cells) / n < max(cells)   # the longest-first bound
        assert all(p == sorted(p) for p in parts)
    assert partition.split_by_cells(cells, 2) == partition.split_by_cells(list(cells), 2)  # deterministic
    assert partition.split_by_cells(cells, 1) == [list(range(len(cells)))]


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.over_ranks(3.5, 1, None) == 3.5
