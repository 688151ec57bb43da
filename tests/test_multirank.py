"""Host logic of the multi-rank (weak-scaling) benchmark path, on CPU with the
gloo backend and two ranks: each rank advances its own independently seeded
batch of domains (no data-path collective); only the timing (max) and the cell
count (sum) are reduced over ranks."""
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


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = bench.rank_workload(rank)
        total = bench.over_ranks(wl.cells, world, torch, "sum", device="cpu")
        tmax = bench.over_ranks(0.25 + rank, world, torch, "max", device="cpu")
        sides = [(d.nx, d.ny) for d in wl.domains]
        q.put((rank, wl.cells, total, tmax, sides))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_domains_and_reduce_only_metadata():
    pytest.importorskip("torch")
    import multiprocessing as mp
    import bench
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    cells = [r[1] for r in res]
    assert all(r[2] == sum(cells) for r in res)       # value uses the cells of all ranks
    assert all(r[3] == 1.25 for r in res)              # time = max over ranks
    assert res[0][4] != res[1][4]                      # independent batches per rank
    assert res[0][4] == [(d.nx, d.ny) for d in bench.rank_workload(0).domains]  # deterministic


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.over_ranks(3.5, 1, None) == 3.5
