"""The y-slab decomposition plan (paper_1709_09073_gb300/slabs.py) on CPU:
slabs stepped by the oracle, each fed only the 30 edge-row planes its
neighbours send, reproduce the whole-domain oracle bit for bit -- with periodic,
fixed-temperature, zero-gradient and velocity-wall sides and a body force, in
process for three uneven slabs (and for one slab, which keeps the domain's own
y sides), and as two or
three gloo ranks exchanging rows with torch.distributed point-to-point
messages (the same exchange that carries the device-packed rows of slabs on
GPUs over NCCL)."""
import os
import socket

import numpy as np
import pytest

from paper_1709_09073_gb300 import slabs, workloads as W

PERIODIC, ZG, WALL = W.PERIODIC, W.ZERO_GRADIENT, W.FIXED_T_WALL
VW = W.VELOCITY_WALL
CASES = {
    "periodic": ((PERIODIC,) * 4, (1.0,) * 4),
    "x_walls": ((WALL, WALL, PERIODIC, PERIODIC), (0.97, 1.04, 1.0, 1.0)),
    "y_walls_open_x": ((ZG, ZG, WALL, WALL), (1.0, 1.0, 1.03, 0.96)),
    # velocity walls with a body force (Sec. 3.4): channel walls at the slab stack's
    # ends, and walls on the x sides of every slab
    "channel_force": ((PERIODIC, PERIODIC, VW, VW), (1.02,) * 4),
    "x_velocity_walls": ((VW, VW, PERIODIC, PERIODIC), (1.02,) * 4),
}
FORCE = dict(accel=(2e-4, -1e-4), n_wall=1.05)


def test_plan():
    up, down = slabs.planes_up(), slabs.planes_down()
    assert len(up) == len(down) == 30 and not set(up) & set(down)
    for q in up:
        assert np.sin((q // 6) * np.pi / 6) > 0.1
    for q in down:
        assert np.sin((q // 6) * np.pi / 6) < -0.1
    assert slabs.halo_bytes_per_face(8190, 4) == 983040  # one FP32 face of an 8192-wide domain
    b = slabs.slab_bounds(11, 3)
    assert b == [(0, 4), (4, 8), (8, 11)]
    assert slabs.neighbours(0, 3, False) == (None, 1) and slabs.neighbours(2, 3, True) == (1, 0)
    # two periodic ranks border each other on both faces; one slab is the whole domain
    assert slabs.neighbours(0, 2, True) == (1, 1)
    assert slabs.neighbours(0, 1, True) == (None, None)
    assert slabs.slab_bcs((0, 0, 0, 0), 0, 1) == (0, 0, 0, 0)
    assert slabs.slab_bcs((0, 0, 0, 0), 0, 2) == (0, 0, 4, 4)
    assert slabs.slab_bcs((2, 2, 2, 2), 1, 3) == (2, 2, 4, 4)
    assert slabs.slab_bcs((2, 2, 2, 2), 2, 3) == (2, 2, 4, 2)
    assert slabs.slab_bcs((2, 2, 2, 2), 2, 3, internal=1) == (2, 2, 1, 2)
    with pytest.raises(ValueError):
        slabs.slab_bounds(2, 3)


def _setup(orc, name, nx, ny):
    bc, tw = CASES[name]
    extra = FORCE if VW in bc else {}
    spec = W.DomainSpec(nx, ny, 0.85, W.MJ, bc, tw, **extra)
    init = W.random_domain_state(nx, ny, 77, W.MJ, u_amp=0.06)
    return spec, init


def _domain(orc, spec, ny, bc):
    return orc.domain(spec.nx, ny, spec.tau, spec.edf, bc, spec.t_wall, accel=spec.accel, n_wall=spec.n_wall)


def _whole(orc, spec, init, steps):
    dom = _domain(orc, spec, spec.ny, spec.bc)
    f, m, _ = orc.init(dom, init.kind, init.a, init.theta, init.ux, init.uy)
    f, m, _ = orc.run(dom, f, m, steps)
    return f


class _Slab:
    def __init__(self, orc, spec, init, rank, nranks):
        self.orc = orc
        y0, y1 = slabs.slab_bounds(spec.ny, nranks)[rank]
        self.y0, self.y1 = y0, y1
        bc = slabs.slab_bcs(spec.bc, rank, nranks, internal=slabs.ZERO_GRADIENT)
        self.dom = _domain(orc, spec, y1 - y0, bc)
        cut = lambda a: np.ascontiguousarray(a[y0:y1])
        self.f, self.m, _ = orc.init(self.dom, init.kind, cut(init.a), cut(init.theta), cut(init.ux),
                                     cut(init.uy))
        # velocity walls read the full six-plane state of the previous step
        self.full = orc.has_velocity_wall(self.dom)
        if self.full:
            self.m, _ = orc.fields(self.dom, self.f, None, streamed=False)

    def edges(self):
        return self.orc.edge_row(self.dom, self.f, self.m, 0), self.orc.edge_row(self.dom, self.f, self.m, 1)

    def step(self, row_lo, row_hi):
        self.f, mo, _ = self.orc.step_rows(self.dom, self.f, self.m, row_lo, row_hi)
        self.m = mo.copy() if self.full else mo[[0, 2, 3]].copy()


@pytest.mark.parametrize("k", [1, 3])
@pytest.mark.parametrize("name", list(CASES))
def test_uneven_slabs_in_process(orc, name, k):
    nx, ny, steps = 14, 11, 6
    spec, init = _setup(orc, name, nx, ny)
    periodic_y = spec.bc[2] == PERIODIC
    parts = [_Slab(orc, spec, init, r, k) for r in range(k)]
    up, down = slabs.planes_up(), slabs.planes_down()
    for _ in range(steps):
        edges = [p.edges() for p in parts]
        for r, p in enumerate(parts):
            below, above = slabs.neighbours(r, k, periodic_y)
            lo = slabs.unpack(slabs.pack(edges[below][1], up), up, nx) if below is not None else None
            hi = slabs.unpack(slabs.pack(edges[above][0], down), down, nx) if above is not None else None
            p.step(lo, hi)
    got = np.concatenate([p.f for p in parts], axis=1)
    assert np.array_equal(got, _whole(orc, spec, init, steps))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, name, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import torch.distributed as dist
    from oracle import oracle as orc
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        nx, ny, steps = 12, 10, 5
        spec, init = _setup(orc, name, nx, ny)
        part = _Slab(orc, spec, init, rank, world)
        ex = slabs.SlabExchange(rank, world, nx, spec.bc[2] == PERIODIC)
        for _ in range(steps):
            if world == 3:  # packed faces, None toward the domain's ends
                bottom, top = part.edges()
                f = lambda row, planes, keep: (torch.from_numpy(slabs.pack(row, planes)) if keep else None)
                send_lo, send_hi = f(bottom, ex.down, ex.below is not None), f(top, ex.up, ex.above is not None)
                recv_lo = torch.empty((30, nx + 2), dtype=torch.float64) if ex.below is not None else None
                recv_hi = torch.empty((30, nx + 2), dtype=torch.float64) if ex.above is not None else None
                ex.exchange_packed(send_lo, send_hi, recv_lo, recv_hi)
                lo = slabs.unpack(recv_lo.numpy(), ex.up, nx) if recv_lo is not None else None
                hi = slabs.unpack(recv_hi.numpy(), ex.down, nx) if recv_hi is not None else None
            else:
                lo, hi = ex.exchange(*part.edges())
            part.step(lo, hi)
        q.put((rank, part.y0, part.f))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name,world", [("periodic", 2), ("x_walls", 2), ("y_walls_open_x", 3)])
def test_gloo_ranks_match_whole_domain(orc, name, world):
    """Two periodic ranks are each other's neighbour on both faces (messages
    must match in order); three ranks between y walls have open ends."""
    pytest.importorskip("torch")
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, name, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(world)), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got = np.concatenate([r[2] for r in res], axis=1)
    spec, init = _setup(orc, name, 12, 10)
    assert np.array_equal(got, _whole(orc, spec, init, 5))
