"""Device y-slabs (rlbm_pack_edge_rows / rlbm_unpack_ghost_rows and
slabs.DeviceSlab): one domain cut into uneven y-slabs, each fed every step
only the 30 edge-row planes its neighbours send (Eqs. 17-18: the pull reaches
one row) into the ghost row of an RLBM_EXCHANGED side (or of a zero-gradient
placeholder side), reproduces the undivided domain on the GPU bit for bit -- stored
populations and streamed fields -- in every storage format and in both step
kernels, with periodic, fixed-temperature-wall, zero-gradient and
velocity-wall sides and a body force. In process the slabs are domains of one
handle whose packed faces are handed over on the device; across processes two
ranks on the one GPU step their slabs through DeviceSlab over gloo. A packed
face written back into a y-periodic domain's own ghost row leaves its state
unchanged, which pins the face layout to the step kernels' periodic halo."""
import dataclasses
import os
import queue
import socket

import numpy as np
import pytest

from paper_1709_09073_gb300 import slabs, workloads as W

pytestmark = pytest.mark.gpu

P, ZG, WALL, VW = W.PERIODIC, W.ZERO_GRADIENT, W.FIXED_T_WALL, W.VELOCITY_WALL


@pytest.fixture(scope="module")
def R():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1709_09073_gb300 import build, rlbm
    build.build()
    rlbm.load()
    return rlbm


def _slab_specs(spec, bounds, internal=slabs.EXCHANGED):
    n = len(bounds)
    return [dataclasses.replace(spec, ny=y1 - y0, bc=slabs.slab_bcs(spec.bc, r, n, internal))
            for r, (y0, y1) in enumerate(bounds)]


def _cut(init, y0, y1):
    c = lambda a: np.ascontiguousarray(a[y0:y1])
    return W.InitialState(init.kind, c(init.a), c(init.theta), c(init.ux), c(init.uy))


class _InProcess:
    """Stand-in for SlabExchange between slabs of one process: the
    neighbours' packed faces are copied on the device."""

    def __init__(self, parts, below, above):
        self.parts, self.below, self.above = parts, below, above

    def exchange_packed(self, send_lo, send_hi, recv_lo, recv_hi):
        if self.below is not None:
            recv_lo.copy_(self.parts[self.below].send_hi)
        if self.above is not None:
            recv_hi.copy_(self.parts[self.above].send_lo)


def _halo_all(parts):
    # every slab packs before any slab unpacks: the rows sent are this step's
    for p in parts:
        p.pack()
    for p in parts:
        p.ex.exchange_packed(p.send_lo, p.send_hi, p.recv_lo, p.recv_hi)
        p.unpack()


def _whole(R, spec, init, steps, storage, kernel):
    sim = R.Simulation([spec], edf=spec.edf, storage=storage)
    st = sim.init(0, init)
    if kernel is not None:
        sim.select_kernel(kernel)
    sim.step(steps)
    f = sim.get_populations(0)
    out = sim.moments(0)
    st |= sim.sync_status()
    sim.close()
    return f, out, st


def _slabbed(R, spec, init, bounds, steps, storage, kernel, internal=slabs.EXCHANGED):
    specs = _slab_specs(spec, bounds, internal)
    sim = R.Simulation(specs, edf=spec.edf, storage=storage)
    st = 0
    for r, (y0, y1) in enumerate(bounds):
        st |= sim.init(r, _cut(init, y0, y1))
    if kernel is not None:
        sim.select_kernel(kernel)
    periodic_y = spec.bc[2] == P
    parts = []
    for r in range(len(bounds)):
        below, above = slabs.neighbours(r, len(bounds), periodic_y)
        parts.append(slabs.DeviceSlab(sim, r, _InProcess(parts, below, above)))
    for _ in range(steps):
        _halo_all(parts)
        sim.step(1)
    _halo_all(parts)  # the streamed fields read the ghost rows
    f = [sim.get_populations(r) for r in range(len(bounds))]
    outs = [sim.moments(r) for r in range(len(bounds))]
    st |= sim.sync_status()
    sim.close()
    f = np.concatenate([g[:, 1:-1, :] for g in f], axis=1)
    outs = [np.concatenate([o[k] for o in outs], axis=0) for k in range(5)]
    return f, outs, st


CASES = {
    "periodic": ((P, P, P, P), (1.0,) * 4, {}),
    "x_walls": ((WALL, WALL, P, P), (0.97, 1.04, 1.0, 1.0), {}),
    "y_walls_open_x": ((ZG, ZG, WALL, WALL), (1.0, 1.0, 1.03, 0.96), {}),
    "channel_force": ((P, P, VW, VW), (1.02,) * 4, dict(accel=(2e-4, -1e-4), n_wall=1.05)),
    "x_velocity_walls": ((VW, VW, P, P), (1.02,) * 4, dict(n_wall=0.98)),
}


def _check_equal(R, spec, init, bounds, steps, storage, kernel=None, internal=slabs.EXCHANGED):
    f0, out0, st0 = _whole(R, spec, init, steps, storage, kernel)
    f1, out1, st1 = _slabbed(R, spec, init, bounds, steps, storage, kernel, internal)
    assert (st0 & R.RLBM_W_NONPHYSICAL) == 0 and st0 == st1
    assert np.array_equal(f1, f0[:, 1:-1, :])
    for k in range(5):
        assert np.array_equal(out1[k], out0[k]), k
    return out0


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_slabs_bit_exact(R, orc, name):
    bc, tw, extra = CASES[name]
    nx, ny, steps = 23, 13, 12
    spec = W.DomainSpec(nx, ny, 0.85, W.MJ, bc, tw, **extra)
    init = W.random_domain_state(nx, ny, 41, W.MJ, u_amp=0.06)
    out = _check_equal(R, spec, init, [(0, 5), (5, 6), (6, 13)], steps, R.RLBM_F64)
    # and the undivided run is the oracle's
    dom = orc.domain(nx, ny, spec.tau, spec.edf, bc, tw, accel=spec.accel, n_wall=spec.n_wall)
    f, m, _ = orc.init(dom, init.kind, init.a, init.theta, init.ux, init.uy)
    f, m, _ = orc.run(dom, f, m, steps)
    ref, _ = orc.fields(dom, f, m, streamed=True)
    assert np.max(np.abs(out[0] - ref[0]) / ref[0]) <= 1e-12
    assert np.max(np.abs(out[2] - ref[2])) <= 1e-12 * np.max(np.abs(ref[2]))


@pytest.mark.parametrize("edf", [W.FD, W.BE])
def test_fp64_slabs_quantum_statistics(R, edf):
    spec = W.DomainSpec(17, 12, 0.9, edf, (WALL, WALL, P, P), (0.97, 1.04, 1.0, 1.0))
    init = W.random_domain_state(17, 12, 50 + edf, edf, u_amp=0.05)
    _check_equal(R, spec, init, [(0, 4), (4, 8), (8, 12)], 8, R.RLBM_F64)


@pytest.mark.parametrize("storage", ["RLBM_F32", "RLBM_F32DEV", "RLBM_BF16DEV", "RLBM_F16DEV"])
@pytest.mark.parametrize("name", ["periodic", "x_walls", "y_walls_open_x"])
def test_mixed_storage_slabs_bit_exact(R, storage, name):
    bc, tw, _ = CASES[name]
    nx, ny = 37, 14
    spec = W.DomainSpec(nx, ny, 0.8, W.MJ, bc, tw, scale=0.5)
    init = W.random_domain_state(nx, ny, 43, W.MJ, u_amp=0.05)
    _check_equal(R, spec, init, [(0, 6), (6, 7), (7, 14)], 10, getattr(R, storage))


@pytest.mark.parametrize("storage", ["RLBM_F64", "RLBM_F32DEV"])
@pytest.mark.parametrize("name", ["periodic", "x_walls", "channel_force"])
def test_zero_gradient_placeholder_slabs_bit_exact(R, storage, name):
    """The slab sides facing a neighbour as zero-gradient placeholders (the
    step writes copies there, which the next face overwrites) instead of
    RLBM_EXCHANGED sides: the same populations and fields."""
    if name == "channel_force" and storage != "RLBM_F64":
        pytest.skip("velocity walls are FP64 only")
    bc, tw, extra = CASES[name]
    spec = W.DomainSpec(31, 12, 0.85, W.MJ, bc, tw, **extra)
    init = W.random_domain_state(31, 12, 47, W.MJ, u_amp=0.05)
    _check_equal(R, spec, init, [(0, 5), (5, 12)], 8, getattr(R, storage), internal=slabs.ZERO_GRADIENT)


@pytest.mark.parametrize("storage", ["RLBM_F32DEV", "RLBM_F16DEV"])
def test_tma_kernel_slabs_bit_exact(R, storage):
    spec = W.DomainSpec(37, 16, 0.8, W.BE, (WALL, WALL, P, P), (0.97, 1.04, 1.0, 1.0))
    init = W.random_domain_state(37, 16, 44, W.BE, u_amp=0.05)
    _check_equal(R, spec, init, [(0, 8), (8, 16)], 6, getattr(R, storage), kernel=R.RLBM_KERNEL_TMA)


@pytest.mark.parametrize("storage", ["RLBM_F64", "RLBM_F32DEV", "RLBM_BF16DEV"])
def test_face_layout_matches_periodic_halo(R, storage):
    """Packing the top row of a y-periodic domain and unpacking it as the row
    from below (and the bottom row as the row from above) rewrites its ghost
    rows with what the step kernel's periodic halo put there."""
    spec = W.DomainSpec(29, 9, 0.9, W.MJ, (WALL, WALL, P, P), (0.97, 1.04, 1.0, 1.0))
    init = W.random_domain_state(29, 9, 45, W.MJ, u_amp=0.05)
    sim = R.Simulation([spec], edf=W.MJ, storage=getattr(R, storage))
    sim.init(0, init)
    sim.step(3)
    before = sim.get_populations(0)
    lo, hi = sim.edge_row_buffer(0), sim.edge_row_buffer(0)
    assert lo.shape == (30, spec.nx + 2)
    sim.pack_edge_rows(0, lo, hi)
    scratch = before.copy()
    scratch[6:36, 0, :] = -1.0   # spoil the planes the unpack must restore
    scratch[42:72, -1, :] = -1.0
    sim.set_populations(0, scratch)
    sim.unpack_ghost_rows(0, hi, lo)
    after = sim.get_populations(0)
    assert np.array_equal(after, before)
    sim.close()


def test_argument_errors(R):
    import torch
    spec = W.DomainSpec(8, 4, 0.9)
    sim = R.Simulation([spec], edf=W.MJ, storage=R.RLBM_F64)
    buf = sim.edge_row_buffer(0)
    with pytest.raises(R.RlbmError):  # not initialised yet
        sim.pack_edge_rows(0, buf, None)
    sim.init(0, W.random_domain_state(8, 4, 1, W.MJ))
    with pytest.raises(R.RlbmError):
        sim.pack_edge_rows(1, buf, None)
    odd = torch.empty(30 * 10 * 8 + 4, dtype=torch.uint8, device="cuda")[4:]  # misaligned for FP64
    with pytest.raises(R.RlbmError):
        sim.unpack_ghost_rows(0, odd, None)
    sim.pack_edge_rows(0, None, None)  # nothing to do
    assert R.load().rlbm_edge_row_bytes(sim.h, 0) == 30 * 10 * 8
    assert R.load().rlbm_edge_row_bytes(sim.h, 3) == 0
    sim.close()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


RANK_CASE = dict(nx=21, ny=10, steps=7, tau=0.85)


def _rank_spec(name):
    bc, tw, extra = CASES[name]
    c = RANK_CASE
    return (W.DomainSpec(c["nx"], c["ny"], c["tau"], W.MJ, bc, tw, **extra),
            W.random_domain_state(c["nx"], c["ny"], 46, W.MJ, u_amp=0.06))


def _rank_main(rank, world, port, name, storage, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import torch.distributed as dist
    from paper_1709_09073_gb300 import rlbm, slabs as S
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        spec, init = _rank_spec(name)
        y0, y1 = S.slab_bounds(spec.ny, world)[rank]
        sspec = _slab_specs(spec, S.slab_bounds(spec.ny, world))[rank]
        sim = rlbm.Simulation([sspec], edf=spec.edf, storage=storage)
        sim.init(0, _cut(init, y0, y1))
        part = S.DeviceSlab(sim, 0, S.SlabExchange(rank, world, spec.nx, spec.bc[2] == P))
        part.step(RANK_CASE["steps"])
        part.halo()
        f = sim.get_populations(0)[:, 1:-1, :]
        st = sim.sync_status()
        sim.close()
        q.put((rank, f, st))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name,storage", [("periodic", 0), ("x_walls", 4)])
def test_two_ranks_device_slabs(R, name, storage):
    """Two processes on the one GPU, each stepping its slab with DeviceSlab;
    device faces travel over gloo through host memory. No kernel waits on the
    other process: each exchange is complete on the host before the next
    launch."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, name, storage, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = []
    try:
        while len(res) < 2:
            try:
                res.append(q.get(timeout=5))
            except queue.Empty:
                dead = [p.exitcode for p in procs if p.exitcode not in (None, 0)]
                assert not dead, "a rank failed: exit codes %s" % dead
    finally:
        for p in procs:
            p.join(timeout=120)
            if p.exitcode is None:
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    res.sort(key=lambda r: r[0])
    spec, init = _rank_spec(name)
    f0, _, _ = _whole(R, spec, init, RANK_CASE["steps"], storage, None)
    got = np.concatenate([r[1] for r in res], axis=1)
    assert np.array_equal(got, f0[:, 1:-1, :])
    assert all(r[2] == 0 for r in res)
