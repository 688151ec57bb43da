"""Host-side plan of a y-slab decomposition of one domain over several ranks
(one GPU each): which rows each rank owns and which populations cross a slab
edge every step.

The pull stencil (Eqs. 17-18) reaches one row: a cell reads row y - 1 only for
the directions with v_y > 0 and row y + 1 only for those with v_y < 0. So each
step a slab sends the 5 directions x 6 shells = 30 planes with v_y > 0 of its
top row to the slab above, and the 30 planes with v_y < 0 of its bottom row to
the slab below, each row with its two x ghost values (x = -1 and x = nx) so
that x walls and x periodicity need nothing more. Rows are [72][nx + 2]
arrays; the planes a neighbour does not need are left NaN.

The exchange below uses torch.distributed point-to-point messages (gloo on the
host, NCCL between GPUs). On a GPU the rows never leave the device: librlbm
packs a slab's two edge rows into [30][nx + 2] faces in the storage encoding
and writes received faces into its ghost rows (DeviceSlab). The batched
benchmark shards whole domains instead and needs none of this.
"""
import numpy as np

N_DIRECTIONS, N_SHELLS = 12, 6


def sign_vy(d):
    """Sign of the y velocity of direction d (phi_d = d pi / 6)."""
    if d % 6 == 0:
        return 0
    return 1 if d < 6 else -1


def planes_up():
    """Population planes q = 6 d + s that the row above reads from a slab's top row."""
    return [6 * d + s for d in range(N_DIRECTIONS) if sign_vy(d) > 0 for s in range(N_SHELLS)]


def planes_down():
    """Planes that the row below reads from a slab's bottom row."""
    return [6 * d + s for d in range(N_DIRECTIONS) if sign_vy(d) < 0 for s in range(N_SHELLS)]


def slab_bounds(ny, nranks):
    """Rows [y0, y1) of each rank, as equal as possible, lower ranks at lower y."""
    if nranks < 1 or ny < nranks:
        raise ValueError("need 1 <= nranks <= ny")
    base, extra = divmod(ny, nranks)
    out, y = [], 0
    for r in range(nranks):
        h = base + (1 if r < extra else 0)
        out.append((y, y + h))
        y += h
    return out


def neighbours(rank, nranks, periodic_y):
    """(rank below, rank above); None at a non-periodic end of the domain, and
    both None for a single slab (it keeps the domain's own y sides)."""
    if nranks == 1:
        return None, None
    below = rank - 1 if rank > 0 else (nranks - 1 if periodic_y else None)
    above = rank + 1 if rank < nranks - 1 else (0 if periodic_y else None)
    return below, above


ZERO_GRADIENT, EXCHANGED = 1, 4


def slab_bcs(bc, rank, nranks, internal=EXCHANGED):
    """Boundary conditions of a slab: x sides as the domain's; a y side that
    borders another slab gets `internal`. EXCHANGED (the device path) has the
    step write nothing there, since the neighbour's face fills that ghost row;
    ZERO_GRADIENT (the oracle, which knows no exchanged side) is a placeholder
    that the face overwrites. A single slab is the whole domain."""
    if nranks == 1:
        return tuple(bc)
    xlo, xhi, ylo, yhi = bc
    periodic_y = ylo == 0
    lo = internal if (periodic_y or rank > 0) else ylo
    hi = internal if (periodic_y or rank < nranks - 1) else yhi
    return (xlo, xhi, lo, hi)


def pack(row, planes):
    """The planes of a [72][nx + 2] edge row that a neighbour needs (contiguous)."""
    return np.ascontiguousarray(row[planes])


def unpack(buf, planes, nx):
    """A received row: the sent planes in place, NaN elsewhere."""
    row = np.full((72, nx + 2), np.nan)
    row[planes] = buf
    return row


class SlabExchange:
    """Point-to-point exchange of edge rows between y-neighbouring ranks."""

    UP, DOWN = 11, 12  # message tags: rows travelling up / down

    def __init__(self, rank, nranks, nx, periodic_y):
        self.rank, self.nranks, self.nx = rank, nranks, nx
        self.below, self.above = neighbours(rank, nranks, periodic_y)
        self.up, self.down = planes_up(), planes_down()

    def exchange_packed(self, send_lo, send_hi, recv_lo, recv_hi):
        """Send the packed faces (send_lo: the bottom row's planes for the slab
        below, send_hi: the top row's for the slab above) and receive the
        neighbours' into recv_lo (from below) and recv_hi (from above). Torch
        tensors on the process group's device (CPU for gloo, the rank's GPU
        for NCCL); faces toward a non-periodic end of the domain are skipped
        and may be None.
        Both sends are posted before both receives, rows travelling up first
        on either side, so that two ranks that are each other's neighbour on
        both faces match their messages in order as well as by tag. Device
        faces over a host-only backend (gloo) are staged through host memory."""
        import torch.distributed as dist
        faces = [t for t in (send_lo, send_hi, recv_lo, recv_hi) if t is not None]
        stage = bool(faces) and faces[0].is_cuda and dist.get_backend() == "gloo"
        if stage:
            dev_lo, dev_hi = recv_lo, recv_hi
            host = lambda t: t.cpu() if t is not None else None
            send_lo, send_hi = host(send_lo), host(send_hi)
            recv_lo, recv_hi = host(recv_lo), host(recv_hi)
        ops = []
        if self.above is not None:
            ops.append(dist.P2POp(dist.isend, send_hi, self.above, tag=self.UP))
        if self.below is not None:
            ops.append(dist.P2POp(dist.isend, send_lo, self.below, tag=self.DOWN))
            ops.append(dist.P2POp(dist.irecv, recv_lo, self.below, tag=self.UP))
        if self.above is not None:
            ops.append(dist.P2POp(dist.irecv, recv_hi, self.above, tag=self.DOWN))
        if ops:
            for r in dist.batch_isend_irecv(ops):
                r.wait()
        if stage:
            if self.below is not None:
                dev_lo.copy_(recv_lo)
            if self.above is not None:
                dev_hi.copy_(recv_hi)

    def exchange(self, bottom_row, top_row):
        """Host rows: send this slab's edge rows ([72][nx + 2] FP64), receive
        the neighbours'; returns (row_lo, row_hi), each None at a
        non-periodic end of the domain."""
        import torch
        shape = (len(self.up), self.nx + 2)
        send_lo = torch.from_numpy(pack(bottom_row, self.down))
        send_hi = torch.from_numpy(pack(top_row, self.up))
        recv_lo = torch.empty(shape, dtype=torch.float64)
        recv_hi = torch.empty(shape, dtype=torch.float64)
        self.exchange_packed(send_lo, send_hi, recv_lo, recv_hi)
        row_lo = unpack(recv_lo.numpy(), self.up, self.nx) if self.below is not None else None
        row_hi = unpack(recv_hi.numpy(), self.down, self.nx) if self.above is not None else None
        return row_lo, row_hi


class DeviceSlab:
    """One y-slab on this process's GPU: domain `domain` of a Simulation
    (paper_1709_09073_gb300.rlbm) built with slab_bcs, its y neighbours
    reached through `exchange` (a SlabExchange over NCCL, or any object with
    the same below/above/exchange_packed). Every step packs the edge rows on
    the device, exchanges them, writes the received rows into the ghost rows
    and steps the Simulation once. The Simulation must run on the current
    torch stream, which orders the NCCL messages after the pack and the
    unpack after the messages."""

    def __init__(self, sim, domain, exchange):
        self.sim, self.domain, self.ex = sim, domain, exchange
        self.send_lo, self.send_hi = sim.edge_row_buffer(domain), sim.edge_row_buffer(domain)
        self.recv_lo, self.recv_hi = sim.edge_row_buffer(domain), sim.edge_row_buffer(domain)

    def pack(self):
        lo = self.send_lo if self.ex.below is not None else None
        hi = self.send_hi if self.ex.above is not None else None
        self.sim.pack_edge_rows(self.domain, lo, hi)

    def unpack(self):
        lo = self.recv_lo if self.ex.below is not None else None
        hi = self.recv_hi if self.ex.above is not None else None
        self.sim.unpack_ghost_rows(self.domain, lo, hi)

    def halo(self):
        """Bring the ghost rows up to date (after init and before each step)."""
        self.pack()
        self.ex.exchange_packed(self.send_lo, self.send_hi, self.recv_lo, self.recv_hi)
        self.unpack()

    def step(self, nsteps=1):
        for _ in range(nsteps):
            self.halo()
            self.sim.step(1)


def halo_bytes_per_face(nx, esize):
    """Bytes one slab sends across one face per step (30 planes of nx + 2 values)."""
    return len(planes_up()) * (nx + 2) * esize

