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
host, NCCL between GPUs); the batched benchmark shards whole domains instead
and needs none of this.
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
    """(rank below, rank above); None at a non-periodic end of the domain."""
    below = rank - 1 if rank > 0 else (nranks - 1 if periodic_y else None)
    above = rank + 1 if rank < nranks - 1 else (0 if periodic_y else None)
    return below, above


def slab_bcs(bc, rank, nranks):
    """Boundary conditions of a slab: x sides as the domain's; a y side that
    borders another slab gets zero-gradient, a placeholder never read because
    that row is supplied by the neighbour."""
    xlo, xhi, ylo, yhi = bc
    periodic_y = ylo == 0
    ZG = 1
    lo = ZG if (periodic_y or rank > 0) else ylo
    hi = ZG if (periodic_y or rank < nranks - 1) else yhi
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

    def exchange(self, bottom_row, top_row):
        """Send this slab's edge rows, receive the neighbours'; returns
        (row_lo, row_hi), each None at a non-periodic end of the domain."""
        import torch
        import torch.distributed as dist
        reqs, recv_lo, recv_hi = [], None, None
        shape = (len(self.up), self.nx + 2)
        if self.above is not None:
            reqs.append(dist.isend(torch.from_numpy(pack(top_row, self.up)), self.above, tag=self.UP))
            recv_hi = torch.empty(shape, dtype=torch.float64)
            reqs.append(dist.irecv(recv_hi, self.above, tag=self.DOWN))
        if self.below is not None:
            reqs.append(dist.isend(torch.from_numpy(pack(bottom_row, self.down)), self.below, tag=self.DOWN))
            recv_lo = torch.empty(shape, dtype=torch.float64)
            reqs.append(dist.irecv(recv_lo, self.below, tag=self.UP))
        for r in reqs:
            r.wait()
        row_lo = unpack(recv_lo.numpy(), self.up, self.nx) if recv_lo is not None else None
        row_hi = unpack(recv_hi.numpy(), self.down, self.nx) if recv_hi is not None else None
        return row_lo, row_hi


def halo_bytes_per_face(nx, esize):
    """Bytes one slab sends across one face per step (30 planes of nx + 2 values)."""
    return len(planes_up()) * (nx + 2) * esize

