"""Split one batch of independent domains across GPUs by cell count.

The domains of a batch (the Taylor-Green and Fourier-flow sweeps over tau of
Secs. 3.2 and 3.3) are independent problems: a rank that owns whole domains
needs no data from any other rank, so the split has no data-path collective.
The cost of a step is proportional to the cells a rank updates, so the domains
are dealt out by the longest-processing-time rule: largest domain first, each
to the rank with the fewest cells so far (ties to the lowest rank). The
heaviest rank then exceeds the mean by less than the largest single domain.
"""


def split_by_cells(cells, nranks):
    """Indices of the domains each of `nranks` ranks owns, from the per-domain
    cell counts `cells`; every rank's list is in the batch's own order."""
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    load = [0] * nranks
    owned = [[] for _ in range(nranks)]
    for i in sorted(range(len(cells)), key=lambda k: (-cells[k], k)):
        r = min(range(nranks), key=lambda k: (load[k], k))
        owned[r].append(i)
        load[r] += cells[i]
    return [sorted(o) for o in owned]


def shard(workload, rank, nranks):
    """The part of a workloads.Workload that `rank` of `nranks` advances, with
    the batch's own name and the indices of its domains in `meta`."""
    from . import workloads as W
    cells = [d.nx * d.ny for d in workload.domains]
    mine = split_by_cells(cells, nranks)[rank]
    meta = dict(workload.meta)
    meta.update({"shard_of": workload.name, "rank": rank, "nranks": nranks, "domains": mine})
    return W.Workload(workload.name, [workload.domains[i] for i in mine], [workload.init[i] for i in mine],
                      workload.steps, meta)
