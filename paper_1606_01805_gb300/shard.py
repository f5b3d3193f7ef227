"""Split of a batch of independent lattices over ranks (one GPU each).

The instances of a screening batch share nothing during a step (each has
its own populations, particles and walls, §2 applied per lattice), so N
ranks take disjoint subsets with no exchange on the data path; the only
collective is the timing's.  The split balances cell updates, the work of
the fluid kernel that dominates a step: instances in decreasing cell count
(ties by index) go one by one to the rank with the fewest cells so far
(ties to the lowest rank).  Every rank computes the same split from the
same list, so no rank needs to hear of another's choice.
"""


def shard_instances(cells, world):
    """Indices of the instances each of `world` ranks takes, given the cell
    count of every instance: a list of `world` sorted index lists, disjoint,
    together every index once."""
    if world < 1:
        raise ValueError("world must be at least 1")
    load = [0] * world
    out = [[] for _ in range(world)]
    for k in sorted(range(len(cells)), key=lambda k: (-int(cells[k]), k)):
        r = min(range(world), key=lambda r: (load[r], r))
        out[r].append(k)
        load[r] += int(cells[k])
    return [sorted(o) for o in out]


def rank_instances(cells, rank, world):
    """This rank's share of `shard_instances(cells, world)`."""
    if not 0 <= rank < world:
        raise ValueError("rank must lie in [0, world)")
    return shard_instances(cells, world)[rank]
