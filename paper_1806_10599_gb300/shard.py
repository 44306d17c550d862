"""Independent RVEs spread over the ranks of a job (one GPU per rank).

A batch of RVEs (gff_batch_run) has no coupling between RVEs: each rank runs
its share as a batch of its own and only the per-RVE results travel, once, to
rank 0 at the end -- no collective on the data path.  The share is a greedy
longest-processing-time assignment on the cost of one Galerkin-operator apply,
n log2 n for n voxels (the transforms' work; the per-voxel constitutive work
adds a term linear in n of the same order, so the ranking is the same).
"""

import math


def rve_cost(shape):
    """Cost model of one RVE: n log2 n, n the voxel count (shape: int edge or (nz, ny, nx))."""
    if isinstance(shape, int):
        n = shape ** 3
    else:
        n = 1
        for s in shape:
            n *= int(s)
    return n * math.log2(max(n, 2))


def assign(shapes, world):
    """RVE indices per rank: the costliest RVE first, each to the rank with the
    least cost so far (ties to the lowest rank); deterministic, so every rank
    computes the same assignment without communicating."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(shapes)), key=lambda i: (-rve_cost(shapes[i]), i))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += rve_cost(shapes[i])
    for p in parts:
        p.sort()
    return parts


def gather_to_rank0(obj, world):
    """Every rank's `obj` on rank 0 (a list in rank order), None elsewhere; [obj] alone for one rank.
    Uses the initialised torch.distributed process group."""
    if world == 1:
        return [obj]
    import torch.distributed as dist

    out = [None] * world if dist.get_rank() == 0 else None
    dist.gather_object(obj, out, dst=0)
    return out


def merge(per_rank, parts, n):
    """Per-RVE results in global order from per-rank lists (per_rank[r][j] belongs to RVE parts[r][j])."""
    res = [None] * n
    for r, items in enumerate(per_rank):
        if len(items) != len(parts[r]):
            raise ValueError("rank %d returned %d results for %d RVEs" % (r, len(items), len(parts[r])))
        for i, v in zip(parts[r], items):
            res[i] = v
    return res
