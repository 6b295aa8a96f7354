"""Placement of independent images on GPUs (one process per GPU). The images of a batch share
nothing (each is its own problem (7), Sec. 4), so a multi-GPU run needs no collective on the
data path: every rank solves its own images.

Images are placed by the longest-processing-time rule on their algorithmic bytes per
iteration, B = 4 n K (4L + 11) (every array of one SALSA iteration read or written once in
FP32): the largest image first, each to the rank with the least work so far (ties to the lowest
rank). The resulting spread between the busiest and the idlest rank is at most the cost of one
image. Pure host logic: no GPU, no library."""
from __future__ import annotations


def iteration_bytes(H: int, W: int, K: int, M: int, elem_bytes: int = 4) -> int:
    """Algorithmic bytes of one SALSA iteration of an H x W image with K classes and a
    (2M+1) x (2M+1) patch: d2 (L K pairs) read and written, d1, d3, d4 read and written, p and
    z read, rhs written, and the z-update's rhs read and z write."""
    L = (2 * M + 1) ** 2
    return elem_bytes * H * W * K * (4 * L + 11)


def partition(costs, world: int):
    """Indices of the items each of `world` ranks takes, by longest processing time first.
    Returns a list of `world` sorted index lists; every index appears exactly once."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]
