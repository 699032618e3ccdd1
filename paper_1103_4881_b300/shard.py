"""Partition of independent work units over ranks (host-side only).

Frames, and serving requests, are independent repetitions of the filter
(Sec. 3.B: the frame is the outermost repetition of the downscaler), so the
path shards with no exchange: every rank takes its own units, reads them from
its own memory and writes its own outputs.  Both partitions below are pure
functions of (units, world, rank), so every rank computes the same split
without talking to the others.
"""
from __future__ import annotations


def frame_range(n_total: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous frame range [start, stop) of `rank`; sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world or n_total < 0:
        raise ValueError("bad world/rank/n_total")
    base, extra = divmod(n_total, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def balance_by_bytes(sizes, world: int) -> list[int]:
    """Owner rank of each unit: units in order, each to the rank with the fewest
    bytes so far (lowest rank on ties).  The final loads differ by at most the
    largest unit."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0] * world
    owner = []
    for s in sizes:
        r = min(range(world), key=lambda k: (load[k], k))
        owner.append(r)
        load[r] += int(s)
    return owner


def shard_requests(requests, world: int, rank: int, nbytes) -> list:
    """The requests `rank` serves: byte-balanced assignment in arrival order,
    nbytes(request) giving each request's input + output bytes."""
    if not 0 <= rank < world:
        raise ValueError("bad world/rank")
    owner = balance_by_bytes([nbytes(r) for r in requests], world)
    return [r for r, o in zip(requests, owner) if o == rank]
