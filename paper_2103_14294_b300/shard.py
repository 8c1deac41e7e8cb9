"""Root sharding for runs over several GPUs (one process per GPU).

Root vertices are independent units of the enumeration (every match is found from exactly one
root, the data vertex bound at position 0 of the matching order), so a job splits into disjoint
root ranges with no exchange on the data path; the per-rank counts add up to the whole count.
Ranges are contiguous in the relabelled ids and balanced by the weight 1 + degree, the same
weight the library uses to cut root chunks for its warps.
"""
from __future__ import annotations

import numpy as np


def shard_bounds(offsets: np.ndarray, world: int) -> list[tuple[int, int]]:
    """`world` contiguous root ranges [r0, r1) covering 0..n-1, each with about the same total
    weight 1 + degree(r). `offsets` is the CSR offset array (n + 1 entries) of the graph whose
    ids the ranges refer to."""
    if world < 1:
        raise ValueError("world must be >= 1")
    off = np.asarray(offsets, dtype=np.int64)
    n = len(off) - 1
    w = np.cumsum(1 + np.diff(off))
    total = int(w[-1]) if n else 0
    cuts = [0]
    for i in range(1, world):
        cuts.append(int(np.searchsorted(w, total * i / world, side="left")) if n else 0)
    cuts.append(n)
    cuts = np.maximum.accumulate(np.minimum(np.asarray(cuts), n))
    return [(int(cuts[i]), int(cuts[i + 1])) for i in range(world)]


def shard_of(offsets: np.ndarray, rank: int, world: int) -> tuple[int, int]:
    """The root range of `rank`."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return shard_bounds(offsets, world)[rank]


def relabelled_offsets(graph) -> np.ndarray:
    """CSR offsets of `graph` after the library's relabelling by (degree, id) ascending: the
    degree sequence in new ids is the sorted degree sequence, so root ranges computed on these
    offsets refer to the ids the library enumerates in."""
    deg = np.sort(np.diff(np.asarray(graph.offsets, dtype=np.int64)), kind="stable")
    return np.concatenate([[0], np.cumsum(deg)]).astype(np.int64)
