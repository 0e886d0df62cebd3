"""Run-range sharding of one search over several processes (one per GPU).

Runs of Algorithm 2 are independent and the row stream is counter-based, so
rank r can search runs [l_r, l_{r+1}) on its own device with
``Context.search_range`` and the ranks' pair lists are merged on the host:
the union of disjoint run ranges covering [0, L) is the whole search.  No
collective touches the data path; the merge gathers the (small) pair lists
once.
"""
from __future__ import annotations

import numpy as np

PAIR_FIELDS = ("j", "k", "agree")


def run_ranges(L: int, world: int):
    """Split runs [0, L) into ``world`` contiguous, disjoint, near-equal ranges."""
    if L < 0 or world < 1:
        raise ValueError("need L >= 0 and world >= 1")
    base, extra = divmod(L, world)
    out, l0 = [], 0
    for r in range(world):
        l1 = l0 + base + (1 if r < extra else 0)
        out.append((l0, l1))
        l0 = l1
    return out


def _as_triples(part) -> np.ndarray:
    if part is None or len(part) == 0:
        return np.zeros((0, 3), dtype=np.int64)
    if part.dtype.names:
        return np.stack([part[f].astype(np.int64) for f in PAIR_FIELDS], axis=1)
    return np.asarray(part, dtype=np.int64).reshape(-1, 3)


def merge_pairs(parts) -> np.ndarray:
    """Union of per-rank results as (j, k, agree) rows sorted by (j, k).

    A pair found by several ranks has the same agreement count everywhere
    (it is a property of the data, eq. def_gamma); the merge keeps one row
    and checks that they agree."""
    rows = np.concatenate([_as_triples(p) for p in parts]) if parts else np.zeros((0, 3), np.int64)
    if len(rows) == 0:
        return rows
    order = np.lexsort((rows[:, 1], rows[:, 0]))
    rows = rows[order]
    first = np.ones(len(rows), dtype=bool)
    first[1:] = (rows[1:, 0] != rows[:-1, 0]) | (rows[1:, 1] != rows[:-1, 1])
    grp = np.cumsum(first) - 1
    uniq = rows[first]
    if not np.array_equal(uniq[grp, 2], rows[:, 2]):
        raise ValueError("ranks disagree on the agreement count of a pair")
    return uniq


def search_sharded(search_range, L: int, rank: int, world: int, gather=None) -> np.ndarray:
    """Search runs [0, L) split over ``world`` ranks.

    ``search_range(l0, l1)`` returns this rank's pairs (a structured array
    with fields j, k, agree, or (j, k, agree) rows); ``gather(obj)`` returns
    the list of every rank's ``obj`` (``torch.distributed.all_gather_object``
    by default).  Every rank returns the merged result."""
    l0, l1 = run_ranges(L, world)[rank]
    mine = _as_triples(search_range(l0, l1) if l1 > l0 else None)
    if gather is None:
        import torch.distributed as dist
        objs = [None] * world
        dist.all_gather_object(objs, mine)
    else:
        objs = gather(mine)
    return merge_pairs(objs)
