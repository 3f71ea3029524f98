"""Velocity-range sharding of one search across processes (one GPU each).

The histograms of different velocities are independent (Sec. 2.1: each trial
velocity is projected and counted on its own), so a search splits into
contiguous v_idx ranges with no exchange step.  Each rank searches its range
(sas_stack with v_begin/v_end); the candidate lists are gathered on the host and
merged by concatenation plus the same total order the library uses:
(distinct desc, raw desc, v_idx asc, by asc, bx asc).  The merged list is
byte-identical to a single search of the whole lattice, and a top-K cut after
the merge equals the single search's top-K when every shard keeps its own top-K.

This module is host logic only; the search itself is whatever `search_fn`
runs (on a GPU: the library's sas_stack).
"""
from __future__ import annotations

from typing import Callable, List, Sequence, Tuple

import numpy as np

CANDIDATE_DTYPE = np.dtype([("v_idx", "<u4"), ("bx", "<u4"), ("by", "<u4"), ("count", "<u4"),
                            ("raw", "<u4"), ("id_len", "<u4"), ("id_off", "<u8")])


def velocity_ranges(n_velocities: int, world: int) -> List[Tuple[int, int]]:
    """Contiguous, balanced [begin, end) ranges of v_idx, one per rank (empty
    ranges when there are more ranks than velocities)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    base, extra = divmod(n_velocities, world)
    out, b = [], 0
    for r in range(world):
        e = b + base + (1 if r < extra else 0)
        out.append((b, e))
        b = e
    return out


def merge(parts: Sequence[Tuple[np.ndarray, np.ndarray]], max_candidates: int = 0):
    """Merge per-shard (candidates, ids) into one list in the total order.

    candidates: structured arrays of CANDIDATE_DTYPE whose id_off index the
    shard's own ids array.  Returns (candidates, ids) with id_off rebuilt."""
    cands = [np.asarray(c, CANDIDATE_DTYPE) for c, _ in parts]
    ids = [np.asarray(i, np.uint32) for _, i in parts]
    if not cands:
        return np.zeros(0, CANDIDATE_DTYPE), np.zeros(0, np.uint32)
    allc = np.concatenate(cands)
    shard = np.concatenate([np.full(len(c), k, np.int64) for k, c in enumerate(cands)])
    # np.lexsort: last key is primary
    order = np.lexsort((allc["bx"], allc["by"], allc["v_idx"],
                        -allc["raw"].astype(np.int64), -allc["count"].astype(np.int64)))
    if max_candidates:
        order = order[:max_candidates]
    out = allc[order].copy()
    src = shard[order]
    lists = [ids[s][int(c["id_off"]):int(c["id_off"]) + int(c["id_len"])] for s, c in zip(src, allc[order])]
    lens = np.array([len(x) for x in lists], np.uint64)
    out["id_off"] = np.concatenate([[0], np.cumsum(lens)[:-1]]).astype(np.uint64) if len(lens) else lens
    out_ids = np.concatenate(lists).astype(np.uint32) if lists else np.zeros(0, np.uint32)
    return out, out_ids


def search_sharded(search_fn: Callable[[int, int], Tuple[np.ndarray, np.ndarray]], n_velocities: int,
                   max_candidates: int = 0, group=None):
    """Run `search_fn(v_begin, v_end) -> (candidates, ids)` on this rank's
    velocity range and merge all ranks' lists on rank 0 (torch.distributed,
    host objects; a gloo group works for any backend's ranks).  Returns the
    merged (candidates, ids) on rank 0 and None elsewhere."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    vb, ve = velocity_ranges(n_velocities, world)[rank]
    mine = search_fn(vb, ve) if ve > vb else (np.zeros(0, CANDIDATE_DTYPE), np.zeros(0, np.uint32))
    gathered = [None] * world if rank == 0 else None
    dist.gather_object(mine, gathered, dst=0, group=group)
    if rank != 0:
        return None
    return merge(gathered, max_candidates)
