"""CPU oracle of ownership selection over a candidate list -- TEST
INFRASTRUCTURE.

The paper deduplicates by peeling: take the best cluster, remove the
detections that contributed to it, and look again (Sec. 2.1 step 3).  The
library's one-pass stand-in gives each detection to the first candidate, in
output order, whose id list contains it (its owner), and keeps candidate i
when it owns at least half of its own detections:

  owner(d) = min{ i : d in ids(i) },
  kept(i)  <=>  2 * #{ d in ids(i) : owner(d) = i } >= |ids(i)|.

A mover's ghost cells (neighbouring velocities and bins that also collect its
detections) find those detections owned by its best cell and drop out.
Parity status: pinned against a set-based brute force in
tests/test_oracle_owned.py.
"""
from __future__ import annotations

import numpy as np


def owned(id_lists) -> np.ndarray:
    """Ascending indices of the kept candidates; id_lists[i] are the ids of
    candidate i, candidates in output order."""
    owner = {}
    for i, ids in enumerate(id_lists):
        for d in ids:
            d = int(d)
            if d not in owner:
                owner[d] = i
    keep = []
    for i, ids in enumerate(id_lists):
        mine = sum(1 for d in ids if owner[int(d)] == i)
        if 2 * mine >= len(ids):
            keep.append(i)
    return np.asarray(keep, np.int64)
