"""CPU oracle of ownership selection over a candidate list -- TEST
INFRASTRUCTURE.

The paper deduplicates by peeling: take the best cluster, remove the
detections that contributed to it, and look again (Sec. 2.1 step 3).  The
library's one-pass stand-in gives each detection to the first candidate, in
output order, whose id list contains it (its owner), and keeps candidate i
when it owns at least half of its own detections:

  owner(d) = min{ i : d in ids(i) },  mine(i) = #{ d in ids(i) : owner(d) = i },
  kept(i)  <=>  2 * mine(i) >= |ids(i)|  or  (n_keep > 0 and mine(i) >= n_keep).

A mover's ghost cells (neighbouring velocities and bins that also collect its
detections) find those detections owned by its best cell and drop out.  The
second clause follows the peel: once the better clusters' detections are gone,
a candidate that still holds n_keep detections (the search's threshold) would
be found again -- a fainter mover crossing a brighter one keeps its cell.
Parity status: pinned against a set-based brute force in
tests/test_oracle_owned.py.
"""
from __future__ import annotations

import numpy as np


def owned(id_lists, n_keep: int = 0) -> np.ndarray:
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
        if 2 * mine >= len(ids) or (n_keep > 0 and mine >= n_keep):
            keep.append(i)
    return np.asarray(keep, np.int64)
