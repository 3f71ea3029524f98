"""CPU oracle of the cluster-finding loop (Sec. 2.1 step 3) -- TEST
INFRASTRUCTURE.

The paper finds clusters in a loop: take the cell of the 3-D histogram
(velocity x bin) with the largest count; stop when it is below N_min;
otherwise the detections that contributed to it form a cluster, they are
removed from the histogram, and the loop continues (the paper outputs the first
1000 clusters).  Counts are distinct epochs (the reading taken throughout),
ties go by the search's total order (distinct desc, raw desc, v_idx, by, bx).

Two plain implementations, checked against each other in
tests/test_oracle_peel.py:

  literal(cat, grid, n_min, k) -- exactly the loop above: after every cluster the
      whole search runs again on the catalog without the removed detections.
  peel(cands, id_lists, epoch, n_min, k) -- the same loop over the search's
      candidate list: removing detections only lowers counts, so every later
      maximum is already a candidate; each round recounts the candidates from
      their remaining ids.

Both return [(v_idx, bx, by, distinct, raw, sorted ids)] in the order found.
Parity status: pinned (literal = peel on random and workload catalogs; hand-built
cases; disjointness, monotone counts and termination invariants).
"""
from __future__ import annotations

import dataclasses

import numpy as np

import oracle


def peel(cands, id_lists, epoch, n_min: int, max_clusters: int = 1000):
    """Cluster finding over a candidate list in output order (cands: records
    with v_idx, bx, by; id_lists[i]: ids of candidate i; epoch[id])."""
    removed = set()
    out = []
    n = len(id_lists)
    while len(out) < max_clusters:
        best, best_key, best_ids = None, None, None
        for i in range(n):
            ids = [int(d) for d in id_lists[i] if int(d) not in removed]
            distinct = len({int(epoch[d]) for d in ids})
            if distinct < n_min:
                continue
            c = cands[i]
            key = (-distinct, -len(ids), int(c["v_idx"]), int(c["by"]), int(c["bx"]))
            if best_key is None or key < best_key:
                best, best_key, best_ids = i, key, ids
        if best is None:
            break
        c = cands[best]
        out.append((int(c["v_idx"]), int(c["bx"]), int(c["by"]), -best_key[0], -best_key[1], sorted(best_ids)))
        removed.update(best_ids)
    return out


def literal(cat, grid, n_min: int, max_clusters: int = 1000):
    """The loop as stated: rerun the search after every removal.  A removed
    detection is moved far outside the domain (its epoch stays in the catalog,
    so the reference epoch t0 -- and with it every projection -- is unchanged,
    as removing points from the histogram leaves the projection alone); valid
    for catalogs whose shifts stay well below 2^28 mpx."""
    x = np.array(cat.x, np.int32)
    y = np.array(cat.y, np.int32)
    far = (1 << 29) - 1
    out = []
    while len(out) < max_clusters:
        sub = dataclasses.replace(cat, x=x, y=y)
        r = oracle.stack(sub, grid, n_min, 0, None, 1)
        if len(r.cands) == 0:
            break
        c = r.cands[0]
        ids = sorted(int(d) for d in r.ids[int(c["id_off"]): int(c["id_off"]) + int(c["id_len"])])
        out.append((int(c["v_idx"]), int(c["bx"]), int(c["by"]), int(c["distinct"]), int(c["raw"]), ids))
        x[ids] = far
        y[ids] = far
    return out
