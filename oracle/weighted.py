"""CPU oracle of likelihood-weighted stacking -- TEST INFRASTRUCTURE.

The paper's discussion proposes accumulating each detection's likelihood instead
of the 0/1 indicator of "detected in this epoch" (Sec. 5, future work).  The
weighted score of a cell (velocity, bin) generalises the distinct-epoch count:

    score = sum over epochs e of  max { w_i : detection i of epoch e in the cell }

with integer weights w_i in [0, 255] (a fixed-point likelihood or S/N); every
w_i = 1 gives the distinct-epoch count.  Candidates are the cells with
score >= s_min, in the order (score desc, raw desc, v_idx, by, bx).

A cell with score >= s_min holds at least ceil(s_min / w_max) distinct epochs,
so the pinned stack oracle's candidate list at that threshold contains every
such cell with its ids; the score is then taken from the ids.

Parity status: pinned (tests/test_oracle_weighted.py: unit weights reduce to
the stack oracle, a pure-Python brute force with its own running maxima,
hand-built cells, monotonicity in the weights).
"""
from __future__ import annotations

import math

import numpy as np

import oracle


def score(ids, epoch, w):
    best = {}
    for i in ids:
        e = int(epoch[i])
        best[e] = max(best.get(e, 0), int(w[i]))
    return sum(best.values())


def stack(cat, grid, w, s_min: int):
    """[(v_idx, bx, by, score, raw, ids)] in output order."""
    w = np.asarray(w)
    if s_min < 1:
        raise ValueError("s_min >= 1")
    if len(w) == 0 or int(w.max()) == 0:
        return []
    n1 = max(1, math.ceil(s_min / int(w.max())))
    r = oracle.stack(cat, grid, n1)
    out = []
    for c, ids in zip(r.cands, r.id_lists()):
        s = score(ids, cat.epoch, w)
        if s >= s_min:
            out.append((int(c["v_idx"]), int(c["bx"]), int(c["by"]), s, int(c["raw"]), [int(i) for i in ids]))
    out.sort(key=lambda c: (-c[3], -c[4], c[0], c[2], c[1]))
    return out
