"""CPU oracle of local-peak selection over a candidate list -- TEST
INFRASTRUCTURE.

A linear mover makes a cluster of candidates: the neighbouring velocities and
bins of its best cell also reach the threshold (Sec. 2.1; the velocity
tolerance of Sec. 2.2 spans several lattice steps).  The paper removes such
duplicates by peeling the best cluster's detections (Sec. 2.1 step 3).  The
library's cheaper stand-in keeps only local peaks:

  candidate i is a peak when no other candidate j of the list, with
  |kx_j - kx_i| <= 1, |ky_j - ky_i| <= 1, |bx_j - bx_i| <= 1 and
  |by_j - by_i| <= 1, precedes it in the output order (j < i; the list is in
  the total order distinct desc, raw desc, v_idx, by, bx).

The first candidate is always a peak; no two peaks are neighbours.
Parity status: pinned against an all-pairs brute force in
tests/test_oracle_peaks.py.
"""
from __future__ import annotations

import numpy as np


def peaks(v_idx, bx, by, nvx: int) -> np.ndarray:
    """Ascending indices of the local peaks of a candidate list given in
    output order (v_idx, bx, by are parallel integer arrays)."""
    v_idx = np.asarray(v_idx, np.int64)
    bx = np.asarray(bx, np.int64)
    by = np.asarray(by, np.int64)
    where = {}
    for i in range(len(v_idx)):
        where[(int(v_idx[i]), int(bx[i]), int(by[i]))] = i
    out = []
    for i in range(len(v_idx)):
        kx, ky = int(v_idx[i]) % nvx, int(v_idx[i]) // nvx
        peak = True
        for dky in (-1, 0, 1):
            for dkx in (-1, 0, 1):
                kx2, ky2 = kx + dkx, ky + dky
                if kx2 < 0 or kx2 >= nvx or ky2 < 0:
                    continue
                v2 = ky2 * nvx + kx2
                for dby in (-1, 0, 1):
                    for dbx in (-1, 0, 1):
                        j = where.get((v2, int(bx[i]) + dbx, int(by[i]) + dby))
                        if j is not None and j < i:
                            peak = False
        if peak:
            out.append(i)
    return np.asarray(out, np.int64)
