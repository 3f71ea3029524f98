"""Pins of the local-peak oracle: an all-pairs brute force over random lists
(written from the definition, with no neighbour table), structural facts, and
a hand-built cluster."""
import numpy as np
import pytest

import oracle
from oracle import peaks as P
from paper_2509_26279_gb300 import workloads as W


def brute(v, bx, by, nvx):
    kx, ky = np.asarray(v) % nvx, np.asarray(v) // nvx
    out = []
    for i in range(len(v)):
        near = ((np.abs(kx - kx[i]) <= 1) & (np.abs(ky - ky[i]) <= 1) &
                (np.abs(np.asarray(bx) - bx[i]) <= 1) & (np.abs(np.asarray(by) - by[i]) <= 1))
        near[i] = False
        if not near[:i].any():
            out.append(i)
    return np.asarray(out, np.int64)


@pytest.mark.parametrize("seed", range(30))
def test_peaks_equal_all_pairs_brute_force(seed):
    rng = np.random.default_rng(seed)
    nvx = int(rng.integers(1, 6))
    nvy = int(rng.integers(1, 6))
    m = min(int(rng.integers(0, 60)), nvx * nvy * 36)   # at most every cell once
    cells = set()
    while len(cells) < m:
        cells.add((int(rng.integers(0, nvx * nvy)), int(rng.integers(0, 6)), int(rng.integers(0, 6))))
    cells = list(cells)
    rng.shuffle(cells)                    # any order is some output order
    v = np.array([c[0] for c in cells], np.int64)
    bx = np.array([c[1] for c in cells], np.int64)
    by = np.array([c[2] for c in cells], np.int64)
    assert np.array_equal(P.peaks(v, bx, by, nvx), brute(v, bx, by, nvx))


def test_hand_built_cluster():
    # a 3x3 block of cells at one velocity plus a far cell; kx wraps must not
    # connect v_idx 2 (kx 2) with v_idx 3 (kx 0 of the next row) when nvx = 3
    cells = [(4, 5, 5), (4, 4, 5), (4, 6, 6), (1, 5, 4), (4, 9, 9), (2, 0, 0), (3, 0, 0)]
    v, bx, by = (np.array(c) for c in zip(*cells))
    got = P.peaks(v, bx, by, 3).tolist()
    # 0 is first; 1, 2 touch 0; 3 (v 1 = kx 1, ky 0) touches v 4 (kx 1, ky 1) at (5, 4);
    # 4 is far; 5 (kx 2, ky 0) and 6 (kx 0, ky 1) are not lattice neighbours
    assert got == [0, 4, 5, 6]


def test_peaks_of_a_search_are_separated_and_cover():
    w = W.tiny()
    cat = W.load(w)
    r = oracle.stack(cat, w.grid, 4)
    c = r.cands
    pk = P.peaks(c["v_idx"], c["bx"], c["by"], w.grid.nvx)
    assert pk[0] == 0 and 0 < len(pk) < len(c)
    nvx = w.grid.nvx
    kx, ky = c["v_idx"].astype(np.int64) % nvx, c["v_idx"].astype(np.int64) // nvx
    bx, by = c["bx"].astype(np.int64), c["by"].astype(np.int64)
    is_pk = np.zeros(len(c), bool)
    is_pk[pk] = True
    for i in range(len(c)):
        near = (np.abs(kx - kx[i]) <= 1) & (np.abs(ky - ky[i]) <= 1) & (np.abs(bx - bx[i]) <= 1) & (np.abs(by - by[i]) <= 1)
        near[i] = False
        if is_pk[i]:
            assert not (near & is_pk).any()          # no two peaks are neighbours
        else:
            assert near[:i].any()                    # every other cell has a better neighbour
