"""Pins of the ownership oracle: a set-based brute force written from the
definition (each candidate checks every earlier candidate), hand-built cases,
and the fact that it removes a mover's ghost cells but keeps its best one."""
import numpy as np
import pytest

import oracle
from oracle import owned as O
from paper_2509_26279_gb300 import workloads as W


def brute(id_lists, n_keep=0):
    keep = []
    for i, ids in enumerate(id_lists):
        earlier = set()
        for j in range(i):
            earlier |= set(int(d) for d in id_lists[j])
        mine = [d for d in ids if int(d) not in earlier]
        if 2 * len(mine) >= len(ids) or (n_keep > 0 and len(mine) >= n_keep):
            keep.append(i)
    return np.asarray(keep, np.int64)


@pytest.mark.parametrize("seed", range(30))
def test_owned_equals_brute_force(seed):
    rng = np.random.default_rng(seed)
    m = int(rng.integers(0, 40))
    lists = [np.unique(rng.integers(0, 50, int(rng.integers(1, 12)))) for _ in range(m)]
    n_keep = int(rng.integers(0, 6))
    assert np.array_equal(O.owned(lists, n_keep), brute(lists, n_keep))


def test_hand_built():
    lists = [[1, 2, 3, 4], [3, 4, 5], [5, 6], [1, 2, 9, 10], [7]]
    # 0 owns all; 1 owns only 5 (1 of 3) -> dropped; 2 owns 6 (5 belongs to 1) -> 1 of 2 kept;
    # 3 owns 9, 10 (2 of 4) -> kept; 4 owns 7 -> kept
    assert O.owned(lists).tolist() == [0, 2, 3, 4]


def test_crossing_mover_keeps_its_cell():
    """Two candidates sharing detections: the later one owns only 4 of its 10,
    so the half rule drops it, but with n_keep = 4 (what it alone still holds
    passes the threshold) it stays -- as the peel would find it again."""
    a = list(range(0, 12))
    b = list(range(6, 12)) + [100, 101, 102, 103]
    assert O.owned([a, b]).tolist() == [0]
    assert O.owned([a, b], n_keep=4).tolist() == [0, 1]
    assert O.owned([a, b], n_keep=5).tolist() == [0]


def test_one_clean_mover_keeps_one_cell():
    """A noiseless linear mover at a lattice velocity: its exact cell (count E)
    comes first and owns every detection; every ghost cell is dropped."""
    w = W.tiny()
    rec = W.FieldRecipe(512, 512, 20, 4.0, 0, 1, (3.0, 3.0), (1.0, 1.0), jitter_px=0.0)
    cat = W.make_catalog(rec, 5)
    r = oracle.stack(cat, w.grid, 3)
    lists = r.id_lists()
    kept = O.owned(lists)
    assert len(r.cands) > 1 and kept.tolist() == [0]
    assert O.owned(lists, n_keep=3).tolist() == [0]   # ghosts hold none of their own
