"""Pins of the ownership oracle: a set-based brute force written from the
definition (each candidate checks every earlier candidate), hand-built cases,
and the fact that it removes a mover's ghost cells but keeps its best one."""
import numpy as np
import pytest

import oracle
from oracle import owned as O
from paper_2509_26279_gb300 import workloads as W


def brute(id_lists):
    keep = []
    for i, ids in enumerate(id_lists):
        earlier = set()
        for j in range(i):
            earlier |= set(int(d) for d in id_lists[j])
        mine = [d for d in ids if int(d) not in earlier]
        if 2 * len(mine) >= len(ids):
            keep.append(i)
    return np.asarray(keep, np.int64)


@pytest.mark.parametrize("seed", range(30))
def test_owned_equals_brute_force(seed):
    rng = np.random.default_rng(seed)
    m = int(rng.integers(0, 40))
    lists = [np.unique(rng.integers(0, 50, int(rng.integers(1, 12)))) for _ in range(m)]
    assert np.array_equal(O.owned(lists), brute(lists))


def test_hand_built():
    lists = [[1, 2, 3, 4], [3, 4, 5], [5, 6], [1, 2, 9, 10], [7]]
    # 0 owns all; 1 owns only 5 (1 of 3) -> dropped; 2 owns 6 (5 belongs to 1) -> 1 of 2 kept;
    # 3 owns 9, 10 (2 of 4) -> kept; 4 owns 7 -> kept
    assert O.owned(lists).tolist() == [0, 2, 3, 4]


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
