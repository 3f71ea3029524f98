"""Pins of the cluster-finding oracle (Sec. 2.1 step 3): the candidate-list
form equals the literal loop that reruns the whole search after each removal,
on random tiny catalogs and the tiny workload; hand-built cases; invariants."""
import numpy as np
import pytest

import oracle
from oracle import peel as PL
from paper_2509_26279_gb300 import workloads as W
from tests import cases


def list_form(cat, grid, n_min, k=1000):
    r = oracle.stack(cat, grid, n_min)
    return PL.peel(r.cands, r.id_lists(), cat.epoch, n_min, k), r


@pytest.mark.parametrize("seed", range(20))
def test_candidate_list_form_equals_literal_loop(seed):
    cat, grid, n_min = cases.random_tiny(seed + 2100, max_n=120, max_side=5)
    got, _ = list_form(cat, grid, n_min)
    assert got == PL.literal(cat, grid, n_min)


def test_tiny_workload_and_cap():
    w = W.tiny()
    cat = W.load(w)
    got, r = list_form(cat, w.grid, 6)
    lit = PL.literal(cat, w.grid, 6)
    assert got == lit and len(got) >= 3
    assert list_form(cat, w.grid, 6, 2)[0] == lit[:2]
    # invariants: disjoint clusters, non-increasing counts, every cluster at threshold,
    # and nothing left at the threshold once the loop stops
    seen = set()
    for a, b in zip(got, got[1:]):
        assert (a[3], a[4]) >= (b[3], b[4])
    for c in got:
        assert c[3] >= 6 and not (set(c[5]) & seen)
        seen |= set(c[5])
    for ids in r.id_lists():
        rest = [d for d in ids if int(d) not in seen]
        assert len({int(cat.epoch[d]) for d in rest}) < 6


def test_one_mover_one_cluster():
    """A noiseless mover on the lattice: one cluster holding all its detections
    (its ghosts lose them), count = E at its exact cell."""
    w = W.tiny()
    rec = W.FieldRecipe(512, 512, 20, 4.0, 0, 1, (3.0, 3.0), (1.0, 1.0), jitter_px=0.0)
    cat = W.make_catalog(rec, 5)
    got, r = list_form(cat, w.grid, 3)
    assert len(r.cands) > 1 and len(got) == 1
    assert got[0][3] == len(set(cat.epoch.tolist())) and got[0][5] == sorted(range(cat.n))


def test_hand_built_shared_detections():
    """Two candidates sharing detections: the second keeps what is left if that
    still reaches the threshold, else it is gone."""
    epoch = np.array([0, 1, 2, 3, 4, 5, 6, 7])
    cands = np.zeros(2, [("v_idx", "<u4"), ("bx", "<u4"), ("by", "<u4")])
    cands["v_idx"] = [5, 6]
    lists = [[0, 1, 2, 3, 4], [3, 4, 5, 6, 7]]
    assert PL.peel(cands, lists, epoch, 3) == [(5, 0, 0, 5, 5, [0, 1, 2, 3, 4]), (6, 0, 0, 3, 3, [5, 6, 7])]
    assert PL.peel(cands, lists, epoch, 4) == [(5, 0, 0, 5, 5, [0, 1, 2, 3, 4])]
