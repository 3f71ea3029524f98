"""Cluster finding (Sec. 2.1 step 3) through the C ABI against the oracle's
candidate-list peel (itself pinned to the literal loop): the same clusters,
counts and ids, in the same order, from both the rounds-of-local-maxima form
and the one-cluster-at-a-time block."""
import numpy as np
import pytest

import oracle
from oracle import peel as PL
from paper_2509_26279_gb300 import workloads as W
from tests import cases

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2509_26279_gb300 import sas  # noqa: E402


def gpu_clusters(res):
    c, ids = res.candidates()
    return [(int(r["v_idx"]), int(r["bx"]), int(r["by"]), int(r["count"]), int(r["raw"]),
             ids[int(r["id_off"]): int(r["id_off"]) + int(r["id_len"])].tolist()) for r in c]


def check(cat, grid, n_min, k=1000, peel_min=None, ks=()):
    """Both forms against the oracle at cut k, then at each extra cut in ks."""
    peel_min = n_min if peel_min is None else peel_min
    res = sas.stack_catalog(sas.Grid(grid), cat, n_min)
    ref = oracle.stack(cat, grid, n_min)
    full = PL.peel(ref.cands, ref.id_lists(), cat.epoch, peel_min, max(k, *ks) if ks else k)
    for cut in (k, *ks):
        want = full[:cut]
        for seq in (False, True):
            got = gpu_clusters(sas.sas_peel(res, peel_min, cut, sequential=seq))
            assert got == want, (cut, seq)
    return full[:k]


@pytest.mark.parametrize("seed", range(30))
def test_peel_random_tiny(seed):
    cat, grid, n_min = cases.random_tiny(seed + 2500)
    check(cat, grid, n_min, ks=(1, 2, 3))


def test_peel_workloads_and_cap():
    w = W.tiny()
    cat = W.load(w)
    assert len(check(cat, w.grid, 4, ks=(1, 2, 5))) > 3
    check(cat, w.grid, 4, peel_min=7)
    ws = W.scaled(W.decam_tno(), frac_noise=0.2, width_px=800, height_px=800, n_movers=60, grid_half=15)
    cl = check(W.load(ws), ws.grid, 12, ks=(1, 7, 20))
    assert len(cl) > 10


def test_peel_full_tno_field_is_one_cluster_per_source():
    """Full-size TNO field: clusters are disjoint, in non-increasing order, and
    each holds mostly one mover's detections (the duplicates of the threshold
    list are gone)."""
    w = W.decam_tno()
    cat = W.load(w)
    res = sas.stack_catalog(sas.Grid(w.grid), cat, w.n_min)
    n_cand = res.info()["n_candidates"]
    cl = gpu_clusters(sas.sas_peel(res, w.n_min))
    assert cl == gpu_clusters(sas.sas_peel(res, w.n_min, sequential=True))
    assert cl[:50] == gpu_clusters(sas.sas_peel(res, w.n_min, 50))
    assert 0 < len(cl) < n_cand / 5
    seen = set()
    for a, b in zip(cl, cl[1:]):
        assert (a[3], a[4]) >= (b[3], b[4])
    for c in cl:
        assert c[3] >= w.n_min and not (set(c[5]) & seen)
        seen |= set(c[5])
    movers = [np.bincount(cat.mover[np.array(c[5])] + 2).argmax() - 2 for c in cl]
    assert sum(m >= 0 for m in movers) >= 0.95 * len(cl)


def test_peel_errors():
    w = W.tiny()
    cat = W.load(w)
    g = sas.Grid(w.grid)
    res = sas.stack_catalog(g, cat, 6)
    with pytest.raises(sas.SasError):
        sas.sas_peel(res, 5)                                  # below the search's threshold
    top = sas.stack_catalog(g, cat, 6, opts=sas.make_opts(max_candidates=3))
    with pytest.raises(sas.SasError):
        sas.sas_peel(top, 6)                                  # a top-K list is incomplete
    pl = sas.sas_peel(res, 6)
    with pytest.raises(sas.SasError):
        sas.sas_peel(pl, 6)                                   # a cluster list has no histogram
    with pytest.raises(sas.SasError):
        sas._check(sas._lib.sas_peel(res._h, 6, 10, 2, None, sas.ctypes.byref(sas._p())))  # unknown flag
    empty = sas.stack_catalog(g, cases.catalog([], [], [], cat.t), 6)
    for seq in (False, True):
        assert sas.sas_peel(empty, 6, sequential=seq).info()["n_candidates"] == 0
        assert sas.sas_peel(res, 1000, sequential=seq).info()["n_candidates"] == 0   # nothing reaches it
