"""Host-side bookkeeping of the vetter evaluation: id-based truth matching and
recall per magnitude bin, against straightforward loops."""
import numpy as np

import oracle
from paper_2509_26279_gb300 import vetting
from paper_2509_26279_gb300 import workloads as W


def test_truth_match_equals_loop():
    w = W.tiny()
    cat = W.load(w)
    r = oracle.stack(cat, w.grid, 4)
    c = np.zeros(len(r.cands), [("id_len", "<u4"), ("id_off", "<u8")])
    c["id_len"], c["id_off"] = r.cands["id_len"], r.cands["id_off"]
    got = vetting.truth_match(c, np.asarray(r.ids), cat.mover)
    for i in range(len(c)):
        ids = r.ids[c["id_off"][i]: c["id_off"][i] + c["id_len"][i]]
        m = cat.mover[ids]
        best, arg = 0, -1
        for k in set(m[m >= 0].tolist()):
            n = int((m == k).sum())
            if n > best:
                best, arg = n, k
        want = arg if 2 * best >= len(ids) and arg >= 0 else -1
        assert got[i] == want
    assert (got >= 0).any() and (got < 0).any()


def test_recall_bins():
    mv = np.zeros(5, W.MOVER_DTYPE)
    mv["mag"] = [23.1, 23.4, 24.9, 26.4, 26.5]
    r = vetting.recall_by_mag(np.array([1, 3]), mv)
    assert r["total"] == [2, 0, 0, 1, 0, 0, 2]
    assert r["found"] == [1, 0, 0, 0, 0, 0, 1]
    assert vetting.n_low(20) == 5 and vetting.n_low(100) == 8 and vetting.n_low(150) == 11
