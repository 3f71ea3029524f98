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


def test_noise_floor_is_the_poisson_tail_crossing():
    """The noise floor is the smallest k whose expected count of (lattice point,
    3 x 3 super-bin) pairs with >= k noise detections is below the budget:
    checked against scipy's Poisson survival function, and monotone in the
    detection count and the budget."""
    from scipy.stats import poisson
    g = W.batched_fields(1)[0].grid
    n_sb = -(-g.nbx // 3) * -(-g.nby // 3)
    pairs = n_sb * g.nvx * g.nvy
    for n in (1_000, 50_000, 300_000, 1_000_000):
        k = vetting.noise_floor(n, g, budget=5e4)
        lam = n / n_sb
        assert poisson.sf(k - 1, lam) * pairs <= 5e4 * (1 + 1e-9)
        if k > 1:
            assert poisson.sf(k - 2, lam) * pairs > 5e4
    ks = [vetting.noise_floor(n, g) for n in (1e4, 1e5, 1e6, 4e6)]
    assert ks == sorted(ks)
    assert vetting.noise_floor(300_000, g, budget=1e3) >= vetting.noise_floor(300_000, g, budget=1e6)


def test_lowered_threshold_between_floor_and_n_min():
    g = W.batched_fields(1)[0].grid
    for E, n_min, n in ((100, 25, 400_000), (24, 6, 90_000), (150, 38, 1_200_000), (20, 5, 20_000)):
        lo = vetting.lowered_threshold(E, n_min, n, g, 6)
        assert lo <= n_min
        assert lo == n_min or lo >= -(-E // 6)
        assert lo == n_min or lo >= vetting.noise_floor(n, g)
    # a long, sparse field gets its full lowering; a short dense one none
    assert vetting.lowered_threshold(100, 25, 400_000, g, 6) == 17
    assert vetting.lowered_threshold(24, 6, 90_000, g, 6) == 6
