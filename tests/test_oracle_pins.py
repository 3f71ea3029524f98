"""Pins for the CPU oracle (oracle/sas_oracle.c): it must agree with things fixed
independently of it -- hand-computed cases, a separately written brute force,
invariants of the definition and the noise statistics of Sec. 2.2."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import brute
from paper_2509_26279_gb300 import workloads as W
from tests import cases

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_built.json")


def load_golden():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


def golden_inputs(case):
    cat = cases.catalog(case["x"], case["y"], case["epoch"], case["t"], case["tph"])
    g = dict(case["grid"])
    g.setdefault("speed_min", 0)
    g.setdefault("speed_max", 0)
    return cat, W.GridSpec(**g), case["n_min"]


def oracle_tuples(res):
    return cases.as_tuples(res.cands, res.id_lists())


@pytest.mark.parametrize("case", load_golden(), ids=lambda c: c["name"])
def test_golden_hand_built(case):
    cat, grid, n_min = golden_inputs(case)
    got = oracle_tuples(oracle.stack(cat, grid, n_min))
    want = [tuple(c[:5]) + (list(c[5]),) for c in case["expected"]]
    assert got == want
    bf, _ = brute.search(cat.x, cat.y, cat.epoch, cat.t, cat.ticks_per_hour, grid, n_min)
    assert [tuple(c[:5]) + (list(c[5]),) for c in bf] == want


@pytest.mark.parametrize("seed", range(60))
def test_oracle_equals_brute_force(seed):
    cat, grid, n_min = cases.random_tiny(seed)
    res = oracle.stack(cat, grid, n_min)
    bf, pairs = brute.search(cat.x, cat.y, cat.epoch, cat.t, cat.ticks_per_hour, grid, n_min)
    assert oracle_tuples(res) == [tuple(c[:5]) + (list(c[5]),) for c in bf]
    assert res.n_pairs == pairs


def test_oracle_equals_brute_force_tiny_workload_subgrid():
    w = W.tiny()
    cat = W.load(w)
    g = W.GridSpec(**{**w.grid.__dict__, "nvx": 5, "nvy": 4, "vx0": -2000, "vy0": 1000})
    res = oracle.stack(cat, g, 4)
    bf, pairs = brute.search(cat.x, cat.y, cat.epoch, cat.t, cat.ticks_per_hour, g, 4)
    assert oracle_tuples(res) == [tuple(c[:5]) + (list(c[5]),) for c in bf]
    assert res.n_pairs == pairs


def _mover_catalog(E, vx, vy, x0, y0, tph=3600, step=3600, noise=0, seed=0, field=200_000):
    t = np.arange(E, dtype=np.int64) * step
    x = [x0 + (vx * int(tt)) // tph for tt in t]
    y = [y0 + (vy * int(tt)) // tph for tt in t]
    ep = list(range(E))
    rng = np.random.default_rng(seed)
    for e in range(E):
        for _ in range(noise):
            x.append(int(rng.integers(0, field))); y.append(int(rng.integers(0, field)))
            ep.append(e)
    return cases.catalog(x, y, ep, t, tph)


@pytest.mark.parametrize("kx,ky", [(3, 3), (0, 6), (6, 1), (2, 5)])
def test_linear_mover_found_at_its_velocity(kx, ky):
    """One mover, velocity on the lattice, v*dt an exact multiple of TPH, start
    at a bin centre: exactly one cell reaches count E, at its own v_idx, holding
    all its detections (Eq. 1-2 give zero residual at the true velocity)."""
    E, w = 12, 2000
    grid = W.GridSpec(vx0=-3000, vy0=-3000, dvx=1000, dvy=1000, nvx=7, nvy=7,
                      x_min=0, y_min=0, nbx=100, nby=100, bin=w)
    vx, vy = -3000 + 1000 * kx, -3000 + 1000 * ky
    cat = _mover_catalog(E, vx, vy, 101_000, 99_000, noise=0)
    res = oracle.stack(cat, grid, E)
    assert oracle_tuples(res) == [(ky * 7 + kx, 50, 49, E, E, list(range(E)))]
    # with sparse noise on top the mover's cell is still there with all its ids
    cat2 = _mover_catalog(E, vx, vy, 101_000, 99_000, noise=5, seed=kx * 7 + ky)
    res2 = oracle.stack(cat2, grid, E)
    assert (ky * 7 + kx, 50, 49) in [(int(c["v_idx"]), int(c["bx"]), int(c["by"])) for c in res2.cands]
    top = res2.cands[0]
    assert int(top["distinct"]) == E
    assert set(range(E)) <= set(int(i) for i in res2.id_lists()[0])


def _domain_grid_all(cat, bin_mpx, nv=3, step=500):
    """A lattice and a domain wide enough that every projection is inside it."""
    half = (nv - 1) // 2
    ext = step * half * int(cat.t.max() - cat.t.min()) // cat.ticks_per_hour + 2 * bin_mpx
    x_min = int(cat.x.min()) - ext
    y_min = int(cat.y.min()) - ext
    nbx = (int(cat.x.max()) + ext - x_min) // bin_mpx + 1
    nby = (int(cat.y.max()) + ext - y_min) // bin_mpx + 1
    return W.GridSpec(vx0=-half * step, vy0=-half * step, dvx=step, dvy=step, nvx=nv, nvy=nv,
                      x_min=x_min, y_min=y_min, nbx=nbx, nby=nby, bin=bin_mpx)


def test_raw_counts_sum_to_in_domain_detections():
    """Every detection lands in exactly one bin per velocity when the domain
    covers all projections: sum_b raw = n, and sum_b distinct <= n with equality
    iff no two detections of one epoch share a bin."""
    w = W.tiny()
    cat = W.load(w)
    grid = _domain_grid_all(cat, 4000)
    for (vx, vy) in [(0, 0), (-500, 500), (500, 0)]:
        dist, raw = oracle.histogram(cat, grid, vx, vy)
        assert int(raw.sum()) == cat.n
        assert int(dist.sum()) <= cat.n
    # one detection per epoch, far apart -> equality
    cat1 = cases.catalog([i * 100_000 for i in range(20)], [5] * 20, list(range(20)),
                         np.arange(20) * 600)
    g1 = _domain_grid_all(cat1, 1000)
    d1, r1 = oracle.histogram(cat1, g1, 500, -500)
    assert int(d1.sum()) == int(r1.sum()) == 20
    assert oracle.stack(cat1, g1, 1).n_pairs == 20 * 9


def test_duplicating_detections():
    """Duplicating every detection in place leaves distinct counts unchanged,
    doubles raw counts and lists both copies."""
    for seed in range(5):
        cat, grid, n_min = cases.random_tiny(1000 + seed)
        n = cat.n
        dup = cases.catalog(np.concatenate([cat.x, cat.x]), np.concatenate([cat.y, cat.y]),
                            np.concatenate([cat.epoch, cat.epoch]), cat.t, cat.ticks_per_hour)
        a = oracle_tuples(oracle.stack(cat, grid, n_min))
        b = oracle_tuples(oracle.stack(dup, grid, n_min))
        assert len(a) == len(b)
        exp = sorted([(v, bx, by, d, 2 * r, sorted(ids + [i + n for i in ids]))
                      for (v, bx, by, d, r, ids) in a], key=lambda c: (-c[3], -c[4], c[0], c[2], c[1]))
        assert b == exp


def test_permutation_invariance():
    for seed in range(5):
        cat, grid, n_min = cases.random_tiny(2000 + seed)
        perm = np.random.default_rng(seed).permutation(cat.n)
        pc = cases.catalog(cat.x[perm], cat.y[perm], cat.epoch[perm], cat.t, cat.ticks_per_hour)
        a = oracle_tuples(oracle.stack(cat, grid, n_min))
        b = oracle_tuples(oracle.stack(pc, grid, n_min))
        b_mapped = [(v, bx, by, d, r, sorted(int(perm[i]) for i in ids)) for (v, bx, by, d, r, ids) in b]
        assert a == b_mapped


def test_translation_invariance():
    """Moving all detections and the domain by k bins changes nothing."""
    for seed in range(5):
        cat, grid, n_min = cases.random_tiny(3000 + seed)
        k, l = 3, -2
        dx, dy = k * grid.bin, l * grid.bin
        tc = cases.catalog(cat.x.astype(np.int64) + dx, cat.y.astype(np.int64) + dy, cat.epoch,
                           cat.t, cat.ticks_per_hour)
        tg = W.GridSpec(**{**grid.__dict__, "x_min": grid.x_min + dx, "y_min": grid.y_min + dy})
        assert oracle_tuples(oracle.stack(cat, grid, n_min)) == oracle_tuples(oracle.stack(tc, tg, n_min))


def test_time_origin_invariance():
    """Adding a constant to every epoch time leaves t - t0 and the output unchanged."""
    for seed in range(5):
        cat, grid, n_min = cases.random_tiny(4000 + seed)
        tc = cases.catalog(cat.x, cat.y, cat.epoch, cat.t + 123_456_789, cat.ticks_per_hour)
        assert oracle_tuples(oracle.stack(cat, grid, n_min)) == oracle_tuples(oracle.stack(tc, grid, n_min))
        if cat.n:
            assert oracle.t0(tc) == oracle.t0(cat) + 123_456_789


def test_t0_is_earliest_time_in_catalog():
    cat = cases.catalog([0, 0, 0], [0, 0, 0], [2, 3, 1], [-50, 40, 30, 20], 3600)
    assert oracle.t0(cat) == 20   # epoch 0 (t=-50) has no detection


def test_velocity_range_split_is_a_partition():
    """Searching disjoint lattice ranges and merging in the output order gives
    the whole search (each velocity's histogram is independent, Sec. 2.1 step 2)."""
    cat, grid, n_min = cases.random_tiny(77, max_side=7)
    nv = grid.nvx * grid.nvy
    full = oracle.stack(cat, grid, n_min)
    parts = [oracle.stack(cat, grid, n_min, a, b) for a, b in [(0, nv // 3), (nv // 3, nv)]]
    merged = sorted(sum((oracle_tuples(p) for p in parts), []),
                    key=lambda c: (-c[3], -c[4], c[0], c[2], c[1]))
    assert merged == oracle_tuples(full)
    assert sum(p.n_pairs for p in parts) == full.n_pairs


def test_top_k_is_prefix():
    cat, grid, n_min = cases.random_tiny(5, max_side=7)
    full = oracle_tuples(oracle.stack(cat, grid, 1))
    for k in (1, 3, 10):
        assert oracle_tuples(oracle.stack(cat, grid, 1, max_candidates=k)) == full[:k]


def _binom_pmf(n, k, p):
    return math.comb(n, k) * p ** k * (1 - p) ** (n - k)


@pytest.mark.parametrize("vel", [(0, 0), (1500, -2500)])
def test_noise_distinct_counts_are_binomial(vel):
    """Sec. 2.2: noise peaks are a Poisson/uniform point process, so with n_e
    uniform detections per epoch over a field of B equal bins, a bin is hit in an
    epoch with probability q = 1 - (1 - 1/B)^n_e independently across epochs and
    the distinct-epoch count of an interior cell is Binomial(E, q).  Pearson
    chi-square over the count values."""
    E, ne, nb, w = 24, 1500, 64, 1000
    side = nb * w
    rng = np.random.default_rng(99)
    x = rng.integers(0, side, E * ne); y = rng.integers(0, side, E * ne)
    ep = np.repeat(np.arange(E), ne)
    t = np.arange(E, dtype=np.int64) * 600
    cat = cases.catalog(x, y, ep, t, 3600)
    grid = W.GridSpec(vx0=0, vy0=0, dvx=1, dvy=1, nvx=1, nvy=1, x_min=0, y_min=0,
                      nbx=nb, nby=nb, bin=w)
    dist, raw = oracle.histogram(cat, grid, *vel)
    # interior cells: the source window stays inside the field at every epoch
    span = int(t.max())
    mx = -(-abs(vel[0]) * span // 3600 // w) + 1
    my = -(-abs(vel[1]) * span // 3600 // w) + 1
    inner = dist[my: nb - my, mx: nb - mx].ravel()
    q = 1 - (1 - 1 / (nb * nb)) ** ne
    ks = np.arange(E + 1)
    exp = np.array([_binom_pmf(E, k, q) for k in ks]) * inner.size
    obs = np.bincount(inner, minlength=E + 1).astype(float)
    # merge sparse tails so every expected count >= 5
    lo = 0
    while exp[: lo + 1].sum() < 5: lo += 1
    hi = E
    while exp[hi:].sum() < 5: hi -= 1
    e2 = np.concatenate([[exp[: lo + 1].sum()], exp[lo + 1: hi], [exp[hi:].sum()]])
    o2 = np.concatenate([[obs[: lo + 1].sum()], obs[lo + 1: hi], [obs[hi:].sum()]])
    chi2 = float(((o2 - e2) ** 2 / e2).sum())
    dof = len(e2) - 1
    # 99.9% point of chi-square with dof degrees of freedom (Wilson-Hilferty)
    z = 3.09
    crit = dof * (1 - 2 / (9 * dof) + z * math.sqrt(2 / (9 * dof))) ** 3
    assert chi2 < crit, (chi2, crit, o2, e2)
    assert abs(inner.mean() - E * q) < 0.05 * E * q
