"""Refinement and gathering (Sec. 2.1 steps 4-6) through the C ABI against the
oracle, cluster by cluster: the same status, fit count, subset size, points and
gathered ids, and the same line, residual covariance and determinant bit for
bit (both sides round the exact scatter matrix once and then evaluate the same
IEEE double expressions)."""
import numpy as np
import pytest

import oracle
from oracle import peel as PL
from oracle import refine as R
from paper_2509_26279_gb300 import workloads as W
from tests import cases

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2509_26279_gb300 import sas  # noqa: E402


def rel_times(cat):
    """Per detection: its epoch's time minus t0 (the earliest time over epochs
    that hold detections), ticks."""
    used = np.unique(cat.epoch)
    t0 = int(cat.t[used].min()) if len(used) else 0
    return cat.t[cat.epoch.astype(np.int64)].astype(np.int64) - t0


def same_float(a, b):
    return (np.isnan(a) and np.isnan(b)) or np.float64(a) == np.float64(b)


def compare(cat, tph, clusters, tracks, ids, ks, radius, seed, **kw):
    tt = rel_times(cat)
    x, y = cat.x.astype(np.int64), cat.y.astype(np.int64)
    for k in ks:
        c = clusters[k]
        cl_ids = c[1]
        want = R.refine(cl_ids, tt, x, y, radius, seed, k, **kw)
        g = tracks[k]
        got_ids = ids[int(g["id_off"]): int(g["id_off"]) + int(g["id_len"])].tolist()
        ctx = (k, want.status, int(g["status"]))
        assert int(g["cluster"]) == k
        assert int(g["status"]) == want.status, ctx
        assert int(g["iterations"]) == want.iterations, ctx
        assert int(g["n_points"]) == want.n_points, ctx
        assert got_ids == want.ids, ctx
        if want.iterations == 0:
            continue
        assert int(g["h"]) == want.h, ctx
        assert same_float(g["det"], want.det), (ctx, g["det"], want.det)
        if want.line is None:
            assert np.isnan(g["vx"]) and np.isnan(g["x0"])
            continue
        ln = want.line
        assert same_float(g["vx"], ln.vxt * np.float64(tph)), (ctx, g["vx"], ln.vxt * tph)
        assert same_float(g["vy"], ln.vyt * np.float64(tph)), ctx
        assert same_float(g["x0"], ln.x0) and same_float(g["y0"], ln.y0), ctx
        assert all(same_float(g[f], v) for f, v in zip(("res_xx", "res_xy", "res_yy"), ln.res)), ctx


def clusters_of(res):
    c, ids = res.candidates()
    return [(c[i], ids[int(c[i]["id_off"]): int(c[i]["id_off"]) + int(c[i]["id_len"])].tolist())
            for i in range(len(c))]


FAST = dict(n_starts=30, n_best=3, max_csteps=20, max_iter=4)


@pytest.mark.parametrize("seed", range(20))
def test_refine_random_tiny_candidates(seed):
    """Every candidate of a small random search (duplicates, exact ties, odd
    bins and clocks) as a cluster."""
    cat, grid, n_min = cases.random_tiny(seed + 3100)
    res = sas.stack_catalog(sas.Grid(grid), cat, n_min)
    cl = clusters_of(res)
    if not cl:
        return
    radius = max(1, grid.bin)
    tr = sas.sas_refine(res, None, seed=seed, radius=radius, **FAST)
    tracks, ids = tr.tracks()
    assert len(tracks) == len(cl)
    compare(cat, cat.ticks_per_hour, cl, tracks, ids, range(min(len(cl), 25)), radius, seed, **FAST)


@pytest.mark.parametrize("seed", range(6))
def test_refine_random_tiny_peel(seed):
    cat, grid, n_min = cases.random_tiny(seed + 3300)
    res = sas.stack_catalog(sas.Grid(grid), cat, n_min)
    pl = sas.sas_peel(res, n_min)
    cl = clusters_of(pl)
    if not cl:
        return
    radius = max(1, grid.bin)
    tracks, ids = sas.sas_refine(res, pl, seed=seed + 1, radius=radius, **FAST).tracks()
    compare(cat, cat.ticks_per_hour, cl, tracks, ids, range(len(cl)), radius, seed + 1, **FAST)


def test_refine_tiny_workload_defaults_recovers_velocities():
    w = W.tiny()
    cat = W.load(w)
    res = sas.stack_catalog(sas.Grid(w.grid), cat, 4)
    pl = sas.sas_peel(res, 4)
    cl = clusters_of(pl)
    tracks, ids = sas.sas_refine(res, pl, seed=11).tracks()
    compare(cat, cat.ticks_per_hour, cl, tracks, ids, range(len(cl)), w.grid.bin, 11)
    for g in tracks:
        m = cat.mover[ids[int(g["id_off"]): int(g["id_off"]) + int(g["id_len"])]]
        top = np.bincount(m[m >= 0]).argmax() if (m >= 0).any() else -1
        if top >= 0 and g["status"] == sas.TRACK_CONVERGED and (m == top).sum() >= 10:
            mv = cat.movers[top]
            assert abs(g["vx"] - mv["vx"]) < 100 and abs(g["vy"] - mv["vy"]) < 100


def test_refine_scaled_field_sampled_clusters_and_edge_statuses():
    ws = W.scaled(W.decam_tno(), frac_noise=0.2, width_px=800, height_px=800, n_movers=60, grid_half=15)
    cat = W.load(ws)
    res = sas.stack_catalog(sas.Grid(ws.grid), cat, 12)
    pl = sas.sas_peel(res, 12)
    cl = clusters_of(pl)
    assert len(cl) > 20
    kw = dict(n_starts=60, n_best=4, max_csteps=50, max_iter=6)
    tracks, ids = sas.sas_refine(res, pl, seed=7, **kw).tracks()
    compare(cat, cat.ticks_per_hour, cl, tracks, ids, range(0, len(cl), 5), ws.grid.bin, 7, **kw)
    assert (tracks["status"] == sas.TRACK_CONVERGED).mean() > 0.8
    # one fit only, a radius below every residual, a radius that takes in too much
    for extra, radius in ((dict(max_iter=1), ws.grid.bin), ({}, 1), ({}, 400_000)):
        k2 = dict(kw, **extra)
        tracks, ids = sas.sas_refine(res, pl, seed=8, radius=radius, **k2).tracks()
        compare(cat, cat.ticks_per_hour, cl, tracks, ids, range(0, len(cl), 9), radius, 8, **k2)
    assert (tracks["status"] == sas.TRACK_TOO_MANY).any()


def test_refine_full_tno_field_sampled():
    w = W.decam_tno()
    cat = W.load(w)
    res = sas.stack_catalog(sas.Grid(w.grid), cat, w.n_min)
    pl = sas.sas_peel(res, w.n_min)
    cl = clusters_of(pl)
    tracks, ids = sas.sas_refine(res, pl, seed=3).tracks()
    compare(cat, cat.ticks_per_hour, cl, tracks, ids, [0, len(cl) // 2, len(cl) - 1], w.grid.bin, 3)
    assert (tracks["status"] == sas.TRACK_CONVERGED).mean() > 0.9


def test_refine_sees_detections_outside_the_bucket_grid():
    """Detections far outside the search's bucket grid go to the overflow
    bucket: the search is unchanged, and a gather whose radius reaches them
    takes them in."""
    from tests.test_gpu_parity import gpu_tuples, oracle_tuples
    rng = np.random.default_rng(5)
    E = 10
    t = np.arange(E, dtype=np.int64) * 3600
    xs, ys, es = [], [], []
    for e in range(E):                     # one mover at (1000, 500) mpx/h, 100 mpx jitter
        xs.append(10_000 + 1000 * e + int(rng.integers(-100, 100)))
        ys.append(20_000 + 500 * e + int(rng.integers(-100, 100)))
        es.append(e)
        for _ in range(3):                 # noise in the domain
            xs.append(int(rng.integers(0, 40_000))); ys.append(int(rng.integers(0, 40_000))); es.append(e)
    for e in range(5):                     # far outside the grid
        xs.append(-30_000_000 + int(rng.integers(-1000, 1000))); ys.append(int(rng.integers(0, 40_000)))
        es.append(e)
    cat = cases.catalog(xs, ys, es, t)
    grid = W.GridSpec(vx0=-1000, vy0=-1000, dvx=250, dvy=250, nvx=9, nvy=9, x_min=0, y_min=0, nbx=20, nby=20,
                      bin=2000, speed_min=0, speed_max=0)
    res = sas.stack_catalog(sas.Grid(grid), cat, 6)
    assert gpu_tuples(res) == oracle_tuples(oracle.stack(cat, grid, 6))
    pl = sas.sas_peel(res, 6)
    cl = clusters_of(pl)
    assert cl
    for radius in (2000, 40_000_000):
        tracks, ids = sas.sas_refine(res, pl, seed=2, radius=radius).tracks()
        compare(cat, 3600, cl, tracks, ids, range(len(cl)), radius, 2)
    far = set(range(len(xs) - 5, len(xs)))
    assert far & set(ids.tolist())             # the wide gather took the far detections in


def test_refine_errors():
    w = W.tiny()
    cat = W.load(w)
    g = sas.Grid(w.grid)
    res = sas.stack_catalog(g, cat, 6)
    pl = sas.sas_peel(res, 6)
    with pytest.raises(sas.SasError):
        sas.sas_refine(pl, pl)                                  # a cluster list keeps no catalog
    with pytest.raises(sas.SasError):
        sas.sas_refine(res, pl, n_starts=5000)
    other = sas.stack_catalog(g, cases.catalog(cat.x[:100], cat.y[:100], cat.epoch[:100], cat.t), 6)
    with pytest.raises(sas.SasError):
        sas.sas_refine(other, pl)                               # clusters of another catalog
    empty = sas.stack_catalog(g, cases.catalog([], [], [], cat.t), 6)
    tracks, ids = sas.sas_refine(empty).tracks()
    assert len(tracks) == 0 and len(ids) == 0


def test_refine_large_cluster_uses_the_radix_selection():
    """A track buried in close noise: its cluster holds ~600 points, above the
    256 where the C-step switches from rank counting to the binary descent."""
    rng = np.random.default_rng(12)
    E = 100
    t = np.sort(rng.integers(0, 4 * 3600, E)).astype(np.int64)
    xs, ys, es = [], [], []
    for e in range(E):
        bx, by = 50_000 + 1200 * t[e] / 3600, 60_000 - 800 * t[e] / 3600
        xs.append(int(bx + rng.normal(0, 150))); ys.append(int(by + rng.normal(0, 150))); es.append(e)
        for _ in range(6):
            xs.append(int(bx + rng.uniform(-1900, 1900))); ys.append(int(by + rng.uniform(-1900, 1900)))
            es.append(e)
        for _ in range(30):
            xs.append(int(rng.integers(0, 120_000))); ys.append(int(rng.integers(0, 120_000))); es.append(e)
    cat = cases.catalog(xs, ys, es, t)
    grid = W.GridSpec(vx0=-2000, vy0=-2000, dvx=400, dvy=400, nvx=11, nvy=11, x_min=0, y_min=0, nbx=30, nby=30,
                      bin=4000, speed_min=0, speed_max=0)
    res = sas.stack_catalog(sas.Grid(grid), cat, 30)
    pl = sas.sas_peel(res, 30)
    cl = clusters_of(pl)
    assert len(cl[0][1]) > 256
    kw = dict(n_starts=30, n_best=3, max_iter=3)
    tracks, ids = sas.sas_refine(res, pl, seed=1, **kw).tracks()
    compare(cat, 3600, cl, tracks, ids, range(len(cl)), grid.bin, 1, **kw)
    assert tracks[0]["n_points"] > 256
