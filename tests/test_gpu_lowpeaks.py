"""Parity of the two-threshold search (every cell at N_min, plus the cells at
n_low whose super-bin is a tile-local peak of the raw counts) with its CPU
oracle, through the C ABI: candidate records, id arrays and pair counts byte
for byte, single-field and batched, on tiny random searches, every tile shape,
lattice ranges, the speed annulus, wrapped counters and the full TNO field."""
import numpy as np
import pytest

import oracle
from oracle import lowpeaks as LP
from paper_2509_26279_gb300 import workloads as W
from tests import cases

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2509_26279_gb300 import sas  # noqa: E402
from tests.test_gpu_parity import assert_same, gpu_tuples, oracle_tuples  # noqa: E402


def run_two(cat, grid, n_min, n_low, v_begin=0, v_end=None, peaks_only=0, **optkw):
    o = sas.make_opts(n_low=n_low, peaks_only=peaks_only, **optkw)
    if v_end is not None:
        o.v_begin, o.v_end = v_begin, v_end
    res = sas.stack_catalog(sas.Grid(grid), cat, n_min, opts=o)
    info = res.info()
    assert info["n_low"] == (n_low or n_min) and info["peaks_only"] == peaks_only
    ref = LP.search(cat, grid, n_min, n_low or n_min, LP.tiles_of(info), v_begin, v_end,
                    peaks_only=bool(peaks_only))
    return res, ref


@pytest.mark.parametrize("seed", range(60))
def test_random_tiny_catalogs(seed):
    cat, grid, n_min = cases.random_tiny(seed)
    rng = np.random.default_rng(seed + 500)
    n_min += int(rng.integers(0, 3))
    n_low = int(rng.integers(1, n_min + 1))
    res, ref = run_two(cat, grid, n_min, n_low, peaks_only=int(seed % 3 == 0))
    assert_same(res, ref)


def _scaled(seed=5, **kw):
    a = dict(frac_noise=0.03, width_px=500, height_px=600, n_epochs=40, n_movers=30, grid_half=10, seed=seed)
    a.update(kw)
    w = W.scaled(W.decam_tno(), **a)
    return w, W.load(w)


@pytest.mark.parametrize("cfg", [
    dict(), dict(tile_kx=4, tile_ky=1), dict(tile_kx=4, tile_ky=2), dict(tile_kx=8, tile_ky=2),
    dict(tile_kx=8, tile_ky=4), dict(tile_kx=8, tile_ky=8), dict(counter_bits=16), dict(counter_bits=32),
    dict(tile_kx=8, tile_ky=8, counter_bits=16, tile_bx=16, tile_by=12), dict(tile_bx=12, tile_by=8),
    dict(superbin=1), dict(superbin=2), dict(superbin=3, velocity_block=2), dict(superbin=4, velocity_block=4),
])
def test_tile_configurations(cfg):
    """Every tile shape gives the oracle's list for its own tiles (the peak test
    is tile-local, so the list depends on the tiles; the oracle takes them from
    the result), with and without the cells at N_min outside the peaks."""
    w, cat = _scaled()
    res, ref = run_two(cat, w.grid, 10, 6, **cfg)
    plain = oracle.stack(cat, w.grid, 10)
    assert len(ref.cands) > len(plain.cands) > 0
    assert_same(res, ref)
    res, ref_po = run_two(cat, w.grid, 10, 6, peaks_only=1, **cfg)
    assert_same(res, ref_po)
    assert 0 < len(ref_po.cands) < len(ref.cands)


def test_speed_annulus_and_lattice_ranges():
    w, cat = _scaled(seed=8)
    g = W.GridSpec(**{**w.grid.__dict__, "speed_min": 2000, "speed_max": 9000})
    res, ref = run_two(cat, g, 9, 5, tile_kx=8, tile_ky=8)
    assert_same(res, ref)
    res, ref = run_two(cat, g, 9, 5, peaks_only=1, tile_kx=8, tile_ky=8)
    assert_same(res, ref)
    nv = w.grid.nvx * w.grid.nvy
    for k, (a, b) in enumerate([(0, 17), (5, nv // 2), (nv // 3, nv), (nv - 1, nv),
                                (3 * w.grid.nvx + 2, 9 * w.grid.nvx + 5)]):
        res, ref = run_two(cat, w.grid, 9, 5, v_begin=a, v_end=b, peaks_only=k % 2, tile_kx=8, tile_ky=4)
        assert_same(res, ref)


def test_equal_or_zero_n_low_is_the_plain_search():
    w, cat = _scaled(seed=9)
    plain = sas.stack_catalog(sas.Grid(w.grid), cat, 9)
    for n_low in (0, 9):
        res = sas.stack_catalog(sas.Grid(w.grid), cat, 9, opts=sas.make_opts(n_low=n_low))
        assert gpu_tuples(res) == gpu_tuples(plain)
        assert res.info()["n_emitted"] == plain.info()["n_emitted"]


def test_fewer_emissions_than_the_low_search():
    """The peak test runs before any bin is counted: far fewer super-bins are
    emitted than by the one-threshold search at n_low."""
    w, cat = _scaled(seed=10, frac_noise=0.08)
    res, ref = run_two(cat, w.grid, 10, 5)
    assert_same(res, ref)
    low = sas.stack_catalog(sas.Grid(w.grid), cat, 5, opts=sas.make_opts(superbin=res.info()["superbin"]))
    assert res.info()["n_emitted"] * 2 < low.info()["n_emitted"]
    assert res.info()["n_candidates"] < low.info()["n_candidates"]


def test_peaks_only_at_n_min_and_peel_refuses_it():
    """peaks_only without n_low: the peaks at N_min alone, fewer than the plain
    list; cluster finding needs the complete list and refuses it."""
    w, cat = _scaled(seed=12)
    res, ref = run_two(cat, w.grid, 9, 0, peaks_only=1)
    assert_same(res, ref)
    plain = oracle.stack(cat, w.grid, 9)
    assert 0 < len(ref.cands) < len(plain.cands)
    with pytest.raises(sas.SasError):
        sas.sas_peel(res, 9, 100)


def test_counter_wrap_reruns_wider():
    x = [5000] * 300 + [5000] + [9000] * 3
    y = [7000] * 300 + [7000] + [3000] * 3
    ep = [0] * 300 + [1] + [0, 1, 2]
    cat = cases.catalog(x, y, ep, [0, 3600, 7200], 3600)
    grid = W.GridSpec(vx0=-1000, vy0=-1000, dvx=1000, dvy=1000, nvx=3, nvy=3, x_min=0,
                      y_min=0, nbx=16, nby=16, bin=1000)
    res, ref = run_two(cat, grid, 3, 2)
    assert_same(res, ref)
    assert res.info()["counter_bits"] >= 16
    res, ref = run_two(cat, grid, 3, 2, peaks_only=1)
    assert_same(res, ref)


def test_argument_errors():
    w, cat = _scaled(seed=11)
    g = sas.Grid(w.grid)
    with pytest.raises(sas.SasError):
        sas.stack_catalog(g, cat, 5, opts=sas.make_opts(n_low=6))
    wts = np.ones(cat.x.shape[0], np.uint8)
    with pytest.raises(sas.SasError):
        sas.sas_stack_weighted(g, cat.x, cat.y, cat.epoch, wts, cat.t, cat.ticks_per_hour, 5,
                               opts=sas.make_opts(n_low=3))
    with pytest.raises(sas.SasError):
        sas.sas_stack_weighted(g, cat.x, cat.y, cat.epoch, wts, cat.t, cat.ticks_per_hour, 5,
                               opts=sas.make_opts(peaks_only=1))
    with pytest.raises(sas.SasError):
        sas.stack_catalog(g, cat, 5, opts=sas.make_opts(peaks_only=2))


def _dev(cat):
    d = torch.device("cuda")
    return (torch.from_numpy(cat.x).to(d), torch.from_numpy(cat.y).to(d),
            torch.from_numpy(cat.epoch.view(np.int16)).to(d))


def test_batch_fields_match_the_oracle():
    """Uneven small fields in one batch, each at N_min = ceil(E/4) with n_low =
    ceil(E/6) (two of them with n_low off; three with the peaks alone), field
    by field against the oracle with the field's own tiles."""
    rng = np.random.default_rng(77)
    fields, specs, opts = [], [], []
    for i in range(6):
        E = int(rng.integers(20, 151))
        w = W.scaled(W.decam_tno(), frac_noise=float(rng.uniform(0.02, 0.08)), width_px=int(rng.integers(300, 900)),
                     height_px=int(rng.integers(300, 900)), n_epochs=E, n_movers=int(rng.integers(10, 40)),
                     grid_half=int(rng.integers(6, 14)), seed=7700 + i)
        cat = W.load(w)
        n_min, n_low = max(3, -(-E // 4)), (0 if i in (2, 4) else max(2, -(-E // 6)))
        po = int(i in (1, 4, 5))
        x, y, e = _dev(cat)
        fields.append((sas.Grid(w.grid), x, y, e, cat.t, cat.ticks_per_hour, n_min))
        specs.append((w, cat, n_min, n_low, po))
        opts.append(sas.make_opts(n_low=n_low, peaks_only=po, tile_kx=8, tile_ky=8 if i % 2 else 4))
    b = sas.Batch(fields, opts=opts)
    b.run()
    assert b.stats()[1] == 0
    for f, (w, cat, n_min, n_low, po) in enumerate(specs):
        info = b.field_info(f)
        assert info["n_low"] == (n_low or n_min) and info["peaks_only"] == po
        ref = LP.search(cat, w.grid, n_min, n_low or n_min, LP.tiles_of(info), peaks_only=bool(po))
        c, ids = b.candidates(f)
        assert len(c) == len(ref.cands)
        for fg, fo in [("v_idx", "v_idx"), ("bx", "bx"), ("by", "by"), ("count", "distinct"), ("raw", "raw"),
                       ("id_off", "id_off"), ("id_len", "id_len")]:
            assert np.array_equal(c[fg].astype(np.int64), ref.cands[fo].astype(np.int64)), (f, fg)
        assert np.array_equal(ids.astype(np.int64), ref.ids.astype(np.int64))
        assert info["n_pairs"] == ref.n_pairs
    b.destroy()


def test_full_decam_tno_bands():
    """The full TNO field (2048x4096 px, 100 epochs, 111x111 lattice) at N_min
    = 25 and n_low = 17: the whole output is ordered and valid; on bands of
    lattice rows around low-threshold candidates and one random band, the
    list equals the oracle's (its search at n_low over the band, each cell
    kept by the definition with the super-bin counts of the whole lattice); a
    sample of cells recomputed from the definition."""
    w = W.decam_tno()
    cat = W.load(w)
    g = w.grid
    n_min, n_low = w.n_min, -(-w.recipe.n_epochs // 6)
    res = sas.stack_catalog(sas.Grid(g), cat, n_min, opts=sas.make_opts(n_low=n_low))
    info = res.info()
    got = gpu_tuples(res)
    keys = [(-c[3], -c[4], c[0], c[2], c[1]) for c in got]
    assert keys == sorted(keys) and len(set(keys)) == len(keys)
    assert all(c[3] >= n_low and c[4] == len(c[5]) for c in got)
    low_only = [i for i, c in enumerate(got) if c[3] < n_min]
    assert len(low_only) > 100
    rng = np.random.default_rng(3)
    for i in rng.choice(len(got), 20, replace=False):
        v, bx, by, d, r, ids = got[i]
        d2, r2, ids2 = oracle.cell(cat, g, v, bx, by)
        assert (d, r, ids) == (d2, r2, ids2.tolist())
    tiles = LP.tiles_of(info)
    R = LP.SuperbinCounts(cat, g, tiles["s"])
    rows = [got[i][0] // g.nvx for i in rng.choice(low_only, 2, replace=False)] + [int(rng.integers(0, g.nvy))]
    for row in rows:
        a, b = max(0, row - 1) * g.nvx, min(g.nvy, row + 1) * g.nvx
        lo = oracle.stack(cat, g, n_low, a, b, threads=0)
        keep = np.zeros(len(lo.cands), bool)
        for k, c in enumerate(lo.cands):
            v = int(c["v_idx"])
            keep[k] = int(c["distinct"]) >= n_min or LP.is_peak(
                R, v % g.nvx, v // g.nvx, int(c["bx"]) // tiles["s"], int(c["by"]) // tiles["s"], tiles)
        want = oracle_tuples(LP.subset(lo, keep))
        assert [c for c in got if a <= c[0] < b] == want
