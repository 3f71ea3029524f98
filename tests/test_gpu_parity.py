"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

The bar is bit-exactness: candidate lists (v_idx, bx, by, distinct, raw) and
their ascending id lists must equal the oracle's, as must the number of
in-domain (detection, velocity) pairs."""
import numpy as np
import pytest

import oracle
from paper_2509_26279_gb300 import workloads as W
from tests import cases
from tests.test_oracle_pins import golden_inputs, load_golden

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2509_26279_gb300 import sas  # noqa: E402  (raises if libsas.so is missing)


def gpu_tuples(res):
    cands, ids = res.candidates()
    return [(int(c["v_idx"]), int(c["bx"]), int(c["by"]), int(c["count"]), int(c["raw"]),
             ids[c["id_off"]: c["id_off"] + c["id_len"]].tolist()) for c in cands]


def oracle_tuples(r):
    return cases.as_tuples(r.cands, r.id_lists())


def run_both(cat, grid, n_min, opts=None, v_begin=0, v_end=None, max_candidates=0, **kw):
    o = opts or sas.make_opts()
    if v_end is not None:
        o.v_begin, o.v_end = v_begin, v_end
    if max_candidates:
        o.max_candidates = max_candidates
    g = sas.Grid(grid)
    res = sas.stack_catalog(g, cat, n_min, opts=o, **kw)
    ref = oracle.stack(cat, grid, n_min, v_begin, v_end, max_candidates)
    return res, ref


def assert_same(res, ref):
    """Element-by-element equality of the candidate records and id arrays."""
    cands, ids = res.candidates()
    rc = ref.cands
    assert len(cands) == len(rc), (len(cands), len(rc))
    for fg, fo in [("v_idx", "v_idx"), ("bx", "bx"), ("by", "by"), ("count", "distinct"),
                   ("raw", "raw"), ("id_len", "id_len"), ("id_off", "id_off")]:
        a, b = cands[fg].astype(np.int64), rc[fo].astype(np.int64)
        bad = np.nonzero(a != b)[0]
        assert bad.size == 0, f"field {fg} differs first at candidate {bad[0]}: gpu {a[bad[0]]} oracle {b[bad[0]]}"
    assert np.array_equal(ids.astype(np.int64), ref.ids.astype(np.int64))
    assert res.info()["n_pairs"] == ref.n_pairs


@pytest.mark.parametrize("case", load_golden(), ids=lambda c: c["name"])
def test_golden_cases(case):
    cat, grid, n_min = golden_inputs(case)
    res = sas.stack_catalog(sas.Grid(grid), cat, n_min)
    want = [tuple(c[:5]) + (list(c[5]),) for c in case["expected"]]
    assert gpu_tuples(res) == want


@pytest.mark.parametrize("seed", range(80))
def test_random_tiny_catalogs(seed):
    cat, grid, n_min = cases.random_tiny(seed)
    res, ref = run_both(cat, grid, n_min)
    assert_same(res, ref)


def test_tiny_workload():
    w = W.tiny()
    cat = W.load(w)
    res, ref = run_both(cat, w.grid, w.n_min)
    assert len(ref.cands) > 0
    assert_same(res, ref)
    assert res.info()["t0"] == oracle.t0(cat)


@pytest.mark.parametrize("cfg", [
    dict(tile_kx=4, tile_ky=1), dict(tile_kx=4, tile_ky=2), dict(tile_kx=8, tile_ky=2),
    dict(counter_bits=16), dict(counter_bits=32),
    dict(tile_bx=12, tile_by=8), dict(tile_bx=36, tile_by=20, coarse_bins=3),
    dict(coarse_bins=1), dict(coarse_bins=50), dict(tile_kx=8, tile_ky=4),
    dict(tile_kx=8, tile_ky=4, counter_bits=16, tile_bx=20, tile_by=28),
    dict(tile_kx=8, tile_ky=8), dict(tile_kx=8, tile_ky=8, counter_bits=16),
    dict(tile_kx=8, tile_ky=8, counter_bits=32, tile_bx=16, tile_by=12),
])
def test_tile_configurations_agree(cfg):
    """Every tile shape, counter width and bucket size gives the same bytes."""
    w = W.scaled(W.decam_tno(), frac_noise=0.02, width_px=300, height_px=420, n_epochs=40,
                 n_movers=20, grid_half=9, seed=5)
    cat = W.load(w)
    res, ref = run_both(cat, w.grid, 8, opts=sas.make_opts(**cfg))
    assert len(ref.cands) > 0
    assert_same(res, ref)


def test_scaled_tno_many_tiles_ragged():
    """A lattice and domain that are not multiples of the tile: ragged tiles on
    every side; several hundred spatial tiles."""
    w = W.scaled(W.decam_tno(), frac_noise=0.05, width_px=1021, height_px=777, n_movers=60,
                 grid_half=13, seed=11)
    cat = W.load(w)
    res, ref = run_both(cat, w.grid, 12)
    assert len(ref.cands) > 0
    assert_same(res, ref)


def test_scaled_fast_movers():
    w = W.scaled(W.fast_movers(), frac_noise=0.03, width_px=900, height_px=1300, n_movers=30,
                 grid_half=45, seed=3)
    cat = W.load(w)
    res, ref = run_both(cat, w.grid, 10)
    assert len(ref.cands) > 0
    assert_same(res, ref)


def test_speed_annulus_and_lattice_range():
    w = W.scaled(W.decam_tno(), frac_noise=0.03, width_px=500, height_px=600, n_movers=30,
                 grid_half=10, seed=8)
    cat = W.load(w)
    g = W.GridSpec(**{**w.grid.__dict__, "speed_min": 2000, "speed_max": 9000})
    res, ref = run_both(cat, g, 9)
    assert_same(res, ref)
    nv = w.grid.nvx * w.grid.nvy
    for a, b in [(0, 17), (5, nv // 2), (nv // 3, nv), (nv - 1, nv)]:
        res, ref = run_both(cat, w.grid, 9, v_begin=a, v_end=b)
        assert_same(res, ref)


def test_tall_tiles_with_annulus_ranges_and_ragged_edges():
    """8 x 8 velocity tiles (64-bit lattice masks) on the masked paths: speed
    annulus, index ranges that end mid-tile, a lattice that is not a multiple of 8."""
    w = W.scaled(W.decam_tno(), frac_noise=0.03, width_px=500, height_px=600, n_movers=30,
                 grid_half=10, seed=8)
    cat = W.load(w)
    o = sas.make_opts(tile_kx=8, tile_ky=8)
    g = W.GridSpec(**{**w.grid.__dict__, "speed_min": 2000, "speed_max": 9000})
    res, ref = run_both(cat, g, 9, opts=o)
    assert_same(res, ref)
    nv = w.grid.nvx * w.grid.nvy
    for a, b in [(0, 17), (5, nv // 2), (nv // 3, nv), (nv - 1, nv)]:
        res, ref = run_both(cat, w.grid, 9, opts=o, v_begin=a, v_end=b)
        assert_same(res, ref)


def test_top_k():
    w = W.tiny()
    cat = W.load(w)
    full = oracle_tuples(oracle.stack(cat, w.grid, 5))
    for k in (1, 7, 100):
        res = sas.stack_catalog(sas.Grid(w.grid), cat, 5, opts=sas.make_opts(max_candidates=k))
        assert gpu_tuples(res) == full[:k]


def test_counter_wrap_reruns_wider():
    """More than 255 detections of one cell inside one tile wrap an 8-bit
    counter; the library must notice and rerun with 16-bit counters."""
    x = [5000] * 300 + [5000]
    y = [7000] * 300 + [7000]
    ep = [0] * 300 + [1]
    cat = cases.catalog(x, y, ep, [0, 3600], 3600)
    grid = W.GridSpec(vx0=-1000, vy0=-1000, dvx=1000, dvy=1000, nvx=3, nvy=3, x_min=0,
                      y_min=0, nbx=16, nby=16, bin=1000)
    res, ref = run_both(cat, grid, 2)
    assert_same(res, ref)
    assert res.info()["counter_bits"] >= 16


def test_many_candidates_large_sort():
    """N_min = 1: every occupied cell is a candidate (over a million), which
    overflows the first emission list (rerun) and exercises the multi-block sort."""
    w = W.tiny()
    cat = W.load(w)
    res, ref = run_both(cat, w.grid, 1)
    assert len(ref.cands) > 100_000
    assert_same(res, ref)


def test_epoch_extremes():
    rng = np.random.default_rng(0)
    # a single epoch: every velocity sees the same histogram
    n = 500
    cat = cases.catalog(rng.integers(0, 50_000, n), rng.integers(0, 50_000, n), np.zeros(n),
                        [123], 3600)
    grid = W.GridSpec(vx0=-3000, vy0=-3000, dvx=1000, dvy=1500, nvx=7, nvy=5, x_min=0,
                      y_min=0, nbx=25, nby=25, bin=2000)
    res, ref = run_both(cat, grid, 1)
    assert_same(res, ref)
    # 1024 epochs (the maximum), stationary sources plus noise
    E = 1024
    t = np.arange(E, dtype=np.int64) * 10
    xs = np.concatenate([np.full(E, 10_500), rng.integers(0, 40_000, 3000)])
    ys = np.concatenate([np.full(E, 20_500), rng.integers(0, 40_000, 3000)])
    ep = np.concatenate([np.arange(E), rng.integers(0, E, 3000)])
    cat = cases.catalog(xs, ys, ep, t, 3600)
    grid = W.GridSpec(vx0=-2000, vy0=-2000, dvx=1000, dvy=1000, nvx=5, nvy=5, x_min=0,
                      y_min=0, nbx=20, nby=20, bin=2000)
    res, ref = run_both(cat, grid, 40)
    assert_same(res, ref)
    assert gpu_tuples(res)[0][3] >= E


def test_bin_of_one_mpx_and_empty_catalog():
    cat, grid, n_min = cases.random_tiny(7)
    g1 = W.GridSpec(**{**grid.__dict__, "bin": 1, "nbx": 40, "nby": 40})
    res, ref = run_both(cat, g1, 1)
    assert_same(res, ref)
    empty = cases.catalog([], [], [], [0, 100], 3600)
    res = sas.stack_catalog(sas.Grid(grid), empty, 1)
    assert gpu_tuples(res) == []
    assert res.info()["n_pairs"] == 0


def test_device_resident_inputs_match_host_inputs():
    w = W.tiny()
    cat = W.load(w)
    g = sas.Grid(w.grid)
    host = gpu_tuples(sas.stack_catalog(g, cat, w.n_min))
    dx = torch.from_numpy(cat.x).cuda()
    dy = torch.from_numpy(cat.y).cuda()
    de = torch.from_numpy(cat.epoch.astype(np.int16)).cuda()   # same 16-bit payload
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        res = sas.sas_stack(g, dx, dy, de, cat.t, cat.ticks_per_hour, w.n_min, on_device=True,
                            stream=s)
    assert gpu_tuples(res) == host


def test_candidates_into_reused_pinned_host_buffers():
    """candidates(out=...) fills caller-owned page-locked arrays with the same
    bytes as fresh arrays, across results, and refuses buffers that are too
    small or of the wrong type."""
    w = W.tiny()
    cat = W.load(w)
    g = sas.Grid(w.grid)
    res = sas.stack_catalog(g, cat, w.n_min)
    want_c, want_i = res.candidates()
    assert len(want_c) > 0
    hc = torch.empty((len(want_c) + 5) * sas.CANDIDATE_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
    hi = torch.empty(len(want_i) + 7, dtype=torch.int32).pin_memory()
    out = (hc.numpy().view(sas.CANDIDATE_DTYPE), hi.numpy().view(np.uint32))
    for _ in range(2):                     # reuse the same buffers for a second result
        r = sas.stack_catalog(g, cat, w.n_min)
        c, i = r.candidates(out=out)
        assert c.tobytes() == want_c.tobytes() and np.array_equal(i, want_i)
        r.free()
    with pytest.raises(sas.SasError) as ei:
        res.candidates(out=(out[0][:len(want_c) - 1], out[1]))
    assert ei.value.status == sas.SAS_ERR_OVERFLOW
    with pytest.raises(sas.SasError) as ei:
        res.candidates(out=(out[0], out[1].view(np.int32)))
    assert ei.value.status == sas.SAS_ERR_ARG


def test_range_errors():
    g = sas.Grid(W.tiny().grid)
    bad_epoch = cases.catalog([1, 2], [1, 2], [0, 5], [0, 10], 3600)
    with pytest.raises(sas.SasError) as ei:
        sas.stack_catalog(g, bad_epoch, 1)
    assert ei.value.status == sas.SAS_ERR_RANGE
    big = cases.catalog([1 << 29, 2], [1, 2], [0, 1], [0, 10], 3600)
    with pytest.raises(sas.SasError) as ei:
        sas.stack_catalog(g, big, 1)
    assert ei.value.status == sas.SAS_ERR_RANGE
    far = cases.catalog([1, 2], [1, 2], [0, 1], [0, (1 << 31)], 1)  # shift >= 2^28
    with pytest.raises(sas.SasError) as ei:
        sas.stack_catalog(g, far, 1)
    assert ei.value.status == sas.SAS_ERR_RANGE
    # the context is still usable afterwards
    w = W.tiny()
    assert len(gpu_tuples(sas.stack_catalog(g, W.load(w), w.n_min))) > 0


# ---- full-size workloads: exact on a lattice-index sample, sampled cells -----

def _full_size_check(w, n_ranges, n_cells_sample, seed, half=20):
    cat = W.load(w)
    g = sas.Grid(w.grid)
    res = sas.stack_catalog(g, cat, w.n_min)
    got = gpu_tuples(res)
    info = res.info()
    assert len(got) > 0
    # (1) every output is a valid candidate, in order, ids sorted and distinct
    keys = [(-c[3], -c[4], c[0], c[2], c[1]) for c in got]
    assert keys == sorted(keys) and len(set(keys)) == len(keys)
    for c in got:
        assert c[3] >= w.n_min and c[4] == len(c[5]) and c[5] == sorted(set(c[5]))
    # (2) a random sample of candidates recomputed one by one from the definition
    rng = np.random.default_rng(seed)
    for i in rng.choice(len(got), min(n_cells_sample, len(got)), replace=False):
        v, bx, by, d, r, ids = got[i]
        d2, r2, ids2 = oracle.cell(cat, w.grid, v, bx, by)
        assert (d, r, ids) == (d2, r2, ids2.tolist())
    # (3) exact parity on contiguous lattice-index ranges: around randomly chosen
    # candidates (so the check is not vacuous) and one random range
    nv = w.grid.nvx * w.grid.nvy
    centres = [got[i][0] for i in rng.choice(len(got), n_ranges, replace=False)]
    centres.append(int(rng.integers(0, nv)))
    for v in centres:
        a, b = max(0, v - half), min(nv, v + half)
        sub = [c for c in got if a <= c[0] < b]
        ref = oracle.stack(cat, w.grid, w.n_min, a, b)
        assert sub == oracle_tuples(ref)
    return info


def test_full_decam_tno():
    info = _full_size_check(W.decam_tno(), n_ranges=2, n_cells_sample=40, seed=1)
    assert info["n_pairs"] > 3e9


def test_full_decam_tno_whole_list():
    """The whole candidate list and id array of the full TNO field (2048x4096 px,
    100 epochs, 111x111 lattice), byte for byte against the oracle run over all
    host cores (its OpenMP form, equal to the single loop by its own pin)."""
    w = W.decam_tno()
    cat = W.load(w)
    res = sas.stack_catalog(sas.Grid(w.grid), cat, w.n_min)
    ref = oracle.stack(cat, w.grid, w.n_min, threads=0)
    assert len(ref.cands) > 1000 and ref.n_pairs > 3e9
    assert_same(res, ref)


def test_full_fast_movers():
    info = _full_size_check(W.fast_movers(), n_ranges=2, n_cells_sample=30, seed=2)
    assert info["n_pairs"] > 1e11


def test_dense_catalog_multi_pass_staging():
    """More detections in one work unit than the staging area holds: the kernel
    stages and runs the unit in several passes per velocity tile."""
    rng = np.random.default_rng(5)
    E, n = 20, 60_000
    x = rng.integers(0, 120_000, n)
    y = rng.integers(0, 120_000, n)
    ep = rng.integers(0, E, n)
    cat = cases.catalog(x, y, ep, np.arange(E) * 720, 3600)
    grid = W.GridSpec(vx0=-2000, vy0=-2000, dvx=1000, dvy=1000, nvx=5, nvy=5, x_min=0,
                      y_min=0, nbx=60, nby=60, bin=2000)
    res, ref = run_both(cat, grid, 30)
    assert_same(res, ref)
    res, ref = run_both(cat, grid, 30, opts=sas.make_opts(superbin=1, velocity_block=1))
    assert_same(res, ref)


@pytest.mark.parametrize("sb,vb", [(1, 1), (2, 1), (3, 2), (4, 8), (2, 3)])
def test_superbin_and_velocity_block_agree(sb, vb):
    w = W.scaled(W.decam_tno(), frac_noise=0.03, width_px=700, height_px=500, n_movers=40,
                 grid_half=12, seed=21)
    cat = W.load(w)
    res, ref = run_both(cat, w.grid, 10, opts=sas.make_opts(superbin=sb, velocity_block=vb))
    assert len(ref.cands) > 0
    assert_same(res, ref)
    assert res.info()["superbin"] == sb


@pytest.mark.parametrize("nvx", [2, 3, 5, 6, 7, 9])
def test_lattice_edge_inside_a_counter_word(nvx):
    """Lattice widths that end inside a counter word (four 8-bit counters per
    word along kx), on slow lattices where the word's columns are merged into
    at most two reductions: the columns past the edge must neither count nor
    steer a reduction."""
    w = W.scaled(W.decam_tno(), frac_noise=0.2, width_px=600, height_px=500, n_movers=30, grid_half=3,
                 seed=40 + nvx)
    g = w.grid
    grid = W.GridSpec(vx0=g.vx0, vy0=g.vy0, dvx=g.dvx, dvy=g.dvy, nvx=nvx, nvy=g.nvy, x_min=g.x_min,
                      y_min=g.y_min, nbx=g.nbx, nby=g.nby, bin=g.bin)
    cat = W.load(w)
    res, ref = run_both(cat, grid, 6)
    assert len(ref.cands) > 0
    assert_same(res, ref)
