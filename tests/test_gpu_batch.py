"""The batched, graph-replayed search gives every field exactly what sas_stack
gives it, including fields that need the exact fallback."""
import numpy as np
import pytest

import oracle
from paper_2509_26279_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2509_26279_gb300 import sas  # noqa: E402


def _dev(cat):
    d = torch.device("cuda")
    return (torch.from_numpy(cat.x).to(d), torch.from_numpy(cat.y).to(d),
            torch.from_numpy(cat.epoch.view(np.int16)).to(d))


def _fields(n, seed):
    """Uneven small fields: epochs 20..150, noise 2%..8% of the full density."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        E = int(rng.integers(20, 151))
        w = W.scaled(W.decam_tno(), frac_noise=float(rng.uniform(0.02, 0.08)), width_px=int(rng.integers(300, 900)),
                     height_px=int(rng.integers(300, 900)), n_epochs=E, n_movers=int(rng.integers(10, 40)),
                     grid_half=int(rng.integers(6, 14)), seed=seed * 100 + i)
        out.append((w, max(3, -(-E // 4))))
    return out


def _assert_oracle(c, ids, n_pairs, ref):
    """Element-by-element equality of a field's candidates and ids with the oracle's."""
    assert len(c) == len(ref.cands), (len(c), len(ref.cands))
    for fg, fo in [("v_idx", "v_idx"), ("bx", "bx"), ("by", "by"), ("count", "distinct"), ("raw", "raw"),
                   ("id_off", "id_off"), ("id_len", "id_len")]:
        assert np.array_equal(c[fg].astype(np.int64), ref.cands[fo].astype(np.int64)), fg
    assert np.array_equal(ids.astype(np.int64), ref.ids.astype(np.int64))
    assert n_pairs == ref.n_pairs


def _single(grid, cat, n_min):
    r = sas.stack_catalog(grid, cat, n_min)
    c, ids = r.candidates()
    return c, ids, r.info()["n_pairs"]


def test_batch_equals_single_field_search():
    specs = _fields(7, 3)
    fields, refs, orefs = [], [], []
    for w, n_min in specs:
        cat = W.load(w)
        g = sas.Grid(w.grid)
        x, y, e = _dev(cat)
        fields.append((g, x, y, e, cat.t, cat.ticks_per_hour, n_min))
        refs.append(_single(g, cat, n_min))
        orefs.append(oracle.stack(cat, w.grid, n_min))
    b = sas.Batch(fields)
    for rep in range(2):  # two replays of the same graph
        b.run()
        for f, (c_ref, ids_ref, pairs_ref) in enumerate(refs):
            c, ids = b.candidates(f)
            _assert_oracle(c, ids, b.field_info(f)["n_pairs"], orefs[f])
            assert np.array_equal(c, c_ref), (rep, f)
            assert np.array_equal(ids, ids_ref), (rep, f)
            assert b.field_info(f)["n_pairs"] == pairs_ref
    ms, fallbacks = b.stats()
    assert ms > 0 and fallbacks == 0
    b.destroy()


def test_batch_grows_past_its_capacity():
    """A field with far more candidates than the batch's initial per-field
    capacity (32768) makes the run grow its capacities, rebuild the pass and
    replay: every field stays batched and exact."""
    w = W.tiny()
    cat = W.load(w)
    g = sas.Grid(w.grid)
    x, y, e = _dev(cat)
    w2 = _fields(1, 9)[0][0]
    cat2 = W.load(w2)
    g2 = sas.Grid(w2.grid)
    x2, y2, e2 = _dev(cat2)
    b = sas.Batch([(g, x, y, e, cat.t, cat.ticks_per_hour, 2),
                   (g2, x2, y2, e2, cat2.t, cat2.ticks_per_hour, 12)])
    b.run()
    ref = oracle.stack(cat, w.grid, 2)
    c, ids = b.candidates(0)
    assert len(ref.cands) > 32768 and len(c) == len(ref.cands)
    assert np.array_equal(c["count"].astype(np.int64), ref.cands["distinct"].astype(np.int64))
    assert np.array_equal(ids.astype(np.int64), ref.ids.astype(np.int64))
    c2, ids2, _ = _single(g2, cat2, 12)
    cb, idsb = b.candidates(1)
    assert np.array_equal(cb, c2) and np.array_equal(idsb, ids2)
    assert b.stats()[1] == 0 and b.rebuilds >= 1
    # a second run replays the grown pass without rebuilding
    b.run()
    assert b.stats()[1] == 0 and b.rebuilds == 1
    c, ids = b.candidates(0)
    assert np.array_equal(ids.astype(np.int64), ref.ids.astype(np.int64))
    b.destroy()


def test_batch_sorts_large_fields_without_fallback():
    """12,838 candidates (more than one shared-memory sort) stay in the batch:
    the segmented sort orders them exactly like the single-field path."""
    w = W.tiny()
    cat = W.load(w)
    g = sas.Grid(w.grid)
    x, y, e = _dev(cat)
    w2 = _fields(1, 9)[0][0]
    cat2 = W.load(w2)
    g2 = sas.Grid(w2.grid)
    x2, y2, e2 = _dev(cat2)
    b = sas.Batch([(g, x, y, e, cat.t, cat.ticks_per_hour, 3),
                   (g2, x2, y2, e2, cat2.t, cat2.ticks_per_hour, 12)])
    for _ in range(2):
        b.run()
        ref = oracle.stack(cat, w.grid, 3)
        c, ids = b.candidates(0)
        assert len(ref.cands) > 8192 and len(c) == len(ref.cands)
        for fg, fo in [("v_idx", "v_idx"), ("bx", "bx"), ("by", "by"), ("count", "distinct"),
                       ("raw", "raw"), ("id_len", "id_len"), ("id_off", "id_off")]:
            assert np.array_equal(c[fg].astype(np.int64), ref.cands[fo].astype(np.int64)), fg
        assert np.array_equal(ids.astype(np.int64), ref.ids.astype(np.int64))
        c2, ids2, _ = _single(g2, cat2, 12)
        cb, idsb = b.candidates(1)
        assert np.array_equal(cb, c2) and np.array_equal(idsb, ids2)
    assert b.stats()[1] == 0
    b.destroy()


def test_autotune_returns_a_valid_faster_config():
    w = W.scaled(W.decam_tno(), frac_noise=0.05, width_px=700, height_px=500, n_movers=40,
                 grid_half=12, seed=21)
    cat = W.load(w)
    g = sas.Grid(w.grid)
    x, y, e = _dev(cat)
    best, ms = sas.sas_autotune(g, x, y, e, cat.t, cat.ticks_per_hour, 10, reps=2)
    assert best.superbin in (1, 2, 3, 4) and best.velocity_block in (0, 2, 4) and ms > 0
    assert (best.tile_kx, best.tile_ky) in ((8, 8), (8, 4)) and best.tile_bx in (0, 32, 64)
    r = sas.stack_catalog(g, cat, 10, opts=best)
    c, ids = r.candidates()
    c0, ids0, _ = _single(g, cat, 10)
    assert np.array_equal(c, c0) and np.array_equal(ids, ids0)


def test_batch_with_per_field_tuned_options():
    """Fields of one batch with different super-bin sizes and velocity blocks
    (as the autotuner's per-size-class cache hands them out) still equal their
    single-field searches."""
    specs = _fields(6, 11)
    fields, refs, opts = [], [], []
    for i, (w, n_min) in enumerate(specs):
        cat = W.load(w)
        g = sas.Grid(w.grid)
        x, y, e = _dev(cat)
        fields.append((g, x, y, e, cat.t, cat.ticks_per_hour, n_min))
        o = sas.make_opts(superbin=1 + i % 3, velocity_block=[1, 2, 4, 8][i % 4])
        opts.append(o)
        r = sas.stack_catalog(g, cat, n_min, opts=o)
        refs.append(r.candidates())
    b = sas.Batch(fields, opts=opts)
    b.run()
    for f, (c_ref, ids_ref) in enumerate(refs):
        c, ids = b.candidates(f)
        assert np.array_equal(c, c_ref) and np.array_equal(ids, ids_ref), f


def test_full_size_uneven_fields_with_tuned_options_match_oracle():
    """Four of the 60 full-size uneven fields (2048x4096 px, 111x111 lattice):
    the fewest epochs, the most epochs, the most detections and the median
    detection count, each with the autotuner's options for its size class, in
    one batch; every field's candidates, ids and pair count byte for byte
    against the oracle (OpenMP form over all host cores)."""
    from paper_2509_26279_gb300 import tuning, vetting
    ws = W.batched_fields(60)
    load = [w.recipe.n_epochs * w.recipe.noise_per_epoch for w in ws]
    pick = {int(np.argmin([w.recipe.n_epochs for w in ws])), int(np.argmax([w.recipe.n_epochs for w in ws])),
            int(np.argmax(load)), int(np.argsort(load)[len(load) // 2])}
    dev = torch.device("cuda")
    fields = [vetting.Field(ws[i], dev) for i in sorted(pick)]
    cache = tuning.TuneCache()
    opts = []
    for f in fields:
        cache.tune(f)
        opts.append(cache.opts_for(f))
    b = sas.Batch([(f.grid, f.dx, f.dy, f.de, f.cat.t, f.cat.ticks_per_hour, f.w.n_min) for f in fields], opts=opts)
    b.run()
    assert b.stats()[1] == 0  # no field left the batch
    for k, f in enumerate(fields):
        ref = oracle.stack(f.cat, f.w.grid, f.w.n_min, threads=0)
        c, ids = b.candidates(k)
        assert len(ref.cands) > 100
        _assert_oracle(c, ids, b.field_info(k)["n_pairs"], ref)
    b.destroy()


def test_batch_mixes_tile_shapes_and_counter_widths():
    """One batch whose fields need different stack kernels -- 8 x 8 and 8 x 4
    velocity tiles, and 16-bit counters for fields whose brightest mover could
    wrap an 8-bit counter (many epochs, low threshold) -- runs one persistent
    launch per kernel and still equals the oracle field by field, with no
    field recomputed on the single-field path."""
    # (epochs, N_min, movers, noise fraction, tile_ky): 150 and 140 epochs at
    # N_min 20 and 12 could pass 128 + N_min detections in a super-bin
    specs = [(150, 20, 3, 0.03, 8), (60, 15, 20, 0.05, 8), (140, 12, 3, 0.02, 4), (90, 23, 20, 0.05, 4)]
    fields, orefs, opts = [], [], []
    for i, (E, n_min, movers, frac, ky) in enumerate(specs):
        w = W.scaled(W.decam_tno(), frac_noise=frac, width_px=600, height_px=500, n_epochs=E, n_movers=movers,
                     grid_half=10, seed=1700 + i)
        cat = W.load(w)
        g = sas.Grid(w.grid)
        x, y, e = _dev(cat)
        fields.append((g, x, y, e, cat.t, cat.ticks_per_hour, n_min))
        opts.append(sas.make_opts(tile_kx=8, tile_ky=ky))
        orefs.append(oracle.stack(cat, w.grid, n_min))
    b = sas.Batch(fields, opts=opts)
    b.run()
    widths = set()
    for f, ref in enumerate(orefs):
        c, ids = b.candidates(f)
        info = b.field_info(f)
        widths.add((info["tile_ky"], info["counter_bits"]))
        _assert_oracle(c, ids, info["n_pairs"], ref)
    assert widths == {(8, 16), (8, 8), (4, 16), (4, 8)}, widths
    assert b.stats()[1] == 0
    b.destroy()
