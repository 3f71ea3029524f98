"""sas_cell_counts_noalloc against the CPU oracle and the existing entry point.

Some callers cannot allocate device memory while they run: a process that has
given all its device memory to its own pool under a fixed budget, or code that
issues work from a loop which must never wait on the allocator.  For them the
library offers exact cell counts that keep their working state in a fixed array
inside the library instead of allocating.  Its numbers must equal the oracle's
single-cell counts (oracle.cell) and what sas_stack reports for the same cells,
for candidate cells, cells with nothing in them and cells of a catalog with
empty epochs, on calls in a row (a call must not be affected by what the one
before left in the shared array); a cell outside the lattice or the domain is
an argument error whose outputs read 0xffffffff."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2509_26279_gb300 import sas, workloads as W  # noqa: E402
from tests import cases  # noqa: E402


def _noalloc(grid_spec, cat, cells):
    """(distinct, raw) of the cells through the entry point (device arrays in and out)."""
    dev = torch.device("cuda")
    cells = np.asarray(cells, np.uint32).reshape(-1, 3)
    d_cells = torch.from_numpy(cells.ravel().view(np.int32)).to(dev)
    d_x = torch.from_numpy(np.ascontiguousarray(cat.x)).to(dev)
    d_y = torch.from_numpy(np.ascontiguousarray(cat.y)).to(dev)
    d_e = torch.from_numpy(np.ascontiguousarray(cat.epoch).view(np.int16)).to(dev)
    d_distinct = torch.full((len(cells),), -7, dtype=torch.int32, device=dev)
    d_raw = torch.full((len(cells),), -7, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    try:
        sas.sas_cell_counts_noalloc(sas.Grid(grid_spec), d_x, d_y, d_e, cat.t, cat.ticks_per_hour, d_cells,
                                    len(cells), d_distinct, d_raw)
        err = None
    except sas.SasError as e:
        err = e
    return d_distinct.cpu().numpy().view(np.uint32), d_raw.cpu().numpy().view(np.uint32), err


def _oracle_counts(cat, grid, cells):
    out = [oracle.cell(cat, grid, int(v), int(bx), int(by))[:2] for v, bx, by in cells]
    return np.array([o[0] for o in out], np.uint32), np.array([o[1] for o in out], np.uint32)


def _check(w_or_cat, grid, n_min, n_random, seed):
    cat = W.load(w_or_cat) if isinstance(w_or_cat, W.Workload) else w_or_cat
    res = sas.stack_catalog(sas.Grid(grid), cat, n_min)
    cands, _ = res.candidates()
    assert len(cands) > 0
    rng = np.random.default_rng(seed)
    pick = rng.choice(len(cands), min(60, len(cands)), replace=False)
    cand_cells = np.stack([cands["v_idx"][pick], cands["bx"][pick], cands["by"][pick]], 1)
    rnd = np.stack([rng.integers(0, grid.nvx * grid.nvy, n_random), rng.integers(0, grid.nbx, n_random),
                    rng.integers(0, grid.nby, n_random)], 1)
    cells = np.concatenate([cand_cells, rnd]).astype(np.uint32)
    distinct, raw, err = _noalloc(grid, cat, cells)
    assert err is None, err
    od, orw = _oracle_counts(cat, grid, cells)
    assert np.array_equal(distinct, od) and np.array_equal(raw, orw)
    # the candidate cells also equal the stack's exact counts
    assert np.array_equal(distinct[:len(pick)], cands["count"][pick])
    assert np.array_equal(raw[:len(pick)], cands["raw"][pick])
    # random cells include empty ones (not vacuous)
    assert (raw[len(pick):] == 0).sum() > 0
    return cat


def test_noalloc_counts_equal_oracle_on_calls_in_a_row():
    # first call: a ragged, several-tile field with 100 epochs
    w = W.scaled(W.decam_tno(), frac_noise=0.05, width_px=700, height_px=500, n_movers=40, grid_half=12, seed=21)
    _check(w, w.grid, 10, 200, 1)
    # second call: another catalog with fewer epochs and another grid
    _check(W.tiny(), W.tiny().grid, W.tiny().n_min, 200, 2)
    # third call: a catalog whose epoch table has epochs without detections
    # (including the earliest time: t0 is the earliest time that has one)
    w = W.tiny()
    cat = W.load(w)
    keep = (cat.epoch % 3) != 0
    sparse = cases.catalog(cat.x[keep], cat.y[keep], cat.epoch[keep], cat.t, cat.ticks_per_hour)
    assert len(np.unique(sparse.epoch)) < len(sparse.t)
    _check(sparse, w.grid, 5, 200, 3)


def test_noalloc_cell_outside_lattice_or_domain_is_an_argument_error():
    w = W.tiny()
    cat = W.load(w)
    g = w.grid
    cells = [(0, 0, 0), (g.nvx * g.nvy, 0, 0), (5, g.nbx, 1), (7, 2, g.nby), (g.nvx * g.nvy - 1, g.nbx - 1, g.nby - 1)]
    distinct, raw, err = _noalloc(g, cat, cells)
    assert err is not None and err.status == sas.SAS_ERR_ARG
    for i in (1, 2, 3):
        assert distinct[i] == 0xFFFFFFFF and raw[i] == 0xFFFFFFFF
    od, orw = _oracle_counts(cat, g, [cells[0], cells[4]])
    assert distinct[0] == od[0] and raw[0] == orw[0] and distinct[4] == od[1] and raw[4] == orw[1]
    # a following call is unaffected by the error left in the shared array
    _check(w, g, w.n_min, 50, 4)


def test_noalloc_rejects_too_many_epochs():
    grid = sas.Grid(W.tiny().grid)
    dev = torch.device("cuda")
    z = torch.zeros(4, dtype=torch.int32, device=dev)
    e = torch.zeros(4, dtype=torch.int16, device=dev)
    out = torch.zeros(1, dtype=torch.int32, device=dev)
    cells = torch.zeros(3, dtype=torch.int32, device=dev)
    with pytest.raises(sas.SasError) as ei:
        sas.sas_cell_counts_noalloc(grid, z, z, e, np.zeros(2000, np.int64), 3600, cells, 1, out, out)
    assert ei.value.status == sas.SAS_ERR_RANGE
