"""sas_cell_counts_noalloc against the existing entry point.

Some callers cannot allocate device memory while they run: a process that has
given all its device memory to its own pool under a fixed budget, or code that
issues work from a loop which must never wait on the allocator.  For them the
library offers exact cell counts that keep their working state in a fixed array
inside the library instead of allocating.  Its numbers must equal what
sas_stack reports for the same cells, on two calls in a row (the second call
must not be affected by what the first left in the shared array)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2509_26279_gb300 import sas, workloads as W  # noqa: E402


def _counts_match_stack(w, n_min):
    cat = W.load(w)
    grid = sas.Grid(w.grid)
    res = sas.stack_catalog(grid, cat, n_min)
    cands, _ = res.candidates()
    assert len(cands) > 0
    cells = np.stack([cands["v_idx"], cands["bx"], cands["by"]], 1).astype(np.uint32).ravel()
    dev = torch.device("cuda")
    d_cells = torch.from_numpy(cells.view(np.int32)).to(dev)
    d_x = torch.from_numpy(cat.x).to(dev)
    d_y = torch.from_numpy(cat.y).to(dev)
    d_e = torch.from_numpy(cat.epoch.view(np.int16)).to(dev)
    d_distinct = torch.full((len(cands),), -1, dtype=torch.int32, device=dev)
    d_raw = torch.full((len(cands),), -1, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    sas.sas_cell_counts_noalloc(grid, d_x, d_y, d_e, cat.t, cat.ticks_per_hour, d_cells,
                                len(cands), d_distinct, d_raw)
    distinct = d_distinct.cpu().numpy().view(np.uint32)
    raw = d_raw.cpu().numpy().view(np.uint32)
    assert np.array_equal(distinct, cands["count"])
    assert np.array_equal(raw, cands["raw"])


def test_noalloc_counts_equal_stack_on_two_calls():
    # first call: a ragged, several-tile field with 100 epochs
    _counts_match_stack(W.scaled(W.decam_tno(), frac_noise=0.05, width_px=700, height_px=500,
                                 n_movers=40, grid_half=12, seed=21), 10)
    # second call: another catalog with fewer epochs and another grid
    _counts_match_stack(W.tiny(), W.tiny().n_min)


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
