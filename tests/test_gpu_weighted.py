"""Weighted stacking through the C ABI against the oracle: the same cells,
scores, raw counts and ids in the same order (integer arithmetic: bit-exact)."""
import numpy as np
import pytest

from oracle import weighted as WT
from paper_2509_26279_gb300 import workloads as W
from tests import cases

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2509_26279_gb300 import sas  # noqa: E402


def gpu_tuples(res):
    c, ids = res.candidates()
    return [(int(r["v_idx"]), int(r["bx"]), int(r["by"]), int(r["count"]), int(r["raw"]),
             ids[int(r["id_off"]): int(r["id_off"]) + int(r["id_len"])].tolist()) for r in c]


def run(cat, grid, w, s_min, **kw):
    return sas.sas_stack_weighted(sas.Grid(grid), cat.x, cat.y, cat.epoch, w, cat.t, cat.ticks_per_hour, s_min,
                                  **kw)


@pytest.mark.parametrize("seed", range(30))
def test_weighted_random_tiny(seed):
    cat, grid, n_min = cases.random_tiny(seed + 5100)
    rng = np.random.default_rng(seed)
    w = rng.integers(0, 256, len(cat.x)).astype(np.uint8) if seed % 3 else \
        rng.integers(1, 5, len(cat.x)).astype(np.uint8)
    s_min = int(rng.integers(1, 4 * (int(w.max()) if len(w) else 1) + 2))
    assert gpu_tuples(run(cat, grid, w, s_min)) == WT.stack(cat, grid, w, s_min)


def test_unit_weights_match_the_plain_search():
    w = W.tiny()
    cat = W.load(w)
    plain = sas.stack_catalog(sas.Grid(w.grid), cat, 5)
    c, ids = plain.candidates()
    want = [(int(r["v_idx"]), int(r["bx"]), int(r["by"]), int(r["count"]), int(r["raw"]),
             ids[int(r["id_off"]): int(r["id_off"]) + int(r["id_len"])].tolist()) for r in c]
    assert gpu_tuples(run(cat, w.grid, np.ones(len(cat.x), np.uint8), 5)) == want


@pytest.mark.parametrize("cb", [8, 16, 32])
def test_weighted_scaled_field_every_counter_width(cb):
    """A TNO-like field with S/N-like weights (noise near threshold, movers
    brighter); counter wraps force reruns with wider counters on the way."""
    ws = W.scaled(W.decam_tno(), frac_noise=0.2, width_px=600, height_px=600, n_movers=40, grid_half=10)
    cat = W.load(ws)
    rng = np.random.default_rng(3)
    w = np.where(cat.mover >= 0, rng.integers(40, 120, len(cat.x)), rng.integers(20, 45, len(cat.x))).astype(np.uint8)
    s_min = 12 * 60
    got = gpu_tuples(run(cat, ws.grid, w, s_min, opts=sas.make_opts(counter_bits=cb)))
    assert got == WT.stack(cat, ws.grid, w, s_min)
    assert len(got) > 10


def test_weighted_device_inputs_and_refine():
    w = W.tiny()
    cat = W.load(w)
    wt = np.random.default_rng(1).integers(1, 30, len(cat.x)).astype(np.uint8)
    dev = torch.device("cuda", 0)
    dx, dy = torch.from_numpy(cat.x).to(dev), torch.from_numpy(cat.y).to(dev)
    de = torch.from_numpy(cat.epoch.view(np.int16)).to(dev)
    dw = torch.from_numpy(wt).to(dev)
    res = sas.sas_stack_weighted(sas.Grid(w.grid), dx, dy, de, dw, cat.t, cat.ticks_per_hour, 60, on_device=True)
    assert gpu_tuples(res) == WT.stack(cat, w.grid, wt, 60)
    with pytest.raises(sas.SasError):
        sas.sas_peel(res, 60)                    # recounts are distinct epochs
    tracks, _ = sas.sas_refine(res, None, n_starts=20, max_iter=2).tracks()
    assert len(tracks) == res.info()["n_candidates"]
