"""Velocity-range shards searched by the CUDA path (one process, shards in
turn) merge into the same bytes as one search of the whole lattice."""
import numpy as np
import pytest

from paper_2509_26279_gb300 import shard
from paper_2509_26279_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2509_26279_gb300 import sas  # noqa: E402


@pytest.mark.parametrize("world,k", [(2, 0), (5, 0), (3, 50)])
def test_shards_merge_to_single_search(world, k):
    w = W.scaled(W.decam_tno(), frac_noise=0.1)
    cat = W.load(w)
    g = sas.Grid(w.grid)
    nv = w.grid.nvx * w.grid.nvy
    full_c, full_i = sas.stack_catalog(g, cat, 12, opts=sas.make_opts(max_candidates=k)).candidates()
    parts = []
    for b, e in shard.velocity_ranges(nv, world):
        r = sas.stack_catalog(g, cat, 12, opts=sas.make_opts(v_begin=b, v_end=e, max_candidates=k))
        parts.append(r.candidates())
    c, i = shard.merge(parts, k)
    assert len(full_c) > 20
    assert c.tobytes() == np.asarray(full_c, shard.CANDIDATE_DTYPE).tobytes()
    assert np.array_equal(i, full_i)
