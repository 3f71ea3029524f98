"""The oracle's OpenMP form (velocity chunks in parallel, merged in the total
order) must give exactly what its single loop over velocities gives: the
velocities' histograms are independent (Sec. 2.1 step 2), so splitting the
lattice changes no candidate, id or pair count."""
import numpy as np
import pytest

import oracle
from paper_2509_26279_gb300 import workloads as W
from tests import cases


def _same(a, b):
    assert np.array_equal(a.cands, b.cands)
    assert np.array_equal(a.ids, b.ids)
    assert a.n_pairs == b.n_pairs


@pytest.mark.parametrize("seed", range(24))
@pytest.mark.parametrize("threads", [2, 5, 0])
def test_openmp_equals_single_loop_on_random_catalogs(seed, threads):
    cat, grid, n_min = cases.random_tiny(seed)
    _same(oracle.stack(cat, grid, n_min, threads=threads), oracle.stack(cat, grid, n_min))


def test_openmp_equals_single_loop_on_a_workload_with_ranges_and_top_k():
    w = W.tiny()
    cat = W.load(w)
    nv = w.grid.nvx * w.grid.nvy
    for a, b, k in [(0, nv, 0), (17, nv - 30, 0), (0, nv, 3), (100, 101, 0), (5, 5, 0)]:
        _same(oracle.stack(cat, w.grid, w.n_min, a, b, k, threads=4),
              oracle.stack(cat, w.grid, w.n_min, a, b, k))


def test_thread_count_is_reported():
    assert oracle.threads() >= 1
