"""Pins of the weighted-stacking oracle: unit weights reduce to the stack
oracle, an independent pure-Python brute force (its own projection and running
per-epoch maxima), hand-built cells, and monotonicity in the weights."""
import numpy as np
import pytest

import oracle
from oracle import weighted as WT
from tests import cases


def brute(cat, grid, w, s_min):
    t = [int(v) for v in cat.t]
    ep = [int(e) for e in cat.epoch]
    t_ref = min(t[e] for e in ep) if ep else 0
    cells = {}
    for ky in range(grid.nvy):
        for kx in range(grid.nvx):
            vx, vy = grid.vx0 + kx * grid.dvx, grid.vy0 + ky * grid.dvy
            if (grid.speed_min, grid.speed_max) != (0, 0):
                s2 = vx * vx + vy * vy
                if s2 < grid.speed_min ** 2 or s2 > grid.speed_max ** 2:
                    continue
            for i in range(len(ep)):
                dt = t[ep[i]] - t_ref
                bx = (int(cat.x[i]) - (vx * dt) // cat.ticks_per_hour - grid.x_min) // grid.bin
                by = (int(cat.y[i]) - (vy * dt) // cat.ticks_per_hour - grid.y_min) // grid.bin
                if 0 <= bx < grid.nbx and 0 <= by < grid.nby:
                    mx, ids = cells.setdefault((ky * grid.nvx + kx, bx, by), ({}, []))
                    mx[ep[i]] = max(mx.get(ep[i], 0), int(w[i]))
                    ids.append(i)
    out = [(v, bx, by, sum(mx.values()), len(ids), sorted(ids)) for (v, bx, by), (mx, ids) in cells.items()
           if sum(mx.values()) >= s_min]
    out.sort(key=lambda c: (-c[3], -c[4], c[0], c[2], c[1]))
    return out


@pytest.mark.parametrize("seed", range(25))
def test_against_brute_force(seed):
    cat, grid, n_min = cases.random_tiny(seed + 4100, max_n=90, max_side=5)
    rng = np.random.default_rng(seed)
    w = rng.integers(0, 256, len(cat.x)) if seed % 3 else rng.integers(1, 4, len(cat.x))
    s_min = int(rng.integers(1, 3 * max(1, int(w.max()) if len(w) else 1)))
    assert WT.stack(cat, grid, w, s_min) == brute(cat, grid, w, s_min)


@pytest.mark.parametrize("seed", range(10))
def test_unit_weights_are_distinct_counts(seed):
    cat, grid, n_min = cases.random_tiny(seed + 4300)
    ref = oracle.stack(cat, grid, n_min)
    want = cases.as_tuples(ref.cands, ref.id_lists())
    assert WT.stack(cat, grid, np.ones(len(cat.x), np.uint8), n_min) == want


def test_hand_built_cell():
    # one mover at rest over 4 epochs with weights 5, 9, 3, 7 plus a second
    # detection in epoch 1 (weight 8, same bin): score 5 + 9 + 3 + 7, raw 5
    from paper_2509_26279_gb300.workloads import GridSpec
    x = [100, 100, 150, 100, 100]
    y = [100, 100, 120, 100, 100]
    e = [0, 1, 1, 2, 3]
    w = [5, 9, 8, 3, 7]
    cat = cases.catalog(x, y, e, [0, 3600, 7200, 10800])
    grid = GridSpec(vx0=0, vy0=0, dvx=1, dvy=1, nvx=1, nvy=1, x_min=0, y_min=0, nbx=4, nby=4, bin=200,
                    speed_min=0, speed_max=0)
    assert WT.stack(cat, grid, w, 24) == [(0, 0, 0, 24, 5, [0, 1, 2, 3, 4])]
    assert WT.stack(cat, grid, w, 25) == []
    w2 = [5, 1, 8, 3, 7]        # the duplicate now carries its epoch's maximum
    assert WT.stack(cat, grid, w2, 1)[0][3] == 5 + 8 + 3 + 7


def test_scores_grow_with_the_weights():
    cat, grid, n_min = cases.random_tiny(4500)
    rng = np.random.default_rng(1)
    w = rng.integers(0, 100, len(cat.x))
    lo = {c[:3]: c[3] for c in WT.stack(cat, grid, w, 1)}
    w2 = w + rng.integers(0, 50, len(cat.x))
    hi = {c[:3]: c[3] for c in WT.stack(cat, grid, w2, 1)}
    assert all(hi[k] >= v for k, v in lo.items())
