"""Seeded edge-case catalogs for parity tests (inputs only; no stacking arithmetic)."""
from __future__ import annotations

import numpy as np

from paper_2509_26279_gb300.workloads import Catalog, GridSpec, MOVER_DTYPE


def catalog(x, y, epoch, t, tph=3600, mover=None) -> Catalog:
    x = np.asarray(x, np.int32)
    return Catalog(x=x, y=np.asarray(y, np.int32), epoch=np.asarray(epoch, np.uint16),
                   t=np.asarray(t, np.int64), ticks_per_hour=int(tph),
                   mover=np.full(x.shape[0], -1, np.int32) if mover is None else np.asarray(mover, np.int32),
                   movers=np.zeros(0, MOVER_DTYPE), width_px=0, height_px=0)


def random_tiny(seed: int, max_n: int = 160, max_e: int = 70, max_side: int = 7):
    """A small random search with the awkward parts switched on at random:
    unsorted and repeated epoch times, unused epochs, negative lattice steps and
    origins, negative domain origin, detections on and around domain edges,
    same-epoch duplicates, odd bin sizes, odd ticks-per-hour, speed annulus."""
    rng = np.random.default_rng(seed)
    E = int(rng.integers(1, max_e + 1))
    tph = int(rng.choice([3600, 1000, 7, 86400]))
    t = rng.integers(-5 * tph, 5 * tph, E).astype(np.int64)
    if rng.random() < 0.3:
        t = np.sort(t)
    w = int(rng.choice([1, 3, 7, 1000, 2000, 4999]))
    nbx, nby = int(rng.integers(1, 12)), int(rng.integers(1, 12))
    x_min, y_min = int(rng.integers(-20, 20)) * w // 3, int(rng.integers(-20, 20)) * w // 3
    span_x, span_y = nbx * w, nby * w
    dv_scale = max(1, (w * tph) // max(1, int(t.max() - t.min()) if E > 1 else 1))
    nvx, nvy = int(rng.integers(1, max_side + 1)), int(rng.integers(1, max_side + 1))
    dvx = int(rng.integers(-3, 4)) * dv_scale or dv_scale
    dvy = int(rng.integers(-3, 4)) * dv_scale or -dv_scale
    vx0 = -dvx * (nvx // 2) + int(rng.integers(-2, 3))
    vy0 = -dvy * (nvy // 2) + int(rng.integers(-2, 3))
    smin = smax = 0
    if rng.random() < 0.25:
        vmax = max(abs(vx0), abs(vx0 + (nvx - 1) * dvx)) + max(abs(vy0), abs(vy0 + (nvy - 1) * dvy))
        smin, smax = int(rng.integers(0, vmax // 2 + 1)), int(rng.integers(vmax // 2, vmax + 2))
    grid = GridSpec(vx0=vx0, vy0=vy0, dvx=dvx, dvy=dvy, nvx=nvx, nvy=nvy, x_min=x_min,
                    y_min=y_min, nbx=nbx, nby=nby, bin=w, speed_min=smin, speed_max=smax)
    n = int(rng.integers(0, max_n + 1))
    used = rng.integers(0, E, max(1, E // 2 + 1))          # some epochs stay empty
    ep = rng.choice(used, n).astype(np.int64)
    x = rng.integers(x_min - w, x_min + span_x + w, n)
    y = rng.integers(y_min - w, y_min + span_y + w, n)
    edge = rng.random(n) < 0.2                              # exactly on bin edges
    x[edge] = x_min + rng.integers(0, nbx + 1, edge.sum()) * w - rng.integers(0, 2, edge.sum())
    if n > 4 and rng.random() < 0.5:                        # same-epoch duplicates
        k = int(rng.integers(1, n // 2))
        src = rng.integers(0, n, k)
        x = np.concatenate([x, x[src]]); y = np.concatenate([y, y[src]])
        ep = np.concatenate([ep, ep[src]])
    n_min = int(rng.integers(1, max(2, min(E, 6)) + 1))
    return catalog(x, y, ep, t, tph), grid, n_min


def as_tuples(cands, id_lists):
    return [(int(c["v_idx"]), int(c["bx"]), int(c["by"]), int(c["distinct"]), int(c["raw"]),
             [int(i) for i in ids]) for c, ids in zip(cands, id_lists)]
