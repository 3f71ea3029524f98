"""Brute-force shift-and-stack in pure Python -- TEST INFRASTRUCTURE (tiny inputs).

A second formulation of Sec. 2.1 steps 1-3, written independently of
sas_oracle.c: Python integers (unbounded, '//' is the mathematical floor), one
dictionary keyed by (v_idx, bx, by) holding the set of epochs and the list of
detection ids.  It exists to pin the C oracle, not to be fast.
"""
from __future__ import annotations


def search(x, y, epoch, t, tph, grid, n_min):
    """Return (candidates, n_pairs); candidates is a list of
    (v_idx, bx, by, distinct, raw, ids) in the output order
    distinct desc, raw desc, v_idx asc, by asc, bx asc."""
    x = [int(a) for a in x]
    y = [int(a) for a in y]
    epoch = [int(a) for a in epoch]
    t = [int(a) for a in t]
    t_ref = min(t[e] for e in epoch) if epoch else 0   # Sec. 2.1 step 1
    cells = {}
    n_pairs = 0
    for ky in range(grid.nvy):
        for kx in range(grid.nvx):
            vx = grid.vx0 + kx * grid.dvx
            vy = grid.vy0 + ky * grid.dvy
            if (grid.speed_min, grid.speed_max) != (0, 0):
                s2 = vx * vx + vy * vy
                if s2 < grid.speed_min ** 2 or s2 > grid.speed_max ** 2:
                    continue
            v_idx = ky * grid.nvx + kx
            for i in range(len(x)):
                dt = t[epoch[i]] - t_ref
                px = x[i] - (vx * dt) // tph          # position at the reference epoch
                py = y[i] - (vy * dt) // tph
                bx = (px - grid.x_min) // grid.bin
                by = (py - grid.y_min) // grid.bin
                if 0 <= bx < grid.nbx and 0 <= by < grid.nby:
                    n_pairs += 1
                    ep, ids = cells.setdefault((v_idx, bx, by), (set(), []))
                    ep.add(epoch[i])
                    ids.append(i)
    out = []
    for (v_idx, bx, by), (ep, ids) in cells.items():
        if len(ep) >= n_min:
            out.append((v_idx, bx, by, len(ep), len(ids), sorted(ids)))
    out.sort(key=lambda c: (-c[3], -c[4], c[0], c[2], c[1]))
    return out, n_pairs
