"""CPU oracle of the two-threshold search with tile-local super-bin peaks --
TEST INFRASTRUCTURE.

Below the paper's threshold N_min (Sec. 2.1 step 3) a fainter mover is still
a cell with many distinct epochs, but a lowered threshold n_low also admits
every neighbouring velocity and bin of each bright mover and of each noise
alignment (the velocity tolerance of Sec. 2.2 spans several lattice steps).
The library's extension keeps, besides every cell with >= N_min distinct
epochs, the cells with >= n_low distinct epochs whose super-bin is a peak of
the raw counts within its tile.  Definitions, in the order they are used:

  super-bin B = (sbx, sby): the S x S bins bx in [S sbx, S sbx + S),
      by in [S sby, S sby + S) of the histogram domain (Sec. 2.1 step 2);
  R(v, B): the detections whose projection at lattice point v lands in one
      of B's bins (the raw counts of Sec. 2.1 step 2 summed over B); 0 for a
      lattice point outside the searched set (index range, speed bounds);
  tiles: lattice point (kx, ky) lies in velocity tile
      (kx // KX, (ky - ky_lo) // KY) with ky_lo = v_begin // nvx, super-bin
      B in spatial tile (sbx // TX, sby // TY);
  peak: B at v is a tile-local peak when no (v', B') in the same velocity
      tile and the same spatial tile, with every one of |kx' - kx|,
      |ky' - ky|, |sbx' - sbx|, |sby' - sby| at most 1, has
      R(v', B') > R(v, B);
  result: every cell (v, bx, by) with distinct >= N_min, and every cell with
      distinct >= n_low whose super-bin (bx // S, by // S) at v is a peak, in
      the search's output order (distinct desc, raw desc, v_idx, by, bx);
  peaks only: the cells with distinct >= n_low whose super-bin is a peak,
      and no others (the cells at or above N_min elsewhere, the neighbourhood
      a mover raises around its best cells, are left out as well).

R is taken from the oracle's dense raw histograms (oracle.histogram), the
cells and their ids from the oracle's search at n_low (oracle.stack); no code
is shared with the library.

Parity status: pinned in tests/test_oracle_lowpeaks.py (a pure-Python brute
force over dictionaries of epoch sets with its own neighbourhood loop, the
special cases n_low = N_min and one-point tiles, containment between the
plain searches at N_min and n_low, and hand-built movers).
"""
from __future__ import annotations

import numpy as np

from . import OracleResult, histogram, stack


def velocity_active(grid, kx: int, ky: int, v_begin: int, v_end: int) -> bool:
    """Whether lattice point (kx, ky) is searched: index in [v_begin, v_end)
    and, with speed bounds, speed_min^2 <= vx^2 + vy^2 <= speed_max^2."""
    v = ky * grid.nvx + kx
    if not (v_begin <= v < v_end):
        return False
    if (grid.speed_min, grid.speed_max) == (0, 0):
        return True
    vx = grid.vx0 + kx * grid.dvx
    vy = grid.vy0 + ky * grid.dvy
    s2 = vx * vx + vy * vy
    return grid.speed_min ** 2 <= s2 <= grid.speed_max ** 2


class SuperbinCounts:
    """R(v, B) for the lattice points asked for, one dense [nsy, nsx] array
    per lattice point, computed on first use."""

    def __init__(self, cat, grid, s: int, v_begin: int = 0, v_end: int | None = None):
        self.cat, self.grid, self.s = cat, grid, int(s)
        self.v_begin = int(v_begin)
        self.v_end = int(grid.nvx * grid.nvy if v_end is None else v_end)
        self.nsx = -(-grid.nbx // self.s)
        self.nsy = -(-grid.nby // self.s)
        self._cache = {}

    def at(self, kx: int, ky: int) -> np.ndarray:
        key = (kx, ky)
        if key not in self._cache:
            g, s = self.grid, self.s
            r = np.zeros((self.nsy, self.nsx), np.int64)
            if velocity_active(g, kx, ky, self.v_begin, self.v_end):
                _, raw = histogram(self.cat, g, g.vx0 + kx * g.dvx, g.vy0 + ky * g.dvy)
                pad = np.zeros((self.nsy * s, self.nsx * s), np.int64)
                pad[: g.nby, : g.nbx] = raw
                r = pad.reshape(self.nsy, s, self.nsx, s).sum(axis=(1, 3))
            self._cache[key] = r
        return self._cache[key]


def is_peak(R: SuperbinCounts, kx: int, ky: int, sbx: int, sby: int, tiles: dict) -> bool:
    """Tile-local peak test of super-bin (sbx, sby) at lattice point (kx, ky);
    tiles = {"kx": KX, "ky": KY, "bx": TX, "by": TY}."""
    g = R.grid
    ky_lo = R.v_begin // g.nvx
    vt = (kx // tiles["kx"], (ky - ky_lo) // tiles["ky"])
    st = (sbx // tiles["bx"], sby // tiles["by"])
    me = R.at(kx, ky)[sby, sbx]
    for ky2 in (ky - 1, ky, ky + 1):
        for kx2 in (kx - 1, kx, kx + 1):
            if not (0 <= kx2 < g.nvx and 0 <= ky2 < g.nvy):
                continue
            if (kx2 // tiles["kx"], (ky2 - ky_lo) // tiles["ky"]) != vt:
                continue
            r = R.at(kx2, ky2)
            for sby2 in (sby - 1, sby, sby + 1):
                for sbx2 in (sbx - 1, sbx, sbx + 1):
                    if not (0 <= sbx2 < R.nsx and 0 <= sby2 < R.nsy):
                        continue
                    if (sbx2 // tiles["bx"], sby2 // tiles["by"]) != st:
                        continue
                    if r[sby2, sbx2] > me:
                        return False
    return True


def subset(res: OracleResult, keep: np.ndarray) -> OracleResult:
    """The candidates of res where keep is True, in the same order, with their
    id lists copied into a new id array."""
    c = res.cands[keep].copy()
    parts = [res.ids[int(a["id_off"]): int(a["id_off"]) + int(a["id_len"])] for a in c]
    off = np.cumsum([0] + [len(p) for p in parts])[:-1]
    c["id_off"] = off
    ids = np.concatenate(parts) if parts else np.zeros(0, res.ids.dtype)
    return OracleResult(c, ids, res.n_pairs)


def search(cat, grid, n_min: int, n_low: int, tiles: dict, v_begin: int = 0, v_end: int | None = None,
           threads: int = 1, peaks_only: bool = False) -> OracleResult:
    """The two-threshold search: oracle.stack at n_low, then each cell kept when
    distinct >= n_min (unless peaks_only) or its super-bin is a tile-local
    peak.  tiles = {"kx", "ky", "bx", "by", "s"} (velocity tile, spatial tile
    in super-bins, super-bin side in bins)."""
    if v_end is None:
        v_end = grid.nvx * grid.nvy
    low = stack(cat, grid, n_low, v_begin, v_end, threads=threads)
    if n_low >= n_min and not peaks_only:
        return low
    R = SuperbinCounts(cat, grid, tiles["s"], v_begin, v_end)
    keep = np.zeros(len(low.cands), bool)
    peak_of = {}
    for i, c in enumerate(low.cands):
        if int(c["distinct"]) >= n_min and not peaks_only:
            keep[i] = True
            continue
        v = int(c["v_idx"])
        kx, ky = v % grid.nvx, v // grid.nvx
        sb = (int(c["bx"]) // tiles["s"], int(c["by"]) // tiles["s"])
        key = (v, sb)
        if key not in peak_of:
            peak_of[key] = is_peak(R, kx, ky, sb[0], sb[1], tiles)
        keep[i] = peak_of[key]
    return subset(low, keep)


def tiles_of(info: dict) -> dict:
    """The tile geometry a search ran with, from its result info."""
    return {"kx": int(info["tile_kx"]), "ky": int(info["tile_ky"]), "bx": int(info["tile_bx"]),
            "by": int(info["tile_by"]), "s": int(info["superbin"])}
