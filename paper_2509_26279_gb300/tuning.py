"""Per-size-class tile choices from the autotuner, cached as JSON.

sas_autotune times the whole search for each velocity tile (lattice points
per tile) x bin tile (super-bin side, spatial tile width) x velocity block on
one field and returns the fastest.  Fields of similar shape -- the same
lattice and bin, similar epoch count, detection density and threshold -- share
the answer, so a batch of many uneven fields is tuned once per size class and
each field takes its class's options.  The cache is a JSON object
{class key: {"tile_kx": kx, "tile_ky": ky, "superbin": s, "tile_bx": bx,
"tile_by": by, "velocity_block": b, "ms": t, "planner_ms": t0, "device": name}}
(0: the planner's choice for that field; planner_ms: the planner's own options
timed the same way on the same field)
that can be written to disk and reused across runs on the same GPU model.

Host logic only: the timing runs in the library (sas_autotune).
"""
from __future__ import annotations

import json
import math
import os
from typing import Dict, Optional

import numpy as np


OPTION_KEYS = ("tile_kx", "tile_ky", "superbin", "tile_bx", "tile_by", "velocity_block")


def shape_of(entry: dict) -> str:
    """A cache entry's choice as text: velocity tile x bin tile, velocity block."""
    return (f"{entry.get('tile_kx', 0)}x{entry.get('tile_ky', 0)} lattice points, super-bin {entry['superbin']}, "
            f"tile_bx {entry.get('tile_bx', 0) or 'planner'}, velocity block {entry['velocity_block'] or 'planner'}")


def size_class(n_epochs: int, n_detections: int, grid, n_min: int) -> str:
    """Class key: epochs in steps of 32, detections per epoch in octaves,
    lattice shape, bin, threshold as a fraction of the epochs in eighths."""
    e_cls = -(-n_epochs // 32)
    d_cls = int(round(math.log2(max(1.0, n_detections / max(1, n_epochs)))))
    f_cls = min(8, (8 * n_min) // max(1, n_epochs))
    return f"E{e_cls}-d{d_cls}-v{grid.nvx}x{grid.nvy}-b{grid.bin}-f{f_cls}"


class TuneCache:
    """Autotuned options per size class, optionally backed by a JSON file."""

    def __init__(self, path: Optional[str] = None):
        self.path = path
        self.entries: Dict[str, dict] = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.entries = json.load(f)

    def save(self, path: Optional[str] = None):
        path = path or self.path
        if not path:
            raise ValueError("no path to save the tuning cache to")
        d = os.path.dirname(os.path.abspath(path))
        os.makedirs(d, exist_ok=True)
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(self.entries, f, indent=1, sort_keys=True)
        os.replace(tmp, path)

    def lookup(self, key: str):
        return self.entries.get(key)

    def tune(self, field, device_name: str = "", reps: int = 3, base=None, tag: str = "") -> dict:
        """Entry of field's class, measured with sas_autotune if missing.
        field: an object with grid (sas.Grid), w (workload: grid spec, n_min),
        cat, dx, dy, de (device catalog) and E -- e.g. vetting.Field.  base:
        sas_opts the search runs with besides the tiles (e.g. n_low and
        peaks_only, which change what the tiles cost); tag: prefix of the class
        key that keeps such entries apart."""
        from . import sas
        key = tag + size_class(field.E, field.cat.n, field.w.grid, field.w.n_min)
        if key not in self.entries:
            best, ms = sas.sas_autotune(field.grid, field.dx, field.dy, field.de, field.cat.t,
                                        field.cat.ticks_per_hour, field.w.n_min, base=base, reps=reps)
            # the planner's own choice on the same field, timed the same way (device
            # time of the whole search, median of reps after one warm-up)
            ts = []
            for r in range(reps + 1):
                res = sas.sas_stack(field.grid, field.dx, field.dy, field.de, field.cat.t,
                                    field.cat.ticks_per_hour, field.w.n_min, on_device=True, opts=base)
                if r:
                    ts.append(res.info()["ms_total"])
                res.free()
            self.entries[key] = {"tile_kx": int(best.tile_kx), "tile_ky": int(best.tile_ky),
                                 "superbin": int(best.superbin), "tile_bx": int(best.tile_bx),
                                 "tile_by": int(best.tile_by), "velocity_block": int(best.velocity_block),
                                 "ms": round(float(ms), 4), "planner_ms": round(float(sorted(ts)[len(ts) // 2]), 4),
                                 "device": device_name}
        return self.entries[key]

    def opts_for(self, field, tag: str = ""):
        """sas_opts for a field from its class entry (planner defaults if none)."""
        from . import sas
        e = self.lookup(tag + size_class(field.E, field.cat.n, field.w.grid, field.w.n_min))
        if e is None:
            return sas.make_opts()
        return sas.make_opts(**{k: e.get(k, 0) for k in OPTION_KEYS})
