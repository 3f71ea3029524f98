"""Seeded synthetic detection catalogs shaped like the paper's DECam searches.

This module only draws inputs: positions, epochs, times and the truth table of
injected movers.  It holds none of the stacking arithmetic (no projection, no
binning, no counting), so both the CUDA path and the CPU oracle can consume the
same arrays without sharing any of the method.

Units (fixed-point, so that shift-and-bin is pure integer work):
  * positions  : int32 milli-pixels (mpx) in a local tangent plane (x = RA-like,
                 y = Dec-like), Eq. 1-2 of Sec. 2;
  * velocities : int32 milli-pixels per hour (mpx/h);
  * times      : int64 ticks, ``ticks_per_hour`` = 3600 (seconds); the time of an
                 exposure is its midpoint (Sec. 3.2).

Workload recipes (field geometry from Sec. 3.1-3.3: one 2048x4096 CCD, ~100
exposures over ~4 h, TNO and MBA rate ranges of Sec. 3.3 converted at
0.263 arcsec/px):

  tiny            512x512 px, 20 epochs / 4 h, 200 noise/epoch, 3 movers 1-10 px/h,
                  p=0.6, 0.5 px jitter; lattice 21x21 step 1000 mpx/h; bin 4 px; N_min 8
  decam_tno       2048x4096 px, 100 epochs / 4 h, 3000 noise/epoch, 200 movers
                  0.5-20 px/h, m~U[23,25.5], p 0.9->0.3 linear in m; lattice 111x111
                  step 364 mpx/h (+-20.02 px/h); bin 2 px; N_min 25
  fast_movers     same CCD, 60 epochs / 1.5 h, 5000 noise/epoch, 100 movers 20-300 px/h;
                  lattice 1001x1001 step 600 mpx/h (+-300 px/h); bin 3 px; N_min 15
  batched_fields  60 CCD fields, epochs U{20..150} over 4 h, noise/epoch log-U[1e3,8e3],
                  movers and lattice as decam_tno; bin 2 px; N_min = ceil(E/4)
  vetter_fields   as batched_fields with magnitudes U[23,26.5] (p 0.9 -> 0.06)
"""
from __future__ import annotations

import dataclasses
import hashlib
import math
from typing import List, Optional

import numpy as np

TICKS_PER_HOUR = 3600
MPX = 1000  # milli-pixels per pixel


@dataclasses.dataclass(frozen=True)
class GridSpec:
    """Velocity lattice and histogram domain (the search set V of Sec. 2.1 and the
    bin size Delta-x).  Lattice point (kx, ky) has velocity (vx0 + kx*dvx,
    vy0 + ky*dvy) mpx/h and index v_idx = ky*nvx + kx.  The histogram domain is
    [x_min, x_min + nbx*bin) x [y_min, y_min + nby*bin) mpx with half-open bins.
    speed_min/speed_max (mpx/h) select an annulus of the lattice; 0, 0 means all."""
    vx0: int
    vy0: int
    dvx: int
    dvy: int
    nvx: int
    nvy: int
    x_min: int
    y_min: int
    nbx: int
    nby: int
    bin: int
    speed_min: int = 0
    speed_max: int = 0

    @property
    def n_velocities(self) -> int:
        return self.nvx * self.nvy


@dataclasses.dataclass
class Catalog:
    """Structure-of-arrays detection catalog C = [x_i, y_i, t_i] (Sec. 2.1).
    ``epoch[i]`` indexes ``t``; ``mover[i]`` is the injected mover that made
    detection i, -1 for a noise peak or STATIC (-2) for a stationary artifact
    (truth, not an input of the method)."""
    x: np.ndarray          # int32 [n]
    y: np.ndarray          # int32 [n]
    epoch: np.ndarray      # uint16 [n]
    t: np.ndarray          # int64 [E]
    ticks_per_hour: int
    mover: np.ndarray      # int32 [n]
    movers: np.ndarray     # structured [n_movers]: x0, y0, vx, vy (mpx, mpx/h), mag, p
    width_px: int
    height_px: int

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    @property
    def n_epochs(self) -> int:
        return int(self.t.shape[0])

    def sha256(self) -> str:
        h = hashlib.sha256()
        for a in (self.x, self.y, self.epoch, self.t):
            h.update(np.ascontiguousarray(a).tobytes())
        return h.hexdigest()


@dataclasses.dataclass(frozen=True)
class FieldRecipe:
    width_px: int
    height_px: int
    n_epochs: int
    span_h: float
    noise_per_epoch: int
    n_movers: int
    speed_px_h: tuple          # (lo, hi) uniform speed, random direction
    p_detect: tuple            # (p_bright, p_faint) linear in magnitude over mag range
    mag_range: tuple = (23.0, 25.5)
    jitter_px: float = 0.5
    n_static: int = 0          # stationary artifacts (fixed position, detected with p_static)
    p_static: tuple = (0.5, 1.0)


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    recipe: FieldRecipe
    grid: GridSpec
    n_min: int
    seed: int


STATIC = -2  # Catalog.mover value of a stationary artifact's detection

MOVER_DTYPE = np.dtype([("x0", "f8"), ("y0", "f8"), ("vx", "f8"), ("vy", "f8"),
                        ("mag", "f8"), ("p", "f8")])


def epoch_times(n_epochs: int, span_h: float) -> np.ndarray:
    """Evenly spaced exposure midpoints t_e = floor(e*T/(E-1)) seconds."""
    span = int(round(span_h * TICKS_PER_HOUR))
    if n_epochs == 1:
        return np.zeros(1, np.int64)
    e = np.arange(n_epochs, dtype=np.int64)
    return (e * span) // (n_epochs - 1)


def make_catalog(recipe: FieldRecipe, seed: int, mag_range: Optional[tuple] = None) -> Catalog:
    """Draw one field: uniform noise peaks per epoch plus linear movers (Eq. 1-2)
    detected per epoch with probability p(m), with Gaussian astrometric jitter."""
    rng = np.random.default_rng(seed)
    W, H, E = recipe.width_px * MPX, recipe.height_px * MPX, recipe.n_epochs
    t = epoch_times(E, recipe.span_h)
    mr = mag_range or recipe.mag_range
    nm = recipe.n_movers
    movers = np.zeros(nm, MOVER_DTYPE)
    movers["x0"] = rng.uniform(0, W, nm)
    movers["y0"] = rng.uniform(0, H, nm)
    speed = rng.uniform(recipe.speed_px_h[0], recipe.speed_px_h[1], nm) * MPX
    ang = rng.uniform(0, 2 * np.pi, nm)
    movers["vx"] = speed * np.cos(ang)
    movers["vy"] = speed * np.sin(ang)
    movers["mag"] = rng.uniform(mr[0], mr[1], nm)
    pb, pf = recipe.p_detect
    lo, hi = recipe.mag_range
    frac = np.clip((movers["mag"] - lo) / (hi - lo), 0.0, None) if hi > lo else np.zeros(nm)
    movers["p"] = np.clip(pb + (pf - pb) * frac, 0.0, 1.0)

    # stationary artifacts draw from their own stream, so fields without them
    # are unchanged
    ns = recipe.n_static
    if ns:
        srng = np.random.default_rng([seed, 7919])
        sx0 = srng.uniform(0, W, ns)
        sy0 = srng.uniform(0, H, ns)
        sp = srng.uniform(recipe.p_static[0], recipe.p_static[1], ns)

    xs, ys, es, ms = [], [], [], []
    t0 = t.min()
    for e in range(E):
        nn = recipe.noise_per_epoch
        xe = rng.integers(0, W, nn, dtype=np.int64)
        ye = rng.integers(0, H, nn, dtype=np.int64)
        me = np.full(nn, -1, np.int64)
        if nm:
            dt_h = (t[e] - t0) / TICKS_PER_HOUR
            px = movers["x0"] + movers["vx"] * dt_h + rng.normal(0, recipe.jitter_px * MPX, nm)
            py = movers["y0"] + movers["vy"] * dt_h + rng.normal(0, recipe.jitter_px * MPX, nm)
            det = rng.random(nm) < movers["p"]
            px, py = np.rint(px).astype(np.int64), np.rint(py).astype(np.int64)
            inside = det & (px >= 0) & (px < W) & (py >= 0) & (py < H)
            idx = np.nonzero(inside)[0]
            xe = np.concatenate([xe, px[idx]])
            ye = np.concatenate([ye, py[idx]])
            me = np.concatenate([me, idx])
        if ns:
            det = srng.random(ns) < sp
            qx = np.rint(sx0 + srng.normal(0, recipe.jitter_px * MPX, ns)).astype(np.int64)
            qy = np.rint(sy0 + srng.normal(0, recipe.jitter_px * MPX, ns)).astype(np.int64)
            keep = det & (qx >= 0) & (qx < W) & (qy >= 0) & (qy < H)
            xe = np.concatenate([xe, qx[keep]])
            ye = np.concatenate([ye, qy[keep]])
            me = np.concatenate([me, np.full(int(keep.sum()), STATIC, np.int64)])
        perm = rng.permutation(xe.shape[0])   # catalog order shuffled within an epoch
        xs.append(xe[perm]); ys.append(ye[perm]); ms.append(me[perm])
        es.append(np.full(xe.shape[0], e, np.int64))
    return Catalog(
        x=np.concatenate(xs).astype(np.int32), y=np.concatenate(ys).astype(np.int32),
        epoch=np.concatenate(es).astype(np.uint16), t=t, ticks_per_hour=TICKS_PER_HOUR,
        mover=np.concatenate(ms).astype(np.int32), movers=movers,
        width_px=recipe.width_px, height_px=recipe.height_px)


def field_grid(width_px: int, height_px: int, bin_mpx: int, step: int, half: int) -> GridSpec:
    """Square lattice k in [-half, half] with the given step, over the field at t0."""
    n = 2 * half + 1
    return GridSpec(vx0=-half * step, vy0=-half * step, dvx=step, dvy=step, nvx=n, nvy=n,
                    x_min=0, y_min=0, nbx=-(-width_px * MPX // bin_mpx),
                    nby=-(-height_px * MPX // bin_mpx), bin=bin_mpx)


BASE_SEED = 20250926


def tiny() -> Workload:
    r = FieldRecipe(512, 512, 20, 4.0, 200, 3, (1.0, 10.0), (0.6, 0.6))
    return Workload("tiny", r, field_grid(512, 512, 4000, 1000, 10), 8, BASE_SEED + 1)


def decam_tno() -> Workload:
    r = FieldRecipe(2048, 4096, 100, 4.0, 3000, 200, (0.5, 20.0), (0.9, 0.3))
    return Workload("decam_tno", r, field_grid(2048, 4096, 2000, 364, 55), 25, BASE_SEED + 2)


def fast_movers() -> Workload:
    r = FieldRecipe(2048, 4096, 60, 1.5, 5000, 100, (20.0, 300.0), (0.9, 0.3))
    return Workload("fast_movers", r, field_grid(2048, 4096, 3000, 600, 500), 15, BASE_SEED + 3)


def batched_fields(n_fields: int = 60, seed: int = BASE_SEED + 4) -> List[Workload]:
    """Uneven fields: epochs U{20..150}, noise/epoch log-uniform in [1e3, 8e3]."""
    rng = np.random.default_rng(seed)
    out = []
    for f in range(n_fields):
        E = int(rng.integers(20, 151))
        noise = int(round(math.exp(rng.uniform(math.log(1e3), math.log(8e3)))))
        r = FieldRecipe(2048, 4096, E, 4.0, noise, 200, (0.5, 20.0), (0.9, 0.3))
        out.append(Workload(f"batched_fields[{f}]", r, field_grid(2048, 4096, 2000, 364, 55),
                            -(-E // 4), seed * 1000 + f))
    return out


def vetter_fields(n_fields: int, seed: int = BASE_SEED + 5) -> List[Workload]:
    """Fields for training and judging the candidate vetter: the geometry,
    lattice and bin of decam_tno with the batched spread of epochs (U{20..150})
    and noise (log-U[1e3, 8e3]); mover magnitudes extended to U[23, 26.5] with
    the same detection-probability slope (p = 0.9 at m = 23 down to 0.06 at
    m = 26.5).  n_min is the plain threshold ceil(E/4).  (Stationary artifacts
    are left out: a count stamp holds no absolute velocity, so a source at rest
    looks like a mover at its own velocity; the search's speed annulus is what
    excludes them.)"""
    rng = np.random.default_rng(seed)
    out = []
    for f in range(n_fields):
        E = int(rng.integers(20, 151))
        noise = int(round(math.exp(rng.uniform(math.log(1e3), math.log(8e3)))))
        r = FieldRecipe(2048, 4096, E, 4.0, noise, 200, (0.5, 20.0), (0.9, 0.06),
                        mag_range=(23.0, 26.5))
        out.append(Workload(f"vetter_fields[{f}]", r, field_grid(2048, 4096, 2000, 364, 55),
                            -(-E // 4), seed * 1000 + f))
    return out


def scaled(w: Workload, frac_noise: float = 1.0, n_epochs: Optional[int] = None,
           width_px: Optional[int] = None, height_px: Optional[int] = None,
           n_movers: Optional[int] = None, grid_half: Optional[int] = None,
           seed: Optional[int] = None) -> Workload:
    """A smaller copy of a workload (same structure) for parity tests."""
    r = w.recipe
    r2 = dataclasses.replace(
        r, noise_per_epoch=int(round(r.noise_per_epoch * frac_noise)),
        n_epochs=n_epochs or r.n_epochs, width_px=width_px or r.width_px,
        height_px=height_px or r.height_px,
        n_movers=r.n_movers if n_movers is None else n_movers)
    g = w.grid
    half = (g.nvx - 1) // 2 if grid_half is None else grid_half
    g2 = field_grid(r2.width_px, r2.height_px, g.bin, g.dvx, half)
    return Workload(w.name + "_scaled", r2, g2, w.n_min, w.seed if seed is None else seed)


def snr_weights(cat: Catalog, nu_th: float = 5.0, scale: float = 8.0, seed: int = BASE_SEED + 6) -> np.ndarray:
    """Synthetic detection weights for weighted stacking: round(scale * S/N),
    clipped to [0, 255].  A mover detected with probability p has true S/N
    nu = nu_th + sqrt(2) erfcinv(2 (1 - p)) (so that P(observed >= nu_th) = p)
    and observed S/N nu + N(0, 1) redrawn until it is >= nu_th; a noise peak's
    observed S/N is nu_th + an exponential tail with rate nu_th (the shape of
    a Gaussian field's peak heights far above nu_th).  Inputs only."""
    from scipy.special import erfcinv
    rng = np.random.default_rng(seed)
    n = len(cat.x)
    nu_obs = nu_th + rng.exponential(1.0 / nu_th, n)
    mv = np.nonzero(cat.mover >= 0)[0]
    if len(mv) and len(cat.movers):
        p = np.clip(cat.movers["p"][cat.mover[mv]], 1e-6, 1 - 1e-6)
        nu = nu_th + np.sqrt(2.0) * erfcinv(2.0 * (1.0 - p))
        obs = nu + rng.standard_normal(len(mv))
        bad = obs < nu_th
        while bad.any():
            obs[bad] = nu[bad] + rng.standard_normal(int(bad.sum()))
            bad = obs < nu_th
        nu_obs[mv] = obs
    return np.clip(np.rint(scale * nu_obs), 0, 255).astype(np.uint8)


def load(w: Workload) -> Catalog:
    return make_catalog(w.recipe, w.seed)
