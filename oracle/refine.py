"""CPU oracle of refinement and gathering (Sec. 2.1 steps 4-6) -- TEST
INFRASTRUCTURE.

Each cluster's detections are points z = (t, x, y): t the epoch's time minus the
reference epoch t0 in ticks, x and y in mpx, all integers.  Refinement fits a
linear trajectory by multivariate regression of Y = (x, y) on X = t (Sec. 2.1,
the regression equations), with the mean and covariance taken from the Minimum
Covariance Determinant subset (the robust estimate the paper prescribes),
found by FAST-MCD (Rousseeuw & Van Driessen 1999): random (d+1)-subsets,
C-steps, the best starts iterated to convergence.  Gathering collects every
detection of the catalog within the radius of the fitted line at its own epoch;
the two repeat until the gathered set no longer changes.

Arithmetic (both sides take every decision in the same precision): the moment
sums of a subset are exact integers (Python ints here), and so is the scatter
matrix S = m * sum(z z^T) - sum(z) sum(z)^T; its entries are rounded to float64
once, and every later quantity is a fixed float64 expression, evaluated in the
order written below with IEEE rounding after every operation (no fused
multiply-add).  A C-step ranks the points by q = u^T adj(S) u, u = m z - sum(z)
(an exact integer vector): for det(S) > 0 that is the squared Mahalanobis
distance times a positive constant, so the ranking is the MCD's.  Ranks order
(q, index); q is compared through its order-preserving 64-bit key.

Random draws come from a counter-based SplitMix64 (Steele, Lea & Flood 2014):
word j of start s of cluster k in refinement iteration it is
    mix(key + (j+1) g),  key = mix(mix(mix(seed + (k+1) g) + (it+1) g) + (s+1) g)
(g = 0x9E3779B97F4A7C15, mix = SplitMix64's output function, arithmetic mod
2^64).  A start's subset is a partial Fisher-Yates shuffle of 0..n-1 whose
step j swaps position j with j + word_j mod (n - j).

Readings (where the paper is silent): h = floor((n + d + 1)/2) with d = 3;
clusters with fewer than d + 2 points are fitted by least squares on all of
them; a start whose subset stays singular (det <= 0) up to h points is an
exact fit and keeps that subset; C-steps stop at the first step that does not
lower det; the raw MCD subset (no consistency factor, no reweighting) gives the
mean and covariance; gathered = squared distance to the line's position at the
detection's epoch <= radius^2; iteration stops when the gathered set equals the
fitted one, or after max_iter fits.

Parity status: pinned (tests/test_oracle_refine.py: SplitMix64 test vector,
least squares against numpy.linalg.lstsq, exact MCD by enumeration on small
sets, C-step monotonicity, robust recovery under 40 % outliers, gathering
against a brute-force scan).
"""
from __future__ import annotations

import dataclasses

import numpy as np

M64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15
D = 3

# status codes (the library's SAS_TRACK_* values)
CONVERGED, MAX_ITER, DEGENERATE, TOO_MANY = 0, 1, 2, 3


def mix64(z: int) -> int:
    """SplitMix64's output function."""
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def splitmix64(seed: int, count: int):
    """The generator as published: state += g, output mix(state)."""
    s, out = seed & M64, []
    for _ in range(count):
        s = (s + GOLDEN) & M64
        out.append(mix64(s))
    return out


def start_key(seed: int, k: int, it: int, s: int) -> int:
    a = mix64((seed + (k + 1) * GOLDEN) & M64)
    b = mix64((a + (it + 1) * GOLDEN) & M64)
    return mix64((b + (s + 1) * GOLDEN) & M64)


def word(key: int, j: int) -> int:
    return mix64((key + (j + 1) * GOLDEN) & M64)


# ---- exact moments and the fixed float64 expressions ---------------------------

@dataclasses.dataclass
class Fit:
    m: int
    sums: tuple          # (T, X, Y) exact
    S: tuple             # (s00, s01, s02, s11, s12, s22) float64 of the exact scatter
    S_exact: tuple
    adj: tuple           # (a00, a01, a02, a11, a12, a22)
    det: float


def fit(pts, members) -> Fit:
    """Exact moments of the subset, scatter S rounded once, adjugate and
    determinant by the fixed expressions."""
    t = [int(pts[i][0]) for i in members]
    x = [int(pts[i][1]) for i in members]
    y = [int(pts[i][2]) for i in members]
    m = len(members)
    T, X, Y = sum(t), sum(x), sum(y)

    def sc(a, b, sa, sb):
        return m * sum(p * q for p, q in zip(a, b)) - sa * sb

    Se = (sc(t, t, T, T), sc(t, x, T, X), sc(t, y, T, Y), sc(x, x, X, X), sc(x, y, X, Y), sc(y, y, Y, Y))
    s00, s01, s02, s11, s12, s22 = (np.float64(float(v)) for v in Se)
    a00 = s11 * s22 - s12 * s12
    a01 = s02 * s12 - s01 * s22
    a02 = s01 * s12 - s02 * s11
    a11 = s00 * s22 - s02 * s02
    a12 = s01 * s02 - s00 * s12
    a22 = s00 * s11 - s01 * s01
    det = (s00 * a00 + s01 * a01) + s02 * a02
    return Fit(m, (T, X, Y), (s00, s01, s02, s11, s12, s22), Se, (a00, a01, a02, a11, a12, a22), det)


def order_key(q: np.ndarray) -> np.ndarray:
    """Order-preserving map of float64 to uint64."""
    b = np.asarray(q, np.float64).view(np.uint64)
    neg = (b >> np.uint64(63)) == np.uint64(1)
    return np.where(neg, ~b, b | np.uint64(1 << 63))


def c_rank(pts_arr, F: Fit) -> np.ndarray:
    """q_i = u_i^T adj(S) u_i for every point, in the fixed order
    w_r = (a_r0 u0 + a_r1 u1) + a_r2 u2,  q = (u0 w0 + u1 w1) + u2 w2."""
    T, X, Y = F.sums
    m = F.m
    u0 = (m * pts_arr[:, 0] - T).astype(np.float64)   # exact: |u| < 2^53 (int64 products)
    u1 = (m * pts_arr[:, 1] - X).astype(np.float64)
    u2 = (m * pts_arr[:, 2] - Y).astype(np.float64)
    a00, a01, a02, a11, a12, a22 = F.adj
    w0 = (a00 * u0 + a01 * u1) + a02 * u2
    w1 = (a01 * u0 + a11 * u1) + a12 * u2
    w2 = (a02 * u0 + a12 * u1) + a22 * u2
    return (u0 * w0 + u1 * w1) + u2 * w2


def c_select(pts_arr, F: Fit, h: int):
    """The h points of smallest (q, index)."""
    key = order_key(c_rank(pts_arr, F))
    order = np.lexsort((np.arange(len(key)), key))
    return sorted(int(i) for i in order[:h])


def run_start(pts, pts_arr, h, key, max_steps):
    """One FAST-MCD start: the (d+1)-subset drawn from the counter words
    (extended one draw at a time while singular), the h nearest points, then
    C-steps while det decreases (at most max_steps)."""
    n = len(pts)
    perm = list(range(n))
    j = 0

    def draw():
        nonlocal j
        r = j + word(key, j) % (n - j)
        perm[j], perm[r] = perm[r], perm[j]
        j += 1

    for _ in range(D + 1):
        draw()
    F = fit(pts, perm[:j])
    while F.det <= 0 and j < h:
        draw()
        F = fit(pts, perm[:j])
    if F.det <= 0:
        H = sorted(perm[:j])
        return H, F
    H = c_select(pts_arr, F, h)
    F = fit(pts, H)
    for _ in range(max_steps):
        if F.det <= 0:
            break
        H2 = c_select(pts_arr, F, h)
        F2 = fit(pts, H2)
        if not F2.det < F.det:
            break
        H, F = H2, F2
    return H, F


def fast_mcd(pts, seed, k, it, n_starts=500, n_best=10, max_csteps=100):
    """FAST-MCD (small-sample form): every start takes two C-steps; the n_best
    lowest determinants (ties: lower start index) continue to convergence; the
    lowest final determinant wins (ties: lower start index).  Returns (h-subset,
    Fit).  Fewer than d + 2 points: all of them."""
    n = len(pts)
    if n < D + 2:
        H = list(range(n))
        return H, fit(pts, H)
    h = (n + D + 1) // 2
    pts_arr = np.array(pts, dtype=np.int64)
    dets = []
    for s in range(n_starts):
        _, F = run_start(pts, pts_arr, h, start_key(seed, k, it, s), 2)
        dets.append((float(F.det), s))
    best = sorted(dets)[:n_best]
    final = []
    for _, s in best:
        H, F = run_start(pts, pts_arr, h, start_key(seed, k, it, s), max_csteps)
        final.append((float(F.det), s, H, F))
    final.sort(key=lambda r: (r[0], r[1]))
    return final[0][2], final[0][3]


# ---- the line, gathering, the loop -------------------------------------------

@dataclasses.dataclass
class Line:
    vxt: float      # mpx per tick
    vyt: float
    x0: float       # mpx at t = 0 (the reference epoch)
    y0: float
    res: tuple      # residual covariance (xx, xy, yy) of the subset, mpx^2, biased


def line_of(F: Fit):
    """Regression on the subset: slope = S_tx / S_tt, intercept from the
    subset means, residual covariance S_YY - S_YX S_XX^-1 S_XY over m^2.
    None when S_tt = 0 (a single epoch: no slope)."""
    s00, s01, s02, s11, s12, s22 = F.S
    if F.S_exact[0] == 0:
        return None
    T, X, Y = F.sums
    m = np.float64(F.m)
    vxt = s01 / s00
    vyt = s02 / s00
    x0 = (np.float64(X) - vxt * np.float64(T)) / m
    y0 = (np.float64(Y) - vyt * np.float64(T)) / m
    mm = m * m
    res = ((s11 - vxt * s01) / mm, (s12 - vxt * s02) / mm, (s22 - vyt * s02) / mm)
    return Line(vxt, vyt, x0, y0, res)


def gather(line: Line, t_ticks, x, y, radius: int):
    """Ids of every detection within the radius of the line at its epoch:
    p = x0 + vxt t, r = x - p, (rx rx + ry ry) <= radius^2."""
    tt = np.asarray(t_ticks, np.float64)
    px = line.x0 + line.vxt * tt
    py = line.y0 + line.vyt * tt
    rx = np.asarray(x, np.float64) - px
    ry = np.asarray(y, np.float64) - py
    d2 = rx * rx + ry * ry
    r2 = np.float64(radius) * np.float64(radius)
    return [int(i) for i in np.nonzero(d2 <= r2)[0]]


@dataclasses.dataclass
class Track:
    status: int
    iterations: int
    line: Line | None
    det: float
    h: int
    n_points: int        # points of the last fit
    ids: list            # the last gathering (the cluster's ids when nothing was fitted)


def refine(ids, t_ticks, x, y, radius, seed, k, max_iter=10, n_starts=500, n_best=10, max_csteps=100,
           max_points=1024):
    """Steps 4-6 for cluster k: fit, gather, repeat until the gathered set is
    the fitted set (at most max_iter fits).  t_ticks, x, y are per detection id
    (the whole catalog)."""
    P = sorted(int(i) for i in ids)
    line, det, h, it = None, 0.0, 0, 0
    if len(P) > max_points:
        return Track(TOO_MANY, 0, None, 0.0, 0, len(P), P)
    for it in range(max_iter):
        pts = [(int(t_ticks[i]), int(x[i]), int(y[i])) for i in P]
        H, F = fast_mcd(pts, seed, k, it, n_starts, n_best, max_csteps)
        ln = line_of(F)
        if ln is None:
            return Track(DEGENERATE, it + 1, None, float(F.det), len(H), len(P), P)
        line, det, h = ln, float(F.det), len(H)
        G = gather(ln, t_ticks, x, y, radius)
        n_fit = len(P)
        if G == P:
            return Track(CONVERGED, it + 1, line, det, h, n_fit, G)
        if len(G) > max_points:
            return Track(TOO_MANY, it + 1, line, det, h, n_fit, P)
        if len(G) < 2:
            return Track(DEGENERATE, it + 1, line, det, h, n_fit, G)
        P = G
    return Track(MAX_ITER, max_iter, line, det, h, n_fit, P)


def exact_mcd_det(pts):
    """The exact MCD by enumeration of every h-subset (small n only): the
    minimum determinant of the exact integer scatter matrix (m^2 cov)."""
    from itertools import combinations
    n = len(pts)
    h = (n + D + 1) // 2
    best = None
    for H in combinations(range(n), h):
        F = fit(pts, list(H))
        s = F.S_exact
        det = (s[0] * (s[3] * s[5] - s[4] * s[4]) - s[1] * (s[1] * s[5] - s[4] * s[2])
               + s[2] * (s[1] * s[4] - s[3] * s[2]))
        if best is None or det < best[0]:
            best = (det, list(H))
    return best
