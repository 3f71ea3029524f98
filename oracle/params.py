"""CPU oracle of the search-parameter relations (Sec. 2.2) -- TEST
INFRASTRUCTURE.

* velocity_count: size of the velocity set that keeps every object of the
  target range within dx of some hypothesis over a baseline dt (Eq. v_size):
  each axis is stepped by dv = dx / dt.
* n_stacks = |V| * Omega / dx^2 (Eq. N_stacks); the false-positive budget is
  eps = N_false / N_stacks.
* peak_density(z, a): surface density of noise peaks per unit detection
  statistic z, for white sky noise under a Gaussian window of width a (PSF
  detection).  The printed closed form is garbled (it integrates to 0.85/a^2
  and goes negative), so this takes the quantity it stands for from its
  definition: the Kac-Rice density of local maxima of a 2-D isotropic Gaussian
  field at height z (spectral moments of that field: gamma = 1/sqrt(2),
  sigma2^2 / sigma1^2 = 2 / a^2), written out as a 2-D integral over the
  Hessian's trace and anisotropy.
* peaks_above(nu_th, a) = integral of peak_density from nu_th to infinity
  (Eq. n_pk_above); noise_rate sums it over epochs for a square bin of side dx.
* poisson_sf / choose_n_min: N_noise ~ Pois(Lambda); the smallest N_min with
  P(N_noise >= N_min) <= eps.
* p_signal: one epoch's probability that a source of S/N nu is detected above
  nu_th and lands in the square bin of side dx centred on its position
  (positional sigma^2 = 2 a^2 / nu^2 per axis); signal_tail: P(N_signal >= k)
  over epochs (Poisson-binomial).
* dx_scan: per bin size, E[N_signal], E[N_noise] and the N_min that the
  false-positive budget N_false / N_stacks requires (the paper's recipe for
  choosing dx and N_min).

Parity status: pinned (tests/test_oracle_params.py: Longuet-Higgins's total
density of maxima, a simulated smoothed random field, a lattice count,
scipy.stats.poisson, Monte Carlo of detection and binning, brute-force
Poisson-binomial).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate

GAMMA = 1.0 / math.sqrt(2.0)


def velocity_count(vmin_x, vmax_x, vmin_y, vmax_y, dx, dt):
    dv = dx / dt
    return ((vmax_x - vmin_x) / dv) * ((vmax_y - vmin_y) / dv)


def n_stacks(n_velocities, omega, dx):
    return n_velocities * omega / (dx * dx)


def peak_density(z, a=1.0):
    """Kac-Rice: p_f(z) * p_grad(0) * E[|det H| ; H < 0 | f = z].  In units of
    sigma2: the trace T = -(h11 + h22) given f = z is N(gamma z, 1 - gamma^2);
    the anisotropy D = |(h11 - h22, 2 h12)| is Rayleigh with density
    2 d exp(-d^2); H < 0 iff T > D, and det H = (T^2 - D^2) / 4.  With
    p_grad(0) = 1 / (pi sigma1^2) and sigma2^2 / sigma1^2 = 2 / a^2."""
    mu, s = GAMMA * z, math.sqrt(1.0 - GAMMA * GAMMA)

    def f(t, d):
        pt = math.exp(-0.5 * ((t - mu) / s) ** 2) / (s * math.sqrt(2 * math.pi))
        return (t * t - d * d) / 4.0 * pt * 2.0 * d * math.exp(-d * d)

    e, _ = integrate.dblquad(f, 0.0, 10.0, lambda d: d, lambda d: max(d, mu) + 12.0 * s,
                             epsabs=1e-13, epsrel=1e-10)
    pz = math.exp(-0.5 * z * z) / math.sqrt(2 * math.pi)
    return pz * (2.0 / (math.pi * a * a)) * e


def peaks_above(nu_th, a=1.0):
    v, _ = integrate.quad(lambda z: peak_density(z, a), nu_th, max(nu_th, 0.0) + 14.0, epsabs=1e-14,
                          epsrel=1e-9, limit=200)
    return v


def noise_rate(nu_th, a_list, dx):
    lam1 = peaks_above(nu_th, 1.0)   # per a^2
    return sum(lam1 * (dx / a) ** 2 for a in a_list)


def poisson_sf(k, lam):
    """P(N >= k) for N ~ Pois(lam), summing the pmf (upward tail when k > lam)."""
    if k <= 0:
        return 1.0
    if lam == 0:
        return 0.0
    logpmf = lambda j: -lam + j * math.log(lam) - math.lgamma(j + 1)
    if k > lam:
        total, j = 0.0, k
        while True:
            t = math.exp(logpmf(j))
            total += t
            if t == 0.0 or (t < total * 1e-17 and j > lam):   # terms only shrink past lam
                break
            j += 1
        return total
    return 1.0 - sum(math.exp(logpmf(j)) for j in range(k))


def choose_n_min(lam, eps):
    k = 0
    while poisson_sf(k, lam) > eps:
        k += 1
    return k


def p_signal(nu, nu_th, a, dx):
    det = 0.5 * math.erfc((nu_th - nu) / math.sqrt(2.0))
    inside = math.erf(dx * nu / (4.0 * a)) ** 2
    return det * inside


def signal_tail(p_list, k):
    """P(sum of independent Bernoulli(p_i) >= k), by the counting recursion."""
    dist = [1.0]
    for p in p_list:
        nxt = [0.0] * (len(dist) + 1)
        for j, q in enumerate(dist):
            nxt[j] += q * (1 - p)
            nxt[j + 1] += q * p
        dist = nxt
    return float(sum(dist[k:])) if k < len(dist) else 0.0


def dx_scan(nu, nu_th, a_list, dx_list, dv, dt, omega, n_false):
    """For each bin size dx: (dx, E[N_signal], E[N_noise], N_min), N_min the
    smallest threshold with P(N_noise >= N_min) <= N_false / N_stacks, where
    N_stacks = (dt dv / dx)^2 omega / dx^2 (Eq. v_size with equal axis ranges,
    Eq. N_stacks).  An object is recoverable where E[N_signal] > E[N_noise] and
    E[N_signal] + E[N_noise] >= N_min."""
    lam1 = peaks_above(nu_th, 1.0)
    out = []
    for dx in dx_list:
        es = sum(p_signal(nu, nu_th, a, dx) for a in a_list)
        en = sum(lam1 * (dx / a) ** 2 for a in a_list)
        ns = n_stacks((dt * dv / dx) ** 2, omega, dx)
        out.append((dx, es, en, choose_n_min(en, n_false / ns)))
    return out
