"""Pins of the search-parameter oracle (Sec. 2.2) against facts outside it:
Longuet-Higgins's density of maxima of a Gaussian surface, a simulated smoothed
white-noise field, a lattice count, scipy's Poisson and binomial tails, Monte
Carlo of detection and binning, brute-force enumeration, and the paper's
statement that objects of S/N 0.5 are not recoverable at any bin size."""
import itertools
import math

import numpy as np
import pytest
from scipy import integrate, stats

from oracle import params as P


def test_total_density_of_maxima_is_longuet_higgins():
    # a Gaussian surface has sigma2^2 / (8 sqrt(3) pi sigma1^2) maxima per unit
    # area; white noise under a Gaussian window of width a: sigma2^2/sigma1^2 = 2/a^2
    for a in (1.0, 2.5):
        tot, _ = integrate.quad(lambda z: P.peak_density(z, a), -12, 14, limit=200)
        assert tot == pytest.approx(2.0 / (a * a) / (8 * math.sqrt(3) * math.pi), rel=1e-6)


def test_peak_heights_of_a_simulated_field():
    rng = np.random.default_rng(0)
    n, a = 512, 3.0
    k = np.fft.fftfreq(n) * 2 * np.pi
    k2 = k[:, None] ** 2 + k[None, :] ** 2
    edges = np.linspace(-1, 5, 7)
    cnt, area = np.zeros(6), 0
    for _ in range(4):
        f = np.real(np.fft.ifft2(np.fft.fft2(rng.normal(size=(n, n))) * np.exp(-k2 * a * a / 2)))
        f /= f.std()
        c = f[1:-1, 1:-1]
        m = np.ones_like(c, bool)
        for dx, dy in itertools.product((-1, 0, 1), repeat=2):
            if dx or dy:
                m &= c > f[1 + dx:n - 1 + dx, 1 + dy:n - 1 + dy]
        cnt += np.histogram(c[m], edges)[0]
        area += c.size
    for j in range(1, 5):      # bins with hundreds to thousands of peaks
        want, _ = integrate.quad(lambda z: P.peak_density(z, a), edges[j], edges[j + 1])
        tol = 3.0 / math.sqrt(cnt[j]) + 0.03          # Poisson scatter + grid discretisation
        assert cnt[j] / area == pytest.approx(want, rel=tol), (j, cnt[j])


def test_velocity_count_is_the_lattice_size():
    dx, dt = 2.0, 4.0          # px, h: dv = 0.5 px/h
    vs = np.arange(-10.0, 10.0, dx / dt)
    assert P.velocity_count(-10, 10, -10, 10, dx, dt) == len(vs) ** 2
    assert P.n_stacks(P.velocity_count(0, 5, 0, 3, dx, dt), 1000.0 * 2000.0, dx) == \
        pytest.approx((5 / 0.5) * (3 / 0.5) * 1000 * 2000 / 4)


@pytest.mark.parametrize("lam", [0.0, 0.3, 4.0, 37.5, 250.0])
def test_poisson_tail_against_scipy(lam):
    for k in range(0, int(lam * 2 + 30), 3):
        want = stats.poisson.sf(k - 1, lam) if lam > 0 else float(k <= 0)
        assert P.poisson_sf(k, lam) == pytest.approx(want, rel=1e-9, abs=1e-300)
    assert P.poisson_sf(2000, lam) == pytest.approx(stats.poisson.sf(1999, lam), abs=1e-300)   # underflowing tail
    if lam > 0:
        for eps in (1e-3, 1e-9):
            n = P.choose_n_min(lam, eps)
            assert stats.poisson.sf(n - 1, lam) <= eps < stats.poisson.sf(n - 2, lam)


def test_detection_and_binning_probability_by_monte_carlo():
    rng = np.random.default_rng(3)
    m = 400_000
    for nu, nu_th, a, dx in [(3.0, 2.5, 1.0, 1.5), (6.0, 5.0, 2.0, 1.0), (1.5, 1.0, 1.0, 4.0)]:
        sig = math.sqrt(2.0) * a / nu
        hit = (rng.normal(nu, 1.0, m) >= nu_th) & (np.abs(rng.normal(0, sig, m)) <= dx / 2) & \
              (np.abs(rng.normal(0, sig, m)) <= dx / 2)
        p = P.p_signal(nu, nu_th, a, dx)
        assert hit.mean() == pytest.approx(p, abs=4 * math.sqrt(p * (1 - p) / m) + 1e-4)


def test_signal_tail_brute_force_and_binomial():
    rng = np.random.default_rng(4)
    p = rng.uniform(0, 1, 9).tolist()
    for k in range(11):
        brute = sum(np.prod([p[i] if b[i] else 1 - p[i] for i in range(9)])
                    for b in itertools.product((0, 1), repeat=9) if sum(b) >= k)
        assert P.signal_tail(p, k) == pytest.approx(brute, abs=1e-14)
    assert P.signal_tail([0.3] * 40, 15) == pytest.approx(stats.binom.sf(14, 40, 0.3), rel=1e-10)


def test_faint_objects_are_not_recoverable_at_any_bin_size():
    """S/N 0.5: expected signal never beats expected noise (the paper's remark on its figure)."""
    for nu_th in (1.0, 2.0, 3.0, 4.0):
        rows = P.dx_scan(0.5, nu_th, [1.0] * 20, np.linspace(0.1, 10, 40), dv=3.0, dt=4.0, omega=162 * 3600.0,
                         n_false=100)
        assert all(es < en for _, es, en, _ in rows)
    rows = P.dx_scan(6.0, 4.0, [1.0] * 20, [0.5, 1.0, 2.0, 4.0], dv=3.0, dt=4.0, omega=162 * 3600.0, n_false=100)
    assert any(es > en and es + en >= nmin for _, es, en, nmin in rows)
