"""The library's parameter functions (host code behind the C ABI) against the
oracle of Sec. 2.2.  No device is needed."""
import math

import numpy as np
import pytest

from oracle import params as P

sas = pytest.importorskip("paper_2509_26279_gb300.sas")
L = sas.params


def test_velocity_count_and_stacks():
    assert L.velocity_count(-3, 5, 0, 2, 1.5, 4.0) == pytest.approx(P.velocity_count(-3, 5, 0, 2, 1.5, 4.0), rel=1e-15)
    assert L.n_stacks(1234.0, 5e6, 2.0) == pytest.approx(P.n_stacks(1234.0, 5e6, 2.0), rel=1e-15)


@pytest.mark.parametrize("z", [-3.0, -1.0, 0.0, 0.7, 2.0, 4.5, 7.0])
def test_peak_density(z):
    for a in (1.0, 1.7):
        assert L.peak_density(z, a) == pytest.approx(P.peak_density(z, a), rel=1e-8, abs=1e-300)


@pytest.mark.parametrize("nu_th", [-2.0, 0.0, 1.5, 3.0, 5.0])
def test_peaks_above_and_noise_rate(nu_th):
    assert L.peaks_above(nu_th, 2.0) == pytest.approx(P.peaks_above(nu_th, 2.0), rel=1e-8)
    a = [0.9, 1.1, 1.3, 1.0]
    assert L.noise_rate(nu_th, a, 2.5) == pytest.approx(P.noise_rate(nu_th, a, 2.5), rel=1e-8)


def test_poisson_and_n_min():
    for lam in (0.0, 0.2, 3.3, 41.0, 400.0):
        for k in (0, 1, 2, 5, 20, 60, 500):
            assert L.poisson_sf(k, lam) == pytest.approx(P.poisson_sf(k, lam), rel=1e-12, abs=1e-300)
        for eps in (0.5, 1e-4, 1e-12):
            assert L.choose_n_min(lam, eps) == P.choose_n_min(lam, eps)


def test_signal_terms_and_scan():
    assert L.p_signal(3.0, 2.0, 1.2, 2.0) == pytest.approx(P.p_signal(3.0, 2.0, 1.2, 2.0), rel=1e-14)
    p = np.random.default_rng(1).uniform(0, 1, 60)
    for k in (0, 10, 30, 59, 61):
        assert L.signal_tail(p, k) == pytest.approx(P.signal_tail(p.tolist(), k), rel=1e-12, abs=1e-300)
    args = (4.0, 3.0, [1.0, 1.2] * 10, [0.5, 1.0, 2.0, 3.5], 3.0, 4.0, 162 * 3600.0, 100.0)
    for g, w in zip(L.dx_scan(*args), P.dx_scan(*args)):
        assert g[0] == w[0] and g[3] == w[3]
        assert g[1] == pytest.approx(w[1], rel=1e-13) and g[2] == pytest.approx(w[2], rel=1e-8)


def test_n_min_far_into_the_tail_and_range_limits():
    # binary search: large rates finish quickly and agree with scipy's tail
    from scipy import stats
    for lam, eps in [(5e4, 1e-12), (3e6, 1e-9)]:
        k = L.choose_n_min(lam, eps)
        assert stats.poisson.sf(k - 1, lam) <= eps < stats.poisson.sf(k - 2, lam)
    with pytest.raises(sas.SasError):
        L.choose_n_min(2e7, 0.1)
    with pytest.raises(sas.SasError):
        L.signal_tail(np.full(70000, 0.5), 3)


def test_argument_errors():
    with pytest.raises(sas.SasError):
        L.peaks_above(1.0, 0.0)
    with pytest.raises(sas.SasError):
        L.choose_n_min(-1.0, 0.1)
    with pytest.raises(sas.SasError):
        L.signal_tail([0.5, 1.5], 1)
    with pytest.raises(sas.SasError):
        L.velocity_count(3, 1, 0, 1, 1, 1)
