"""Pins of the refinement oracle (Sec. 2.1 steps 4-6) against facts outside it:
the published SplitMix64 output, numpy's least squares, exact integer
determinants, Mahalanobis distances from numpy's inverse, the exact MCD by
enumeration, the C-step theorem, robust recovery under outliers, and an exact
rational gather."""
from fractions import Fraction
from itertools import combinations

import numpy as np
import pytest

import sys
import types

from oracle import refine as REFINE


def cloud(rng, n, n_out=0, v=(350.0, -120.0), jitter=500.0, t_span=14400):
    """n points of a linear mover (t ticks, x/y mpx) plus n_out uniform outliers."""
    t = np.sort(rng.integers(0, t_span, n + n_out))
    x = 1_000_000 + v[0] * t / 3600.0 + rng.normal(0, jitter, len(t))
    y = 2_000_000 + v[1] * t / 3600.0 + rng.normal(0, jitter, len(t))
    out = rng.choice(len(t), n_out, replace=False)
    x[out] = rng.uniform(0.9e6, 1.1e6, n_out)
    y[out] = rng.uniform(1.9e6, 2.1e6, n_out)
    return [(int(a), int(round(b)), int(round(c))) for a, b, c in zip(t, x, y)], set(int(i) for i in out)


def exact_det(s):
    return (s[0] * (s[3] * s[5] - s[4] * s[4]) - s[1] * (s[1] * s[5] - s[4] * s[2])
            + s[2] * (s[1] * s[4] - s[3] * s[2]))


def pin_splitmix64_published_vector(R):
    assert R.splitmix64(0, 3) == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def pin_counter_words_are_splitmix64_outputs(R):
    """mix(state + (c+1) g) is output c+1 of the generator started at state, so
    the key chain and the draws are nested generator outputs."""
    def nth(state, c):
        return R.splitmix64(state, c)[-1]
    for seed, k, it, s, j in [(0, 0, 0, 0, 0), (5, 3, 1, 7, 2), (2**64 - 1, 11, 4, 499, 9)]:
        key = nth(nth(nth(seed, k + 1), it + 1), s + 1)
        assert R.start_key(seed, k, it, s) == key
        assert R.word(key, j) == nth(key, j + 1)


def pin_scatter_determinant_and_adjugate_against_exact_and_numpy(R):
    rng = np.random.default_rng(1)
    for _ in range(20):
        pts, _ = cloud(rng, int(rng.integers(5, 40)))
        H = list(range(len(pts)))
        F = R.fit(pts, H)
        assert F.det == pytest.approx(float(exact_det(F.S_exact)), rel=1e-10)
        z = np.array(pts, np.float64)
        cov = np.cov(z.T, bias=True) * len(pts) ** 2           # S = m^2 * biased covariance
        np.testing.assert_allclose(np.array(F.S), cov[np.triu_indices(3)], rtol=1e-9)
        adj = np.array([[F.adj[0], F.adj[1], F.adj[2]], [F.adj[1], F.adj[3], F.adj[4]],
                        [F.adj[2], F.adj[4], F.adj[5]]])
        np.testing.assert_allclose(adj, np.linalg.inv(cov) * np.linalg.det(cov), rtol=1e-6)


def pin_rank_is_mahalanobis_up_to_a_positive_constant(R):
    rng = np.random.default_rng(2)
    pts, _ = cloud(rng, 30, 5)
    F = R.fit(pts, list(range(0, 30, 2)))
    z = np.array(pts, np.float64)
    sub = z[0:30:2]
    mu = sub.mean(0)
    d2 = np.einsum("ij,jk,ik->i", z - mu, np.linalg.inv(np.cov(sub.T, bias=True)), z - mu)
    q = R.c_rank(np.array(pts, np.int64), F)
    ratio = q / d2
    assert np.all(ratio > 0)
    np.testing.assert_allclose(ratio, ratio[0], rtol=1e-6)


def pin_least_squares_special_case(R):
    rng = np.random.default_rng(3)
    for n in (2, 3, 4, 12, 80):
        pts, _ = cloud(rng, n)
        ln = R.line_of(R.fit(pts, list(range(n))))
        z = np.array(pts, np.float64)
        A = np.c_[np.ones(n), z[:, 0]]
        (cx, bx), *_ = np.linalg.lstsq(A, z[:, 1], rcond=None)
        (cy, by), *_ = np.linalg.lstsq(A, z[:, 2], rcond=None)
        assert ln.vxt == pytest.approx(bx, rel=1e-9, abs=1e-12)
        assert ln.vyt == pytest.approx(by, rel=1e-9, abs=1e-12)
        assert ln.x0 == pytest.approx(cx, rel=1e-9)
        assert ln.y0 == pytest.approx(cy, rel=1e-9)
        rx = z[:, 1] - (cx + bx * z[:, 0])
        ry = z[:, 2] - (cy + by * z[:, 0])
        assert ln.res[0] == pytest.approx(np.mean(rx * rx), rel=1e-6, abs=1e-6)
        assert ln.res[1] == pytest.approx(np.mean(rx * ry), rel=1e-6, abs=1e-6)
        assert ln.res[2] == pytest.approx(np.mean(ry * ry), rel=1e-6, abs=1e-6)


def pin_single_epoch_has_no_line(R):
    pts = [(100, 5, 7), (100, 9, 1), (100, 3, 3)]
    assert R.line_of(R.fit(pts, [0, 1, 2])) is None


def pin_fast_mcd_finds_the_exact_mcd_on_small_sets(R):
    rng = np.random.default_rng(4)
    hits = 0
    for trial in range(12):
        n = int(rng.integers(8, 12))
        pts, _ = cloud(rng, n - 3, 3)
        det_min, _ = R.exact_mcd_det(pts)
        H, F = R.fast_mcd(pts, seed=trial, k=0, it=0, n_starts=200)
        got = exact_det(F.S_exact)
        assert len(H) == (n + 4) // 2
        assert got >= det_min
        hits += got == det_min
    assert hits >= 11


def pin_c_step_never_raises_the_determinant(R):
    rng = np.random.default_rng(5)
    for _ in range(30):
        pts, _ = cloud(rng, 40, 15)
        arr = np.array(pts, np.int64)
        h = (len(pts) + 4) // 2
        H = sorted(rng.choice(len(pts), h, replace=False).tolist())
        F = R.fit(pts, H)
        H2 = R.c_select(arr, F, h)
        F2 = R.fit(pts, H2)
        assert exact_det(F2.S_exact) <= exact_det(F.S_exact)


def pin_result_is_a_c_step_fixed_point(R):
    """FAST-MCD iterates its best starts to convergence: one more C-step from
    the returned subset cannot lower the determinant."""
    rng = np.random.default_rng(11)
    for trial in range(6):
        pts, _ = cloud(rng, 45, 30, v=(3500.0, -1200.0), jitter=300.0)
        H, F = R.fast_mcd(pts, seed=trial, k=2, it=1, n_starts=20, n_best=3)
        arr = np.array(pts, np.int64)
        H2 = R.c_select(arr, R.fit(pts, H), len(H))
        assert exact_det(R.fit(pts, H2).S_exact) >= exact_det(R.fit(pts, H).S_exact)


def pin_draws_are_distinct_and_spread(R):
    key = R.start_key(7, 3, 0, 11)
    n = 50
    perm = list(range(n))
    for j in range(n):
        r = j + R.word(key, j) % (n - j)
        perm[j], perm[r] = perm[r], perm[j]
    assert sorted(perm) == list(range(n))
    firsts = [R.word(R.start_key(7, 3, 0, s), 0) % n for s in range(2000)]
    counts = np.bincount(firsts, minlength=n)
    assert counts.min() > 10 and counts.max() < 80


def pin_robust_fit_recovers_the_mover_where_least_squares_fails(R):
    rng = np.random.default_rng(6)
    v = (3500.0, -1200.0)     # slope error of the 30-point subset ~ 300 / (1.15 h * 5.5) ~ 50 mpx/h
    pts, out = cloud(rng, 60, 40, v=v, jitter=300.0)
    _, F = R.fast_mcd(pts, seed=1, k=0, it=0)
    ln = R.line_of(F)
    ls = R.line_of(R.fit(pts, list(range(len(pts)))))
    assert ln.vxt * 3600 == pytest.approx(v[0], abs=200)
    assert ln.vyt * 3600 == pytest.approx(v[1], abs=200)
    assert abs(ls.vxt * 3600 - v[0]) > 0.1 * abs(v[0]) or abs(ls.vyt * 3600 - v[1]) > 0.1 * abs(v[1])


def pin_exact_fit_subset_is_kept(R):
    """Points in one plane (y constant): every subset is singular, so each start
    keeps its first h draws, all tie at det 0, and start 0 wins."""
    rng = np.random.default_rng(7)
    n = 13
    pts = [(int(t), int(1000 + 0.3 * t + rng.integers(-50, 50)), 500) for t in rng.integers(0, 14400, n)]
    H, F = R.fast_mcd(pts, seed=3, k=0, it=0, n_starts=50)
    h = (n + 4) // 2
    key = R.start_key(3, 0, 0, 0)
    perm = list(range(n))
    for j in range(h):
        r = j + R.word(key, j) % (n - j)
        perm[j], perm[r] = perm[r], perm[j]
    assert F.det == 0 and exact_det(F.S_exact) == 0
    assert H == sorted(perm[:h])
    ln = R.line_of(F)
    z = np.array([pts[i] for i in H], np.float64)
    b, *_ = np.linalg.lstsq(np.c_[np.ones(h), z[:, 0]], z[:, 1], rcond=None)
    assert ln.vyt == 0 and ln.vxt == pytest.approx(b[1], rel=1e-9)


def pin_gather_against_exact_rationals(R):
    rng = np.random.default_rng(8)
    n = 4000
    t = rng.integers(0, 14400, n)
    x = rng.integers(-10_000, 10_000, n)
    y = rng.integers(-10_000, 10_000, n)
    ln = R.Line(0.37, -0.21, 120.5, -33.25, (0, 0, 0))
    radius = 2000
    got = R.gather(ln, t, x, y, radius)
    want = []
    for i in range(n):
        px = Fraction(ln.x0) + Fraction(ln.vxt) * int(t[i])
        py = Fraction(ln.y0) + Fraction(ln.vyt) * int(t[i])
        d2 = (int(x[i]) - px) ** 2 + (int(y[i]) - py) ** 2
        if abs(d2 - radius * radius) > 1e-3:
            assert (i in set(got)) == (d2 <= radius * radius)
        if d2 <= radius * radius:
            want.append(i)
    assert 50 < len(got) < n
    assert abs(len(got) - len(want)) <= 1


def pin_refine_converges_on_a_noisy_cluster(R):
    rng = np.random.default_rng(9)
    E = 40
    te = np.sort(rng.integers(0, 14400, E))
    # The MCD of (t, x, y) also favours points close in time: its h-subset may span
    # ~1.5 h (std 0.4 h), so with 100 mpx jitter the slope error is ~100/(0.4*4.9) ~ 50 mpx/h.
    v = (3640.0, -1820.0)
    # one mover (one detection per epoch, 100 mpx jitter) plus uniform noise
    tt, xx, yy, mover = [], [], [], []
    for e in range(E):
        tt.append(te[e]); xx.append(int(500_000 + v[0] * te[e] / 3600 + rng.normal(0, 100)))
        yy.append(int(700_000 + v[1] * te[e] / 3600 + rng.normal(0, 100))); mover.append(True)
        for _ in range(30):
            tt.append(te[e]); xx.append(int(rng.integers(480_000, 540_000)))
            yy.append(int(rng.integers(680_000, 720_000))); mover.append(False)
    tt, xx, yy, mover = map(np.array, (tt, xx, yy, mover))
    truth = np.nonzero(mover)[0]
    # a rough cluster: 70 % of the mover plus some noise near it
    start = sorted(rng.choice(truth, 28, replace=False).tolist()
                   + rng.choice(np.nonzero(~mover)[0], 6, replace=False).tolist())
    tr = R.refine(start, tt, xx, yy, radius=2000, seed=5, k=0, n_starts=100)
    assert tr.status == R.CONVERGED
    assert set(truth.tolist()) <= set(tr.ids)
    # noise inside the 2000 mpx disk: 40 epochs * 30 * pi 2000^2 / (60000 * 40000) ~ 6.3 expected
    assert len(tr.ids) - len(truth) <= 15
    assert tr.line.vxt * 3600 == pytest.approx(v[0], abs=250)
    assert tr.line.vyt * 3600 == pytest.approx(v[1], abs=250)


def pin_refine_edge_cases(R):
    tt = np.array([0, 0, 0]); xx = np.array([1, 2, 3]); yy = np.array([4, 5, 6])
    tr = R.refine([0, 1, 2], tt, xx, yy, radius=10, seed=0, k=0)
    assert tr.status == R.DEGENERATE and tr.line is None
    tr = R.refine(list(range(3)), tt, xx, yy, radius=10, seed=0, k=0, max_points=2)
    assert tr.status == R.TOO_MANY and tr.ids == [0, 1, 2]


PINS = [v for k, v in sorted(globals().items()) if k.startswith("pin_")]


@pytest.mark.parametrize("pin", PINS, ids=lambda f: f.__name__[4:])
def test_pin(pin):
    pin(REFINE)


# Each mutant is the oracle's source with one plausible mistake; it must fail a pin.
MUTANTS = {
    "adjugate_sign": ("a01 = s02 * s12 - s01 * s22", "a01 = s01 * s22 - s02 * s12"),
    "adjugate_index": ("a12 = s01 * s02 - s00 * s12", "a12 = s01 * s02 - s00 * s11"),
    "det_dropped_term": ("det = (s00 * a00 + s01 * a01) + s02 * a02", "det = s00 * a00 + s01 * a01"),
    "rank_transposed": ("w2 = (a02 * u0 + a12 * u1) + a22 * u2", "w2 = (a02 * u0 + a12 * u2) + a22 * u1"),
    "rank_uncentred": ("u1 = (m * pts_arr[:, 1] - X)", "u1 = (m * pts_arr[:, 1] - 0 * X)"),
    "select_largest": ("return sorted(int(i) for i in order[:h])", "return sorted(int(i) for i in order[-h:])"),
    "h_off_by_one": ("h = (n + D + 1) // 2\n    pts_arr", "h = (n + D) // 2\n    pts_arr"),
    "cstep_accepts_increase": ("if not F2.det < F.det:", "if F2.det < F.det:"),
    "best_is_largest": ("best = sorted(dets)[:n_best]", "best = sorted(dets)[-n_best:]"),
    "slope_swapped": ("vxt = s01 / s00", "vxt = s02 / s00"),
    "intercept_sign": ("x0 = (np.float64(X) - vxt * np.float64(T)) / m", "x0 = (np.float64(X) + vxt * np.float64(T)) / m"),
    "residual_term": ("(s12 - vxt * s02) / mm", "(s12 - vyt * s02) / mm"),
    "gather_sign": ("ry = np.asarray(y, np.float64) - py", "ry = np.asarray(y, np.float64) + py"),
    "gather_strict_radius": ("d2 <= r2", "d2 < r2 - 1e6"),
    "mix_constant": ("0x94D049BB133111EB", "0x94D049BB133111EA"),
    "key_order": ("b = mix64((a + (it + 1) * GOLDEN) & M64)", "b = mix64((a + (it + 2) * GOLDEN) & M64)"),
    "draw_range": ("r = j + word(key, j) % (n - j)", "r = j + word(key, j) % (n - j - 1 or 1)"),
    "second_moment_scale": ("return m * sum(p * q for p, q in zip(a, b)) - sa * sb",
                            "return (m - 1) * sum(p * q for p, q in zip(a, b)) - sa * sb"),
}


def _mutant(name):
    src = open(REFINE.__file__).read()
    old, new = MUTANTS[name]
    old, new = old.replace("\\n", "\n"), new.replace("\\n", "\n")
    assert src.count(old) == 1, name
    mod = types.ModuleType(f"refine_mutant_{name}")
    mod.__file__ = REFINE.__file__
    sys.modules[mod.__name__] = mod          # dataclasses look their module up
    try:
        exec(compile(src.replace(old, new), f"<{name}>", "exec"), mod.__dict__)
    finally:
        del sys.modules[mod.__name__]
    return mod


def _fails(pin, mod):
    try:
        pin(mod)
    except Exception:
        return True
    return False


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_fails_a_pin(name):
    mod = _mutant(name)
    assert any(_fails(pin, mod) for pin in PINS), f"mutant {name} passes every pin"
