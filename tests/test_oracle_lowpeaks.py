"""Pins of the two-threshold oracle (tile-local super-bin peaks): a pure-Python
brute force over the brute-force search's cells (its own super-bin sums and an
all-pairs neighbourhood test, no dense histograms), the special cases that
reduce to the one-threshold search, containment between the plain searches,
hand-built movers, and planted mistakes that those pins must catch."""
import numpy as np
import pytest

import oracle
from oracle import brute
from oracle import lowpeaks as LP
from paper_2509_26279_gb300 import workloads as W
from tests import cases


def brute_two(cat, grid, n_min, n_low, tiles, v_begin, v_end, peaks_only=False):
    """Every nonempty cell from the brute-force search, R as sums of raw counts
    over each super-bin, the peak test against every other super-bin."""
    cells, _ = brute.search(cat.x, cat.y, cat.epoch, cat.t, cat.ticks_per_hour, grid, 1)
    cells = [c for c in cells if v_begin <= c[0] < v_end]
    s = tiles["s"]
    R = {}
    for v, bx, by, d, raw, ids in cells:
        k = (v % grid.nvx, v // grid.nvx, bx // s, by // s)
        R[k] = R.get(k, 0) + raw
    keys = np.array(list(R.keys()), np.int64).reshape(-1, 4)
    vals = np.array(list(R.values()), np.int64)
    ky_lo = v_begin // grid.nvx
    size = np.array([tiles["kx"], tiles["ky"], tiles["bx"], tiles["by"]])
    shift = np.array([0, ky_lo, 0, 0])
    tile = (keys - shift) // size

    def peak(k):
        k = np.asarray(k)
        me = R[tuple(k)]
        near = (np.abs(keys - k) <= 1).all(axis=1) & (tile == (k - shift) // size).all(axis=1)
        return not (near & (vals > me)).any()

    out = []
    for c in cells:
        v, bx, by, d = c[0], c[1], c[2], c[3]
        plain = d >= n_min and not peaks_only
        if plain or (d >= n_low and peak((v % grid.nvx, v // grid.nvx, bx // s, by // s))):
            out.append(c)
    return out


def tuples(res):
    return cases.as_tuples(res.cands, res.id_lists())


def random_tiles(rng):
    return {"kx": int(rng.choice([1, 2, 4, 8])), "ky": int(rng.choice([1, 2, 4])),
            "bx": int(rng.choice([1, 2, 3, 7])), "by": int(rng.choice([1, 2, 3, 7])),
            "s": int(rng.choice([1, 2, 3, 4]))}


def random_case(seed):
    cat, grid, n_min = cases.random_tiny(seed)
    rng = np.random.default_rng(seed + 7000)
    n_min = n_min + int(rng.integers(0, 3))
    n_low = int(rng.integers(1, n_min + 1))
    nv = grid.nvx * grid.nvy
    v_begin, v_end = 0, nv
    if rng.random() < 0.4:
        v_begin = int(rng.integers(0, nv))
        v_end = int(rng.integers(v_begin, nv + 1))
    return cat, grid, n_min, n_low, random_tiles(rng), v_begin, v_end, bool(rng.random() < 0.35)


def pins_pass(mod) -> bool:
    """Every pin below, run against an oracle module (the real one or a mutant);
    an exception counts as a failed pin."""
    try:
        for seed in range(40):
            cat, grid, n_min, n_low, tiles, vb, ve, po = random_case(seed)
            got = tuples(mod.search(cat, grid, n_min, n_low, tiles, vb, ve, peaks_only=po))
            if got != brute_two(cat, grid, n_min, n_low, tiles, vb, ve, po):
                return False
        return hand_built_holds(mod)
    except Exception:
        return False


@pytest.mark.parametrize("seed", range(40))
def test_equals_brute_force(seed):
    cat, grid, n_min, n_low, tiles, vb, ve, po = random_case(seed)
    got = tuples(LP.search(cat, grid, n_min, n_low, tiles, vb, ve, peaks_only=po))
    assert got == brute_two(cat, grid, n_min, n_low, tiles, vb, ve, po)


@pytest.mark.parametrize("seed", range(10))
def test_equal_thresholds_is_the_plain_search(seed):
    cat, grid, n_min = cases.random_tiny(seed)
    tiles = random_tiles(np.random.default_rng(seed))
    assert tuples(LP.search(cat, grid, n_min, n_min, tiles)) == tuples(oracle.stack(cat, grid, n_min))


@pytest.mark.parametrize("seed", range(10))
def test_one_point_tiles_is_the_low_search(seed):
    # every super-bin alone in its tile has no neighbour: each is a peak
    cat, grid, n_min = cases.random_tiny(seed)
    n_min += 2
    tiles = {"kx": 1, "ky": 1, "bx": 1, "by": 1, "s": int(np.random.default_rng(seed).integers(1, 5))}
    assert tuples(LP.search(cat, grid, n_min, 1, tiles)) == tuples(oracle.stack(cat, grid, 1))
    assert tuples(LP.search(cat, grid, n_min, 1, tiles, peaks_only=True)) == tuples(oracle.stack(cat, grid, 1))


def test_between_the_plain_searches_on_a_field():
    w = W.tiny()
    cat = W.load(w)
    g = w.grid
    n_min, n_low = 8, 4
    tiles = {"kx": 8, "ky": 4, "bx": 32, "by": 16, "s": 2}
    two = tuples(LP.search(cat, g, n_min, n_low, tiles))
    hi = tuples(oracle.stack(cat, g, n_min))
    lo = tuples(oracle.stack(cat, g, n_low))
    key = lambda c: (c[0], c[1], c[2])
    s_two, s_hi, s_lo = {key(c) for c in two}, {key(c) for c in hi}, {key(c) for c in lo}
    assert s_hi <= s_two <= s_lo
    assert len(s_hi) < len(s_two) < len(s_lo)          # adds cells, and prunes some
    # the same order as the plain search, restricted
    assert [c for c in lo if key(c) in s_two] == two


def hand_built():
    """A stationary faint source (6 detections, epochs 0-5) at (105, 105) and a
    stationary bright one (20 detections, epochs 0-19) at (305, 305); t = e
    hours, lattice v = -4..3 mpx/h per axis, bins of 10 mpx."""
    x = [105] * 6 + [305] * 20
    y = [105] * 6 + [305] * 20
    ep = list(range(6)) + list(range(20))
    cat = cases.catalog(x, y, ep, list(range(20)), tph=1)
    grid = W.GridSpec(vx0=-4, vy0=-4, dvx=1, dvy=1, nvx=8, nvy=8, x_min=0, y_min=0, nbx=40, nby=40, bin=10)
    return cat, grid


def hand_built_holds(mod) -> bool:
    cat, grid = hand_built()
    tiles = {"kx": 8, "ky": 8, "bx": 64, "by": 64, "s": 2}
    got = {(c[0], c[1], c[2]): c[3] for c in tuples(mod.search(cat, grid, 10, 5, tiles))}
    only = {(c[0], c[1], c[2]): c[3] for c in tuples(mod.search(cat, grid, 10, 5, tiles, peaks_only=True))}
    v00, v10 = 4 * 8 + 4, 4 * 8 + 5       # (vx, vy) = (0, 0) and (1, 0)
    return (got.get((v00, 10, 10)) == 6      # the faint source at its velocity
            and got.get((v10, 10, 10)) == 6  # and at the next one (equal super-bin count: a tie)
            and got.get((v00, 30, 30)) == 20  # the bright source (plain threshold)
            and got.get((v10, 29, 30)) == 10  # its neighbour at N_min (plain threshold)
            # at v = (1, 0) its 6 detections of epochs 0-5 stay in bin 30, a ghost
            # below N_min whose super-bin holds 6 against 20 at v = (0, 0): pruned
            and (v10, 30, 30) not in got
            # peaks only: the sources' peaks stay; the cell at N_min whose super-bin
            # (bins 28-29: 14 detections) sits next to the 20 at v = (0, 0) goes
            and only.get((v00, 10, 10)) == 6 and only.get((v10, 10, 10)) == 6
            and only.get((v00, 30, 30)) == 20 and (v10, 29, 30) not in only
            and set(only) <= set(got))


def test_hand_built_movers():
    cat, grid = hand_built()
    lo = {(c[0], c[1], c[2]): c[3] for c in tuples(oracle.stack(cat, grid, 5))}
    assert lo[(4 * 8 + 5, 30, 30)] == 6      # the ghost is there at the low threshold
    assert hand_built_holds(LP)


MUTANTS = {
    "ties_dropped": ("if r[sby2, sbx2] > me:",
                     "if r[sby2, sbx2] >= me and (kx2, ky2, sbx2, sby2) != (kx, ky, sbx, sby):"),
    "velocity_tiles_ignored": ('if (kx2 // tiles["kx"], (ky2 - ky_lo) // tiles["ky"]) != vt:', "if False:"),
    "spatial_tiles_ignored": ('if (sbx2 // tiles["bx"], sby2 // tiles["by"]) != st:', "if False:"),
    "tile_rows_from_zero": ("ky_lo = R.v_begin // g.nvx", "ky_lo = 0"),
    "range_not_zeroed": ("    if not (v_begin <= v < v_end):\n        return False\n", ""),
    "superbin_transposed": ('sb = (int(c["bx"]) // tiles["s"], int(c["by"]) // tiles["s"])',
                            'sb = (int(c["by"]) // tiles["s"], int(c["bx"]) // tiles["s"])'),
    "plain_exclusive": ('if int(c["distinct"]) >= n_min and not peaks_only:',
                        'if int(c["distinct"]) > n_min and not peaks_only:'),
    "peaks_only_ignored": ('if int(c["distinct"]) >= n_min and not peaks_only:', 'if int(c["distinct"]) >= n_min:'),
    "neighbourhood_one_sided": ("for kx2 in (kx - 1, kx, kx + 1):", "for kx2 in (kx - 1, kx):"),
    "spatial_one_sided": ("for sby2 in (sby - 1, sby, sby + 1):", "for sby2 in (sby, sby + 1):"),
}


def test_unmutated_oracle_passes_pins():
    assert pins_pass(LP)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name):
    import importlib.util
    import sys
    src = open(LP.__file__).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, name
    spec = importlib.util.spec_from_loader(f"oracle._lowpeaks_{name}", loader=None)
    mod = importlib.util.module_from_spec(spec)
    mod.__package__ = "oracle"
    sys.modules[spec.name] = mod
    try:
        exec(compile(src.replace(old, new), f"<mutant {name}>", "exec"), mod.__dict__)
        assert not pins_pass(mod), f"mutant {name} passes every pin"
    finally:
        del sys.modules[spec.name]
