"""The oracle's pins must be strong enough to catch plausible mistakes.

Each mutant below is the oracle source with one deliberate mistake (a dropped
term, a wrong sign, a transposed operand, an off-by-one).  The mutant is built
on the CPU in a temporary directory and must fail at least one pin: the
hand-computed golden cases, the independent brute force, or the duplicate
invariant."""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from oracle import brute
from tests import cases
from tests.test_oracle_pins import golden_inputs, load_golden, oracle_tuples

SRC = os.path.join(os.path.dirname(oracle.__file__), "sas_oracle.c")

MUTANTS = {
    "truncating_division": ("if ((a % b) != 0 && a < 0) q -= 1;", ""),
    "shift_sign_x": ("int64_t X = (int64_t)xi - sx - x_min;", "int64_t X = (int64_t)xi + sx - x_min;"),
    "transposed_shift_y": ("int64_t Y = (int64_t)yi - sy - y_min;", "int64_t Y = (int64_t)yi - sx - y_min;"),
    "dropped_x_min": ("int64_t X = (int64_t)xi - sx - x_min;", "int64_t X = (int64_t)xi - sx;"),
    "t0_is_max": ("if (t[epoch[i]] < t0) t0 = t[epoch[i]];",
                  "if (t[epoch[i]] > t0 || t0 == INT64_MAX) t0 = t[epoch[i]];"),
    "dropped_t0": ("sx[e] = floor_div(vx * (t[e] - t0), tph);", "sx[e] = floor_div(vx * t[e], tph);"),
    "exclusive_threshold": ("if (d < n_min) continue;", "if (d <= n_min) continue;"),
    "raw_as_distinct": ("c->distinct = d; c->raw = raw[b];", "c->distinct = raw[b]; c->raw = raw[b];"),
    "swapped_bin_output": ("c->bx = (int32_t)(b % nbx); c->by = (int32_t)(b / nbx);",
                           "c->by = (int32_t)(b % nbx); c->bx = (int32_t)(b / nbx);"),
    "raw_ascending": ("if (a->raw != b->raw) return a->raw > b->raw ? -1 : 1;",
                      "if (a->raw != b->raw) return a->raw < b->raw ? -1 : 1;"),
    "transposed_lattice_index": ("const int64_t kx = v % nvx, ky = v / nvx;\n    const int64_t vx = (int64_t)vx0",
                                 "const int64_t ky = v % nvx, kx = v / nvx;\n    const int64_t vx = (int64_t)vx0"),
    "domain_off_by_one": ("if (bx < 0 || bx >= nbx || by < 0 || by >= nby) return -1;",
                          "if (bx < 0 || bx > nbx || by < 0 || by >= nby) return -1;"),
    "epoch_word_dropped": ("      mask[b * words + e / 64] |= (uint64_t)1 << (e % 64);\n    }\n    /* Step 3",
                           "      mask[b * words] |= (uint64_t)1 << (e % 64);\n    }\n    /* Step 3"),
    "wrong_ids": ("tids[c->id_off + c->id_len++] = (int32_t)i;", "tids[c->id_off + c->id_len++] = (int32_t)(i + 1);"),
    "sort_by_before_bx_flipped": ("if (a->by != b->by) return a->by < b->by ? -1 : 1;",
                                  "if (a->by != b->by) return a->by > b->by ? -1 : 1;"),
}


def _pins_pass(lib) -> bool:
    for case in load_golden():
        cat, grid, n_min = golden_inputs(case)
        want = [tuple(c[:5]) + (list(c[5]),) for c in case["expected"]]
        try:
            if oracle_tuples(oracle.stack(cat, grid, n_min, lib=lib)) != want:
                return False
        except RuntimeError:
            return False
    for seed in list(range(30)) + [1000, 1001]:
        cat, grid, n_min = cases.random_tiny(seed)
        bf, pairs = brute.search(cat.x, cat.y, cat.epoch, cat.t, cat.ticks_per_hour, grid, n_min)
        res = oracle.stack(cat, grid, n_min, lib=lib)
        if oracle_tuples(res) != [tuple(c[:5]) + (list(c[5]),) for c in bf] or res.n_pairs != pairs:
            return False
    return True


def _child(so_path: str) -> None:
    """Entry point of the child process: exit 0 iff every pin passes."""
    sys.exit(0 if _pins_pass(oracle.bind(so_path)) else 1)


def _build_mutant(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    mutated = src.replace(old, new)
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"lib{name}.so"
    c.write_text(mutated)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-o", str(so), str(c)])
    return str(so)


def _run_pins_in_child(so_path: str) -> int:
    # A mutant may write out of bounds and abort; run it in its own process.
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = f"from tests.test_oracle_mutants import _child; _child({so_path!r})"
    return subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True,
                          timeout=300).returncode


def test_unmutated_oracle_passes_pins():
    assert _run_pins_in_child(oracle.build()) == 0


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    so = _build_mutant(tmp_path, name, old, new)
    assert _run_pins_in_child(so) != 0, f"mutant {name} passed every pin"
