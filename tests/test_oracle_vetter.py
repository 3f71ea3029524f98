"""Pins for the vetter oracle (oracle/vetter.py): finite differences, closed
forms, and stamps against independently computed histograms."""
import numpy as np
import pytest

import oracle
from oracle import brute, vetter
from paper_2509_26279_gb300 import workloads as W
from tests import cases


def _small_params(seed):
    return vetter.init_params(seed).astype(np.float64) * 0.5 + 0.01


def test_param_count_and_layout():
    assert vetter.N_PARAMS == 187137
    flat = np.arange(vetter.N_PARAMS, dtype=np.float64)
    assert np.array_equal(vetter.flatten(vetter.unflatten(flat)), flat)
    p = vetter.unflatten(flat)
    assert p["conv1.w"].shape == (32, 9, 3, 3) and p["fc1.w"].shape == (64, 2592)
    assert p["fc2.b"][0] == vetter.N_PARAMS - 1


def test_conv_closed_forms():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 3, 7, 6))
    w = np.zeros((4, 3, 3, 3))
    w[1, 2, 0, 2] = 1.0          # picks channel 2 shifted by (0, 2)
    b = np.arange(4.0)
    out = vetter._conv(x, w, b)
    assert out.shape == (2, 4, 5, 4)
    assert np.allclose(out[:, 1], x[:, 2, 0:5, 2:6] + 1.0)
    assert np.allclose(out[:, 0], 0.0) and np.allclose(out[:, 3], 3.0)
    # against a direct triple loop
    w = rng.normal(size=(4, 3, 3, 3))
    ref = np.zeros((2, 4, 5, 4))
    for o in range(4):
        for yy in range(5):
            for xx in range(4):
                ref[:, o, yy, xx] = (x[:, :, yy:yy + 3, xx:xx + 3] * w[o]).sum(axis=(1, 2, 3))
    assert np.allclose(vetter._conv(x, w, np.zeros(4)), ref)


def test_bce_closed_forms():
    assert abs(vetter.bce_with_logits([0.0], [1.0]) - np.log(2)) < 1e-15
    assert abs(vetter.bce_with_logits([0.0], [0.0]) - np.log(2)) < 1e-15
    assert vetter.bce_with_logits([40.0], [1.0]) < 1e-15
    assert abs(vetter.bce_with_logits([-3.0], [1.0]) - np.log1p(np.exp(3.0))) < 1e-12


def test_gradients_match_central_finite_differences():
    """Every layer's gradient against (L(p + h e_i) - L(p - h e_i)) / 2h on a
    random subset of coordinates of every parameter tensor."""
    rng = np.random.default_rng(1)
    flat = _small_params(3)
    st = rng.integers(0, 12, size=(3, 9, 15, 15))
    y = np.array([1.0, 0.0, 1.0])
    loss, g = vetter.gradients(flat, st, y)
    h = 1e-6
    o = 0
    for name, shape in vetter.SHAPES:
        k = int(np.prod(shape))
        for i in rng.choice(k, min(k, 6), replace=False):
            e = np.zeros_like(flat)
            e[o + i] = h
            lp = vetter.bce_with_logits(vetter.forward(flat + e, st)[0], y)
            lm = vetter.bce_with_logits(vetter.forward(flat - e, st)[0], y)
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[o + i]) <= 1e-6 * max(1.0, abs(fd)), (name, i, fd, g[o + i])
        o += k


def test_adam_first_step_closed_form():
    """With zero moments, Adam's first step moves every parameter by lr * sign(g)
    (up to eps)."""
    flat = np.ones(5)
    g = np.array([0.5, -2.0, 1e-3, -1e-4, 3.0])
    new, m, v = vetter.adam_step(flat, np.zeros(5), np.zeros(5), g, 1, 0.01)
    assert np.allclose(new, flat - 0.01 * np.sign(g), atol=1e-6)


def test_bf16_rounding():
    a = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, 3.14159, -0.1], np.float32)
    r = vetter.bf16_round(a)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2 ** -7
    assert abs(r[3] - 3.140625) < 1e-7 and abs(r[4] + 0.10009765625) < 1e-9


def test_stamp_center_is_the_candidate_count():
    w = W.tiny()
    cat = W.load(w)
    res = oracle.stack(cat, w.grid, w.n_min)
    cells = np.stack([res.cands["v_idx"], res.cands["bx"], res.cands["by"]], 1)[:6]
    st = vetter.stamps(cat, w.grid, cells)
    assert np.array_equal(st[:, 4, 7, 7], res.cands["distinct"][:6])


def test_stamps_match_brute_force_counts():
    """Every stamp element equals the distinct count of the brute-force
    histogram of that (velocity, bin), zeros off the lattice and domain."""
    cat, grid, _ = cases.random_tiny(11, max_n=60, max_side=4)
    bf, _ = brute.search(cat.x, cat.y, cat.epoch, cat.t, cat.ticks_per_hour, grid, 1)
    counts = {(c[0], c[1], c[2]): c[3] for c in bf}
    rng = np.random.default_rng(2)
    nv = grid.nvx * grid.nvy
    cells = np.stack([rng.integers(0, nv, 5), rng.integers(0, grid.nbx, 5),
                      rng.integers(0, grid.nby, 5)], 1)
    st = vetter.stamps(cat, grid, cells)
    for c, (v, bx, by) in enumerate(cells):
        kx, ky = v % grid.nvx, v // grid.nvx
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                for i in range(15):
                    for j in range(15):
                        kx2, ky2, xx, yy = kx + dx, ky + dy, bx - 7 + j, by - 7 + i
                        want = 0
                        if 0 <= kx2 < grid.nvx and 0 <= ky2 < grid.nvy:
                            want = counts.get((ky2 * grid.nvx + kx2, xx, yy), 0)
                        assert st[c, (dy + 1) * 3 + dx + 1, i, j] == want


def test_bf16_store_rounds_to_eight_bits():
    a = np.array([0.0, 1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, 1.0 + 2 ** -8 + 2 ** -30, -3.14159, 257.0, 259.0])
    r = vetter.bf16_store(a)
    assert list(r[:4]) == [0.0, 1.0, 1.0, 1.0 + 2 ** -7]
    assert r[4] == 1.0 + 2 ** -7            # just above the tie: rounds up (no double rounding)
    assert r[5] == -3.140625 and r[6] == 256.0 and r[7] == 260.0
    # on float32 inputs it agrees with the float32 -> bfloat16 rounding
    x = np.random.default_rng(0).normal(0, 10, 10000).astype(np.float32)
    assert np.array_equal(vetter.bf16_store(x.astype(np.float64)), vetter.bf16_round(x).astype(np.float64))


def _shift_network(seed):
    """Weights under which every activation is a small integer, exactly
    representable in BF16: each conv output channel copies one input channel
    at one tap (weight 1, bias 0); each fc1 unit sums a few features."""
    rng = np.random.default_rng(seed)
    p = {name: np.zeros(shape) for name, shape in vetter.SHAPES}
    for name, cin in (("conv1.w", 9), ("conv2.w", 32), ("conv3.w", 32)):
        for o in range(32):
            p[name][o, rng.integers(0, cin), rng.integers(0, 3), rng.integers(0, 3)] = 1.0
    for j in range(64):
        p["fc1.w"][j, rng.choice(2592, 20, replace=False)] = 1.0
    p["fc2.w"][:] = rng.choice([-0.5, 0.25, 1.0], 64)
    p["fc2.b"][0] = -3.0
    return vetter.flatten(p)


def test_store_rounding_is_a_no_op_on_representable_activations():
    """With exactly representable activations, BF16 storage changes nothing:
    the rounded forward and backward equal the exact (finite-difference
    pinned) ones bit for bit -- so the rounding touches activations only, not
    weights or deltas."""
    flat = _shift_network(5)
    rng = np.random.default_rng(6)
    st = 16 * rng.integers(0, 3, size=(4, 9, 15, 15))
    y = np.array([1.0, 0.0, 0.0, 1.0])
    l0, a0 = vetter.forward(flat, st)
    l1, a1 = vetter.forward(flat, st, vetter.bf16_store)
    assert np.array_equal(l0, l1)
    assert a0["a4"].max() > 0 and a0["a4"].max() < 256
    g0 = vetter.gradients(flat, st, y)
    g1 = vetter.gradients(flat, st, y, vetter.bf16_store)
    assert g0[0] == g1[0] and np.array_equal(g0[1], g1[1])


def test_store_rounding_applies_at_every_stored_activation():
    flat = _small_params(8)
    st = np.random.default_rng(3).integers(0, 300, size=(3, 9, 15, 15))
    _, a = vetter.forward(flat, st, vetter.bf16_store)
    _, ex = vetter.forward(flat, st)
    for k in ("x0", "a1", "a2", "a3", "a4"):
        assert np.array_equal(a[k], vetter.bf16_store(a[k])), k
        assert not np.array_equal(a[k], ex[k]), k
