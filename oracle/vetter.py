"""CPU oracle of the candidate vetter -- TEST INFRASTRUCTURE (float64 NumPy).

The paper's conclusion (Sec. 5) names better filtering of the search results as
the way to reach fainter objects without drowning in candidates.  The vetter is
that filter: a small convolutional network that scores a candidate from its
count stamp.  This module is the plain definition the GPU kernels are checked
against; it shares nothing with them.

Stamp of candidate (v_idx, bx, by): a 9 x 15 x 15 array of distinct-epoch
counts; plane q = (dy + 1) * 3 + (dx + 1) is the 2-D histogram (Sec. 2.1
step 2) of lattice point (kx + dx, ky + dy), dx, dy in {-1, 0, 1}; element
(i, j) is its bin (bx - 7 + j, by - 7 + i).  Points off the lattice and bins
off the domain count 0.

Network (input x = count / 16):
  conv1 9->32 3x3 valid, ReLU (15 -> 13); conv2 32->32 (13 -> 11), ReLU;
  conv3 32->32 (11 -> 9), ReLU; flatten in (channel, row, column) order;
  fc1 2592 -> 64, ReLU; fc2 64 -> 1 (the logit).
Loss: mean binary cross-entropy with logits.
Arithmetic: float64 throughout.  forward/gradients take an optional `store`
rounding applied where the GPU stores an activation; bf16_round there is the
network's stated precision (BF16 activations, wide accumulation).
Flat parameter layout (float32 on the GPU, float64 here), in this order:
  conv1.w [32,9,3,3], conv1.b [32], conv2.w [32,32,3,3], conv2.b [32],
  conv3.w [32,32,3,3], conv3.b [32], fc1.w [64,2592], fc1.b [64],
  fc2.w [64], fc2.b [1]   -- 187,137 numbers.
Parity status: pinned (central finite differences, closed forms, stamps
against the oracle's histograms and the brute force); see
tests/test_oracle_vetter.py.
"""
from __future__ import annotations

import numpy as np

import oracle

SHAPES = [("conv1.w", (32, 9, 3, 3)), ("conv1.b", (32,)), ("conv2.w", (32, 32, 3, 3)),
          ("conv2.b", (32,)), ("conv3.w", (32, 32, 3, 3)), ("conv3.b", (32,)),
          ("fc1.w", (64, 2592)), ("fc1.b", (64,)), ("fc2.w", (64,)), ("fc2.b", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)
assert N_PARAMS == 187137


def unflatten(flat: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = flat[o:o + k].reshape(shape)
        o += k
    return out


def flatten(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], np.float64).ravel() for name, _ in SHAPES])


def init_params(seed: int) -> np.ndarray:
    """He-normal weights, zero biases (float32 values)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shape in SHAPES:
        if name.endswith(".b"):
            p[name] = np.zeros(shape)
        else:
            fan_in = int(np.prod(shape[1:])) if len(shape) > 1 else shape[0]
            p[name] = rng.normal(0.0, np.sqrt(2.0 / fan_in), shape)
    return flatten(p).astype(np.float32)


# ---- stamps ---------------------------------------------------------------------

def stamps(cat, grid, cells) -> np.ndarray:
    """Count stamps [n, 9, 15, 15] (int) of cells (v_idx, bx, by)."""
    cells = np.asarray(cells, np.int64).reshape(-1, 3)
    out = np.zeros((len(cells), 9, 15, 15), np.int64)
    hist = {}
    for c, (v, bx, by) in enumerate(cells):
        kx, ky = v % grid.nvx, v // grid.nvx
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                kx2, ky2 = kx + dx, ky + dy
                if not (0 <= kx2 < grid.nvx and 0 <= ky2 < grid.nvy):
                    continue
                key = (kx2, ky2)
                if key not in hist:
                    vx = grid.vx0 + kx2 * grid.dvx
                    vy = grid.vy0 + ky2 * grid.dvy
                    hist[key] = oracle.histogram(cat, grid, vx, vy)[0]
                h = hist[key]
                q = (dy + 1) * 3 + (dx + 1)
                for i in range(15):
                    yy = by - 7 + i
                    if not 0 <= yy < grid.nby:
                        continue
                    for j in range(15):
                        xx = bx - 7 + j
                        if 0 <= xx < grid.nbx:
                            out[c, q, i, j] = h[yy, xx]
    return out


# ---- network ----------------------------------------------------------------------

def _conv(x, w, b):
    """Valid 3x3 convolution: x [B, C, H, W], w [O, C, 3, 3] -> [B, O, H-2, W-2]."""
    B, C, H, W = x.shape
    out = np.zeros((B, w.shape[0], H - 2, W - 2))
    for dy in range(3):
        for dx in range(3):
            patch = x[:, :, dy:dy + H - 2, dx:dx + W - 2]          # [B, C, H-2, W-2]
            out += np.einsum("bchw,oc->bohw", patch, w[:, :, dy, dx])
    return out + b[None, :, None, None]


def _conv_back(x, w, g):
    """Gradients of _conv: (dx, dw, db) given upstream g [B, O, H-2, W-2]."""
    B, C, H, W = x.shape
    dx = np.zeros_like(x)
    dw = np.zeros_like(w)
    for dy in range(3):
        for ddx in range(3):
            patch = x[:, :, dy:dy + H - 2, ddx:ddx + W - 2]
            dw[:, :, dy, ddx] = np.einsum("bohw,bchw->oc", g, patch)
            dx[:, :, dy:dy + H - 2, ddx:ddx + W - 2] += np.einsum("bohw,oc->bchw", g, w[:, :, dy, ddx])
    return dx, dw, g.sum(axis=(0, 2, 3))


def forward(flat, stamp_counts, store=None):
    """Logits [B] and the activations needed by backward.

    store: None for exact float64 activations, or a function applied to every
    stored activation (input x0, a1, a2, a3, fc1 output a4) -- bf16_round gives
    the network's stated arithmetic (BF16 activations, wide accumulation); all
    arithmetic stays float64."""
    st = store if store is not None else (lambda a: a)
    p = unflatten(np.asarray(flat, np.float64))
    x0 = st(np.asarray(stamp_counts, np.float64) / 16.0)
    z1 = _conv(x0, p["conv1.w"], p["conv1.b"]); a1 = st(np.maximum(z1, 0))
    z2 = _conv(a1, p["conv2.w"], p["conv2.b"]); a2 = st(np.maximum(z2, 0))
    z3 = _conv(a2, p["conv3.w"], p["conv3.b"]); a3 = st(np.maximum(z3, 0))
    f = a3.reshape(len(x0), -1)
    z4 = f @ p["fc1.w"].T + p["fc1.b"]; a4 = st(np.maximum(z4, 0))
    logit = a4 @ p["fc2.w"] + p["fc2.b"][0]
    return logit, dict(x0=x0, a1=a1, a2=a2, a3=a3, f=f, a4=a4, p=p)


def bce_with_logits(logit, y):
    """Mean binary cross-entropy, written in its numerically stable form."""
    logit = np.asarray(logit, np.float64)
    y = np.asarray(y, np.float64)
    return float(np.mean(np.maximum(logit, 0) - logit * y + np.log1p(np.exp(-np.abs(logit)))))


def backward(flat, act, g_logit):
    """Flat gradient of the loss given dL/dlogit per sample and the activations
    the forward stored (act: x0, a1, a2, a3, a4 as forward returns them):
    back-propagation through those values and their ReLU masks (a > 0)."""
    p = unflatten(np.asarray(flat, np.float64))
    a1, a2, a3, a4 = (np.asarray(act[k], np.float64) for k in ("a1", "a2", "a3", "a4"))
    x0 = np.asarray(act["x0"], np.float64)
    g_logit = np.asarray(g_logit, np.float64)
    g = {}
    g["fc2.w"] = a4.T @ g_logit
    g["fc2.b"] = np.array([g_logit.sum()])
    g4 = np.outer(g_logit, p["fc2.w"]) * (a4 > 0)
    g["fc1.w"] = g4.T @ a3.reshape(len(a3), -1)
    g["fc1.b"] = g4.sum(axis=0)
    g3 = (g4 @ p["fc1.w"]).reshape(a3.shape) * (a3 > 0)
    d2, g["conv3.w"], g["conv3.b"] = _conv_back(a2, p["conv3.w"], g3)
    g2 = d2 * (a2 > 0)
    d1, g["conv2.w"], g["conv2.b"] = _conv_back(a1, p["conv2.w"], g2)
    g1 = d1 * (a1 > 0)
    _, g["conv1.w"], g["conv1.b"] = _conv_back(x0, p["conv1.w"], g1)
    return flatten(g)


def gradients(flat, stamp_counts, y, store=None):
    """(loss, flat gradient of the mean BCE loss).  With store (see forward),
    back-propagation runs through the stored activations: their ReLU masks
    and their values in the weight gradients."""
    logit, a = forward(flat, stamp_counts, store)
    B = len(logit)
    y = np.asarray(y, np.float64)
    g_logit = (1.0 / (1.0 + np.exp(-logit)) - y) / B              # d loss / d logit
    return bce_with_logits(logit, y), backward(flat, a, g_logit)


def adam_step(flat, m, v, grad, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) in float64; returns (flat, m, v)."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return flat - lr * mh / (np.sqrt(vh) + eps), m, v


def bf16_round(a):
    """Round values to float32, then to the nearest bfloat16 (ties to even);
    returns float32 (finite inputs)."""
    a = np.asarray(a, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def bf16_store(a):
    """Round float64 values directly to the nearest bfloat16 (8 significant
    bits, ties to even); returns float64.  The `store` rounding of forward and
    gradients for the network's BF16 activations (normal range)."""
    m, e = np.frexp(np.asarray(a, np.float64))
    return np.ldexp(np.rint(np.ldexp(m, 8)), e - 8)
