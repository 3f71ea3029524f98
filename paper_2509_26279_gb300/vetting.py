"""Training and judging the candidate vetter (the learned filter the paper's
Sec. 5 calls for) on seeded synthetic fields.

Forms compared on the same fields, each reporting its candidate list:
  plain   -- the paper's threshold at the field's N_min (every cell >= N_min);
  low     -- the same threshold lowered to n_low(E) (fainter movers reachable,
             more contaminants);
  owned   -- the lowered threshold after ownership selection (sas_owned: each
             detection belongs to the first candidate containing it; a
             candidate stays when it owns at least half of its detections --
             the one-pass stand-in for the paper's peeling, Sec. 2.1 step 3);
  vetted  -- every candidate the plain threshold accepts (count >= N_min: the
             plain form stays the fallback, so recall is at least plain's in
             every bin) plus the owned candidates below it whose CNN logit
             reaches a threshold chosen on separate calibration fields for a
             target purity;
  vetted_dedup -- the same decision applied to the owned candidates only (one
             candidate per source, as the peel would report).

Truth (never an input of the method): a candidate is matched to mover m when
at least half of its contributing detection ids were made by m; otherwise it
is a contaminant (noise alignments or mixtures).  A mover is
recovered by a form when some reported candidate is matched to it.  Recall is
reported per 0.5-magnitude bin (the completeness-versus-magnitude view of
Sec. 3.4); purity = matched candidates / reported candidates.

All device work runs in the library (search, ownership, stamps, CNN); this module
marshals arrays and does the host-side bookkeeping.
"""
from __future__ import annotations

import math
from typing import Dict, List, Sequence

import numpy as np

from . import workloads as W

MAG_EDGES = np.arange(23.0, 26.5 + 1e-9, 0.5)


PARAMS = [("conv1.w", (32, 9, 3, 3)), ("conv1.b", (32,)), ("conv2.w", (32, 32, 3, 3)), ("conv2.b", (32,)),
          ("conv3.w", (32, 32, 3, 3)), ("conv3.b", (32,)), ("fc1.w", (64, 2592)), ("fc1.b", (64,)),
          ("fc2.w", (64,)), ("fc2.b", (1,))]


def init_params(seed: int) -> np.ndarray:
    """Fresh vetter parameters in the library's flat order: He-normal weights
    (std sqrt(2 / fan_in)), zero biases; float32."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, shape in PARAMS:
        k = int(np.prod(shape))
        if name.endswith(".b"):
            parts.append(np.zeros(k))
        else:
            fan_in = int(np.prod(shape[1:])) if len(shape) > 1 else shape[0]
            parts.append(rng.normal(0.0, math.sqrt(2.0 / fan_in), k))
    return np.concatenate(parts).astype(np.float32)


def n_low(n_epochs: int) -> int:
    """Lowered threshold for the vetted form: E/14, at least 5 (low enough that
    noise alignments appear in numbers; Sec. 2.2's false-positive rate)."""
    return max(5, -(-n_epochs // 14))


def noise_floor(n_detections: int, grid, budget: float = 5e4, superbin: int = 3) -> int:
    """Smallest k for which uniform noise of n_detections over the field is
    expected to fill fewer than `budget` (lattice point, superbin x superbin
    super-bin) pairs with k or more detections (Poisson tail, Sec. 2.2's
    false-positive count): below it a lowered threshold finds noise, not
    fainter movers."""
    n_sb = -(-grid.nbx // superbin) * -(-grid.nby // superbin)
    pairs = float(n_sb) * grid.nvx * grid.nvy
    lam = n_detections / float(n_sb)
    k, below, term = 0, 0.0, math.exp(-lam)   # below = P(X < k), term = P(X = k)
    while (1.0 - below) * pairs > budget:
        below += term
        k += 1
        term *= lam / k
    return max(k, 1)


def lowered_threshold(n_epochs: int, n_min: int, n_detections: int, grid, div: int = 6) -> int:
    """The lowered threshold ceil(E/div), raised to the field's noise floor and
    capped at n_min."""
    return min(n_min, max(-(-n_epochs // div), noise_floor(n_detections, grid)))


def truth_match(cands, ids, mover: np.ndarray) -> np.ndarray:
    """Mover index matched by each candidate (>= 50 % of its ids), else -1."""
    n = len(cands)
    out = np.full(n, -1, np.int64)
    if n == 0:
        return out
    lens = cands["id_len"].astype(np.int64)
    offs = cands["id_off"].astype(np.int64)
    cid = np.repeat(np.arange(n), lens)
    pos = np.repeat(offs - np.concatenate([[0], np.cumsum(lens)[:-1]]), lens) + np.arange(lens.sum())
    m = mover[ids[pos].astype(np.int64)].astype(np.int64)
    sel = m >= 0
    if not sel.any():
        return out
    big = int(m.max()) + 1
    key, cnt = np.unique(cid[sel] * big + m[sel], return_counts=True)
    c_of, m_of = key // big, key % big
    order = np.lexsort((cnt, c_of))                 # per candidate, largest count last
    last = np.r_[c_of[order][1:] != c_of[order][:-1], True]
    c_best, m_best, n_best = c_of[order][last], m_of[order][last], cnt[order][last]
    ok = 2 * n_best >= lens[c_best]
    out[c_best[ok]] = m_best[ok]
    return out


def recall_by_mag(found: np.ndarray, movers) -> Dict[str, list]:
    """Per 0.5-mag bin: number of injected movers and number recovered."""
    mags = movers["mag"]
    b = np.clip(np.digitize(mags, MAG_EDGES) - 1, 0, len(MAG_EDGES) - 2)
    tot = np.bincount(b, minlength=len(MAG_EDGES) - 1)
    rec = np.bincount(b[found], minlength=len(MAG_EDGES) - 1) if len(found) else np.zeros_like(tot)
    return {"total": tot.tolist(), "found": rec.tolist()}


def _recovered(match: np.ndarray, keep: np.ndarray | None = None) -> np.ndarray:
    m = match if keep is None else match[keep]
    return np.unique(m[m >= 0])


class Field:
    """One workload's catalog on the device."""

    def __init__(self, w: W.Workload, device):
        import torch
        from . import sas
        self.w = w
        self.cat = W.load(w)
        self.grid = sas.Grid(w.grid)
        self.dx = torch.from_numpy(self.cat.x).to(device)
        self.dy = torch.from_numpy(self.cat.y).to(device)
        self.de = torch.from_numpy(self.cat.epoch.view(np.int16)).to(device)
        self.E = w.recipe.n_epochs

    def search(self, n_min: int, stream=None):
        from . import sas
        return sas.sas_stack(self.grid, self.dx, self.dy, self.de, self.cat.t, self.cat.ticks_per_hour,
                             n_min, on_device=True, stream=stream)


def owned_stamps(res, device, n_keep: int = 0, stream=None):
    """(kept indices [k] int64 host, stamps [k, 9, 15, 15] device int16 view of
    u16) of the candidates that survive ownership selection (n_keep: the
    search's threshold, see sas_owned)."""
    import torch
    from . import sas
    n = res.info()["n_candidates"]
    idx = torch.empty(max(n, 1), dtype=torch.int32, device=device)
    k = sas.sas_owned(res, idx, n_keep, stream=stream)
    st = torch.empty((max(k, 1), 9, 15, 15), dtype=torch.int16, device=device)
    sas.sas_stamps_indexed(res, idx, k, st, stream=stream)
    return idx[:k].cpu().numpy().astype(np.int64), st[:k]


def training_set(workloads: Sequence[W.Workload], device):
    """Stamps of the owned candidates of each field searched at n_low(E), with
    labels 1 (matched to a mover) or 0; stamps stay on the device."""
    import torch
    stamps, labels = [], []
    for w in workloads:
        f = Field(w, device)
        res = f.search(n_low(f.E))
        cands, ids = res.candidates()
        pk, st = owned_stamps(res, device, n_low(f.E))
        match = truth_match(cands, ids, f.cat.mover)
        stamps.append(st)
        labels.append((match[pk] >= 0).astype(np.float32))
        res.free()
    st = torch.cat(stamps) if stamps else torch.empty((0, 9, 15, 15), dtype=torch.int16, device=device)
    lab = torch.from_numpy(np.concatenate(labels) if labels else np.zeros(0, np.float32)).to(device)
    return st, lab


def train(vetter, stamps, labels, epochs: int = 20, batch: int = 512, lr: float = 1e-3, seed: int = 0):
    """Adam on shuffled mini-batches (the library gathers each batch through an
    index array); returns the mean loss of each epoch."""
    import torch
    n = int(stamps.shape[0])
    gen = np.random.default_rng(seed)
    loss = torch.zeros(1, device=stamps.device)
    hist = []
    for _ in range(epochs):
        perm = torch.from_numpy(gen.permutation(n).astype(np.int32)).to(stamps.device)
        acc = 0.0
        steps = 0
        for b0 in range(0, n, batch):
            nb = min(batch, n - b0)
            vetter.train_step(stamps, labels, nb, lr, loss, index=perm[b0:b0 + nb])
            acc += float(loss.item())
            steps += 1
        hist.append(acc / max(steps, 1))
    return hist


def vetted_keep(counts, logits, plain_n_min: int, threshold: float) -> np.ndarray:
    """The vetted decision for owned candidates: kept when the plain
    threshold accepts them or the CNN scores them at or above threshold."""
    return (np.asarray(counts) >= plain_n_min) | (np.asarray(logits) >= threshold)


def vetted_mask(counts, owned_idx, owned_logits, plain_n_min: int, threshold: float) -> np.ndarray:
    """The vetted form over a whole candidate list: every candidate at or above
    the plain threshold, plus the owned ones the CNN accepts."""
    mask = np.asarray(counts) >= plain_n_min
    owned_idx = np.asarray(owned_idx, np.int64)
    mask[owned_idx[np.asarray(owned_logits) >= threshold]] = True
    return mask


def logits_of(vetter, stamps) -> np.ndarray:
    """CNN logits of device stamps, to the host."""
    import torch
    n = int(stamps.shape[0])
    out = torch.zeros(max(n, 1), device=stamps.device)
    vetter.forward(stamps, n, out)
    return out[:n].cpu().numpy().astype(np.float64)


def calibrate(logits: np.ndarray, labels: np.ndarray, target_purity: float) -> float:
    """Lowest logit threshold whose kept set (logit >= threshold) still has at
    least the target purity, scanning thresholds from the top; +inf when even
    the best-scored candidate is a contaminant."""
    order = np.argsort(-logits, kind="stable")
    lab = np.asarray(labels, np.float64)[order]
    prec = np.cumsum(lab) / np.arange(1, len(lab) + 1)
    ok = np.nonzero(prec >= target_purity)[0]
    if len(ok) == 0:
        return float("inf")
    return float(logits[order][ok[-1]])


def evaluate(vetter, workloads: Sequence[W.Workload], device, threshold: float = 0.0) -> dict:
    """Recall per magnitude bin and purity of the plain, low, owned, vetted and
    vetted_dedup forms."""
    import torch
    nb = len(MAG_EDGES) - 1
    acc = {k: {"total": [0] * nb, "found": [0] * nb, "reported": 0, "matched": 0}
           for k in ("plain", "low", "owned", "vetted", "vetted_dedup")}
    for w in workloads:
        f = Field(w, device)
        movers = f.cat.movers
        rp = f.search(w.n_min)
        cp, ip = rp.candidates()
        mp = truth_match(cp, ip, f.cat.mover)
        rl = f.search(n_low(f.E))
        cl, il = rl.candidates()
        ml = truth_match(cl, il, f.cat.mover)
        pk, st = owned_stamps(rl, device, n_low(f.E))
        logits = torch.zeros(max(len(pk), 1), device=device)
        vetter.forward(st, len(pk), logits)
        lg = logits[:len(pk)].cpu().numpy()
        keep = vetted_keep(cl["count"][pk], lg, w.n_min, threshold)
        sel = {"plain": (mp, None), "low": (ml, None), "owned": (ml[pk], None),
               "vetted": (ml, vetted_mask(cl["count"], pk, lg, w.n_min, threshold)),
               "vetted_dedup": (ml[pk], keep)}
        for k, (m, kp) in sel.items():
            r = recall_by_mag(_recovered(m, kp), movers)
            a = acc[k]
            a["total"] = [x + y for x, y in zip(a["total"], r["total"])]
            a["found"] = [x + y for x, y in zip(a["found"], r["found"])]
            mm = m if kp is None else m[kp]
            a["reported"] += int(len(mm))
            a["matched"] += int((mm >= 0).sum())
        rp.free()
        rl.free()
    for a in acc.values():
        a["recall"] = [fd / t if t else None for fd, t in zip(a["found"], a["total"])]
        a["purity"] = a["matched"] / a["reported"] if a["reported"] else None
    acc["mag_edges"] = MAG_EDGES.tolist()
    return acc
