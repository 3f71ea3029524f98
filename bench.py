#!/usr/bin/env python
"""Benchmark of the catalog shift-and-stack hot path (Sec. 2.1 steps 1-3) on GB300.

One step = one full search (ingest, bucket, shift tables, stack, exact counts,
ordering, contributing ids) over the DECam-CCD-like outer-solar-system field:
2048x4096 px, 100 epochs over 4 h, 3000 noise detections per epoch plus 200
injected movers, a 111x111 velocity lattice (364 mpx/h spacing), 2 px bins,
N_min = 25.  The metric is detection-shifts per second: in-domain
(detection, velocity) pairs processed per second.

  value     device-resident inputs, CUDA events around each step on the stream
            the library launches on, L2 flushed (256 MiB write) between steps
  e2e       the same search through the C ABI with pinned host buffers: the
            host->device copy of the catalog and the device->host copy of the
            candidates and ids (into page-locked arrays allocated once and
            reused) are inside the timed region (wall clock)
  roofline  the stack kernel against the shared-memory atomic peak measured in
            this run by the library's probe (one atomic per detection-shift)

  fields    fields/s of the plain form (one search per field) against the
            batched + vetted form on 60 uneven fields, with recall per
            magnitude bin and purity (after training the vetter, untimed)

  configs   the other search workloads (tiny, fast_movers) measured the same
            way, each with its stack kernel's roofline fraction and the oracle

--impl reference times the CPU oracle (the plain definition; its OpenMP form
over velocity chunks on all host cores) on a bounded lattice sample of the same
workload.  --vetter-timing, --refine-timing and --selection-timing print only
the timing of the vetter's kernels, of refinement, or of the stack kernel with
one threshold and with the peaks alone (the commands the profiles were taken
with).
Multi-GPU (torchrun): each rank searches its own field (weak scaling); the
only collectives are the timing barrier and the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2509_26279_gb300 import workloads as W  # noqa: E402

METRIC = "detection-shifts/s"
UNIT = "det-shifts/s"
L2_FLUSH_BYTES = 256 << 20
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def workload_desc(w: W.Workload, cat) -> dict:
    r, g = w.recipe, w.grid
    return {
        "workload": (f"{w.name}: {r.width_px}x{r.height_px} px, {r.n_epochs} epochs over "
                     f"{r.span_h:g} h, {r.noise_per_epoch} noise/epoch + {r.n_movers} movers, "
                     f"{g.nvx}x{g.nvy} velocity lattice at {g.dvx} mpx/h, bin {g.bin / 1000:g} px, "
                     f"N_min {w.n_min}"),
        "n_detections": int(cat.n),
        "n_velocities": int(g.nvx * g.nvy),
        "seed": int(w.seed),
    }


class ClockSampler:
    """nvidia-smi sampled every 100 ms while the timed region runs."""

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        # raw samples (the summary goes into the bench line): SAS_CLOCKS_DIR, else a temp dir
        import tempfile
        self.path = os.path.join(os.environ.get("SAS_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"sas_clocks_rank{gpu_index}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={CLOCK_FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self) -> dict:
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [q.strip() for q in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for name, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


STACK_SOURCES = ("sas_stack_kernel.cuh", "sas_stack.cu")  # the kernel and its one-threshold instantiations


def stack_source_sha256() -> str:
    """sha256 over the stack kernel's source files, in STACK_SOURCES order."""
    h = hashlib.sha256()
    for name in STACK_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2509_26279_gb300", "csrc", name), "rb").read())
    return h.hexdigest()


def stack_traffic(workload: str):
    """DRAM bytes per stack launch from the committed ncu summary of this
    workload, if it was taken on the current stack kernel source; else None."""
    p = os.path.join(ROOT, "profiles", f"k_stack_{workload}.md")
    if not os.path.exists(p):
        return None
    fields = {}
    for line in open(p):
        k, sep, v = line.strip().partition(":")
        if sep and k in ("stack_source_sha256", "traffic_bytes_per_launch"):
            fields[k] = v.strip()
    h = stack_source_sha256()
    if fields.get("stack_source_sha256") != h or "traffic_bytes_per_launch" not in fields:
        return None
    return int(fields["traffic_bytes_per_launch"])


def host_info() -> dict:
    """The host the CPU baseline ran on: CPU model, logical CPUs, the CPUs this
    process may run on, and the oracle's default OpenMP team."""
    import oracle
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            k, _, v = line.partition(":")
            if k.strip() in ("Model name", "Vendor ID") and v.strip() and v.strip() != "-":
                model = v.strip() if model is None or k.strip() == "Model name" else model
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None and os.path.exists("/proc/cpuinfo"):
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    return {"cpu_model": model, "nproc": os.cpu_count(),
            "affinity": len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else None,
            "oracle_openmp_threads": oracle.threads()}


def cpu_baseline(w: W.Workload, cat, budget_s: float = 15.0) -> dict:
    """The oracle as it stands on the same workload: single thread on whole
    lattice rows, grown until about budget_s / 2 seconds, and its OpenMP form
    (velocity chunks over every core of the team) on a contiguous lattice range
    sized to about the same time.  The main figure is the OpenMP one; both are
    in det-shifts/s (in-domain pairs per second of wall time)."""
    import oracle
    g = w.grid
    nv = g.nvx * g.nvy
    rows, pairs, secs = 0, 0, 0.0
    row = g.nvy // 2
    while secs < budget_s / 2 and rows < g.nvy:
        ky = (row + rows) % g.nvy
        t0 = time.perf_counter()
        r = oracle.stack(cat, g, w.n_min, ky * g.nvx, (ky + 1) * g.nvx)
        secs += time.perf_counter() - t0
        pairs += r.n_pairs
        rows += 1
    single = {"value": pairs / secs, "cores": 1,
              "sample": f"{rows} lattice rows x {g.nvx} velocities ({pairs} detection-shifts in {secs:.1f} s)"}
    thr = oracle.threads()
    per_v = secs / max(1, rows * g.nvx)                       # one velocity, one thread
    n_v = int(min(nv, max(thr, budget_s / 2 / max(per_v, 1e-9) * thr * 0.8)))
    a = max(0, nv // 2 - n_v // 2)
    t0 = time.perf_counter()
    r = oracle.stack(cat, g, w.n_min, a, a + n_v, threads=0)
    secs_mt = time.perf_counter() - t0
    return {"value": r.n_pairs / secs_mt, "unit": UNIT, "cores": thr, "kind": "oracle",
            "sample": f"OpenMP over {thr} threads: lattice indices [{a}, {a + n_v}) of the same field "
                      f"({r.n_pairs} detection-shifts in {secs_mt:.1f} s)",
            "single_thread": single, "host": host_info()}


def fields_section(dev, stream, n_fields: int = 60, train_fields: int = 30, epochs: int = 15,
                   reps: int = 2) -> dict:
    """fields/s on the batched uneven fields (60 CCDs, epochs U{20..150}, noise
    log-U[1e3, 8e3]): the plain form (one sas_stack per field at N_min =
    ceil(E/4)) against the batched + vetted forms (one graph-captured batch
    pass with the autotuner's per-size-class tiles, then ownership selection,
    stamps and the CNN of all fields in one pass, sas_batch_vet): at the plain
    threshold, at a lowered one, with the tile-local super-bin peaks at a
    lowered threshold added to the plain list, and with the peaks alone (the
    cells every mover raises around its best cell pruned before counting);
    recall per 0.5-mag bin and purity of each form's reported candidates.  The
    vetter is trained first (not timed) on separate seeded fields."""
    import torch
    from paper_2509_26279_gb300 import sas, vetting

    t0 = time.perf_counter()
    st, lab = vetting.training_set(W.vetter_fields(train_fields, seed=W.BASE_SEED + 50), dev)
    vt = sas.Vetter(dev.index or 0, 512)
    vt.set_state(vetting.init_params(1))
    hist = vetting.train(vt, st, lab, epochs=epochs, batch=512, lr=1e-3)
    n_train = int(st.shape[0])
    del st, lab
    cst, clab = vetting.training_set(W.vetter_fields(10, seed=W.BASE_SEED + 70), dev)
    tau = vetting.calibrate(vetting.logits_of(vt, cst), clab.cpu().numpy(), 0.95)
    del cst, clab
    train_s = time.perf_counter() - t0

    fields = [vetting.Field(w, dev) for w in W.batched_fields(n_fields)]
    nb = len(vetting.MAG_EDGES) - 1

    def score(per_field):
        tot, fnd, rep, mat = [0] * nb, [0] * nb, 0, 0
        for f, (cands, ids, keep) in zip(fields, per_field):
            m = vetting.truth_match(cands, ids, f.cat.mover)
            if keep is not None:
                m = m[keep]
            r = vetting.recall_by_mag(np.unique(m[m >= 0]), f.cat.movers)
            tot = [a + b for a, b in zip(tot, r["total"])]
            fnd = [a + b for a, b in zip(fnd, r["found"])]
            rep += len(m)
            mat += int((m >= 0).sum())
        return {"recall_by_mag": [round(b / a, 4) if a else None for a, b in zip(tot, fnd)],
                "movers_by_mag": tot, "reported": rep, "purity": round(mat / rep, 4) if rep else None}

    def timed(fn):
        fn()                                   # warm-up
        best = None
        for _ in range(reps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None or ms < best else best
        return best, out

    def plain():
        res = [f.search(f.w.n_min, stream) for f in fields]
        return res

    ms_plain, res = timed(plain)
    plain_out = []
    for r in res:
        c, i = r.candidates()
        plain_out.append((c, i, None))
        r.free()

    # autotuner: one measured sweep per size class (untimed), each field takes its class's options
    from paper_2509_26279_gb300 import tuning
    t1 = time.perf_counter()
    cache = tuning.TuneCache(os.environ.get("SAS_TUNE_CACHE"))
    gpu_name = torch.cuda.get_device_name(dev)
    for f in fields:
        cache.tune(f, gpu_name)
    if cache.path:
        cache.save()
    tune_s = time.perf_counter() - t1
    tuned_opts = [cache.opts_for(f) for f in fields]

    def lowered(div):
        # ceil(E/div), raised to the field's noise floor (vetting.lowered_threshold)
        return lambda f: vetting.lowered_threshold(f.E, f.w.n_min, f.cat.n, f.w.grid, div)

    # the peaks-only form at the lowered threshold gets its own tuning pass: the
    # peak tests and the smaller count stage change what each tile shape costs
    t2 = time.perf_counter()
    po_tag = "peaks_only_e6:"
    for f in fields:
        cache.tune(f, gpu_name, base=sas.make_opts(n_low=lowered(6)(f), peaks_only=1), tag=po_tag)
    tune_po_s = time.perf_counter() - t2
    po_opts = [cache.opts_for(f, po_tag) for f in fields]

    def make_batch(thr, low=None, peaks_only=0, opts_base=None):
        opts = []
        for f, o in zip(fields, opts_base):
            o2 = sas.make_opts(**{k: getattr(o, k) for k, _ in sas.sas_opts._fields_})
            o2.n_low = low(f) if low is not None else 0
            o2.peaks_only = peaks_only
            opts.append(o2)
        return sas.Batch([(f.grid, f.dx, f.dy, f.de, f.cat.t, f.cat.ticks_per_hour, thr(f)) for f in fields],
                         opts=opts, stream=stream)

    planner_opts = [sas.make_opts() for _ in fields]

    def pick_batch(thr, low, peaks_only, tuned):
        """The batch built with the autotuner's per-class tiles or with the
        planner's, whichever replays faster (the tuner times single searches;
        its choice does not always carry over to one pass over all fields).
        Untimed: one warm-up and two timed replays of each."""
        best = None
        for label, ob in (("autotuned", tuned), ("planner", planner_opts)):
            b = make_batch(thr, low, peaks_only, ob)
            b.run(stream)
            ts = []
            for _ in range(2):
                torch.cuda.synchronize()
                t = time.perf_counter()
                b.run(stream)
                ts.append(time.perf_counter() - t)
            if best is None or min(ts) < best[0]:
                if best is not None:
                    best[2].destroy()
                best = (min(ts), label, b)
            else:
                b.destroy()
        return best[2], best[1]

    def vetted_pass(batch, cap):
        fo = torch.empty(cap, dtype=torch.int32, device=dev)
        co = torch.empty(cap, dtype=torch.int32, device=dev)
        lo = torch.empty(cap, dtype=torch.float32, device=dev)

        def run():
            batch.run(stream)
            n = batch.vet(vt, fo, co, lo, cap, stream)
            return fo[:n], co[:n], lo[:n]
        return run

    result = {"workload": f"batched_fields: {n_fields} CCDs 2048x4096 px, epochs U{{20..150}} over 4 h, "
                          f"noise/epoch log-U[1e3,8e3], 200 movers each, 111x111 lattice, bin 2 px",
              "plain": {"form": "one sas_stack per field, N_min = ceil(E/4)", "ms": round(ms_plain, 3),
                        "fields_per_s": round(n_fields / (ms_plain * 1e-3), 2), **score(plain_out)},
              "autotune": {"classes": len(cache.entries), "seconds": round(tune_s + tune_po_s, 1),
                           "choices": {k: tuning.shape_of(v) for k, v in cache.entries.items()},
                           "ms": {k: v["ms"] for k, v in cache.entries.items()},
                           "planner_ms": {k: v.get("planner_ms") for k, v in cache.entries.items()},
                           "rule": "sas_autotune per size class: velocity tile {8x8, 8x4} x super-bin {1..4} x "
                                   "tile_bx {planner, 32, 64} x velocity block {planner, 2, 4}, median of 3"},
              "vetter_training": {"fields": train_fields, "stamps": n_train, "epochs": epochs,
                                  "final_loss": round(hist[-1], 4), "seconds": round(train_s, 1),
                                  "threshold": round(tau, 4),
                                  "threshold_rule": "purity 0.95 on 10 separate calibration fields"}}
    e4 = lambda f: f.w.n_min
    e6 = lambda f: -(-f.E // 6)
    floor_note = " (raised to the field's noise floor: fewer than 5e4 expected noise pairs)"
    for name, thr, low, po, obase, desc in (
            ("batched_vetted", e4, None, 0, tuned_opts, "batch at N_min = ceil(E/4)"),
            ("batched_vetted_e6", e6, None, 0, tuned_opts, "batch at N_min = ceil(E/6)"),
            ("batched_peaks_e6", e4, lowered(6), 0, tuned_opts,
             "batch at N_min = ceil(E/4) plus the cells of tile-local super-bin peaks at n_low = ceil(E/6)"
             + floor_note),
            ("batched_peaksonly_e4", e4, None, 1, tuned_opts,
             "batch keeping only the cells of tile-local super-bin peaks, at N_min = ceil(E/4)"),
            ("batched_peaksonly_e5", e4, lowered(5), 1, po_opts,
             "batch keeping only the cells of tile-local super-bin peaks, at n_low = ceil(E/5)" + floor_note),
            ("batched_peaksonly_e6", e4, lowered(6), 1, po_opts,
             "batch keeping only the cells of tile-local super-bin peaks, at n_low = ceil(E/6)" + floor_note),
            ("batched_peaksonly_e8", e4, lowered(8), 1, po_opts,
             "batch keeping only the cells of tile-local super-bin peaks, at n_low = ceil(E/8)" + floor_note)):
        if name == "batched_vetted_e6":  # the slow one-threshold comparison: the tuned tiles only
            batch, tiles = make_batch(thr, low, po, obase), "autotuned"
        else:
            batch, tiles = pick_batch(thr, low, po, obase)
        batch.run(stream)
        cap = sum(max(batch.field_info(k)["n_candidates"], 1) for k in range(len(fields))) + 1
        ms, (fo, co, lo) = timed(vetted_pass(batch, cap))
        fo, co, lo = fo.cpu().numpy(), co.cpu().numpy(), lo.cpu().numpy()
        per_field, per_field_dedup = [], []
        for k in range(len(fields)):
            c, i = batch.candidates(k)
            sel = fo == k
            idx = co[sel]
            per_field.append((c, i, vetting.vetted_mask(c["count"], idx, lo[sel], fields[k].w.n_min, tau)))
            dd = np.zeros(len(c), bool)
            dd[idx[vetting.vetted_keep(c["count"][idx], lo[sel], fields[k].w.n_min, tau)]] = True
            per_field_dedup.append((c, i, dd))
        _, fallbacks = batch.stats()
        result[name] = {"form": desc + "; every reported candidate with count >= ceil(E/4) kept, plus the "
                                       "ownership-selected candidates below it whose CNN logit >= the "
                                       "calibrated threshold",
                        "tiles": tiles if tiles == "planner" else
                        ("autotuned for this form" if obase is po_opts else "autotuned at N_min"),
                        "ms": round(ms, 3),
                        "fields_per_s": round(n_fields / (ms * 1e-3), 2), "fallbacks": int(fallbacks),
                        "rebuilds": int(batch.rebuilds),
                        "candidates_searched": int(sum(batch.field_info(k)["n_candidates"]
                                                       for k in range(len(fields)))),
                        "superbins_emitted": int(sum(batch.field_info(k)["n_emitted"]
                                                     for k in range(len(fields)))),
                        **score(per_field),
                        "dedup": {"form": "the same decision on the ownership-selected candidates only",
                                  **score(per_field_dedup)}}
        batch.destroy()
    return result


def peel_section(grid, dx, dy, de, cat, w, stream, reps: int = 5) -> dict:
    """Cluster finding (Sec. 2.1 step 3) on one search result of the bench
    workload: time per sas_peel call (setup + the loop + output records), the
    clusters it returns and how they map onto the injected movers."""
    import torch
    from paper_2509_26279_gb300 import sas

    res = sas.sas_stack(grid, dx, dy, de, cat.t, cat.ticks_per_hour, w.n_min, on_device=True, stream=stream)
    n_cand = int(res.info()["n_candidates"])
    ms = []
    for i in range(reps + 2):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pl = sas.sas_peel(res, w.n_min, 1000, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        if i >= 2:
            ms.append(a.elapsed_time(b))
        if i < reps + 1:
            pl.free()
    cands, ids = pl.candidates()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    sq = sas.sas_peel(res, w.n_min, 1000, stream=stream, sequential=True)
    b.record(stream)
    torch.cuda.synchronize()
    ms_seq = a.elapsed_time(b)
    same = len(sq.candidates()[0]) == len(cands)
    sq.free()
    found, pure = set(), 0
    for c in cands:
        m = cat.mover[ids[int(c["id_off"]): int(c["id_off"]) + int(c["id_len"])]]
        top = np.bincount(m[m >= 0]).argmax() if (m >= 0).any() else -1
        if top >= 0 and 2 * int((m == top).sum()) >= len(m):
            pure += 1
            found.add(int(top))
    ep = {}
    for e, mv in zip(cat.epoch[cat.mover >= 0], cat.mover[cat.mover >= 0]):
        ep.setdefault(int(mv), set()).add(int(e))
    findable = sum(len(v) >= w.n_min for v in ep.values())
    # Sec. 2.1 steps 4-6 on the clusters: FAST-MCD regression, gather, repeat
    rms = []
    for i in range(4):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        tr = sas.sas_refine(res, pl, seed=1, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        if i >= 1:
            rms.append(a.elapsed_time(b))
        if i < 3:
            tr.free()
    tracks, tids = tr.tracks()
    tr.free()
    dv_lat, dv_ref = [], []
    vi = cands["v_idx"].astype(np.int64)
    lat_vx = (w.grid.vx0 + (vi % w.grid.nvx) * w.grid.dvx).astype(np.float64)
    lat_vy = (w.grid.vy0 + (vi // w.grid.nvx) * w.grid.dvy).astype(np.float64)
    for j, g in enumerate(tracks):
        m = cat.mover[tids[int(g["id_off"]): int(g["id_off"]) + int(g["id_len"])]]
        if g["status"] != 0 or not (m >= 0).any():
            continue
        top = np.bincount(m[m >= 0]).argmax()
        if 2 * int((m == top).sum()) < len(m):
            continue
        mv = cat.movers[top]
        dv_ref.append(float(np.hypot(g["vx"] - mv["vx"], g["vy"] - mv["vy"])))
        dv_lat.append(float(np.hypot(lat_vx[j] - mv["vx"], lat_vy[j] - mv["vy"])))
    refine = {"form": "FAST-MCD regression of (x, y) on t per cluster (500 starts, 10 best), gather within "
                      "the bin, repeat until the gathered set is fixed (at most 10 fits)",
              "ms": round(statistics.median(rms), 4), "tracks": int(len(tracks)),
              "converged": int((tracks["status"] == 0).sum()),
              "fits_max": int(tracks["iterations"].max()) if len(tracks) else 0,
              "median_dv_mpx_per_h": {"lattice_point": round(float(np.median(dv_lat)), 2) if dv_lat else None,
                                      "refined": round(float(np.median(dv_ref)), 2) if dv_ref else None},
              "timing": "CUDA events around sas_refine, median of 3"}
    pl.free()
    res.free()
    return {"refine": refine,
            "form": "greedy peel over the search's candidates, N_min as the search, at most 1000 clusters; "
                    "rounds of local maxima",
            "ms": round(statistics.median(ms), 4), "ms_one_cluster_per_step": round(ms_seq, 4),
            "same_count_both_forms": same, "candidates_in": n_cand, "clusters": int(len(cands)),
            "clusters_one_mover": pure, "movers_found": len(found), "movers_findable": findable,
            "timing": f"CUDA events around sas_peel on the launching stream, median of {reps}"}


def weighted_section(grid, dx, dy, de, cat, w, stream, dev, reps: int = 5) -> dict:
    """Weighted stacking on the bench field: synthetic S/N weights (8 x S/N,
    noise peaks just above S/N 5, movers from their detection probability),
    threshold 25 epochs' worth of S/N-5 weight; time per search and movers
    recovered against the plain search at N_min = 25."""
    import torch
    from paper_2509_26279_gb300 import sas

    wt = W.snr_weights(cat)
    dw = torch.from_numpy(wt).to(dev)
    s_min = 25 * 40
    ms = []
    for i in range(reps + 2):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r = sas.sas_stack_weighted(grid, dx, dy, de, dw, cat.t, cat.ticks_per_hour, s_min, on_device=True,
                                   stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        if i >= 2:
            ms.append(a.elapsed_time(b))
        if i < reps + 1:
            r.free()

    def movers_of(res):
        c, ids = res.candidates()
        found = set()
        for x in c:
            m = cat.mover[ids[int(x["id_off"]): int(x["id_off"]) + int(x["id_len"])]]
            if (m >= 0).any():
                top = np.bincount(m[m >= 0]).argmax()
                if 2 * int((m == top).sum()) >= len(m):
                    found.add(int(top))
        return len(c), found

    n_w, f_w = movers_of(r)
    info = r.info()
    r.free()
    plain = sas.sas_stack(grid, dx, dy, de, cat.t, cat.ticks_per_hour, w.n_min, on_device=True, stream=stream)
    n_p, f_p = movers_of(plain)
    plain.free()
    return {"form": "score = sum over epochs of the largest weight in the cell; weights round(8 x S/N) with noise "
                    "peaks at S/N 5 + Exp(rate 5) and movers at S/N from their detection probability; "
                    f"s_min = {s_min} (25 epochs at S/N 5)",
            "ms": round(statistics.median(ms), 4), "det_shifts_per_s": info["n_pairs"] / (statistics.median(ms) * 1e-3),
            "candidates": n_w, "movers_found": len(f_w),
            "plain": {"n_min": w.n_min, "candidates": n_p, "movers_found": len(f_p)},
            "movers_only_weighted": len(f_w - f_p), "movers_only_plain": len(f_p - f_w),
            "timing": f"CUDA events around sas_stack_weighted, median of {reps}, inputs on the device"}


def config_entry(name: str, steps: int, warmup: int, dev, stream, flush, peak_ops: float,
                 cpu_budget_s: float) -> dict:
    """One more search workload measured like the main line (device-resident
    inputs, L2 flushed between steps, CUDA events on the library's stream):
    det-shifts/s of the whole search, the stack kernel's mean time and its
    fraction of the in-run reduction peak, and the oracle beside it."""
    import torch
    from paper_2509_26279_gb300 import sas
    w = getattr(W, name)()
    cat = W.load(w)
    grid = sas.Grid(w.grid)
    dx = torch.from_numpy(cat.x).to(dev)
    dy = torch.from_numpy(cat.y).to(dev)
    de = torch.from_numpy(cat.epoch.view(np.int16)).to(dev)

    def step():
        return sas.sas_stack(grid, dx, dy, de, cat.t, cat.ticks_per_hour, w.n_min, on_device=True, stream=stream)

    for _ in range(warmup):
        r = step()
        info0 = r.info()
        r.free()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    stack_ms = []
    for i in range(steps):
        flush.zero_()
        ev[i][0].record(stream)
        r = step()
        ev[i][1].record(stream)
        stack_ms.append(r.info()["ms_stack"])
        r.free()
    torch.cuda.synchronize()
    total = sum(a.elapsed_time(b) for a, b in ev)
    n_pairs = int(info0["n_pairs"])
    achieved = n_pairs / (statistics.mean(stack_ms) * 1e-3)
    out = {"value": n_pairs * steps / (total * 1e-3), "unit": UNIT, "steps": steps, "warmup": warmup,
           "ms_per_step": total / steps, "config": workload_desc(w, cat),
           "n_pairs_per_step": n_pairs, "candidates": int(info0["n_candidates"]),
           "tile": [info0["tile_kx"], info0["tile_ky"], info0["tile_bx"], info0["tile_by"]],
           "superbin": int(info0["superbin"]), "velocity_block": [info0["vblock_x"], info0["vblock_y"]],
           "roofline": {"bound": "smem_atomic", "kernel": "k_stack", "stack_ms": statistics.mean(stack_ms),
                        "achieved": achieved / 1e9, "peak": peak_ops / 1e9, "unit": "Gop/s",
                        "frac": achieved / peak_ops}}
    if cpu_budget_s > 0:
        out["cpu_baseline"] = cpu_baseline(w, cat, cpu_budget_s)
    return out


def vetter_timing(dev, stream, n_forward: int = 32768, batch: int = 4096, reps: int = 5) -> dict:
    """Throughput of the vetter's kernels on random count stamps shaped like
    the search's (Poisson noise plus a central bump): the forward over
    n_forward stamps in one pass (a vetter sized for them) and training steps
    of `batch` stamps, CUDA events on the launching stream, best of reps."""
    import torch
    from paper_2509_26279_gb300 import sas, vetting
    peaks = measured_peaks()
    rng = np.random.default_rng(W.BASE_SEED + 80)
    st = rng.poisson(1.2, size=(n_forward, 9, 15, 15))
    st[:, 4, 6:9, 6:9] += rng.integers(0, 40, size=(n_forward, 3, 3))
    dst = torch.from_numpy(st.astype(np.uint16).view(np.int16)).to(dev)
    lab = torch.from_numpy((rng.random(n_forward) < 0.5).astype(np.float32)).to(dev)
    vt = sas.Vetter(dev.index or 0, batch)                 # training: steps of `batch` stamps
    vt.set_state(vetting.init_params(1))
    vf = sas.Vetter(dev.index or 0, n_forward)             # inference: one pass over all stamps
    vf.set_state(vetting.init_params(1))
    logits = torch.zeros(n_forward, device=dev)
    loss = torch.zeros(1, device=dev)

    def best_ms(fn):
        fn()
        torch.cuda.synchronize()
        best = None
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            best = ms if best is None or ms < best else best
        return best

    fwd_ms = best_ms(lambda: vf.forward(dst, n_forward, logits, stream=stream))
    vf.check()
    trn_ms = best_ms(lambda: vt.train_step(dst, lab, batch, 1e-3, loss, stream=stream))
    vt.check()
    fwd_flop, trn_flop = 4.93e6, 14.8e6       # per stamp, see the header of csrc/sas_vet.cu
    bf16 = peaks.get("bf16_tflops")
    f_tf = n_forward * fwd_flop / (fwd_ms * 1e-3) / 1e12
    t_tf = batch * trn_flop / (trn_ms * 1e-3) / 1e12
    return {"forward": {"stamps": n_forward, "batch": n_forward, "ms": fwd_ms, "stamps_per_s": n_forward / (fwd_ms * 1e-3),
                        "tflops": f_tf, "frac_of_bf16_peak": f_tf / bf16 if bf16 else None},
            "train_step": {"stamps": batch, "ms": trn_ms, "stamps_per_s": batch / (trn_ms * 1e-3),
                           "tflops": t_tf, "frac_of_bf16_peak": t_tf / bf16 if bf16 else None},
            "peak": {"bf16_tflops": bf16, "source": "MEASURED_PEAKS.json (cuBLAS bf16 burst)"},
            "timing": f"CUDA events on the launching stream, best of {reps} after one warm-up"}


def selection_timing(dev, stream, reps: int = 5) -> dict:
    """The stack kernel with one threshold and with the tile-local peaks alone
    on one of the batched uneven fields (100 epochs, 423402 detections, N_min
    = 25; n_low = ceil(E/6) raised to the field's noise floor): device time of
    the kernel (ms_stack, median of reps after one warm-up), super-bins
    emitted, candidates."""
    from paper_2509_26279_gb300 import sas, vetting
    f = vetting.Field(W.batched_fields(60)[0], dev)
    out = {"workload": f"batched_fields[0]: {f.E} epochs, {f.cat.n} detections, 111x111 lattice, N_min {f.w.n_min}"}
    n_low = vetting.lowered_threshold(f.E, f.w.n_min, f.cat.n, f.w.grid, 6)
    for tag, o in (("one_threshold", sas.make_opts()), ("peaks_only", sas.make_opts(n_low=n_low, peaks_only=1))):
        ms = []
        for i in range(reps + 1):
            res = sas.sas_stack(f.grid, f.dx, f.dy, f.de, f.cat.t, f.cat.ticks_per_hour, f.w.n_min, on_device=True,
                                opts=o, stream=stream)
            inf = res.info()
            if i:
                ms.append(inf["ms_stack"])
            res.free()
        out[tag] = {"n_low": int(inf["n_low"]), "ms_stack": round(statistics.median(ms), 4),
                    "superbins_emitted": int(inf["n_emitted"]), "candidates": int(inf["n_candidates"])}
    return out


def refine_timing(dev, stream, reps: int = 5) -> dict:
    """Cluster finding and refinement on one search of the DECam TNO field:
    sas_peel, then sas_refine with one fit round and with the default loop,
    CUDA events on the launching stream, median of reps."""
    import torch
    from paper_2509_26279_gb300 import sas
    w = W.decam_tno()
    cat = W.load(w)
    grid = sas.Grid(w.grid)
    dx, dy = torch.from_numpy(cat.x).to(dev), torch.from_numpy(cat.y).to(dev)
    de = torch.from_numpy(cat.epoch.view(np.int16)).to(dev)
    res = sas.sas_stack(grid, dx, dy, de, cat.t, cat.ticks_per_hour, w.n_min, on_device=True, stream=stream)
    pl = sas.sas_peel(res, w.n_min, 1000, stream=stream)
    out = {"workload": workload_desc(w, cat)["workload"], "clusters": int(pl.info()["n_candidates"])}
    for tag, kw in (("one_fit_round", {"max_iter": 1}), ("default", {})):
        ms = []
        for i in range(reps + 1):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            tr = sas.sas_refine(res, pl, seed=1, stream=stream, **kw)
            b.record(stream)
            torch.cuda.synchronize()
            if i:
                ms.append(a.elapsed_time(b))
            tracks, _ = tr.tracks()
            tr.free()
        out[tag] = {"ms": statistics.median(ms), "tracks": int(len(tracks)),
                    "converged": int((tracks["status"] == 0).sum()),
                    "fits_max": int(tracks["iterations"].max()) if len(tracks) else 0}
    pl.free()
    res.free()
    out["timing"] = f"CUDA events around sas_refine on the launching stream, median of {reps} after one warm-up"
    return out


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p))
        except (OSError, ValueError):
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = W.decam_tno()
    cat = W.load(w)
    import oracle
    g = w.grid
    thr = oracle.threads()
    per_step = 12 * thr                # lattice points per step: about a second on the OpenMP team
    nv = g.nvx * g.nvy
    def step(i):
        a = (nv // 2 + i * per_step) % (nv - per_step)
        t0 = time.perf_counter()
        pairs = oracle.stack(cat, g, w.n_min, a, a + per_step, threads=0).n_pairs
        return pairs, time.perf_counter() - t0
    for i in range(args.warmup):
        step(i)
    tot_p, tot_s = 0, 0.0
    for i in range(args.steps):
        p, s = step(args.warmup + i)
        tot_p += p
        tot_s += s
    v = tot_p / tot_s
    cfg = workload_desc(w, cat)
    cfg["sample"] = f"{per_step} consecutive lattice points of the field per step (OpenMP, {thr} threads)"
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i64",
           "data": "synthetic", "config": cfg,
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": thr, "kind": "oracle",
                            "sample": cfg["sample"], "host": host_info()},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="decam_tno", choices=["decam_tno", "fast_movers", "tiny"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget-s", type=float, default=15.0)
    ap.add_argument("--no-fields", action="store_true", help="skip the fields/s comparison")
    ap.add_argument("--no-configs", action="store_true", help="skip the other search workloads' entries")
    ap.add_argument("--vetter-timing", action="store_true",
                    help="only time the vetter's forward and training kernels and print that line")
    ap.add_argument("--refine-timing", action="store_true",
                    help="only time cluster finding's refinement on the TNO field and print that line")
    ap.add_argument("--selection-timing", action="store_true",
                    help="only time the stack kernel with one threshold and with the peaks alone on one field")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)

    import torch
    from paper_2509_26279_gb300 import sas

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.vetter_timing or args.refine_timing or args.selection_timing:
        stream = torch.cuda.current_stream(dev)
        if rank == 0:
            mode, fn = (("vetter_timing", vetter_timing) if args.vetter_timing else
                        ("refine_timing", refine_timing) if args.refine_timing else
                        ("selection_timing", selection_timing))
            print(json.dumps({"mode": mode, **fn(dev, stream)}), flush=True)
        return 0

    w = getattr(W, args.workload)()
    w = W.Workload(w.name, w.recipe, w.grid, w.n_min, w.seed + 1000 * rank)  # own field per rank
    cat = W.load(w)
    grid = sas.Grid(w.grid)
    stream = torch.cuda.current_stream(dev)
    dx = torch.from_numpy(cat.x).to(dev)
    dy = torch.from_numpy(cat.y).to(dev)
    de = torch.from_numpy(cat.epoch.view(np.int16)).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()

    def dev_step():
        return sas.sas_stack(grid, dx, dy, de, cat.t, cat.ticks_per_hour, w.n_min,
                             on_device=True, stream=stream)

    for _ in range(args.warmup):
        r = dev_step()
        info0 = r.info()
        r.free()
    peak_ops, probe_mhz = sas.sas_probe_shared_reduction_peak(2048, stream)
    atom_ops, atom_mhz = sas.sas_probe_shared_atomic_peak(2048, stream)
    or64_ops, or64_mhz = sas.sas_probe_shared_or64_peak(2048, stream)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    stack_ms, pairs, phases = [], [], []
    launches0 = sas.sas_kernel_launches()
    with ClockSampler(local) as clk:
        barrier()
        for i in range(args.steps):
            flush.zero_()                          # L2 flush, outside the timed step
            ev[i][0].record(stream)
            r = dev_step()
            ev[i][1].record(stream)
            inf = r.info()
            stack_ms.append(inf["ms_stack"])
            phases.append([inf["ms_prep"], inf["ms_stack"], inf["ms_count"], inf["ms_ids"]])
            pairs.append(inf["n_pairs"])
            r.free()
        barrier()
    launches = sas.sas_kernel_launches() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    if dist is not None:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    n_pairs = int(pairs[0])
    assert all(p == n_pairs for p in pairs), "detection-shift count changed between steps"
    value = n_pairs * args.steps * world / (total_ms * 1e-3)

    # end-to-end through host buffers (pinned), copies inside the timed region
    hx = torch.from_numpy(cat.x).pin_memory()
    hy = torch.from_numpy(cat.y).pin_memory()
    he = torch.from_numpy(cat.epoch.view(np.int16)).pin_memory()
    hxn, hyn, hen = hx.numpy(), hy.numpy(), he.numpy().view(np.uint16)
    # page-locked result buffers, allocated once and reused every step (the
    # result sizes are those of the warm-up steps: the search is deterministic)
    nc_cap, ni_cap = max(1, int(info0["n_candidates"])), max(1, int(info0["n_ids"]))
    hc_out = torch.empty(nc_cap * sas.CANDIDATE_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
    hi_out = torch.empty(ni_cap, dtype=torch.int32).pin_memory()
    out_bufs = (hc_out.numpy().view(sas.CANDIDATE_DTYPE), hi_out.numpy().view(np.uint32))
    e2e_s, d2h = 0.0, 0
    for i in range(max(3, args.steps // 2)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = sas.sas_stack(grid, hxn, hyn, hen, cat.t, cat.ticks_per_hour, w.n_min, stream=stream)
        cands, ids = r.candidates(out=out_bufs)
        e2e_s += time.perf_counter() - t0
        d2h = cands.nbytes + ids.nbytes
        r.free()
        n_e2e = i + 1
    e2e_value = n_pairs * n_e2e * world / e2e_s
    h2d = cat.n * 10 + cat.n_epochs * 8

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0
    achieved = n_pairs / (statistics.mean(stack_ms) * 1e-3)
    roof = {"bound": "smem_atomic", "achieved": achieved / 1e9, "peak": peak_ops / 1e9,
            "unit": "Gop/s", "frac": achieved / peak_ops, "traffic": stack_traffic(args.workload),
            "kernel": "k_stack", "stack_ms": statistics.mean(stack_ms),
            "peak_source": f"sas_probe_shared_reduction_peak (conflict-free red.shared.add.u32), this run "
                           f"({probe_mhz:.0f} MHz)",
            "peak_atomic_returning": atom_ops / 1e9,
            "frac_vs_atomic_returning": achieved / atom_ops,
            "peak_atomic_returning_source": f"sas_probe_shared_atomic_peak (conflict-free atomicAdd, old value "
                                            f"used), this run ({atom_mhz:.0f} MHz)",
            "atomic_or_b64": or64_ops / 1e9,
            "atomic_or_b64_source": f"sas_probe_shared_or64_peak (conflict-free 64-bit atomicOr, old value used: "
                                    f"the epoch-bitmask update the kernel replaces by counters), this run "
                                    f"({or64_mhz:.0f} MHz)"}
    cfg = workload_desc(w, cat)
    cfg.update({"l2": "flushed between steps (256 MiB write)", "n_pairs_per_step": n_pairs,
                "candidates": int(info0["n_candidates"]),
                "tile": [info0["tile_kx"], info0["tile_ky"], info0["tile_bx"], info0["tile_by"]],
                "counter_bits": int(info0["counter_bits"]), "superbin": int(info0["superbin"]),
                "velocity_block": [info0["vblock_x"], info0["vblock_y"]],
                "staged_cap": int(info0["staged_cap"]), "emitted": int(info0["n_emitted"]),
                "phase_ms": dict(zip(["prep", "stack", "count_sort", "ids"],
                                     [round(statistics.mean(c), 4) for c in zip(*phases)])),
                "parallelism": f"replicas{world}"})
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "i32", "data": "synthetic",
           "config": cfg, "clocks": clk.summary(),
           "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                   "d2h_bytes_per_step": int(d2h)},
           "gpu_launches": int(launches), "roofline": roof}
    if world == 1:
        out["peel"] = peel_section(grid, dx, dy, de, cat, w, stream)
        out["weighted"] = weighted_section(grid, dx, dy, de, cat, w, stream, dev)
    if world == 1 and not args.no_configs:
        steps_of = {"tiny": 20, "decam_tno": 10, "fast_movers": 3}
        out["configs"] = {
            name: config_entry(name, steps_of[name], args.warmup, dev, stream, flush, peak_ops,
                               0.0 if args.no_cpu_baseline else min(args.cpu_budget_s, 10.0))
            for name in ("tiny", "decam_tno", "fast_movers") if name != args.workload}
    if world == 1 and not args.no_fields:
        out["fields"] = fields_section(dev, stream)
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(w, cat, args.cpu_budget_s)
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
