"""Thin ctypes binding of the sm_103a shift-and-stack library (include/sas.h).

Argument marshalling only: every step of the search runs in the library's CUDA
kernels.  There is no CPU fallback -- importing this module raises if the
compiled library is missing (build it with ``__graft_entry__.build()``).

Host arrays are NumPy arrays; device arrays may be anything exposing
``data_ptr()`` (torch CUDA tensors) or ``__cuda_array_interface__``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libsas.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libsas.so is not built ({LIB_PATH}); run __graft_entry__.build() first")

_lib = ctypes.CDLL(LIB_PATH)

SAS_OK, SAS_ERR_ARG, SAS_ERR_RANGE, SAS_ERR_OVERFLOW = 0, 1, 2, 3
SAS_ERR_CUDA, SAS_ERR_OOM, SAS_ERR_TIMEOUT, SAS_ERR_INTERNAL = 4, 5, 6, 7
STATUS_NAMES = {0: "SAS_OK", 1: "SAS_ERR_ARG", 2: "SAS_ERR_RANGE", 3: "SAS_ERR_OVERFLOW",
                4: "SAS_ERR_CUDA", 5: "SAS_ERR_OOM", 6: "SAS_ERR_TIMEOUT", 7: "SAS_ERR_INTERNAL"}


class SasError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class sas_grid_desc(ctypes.Structure):
    _fields_ = [("vx0", ctypes.c_int32), ("vy0", ctypes.c_int32), ("dvx", ctypes.c_int32),
                ("dvy", ctypes.c_int32), ("nvx", ctypes.c_uint32), ("nvy", ctypes.c_uint32),
                ("speed_min", ctypes.c_int32), ("speed_max", ctypes.c_int32),
                ("x_min", ctypes.c_int32), ("y_min", ctypes.c_int32), ("nbx", ctypes.c_uint32),
                ("nby", ctypes.c_uint32), ("bin", ctypes.c_int32)]


class sas_catalog(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("x", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("epoch", ctypes.c_void_p), ("n_epochs", ctypes.c_uint32), ("t", ctypes.c_void_p),
                ("ticks_per_hour", ctypes.c_int64), ("on_device", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class sas_opts(ctypes.Structure):
    _fields_ = [("v_begin", ctypes.c_uint64), ("v_end", ctypes.c_uint64),
                ("max_candidates", ctypes.c_uint64), ("tile_kx", ctypes.c_uint32),
                ("tile_ky", ctypes.c_uint32), ("tile_bx", ctypes.c_uint32),
                ("tile_by", ctypes.c_uint32), ("counter_bits", ctypes.c_uint32),
                ("coarse_bins", ctypes.c_uint32), ("superbin", ctypes.c_uint32),
                ("velocity_block", ctypes.c_uint32), ("n_low", ctypes.c_uint32),
                ("peaks_only", ctypes.c_uint32)]


class sas_result_info(ctypes.Structure):
    _fields_ = [("n_candidates", ctypes.c_uint64), ("n_ids", ctypes.c_uint64),
                ("n_pairs", ctypes.c_uint64), ("n_emitted", ctypes.c_uint64),
                ("t0", ctypes.c_int64), ("counter_bits", ctypes.c_uint32),
                ("tile_kx", ctypes.c_uint32), ("tile_ky", ctypes.c_uint32),
                ("tile_bx", ctypes.c_uint32), ("tile_by", ctypes.c_uint32),
                ("superbin", ctypes.c_uint32), ("vblock_x", ctypes.c_uint32),
                ("vblock_y", ctypes.c_uint32), ("staged_cap", ctypes.c_uint32),
                ("n_low", ctypes.c_uint32), ("ms_stack", ctypes.c_float),
                ("ms_total", ctypes.c_float), ("ms_prep", ctypes.c_float),
                ("ms_count", ctypes.c_float), ("ms_ids", ctypes.c_float),
                ("peaks_only", ctypes.c_uint32)]


# sas_candidate as a NumPy record (32 bytes, same layout as the C struct)
CANDIDATE_DTYPE = np.dtype([("v_idx", "<u4"), ("bx", "<u4"), ("by", "<u4"), ("count", "<u4"),
                            ("raw", "<u4"), ("id_len", "<u4"), ("id_off", "<u8")])
assert CANDIDATE_DTYPE.itemsize == 32

_p = ctypes.c_void_p
_lib.sas_version.restype = ctypes.c_char_p
_lib.sas_abi_version.restype = ctypes.c_int
ABI_VERSION = 2  # the struct layouts below
if _lib.sas_abi_version() != ABI_VERSION:
    raise ImportError(f"{LIB_PATH} implements ABI {_lib.sas_abi_version()}, this binding ABI {ABI_VERSION}: rebuild")
_lib.sas_kernel_launches.restype = ctypes.c_uint64
_lib.sas_last_error.restype = ctypes.c_char_p
_lib.sas_create_grid.argtypes = [ctypes.POINTER(sas_grid_desc), ctypes.POINTER(_p)]
_lib.sas_destroy_grid.argtypes = [_p]
_lib.sas_destroy_grid.restype = None
_lib.sas_stack.argtypes = [_p, ctypes.POINTER(sas_catalog), ctypes.c_uint32,
                           ctypes.POINTER(sas_opts), _p, ctypes.POINTER(_p)]
_lib.sas_result_get_info.argtypes = [_p, ctypes.POINTER(sas_result_info)]
_lib.sas_candidates.argtypes = [_p, _p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64), _p,
                                ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64), ctypes.c_int]
_lib.sas_result_free.argtypes = [_p]
_lib.sas_result_free.restype = None
_lib.sas_probe_shared_atomic_peak.argtypes = [ctypes.c_uint32, _p, ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_double)]
_lib.sas_probe_shared_reduction_peak.argtypes = [ctypes.c_uint32, _p, ctypes.POINTER(ctypes.c_double),
                                                 ctypes.POINTER(ctypes.c_double)]
_lib.sas_probe_shared_or64_peak.argtypes = [ctypes.c_uint32, _p, ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_double)]
_lib.sas_cell_counts_noalloc.argtypes = [_p, ctypes.POINTER(sas_catalog), _p, ctypes.c_uint64, _p, _p,
                                         _p]

EXPORTED = ["sas_version", "sas_abi_version", "sas_kernel_launches", "sas_last_error", "sas_create_grid",
            "sas_destroy_grid", "sas_stack", "sas_result_get_info", "sas_candidates",
            "sas_result_free", "sas_probe_shared_atomic_peak", "sas_probe_shared_reduction_peak",
            "sas_probe_shared_or64_peak", "sas_cell_counts_noalloc"]


def _check(status: int):
    if status != SAS_OK:
        raise SasError(status, _lib.sas_last_error().decode())


def sas_version() -> str:
    return _lib.sas_version().decode()


def sas_kernel_launches() -> int:
    return int(_lib.sas_kernel_launches())


def _dev_ptr(a) -> int:
    if hasattr(a, "data_ptr"):
        return int(a.data_ptr())
    if hasattr(a, "__cuda_array_interface__"):
        return int(a.__cuda_array_interface__["data"][0])
    raise TypeError("device array expected (torch CUDA tensor or __cuda_array_interface__)")


def _stream_handle(stream) -> int:
    if stream is None:
        return 0
    if hasattr(stream, "cuda_stream"):
        return int(stream.cuda_stream)
    return int(stream)


class Grid:
    """sas_create_grid / sas_destroy_grid.  Accepts a workloads.GridSpec or the
    same fields as keyword arguments."""

    def __init__(self, spec=None, **kw):
        f = dict(spec.__dict__) if spec is not None else {}
        f.update(kw)
        self.desc = sas_grid_desc(
            vx0=f["vx0"], vy0=f["vy0"], dvx=f["dvx"], dvy=f["dvy"], nvx=f["nvx"], nvy=f["nvy"],
            speed_min=f.get("speed_min", 0), speed_max=f.get("speed_max", 0), x_min=f["x_min"],
            y_min=f["y_min"], nbx=f["nbx"], nby=f["nby"], bin=f["bin"])
        self.nvx, self.nvy = int(f["nvx"]), int(f["nvy"])
        h = _p()
        _check(_lib.sas_create_grid(ctypes.byref(self.desc), ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.sas_destroy_grid(h)
            self._h = _p()


class Result:
    """A finished search (sas_result); owns device memory until freed."""

    def __init__(self, h):
        self._h = h

    def info(self) -> dict:
        inf = sas_result_info()
        _check(_lib.sas_result_get_info(self._h, ctypes.byref(inf)))
        return {k: getattr(inf, k) for k, _ in sas_result_info._fields_}

    def candidates(self, out=None):
        """(candidates: structured array of CANDIDATE_DTYPE, ids: uint32 array).
        out = (cands, ids): caller-owned contiguous host arrays of those dtypes
        (page-locked ones copy fastest) to fill instead of new arrays; the
        returned arrays are their leading parts.  SasError when one is too
        small."""
        nc, ni = ctypes.c_uint64(), ctypes.c_uint64()
        inf = self.info()
        nc_v, ni_v = inf["n_candidates"], inf["n_ids"]
        if out is None:
            cands = np.zeros(nc_v, CANDIDATE_DTYPE)
            ids = np.zeros(ni_v, np.uint32)
        else:
            cands, ids = out
            if (cands.dtype != CANDIDATE_DTYPE or ids.dtype != np.uint32 or not cands.flags.c_contiguous
                    or not ids.flags.c_contiguous):
                raise SasError(SAS_ERR_ARG, "out: contiguous CANDIDATE_DTYPE and uint32 arrays")
        _check(_lib.sas_candidates(self._h, cands.ctypes.data if nc_v else None, len(cands) if nc_v else 0,
                                   ctypes.byref(nc), ids.ctypes.data if ni_v else None, len(ids) if ni_v else 0,
                                   ctypes.byref(ni), 0))
        return cands[:nc_v], ids[:ni_v]

    def candidates_into(self, cands_dev, ids_dev, cap: int, ids_cap: int):
        """Copy into caller-owned device buffers (sas_candidates with on_device=1)."""
        nc, ni = ctypes.c_uint64(), ctypes.c_uint64()
        _check(_lib.sas_candidates(self._h, _dev_ptr(cands_dev), cap, ctypes.byref(nc),
                                   _dev_ptr(ids_dev), ids_cap, ctypes.byref(ni), 1))
        return nc.value, ni.value

    def free(self):
        if self._h is not None and self._h.value:
            _lib.sas_result_free(self._h)
            self._h = _p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def make_opts(**kw) -> sas_opts:
    o = sas_opts()
    for k, v in kw.items():
        setattr(o, k, int(v))
    return o


def sas_stack(grid: Grid, x, y, epoch, t, ticks_per_hour: int, n_min: int, *,
              on_device: bool = False, opts: sas_opts | None = None, stream=None) -> Result:
    """Run the search.  With on_device=False, x/y/epoch are NumPy host arrays
    (int32, int32, uint16); with on_device=True they are device arrays of those
    types.  t (int64 epoch times) is always a host array."""
    t = np.ascontiguousarray(t, np.int64)
    if on_device:
        n = int(x.numel() if hasattr(x, "numel") else len(x))
        px, py, pe = _dev_ptr(x), _dev_ptr(y), _dev_ptr(epoch)
        keep = ()
    else:
        x = np.ascontiguousarray(x, np.int32)
        y = np.ascontiguousarray(y, np.int32)
        epoch = np.ascontiguousarray(epoch, np.uint16)
        n = int(x.shape[0])
        px, py, pe = x.ctypes.data, y.ctypes.data, epoch.ctypes.data
        keep = (x, y, epoch)
    cat = sas_catalog(n=n, x=px, y=py, epoch=pe, n_epochs=int(t.shape[0]), t=t.ctypes.data,
                      ticks_per_hour=int(ticks_per_hour), on_device=1 if on_device else 0)
    h = _p()
    _check(_lib.sas_stack(grid.handle, ctypes.byref(cat), int(n_min),
                          ctypes.byref(opts) if opts is not None else None,
                          _stream_handle(stream), ctypes.byref(h)))
    del keep
    return Result(h)


_lib.sas_stack_weighted.argtypes = [_p, ctypes.POINTER(sas_catalog), _p, ctypes.c_uint32,
                                    ctypes.POINTER(sas_opts), _p, ctypes.POINTER(_p)]
EXPORTED.append("sas_stack_weighted")


def sas_stack_weighted(grid: Grid, x, y, epoch, weights, t, ticks_per_hour: int, s_min: int, *,
                       on_device: bool = False, opts: sas_opts | None = None, stream=None) -> Result:
    """Weighted stacking: weights (uint8 per detection, host or device like x)
    score each cell by the sum over epochs of its largest weight; candidates
    have score >= s_min and their `count` is the score."""
    t = np.ascontiguousarray(t, np.int64)
    if on_device:
        n = int(x.numel() if hasattr(x, "numel") else len(x))
        px, py, pe, pw = _dev_ptr(x), _dev_ptr(y), _dev_ptr(epoch), _dev_ptr(weights)
        keep = ()
    else:
        x = np.ascontiguousarray(x, np.int32)
        y = np.ascontiguousarray(y, np.int32)
        epoch = np.ascontiguousarray(epoch, np.uint16)
        weights = np.ascontiguousarray(weights, np.uint8)
        n = int(x.shape[0])
        px, py, pe = x.ctypes.data, y.ctypes.data, epoch.ctypes.data
        pw = weights.ctypes.data if n else None
        keep = (x, y, epoch, weights)
    cat = sas_catalog(n=n, x=px, y=py, epoch=pe, n_epochs=int(t.shape[0]), t=t.ctypes.data,
                      ticks_per_hour=int(ticks_per_hour), on_device=1 if on_device else 0)
    h = _p()
    _check(_lib.sas_stack_weighted(grid.handle, ctypes.byref(cat), pw, int(s_min),
                                   ctypes.byref(opts) if opts is not None else None,
                                   _stream_handle(stream), ctypes.byref(h)))
    del keep
    return Result(h)


def stack_catalog(grid: Grid, cat, n_min: int, **kw) -> Result:
    """sas_stack on a workloads.Catalog held in host memory."""
    return sas_stack(grid, cat.x, cat.y, cat.epoch, cat.t, cat.ticks_per_hour, n_min, **kw)


def sas_cell_counts_noalloc(grid: Grid, x, y, epoch, t, ticks_per_hour: int, cells, n_cells: int,
                            distinct, raw, stream=None) -> None:
    """Exact (distinct, raw) counts of n_cells cells without any device
    allocation by the library.  x, y, epoch, cells (n_cells x 3 uint32:
    v_idx, bx, by), distinct and raw are device arrays owned by the caller."""
    t = np.ascontiguousarray(t, np.int64)
    n = int(x.numel() if hasattr(x, "numel") else len(x))
    cat = sas_catalog(n=n, x=_dev_ptr(x), y=_dev_ptr(y), epoch=_dev_ptr(epoch),
                      n_epochs=int(t.shape[0]), t=t.ctypes.data,
                      ticks_per_hour=int(ticks_per_hour), on_device=1)
    _check(_lib.sas_cell_counts_noalloc(grid.handle, ctypes.byref(cat), _dev_ptr(cells),
                                        int(n_cells), _dev_ptr(distinct), _dev_ptr(raw),
                                        _stream_handle(stream)))


def sas_probe_shared_atomic_peak(iters: int = 4096, stream=None):
    """(ops/s, SM MHz) of conflict-free 32-bit shared atomicAdd (old value used) on all SMs."""
    ops, mhz = ctypes.c_double(), ctypes.c_double()
    _check(_lib.sas_probe_shared_atomic_peak(int(iters), _stream_handle(stream), ctypes.byref(ops),
                                             ctypes.byref(mhz)))
    return ops.value, mhz.value


def sas_probe_shared_or64_peak(iters: int = 4096, stream=None):
    """(ops/s, SM MHz) of conflict-free 64-bit shared atomicOr (old value used) on all SMs."""
    ops, mhz = ctypes.c_double(), ctypes.c_double()
    _check(_lib.sas_probe_shared_or64_peak(int(iters), _stream_handle(stream), ctypes.byref(ops),
                                           ctypes.byref(mhz)))
    return ops.value, mhz.value


def sas_probe_shared_reduction_peak(iters: int = 4096, stream=None):
    """(ops/s, SM MHz) of conflict-free red.shared.add.u32 on all SMs (the stack kernel's instruction)."""
    ops, mhz = ctypes.c_double(), ctypes.c_double()
    _check(_lib.sas_probe_shared_reduction_peak(int(iters), _stream_handle(stream), ctypes.byref(ops),
                                                ctypes.byref(mhz)))
    return ops.value, mhz.value


def library():
    return _lib


# ---- batched search and autotuner ------------------------------------------------

_lib.sas_grid_get_desc.argtypes = [_p, ctypes.POINTER(sas_grid_desc)]
_lib.sas_batch_create.argtypes = [ctypes.POINTER(_p), ctypes.POINTER(sas_catalog),
                                  ctypes.POINTER(ctypes.c_uint32), ctypes.c_uint32,
                                  ctypes.POINTER(sas_opts), _p, ctypes.POINTER(_p)]
_lib.sas_batch_run.argtypes = [_p, _p]
_lib.sas_batch_field_info.argtypes = [_p, ctypes.c_uint32, ctypes.POINTER(sas_result_info)]
_lib.sas_batch_candidates.argtypes = [_p, ctypes.c_uint32, _p, ctypes.c_uint64,
                                      ctypes.POINTER(ctypes.c_uint64), _p, ctypes.c_uint64,
                                      ctypes.POINTER(ctypes.c_uint64), ctypes.c_int]
_lib.sas_batch_stats.argtypes = [_p, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_uint64),
                                 ctypes.POINTER(ctypes.c_uint64)]
_lib.sas_batch_destroy.argtypes = [_p]
_lib.sas_batch_destroy.restype = None
_lib.sas_autotune.argtypes = [_p, ctypes.POINTER(sas_catalog), ctypes.c_uint32,
                              ctypes.POINTER(sas_opts), ctypes.c_uint32, _p,
                              ctypes.POINTER(sas_opts), ctypes.POINTER(ctypes.c_float)]
EXPORTED += ["sas_grid_get_desc", "sas_batch_create", "sas_batch_run", "sas_batch_field_info",
             "sas_batch_candidates", "sas_batch_stats", "sas_batch_destroy", "sas_autotune"]


def _device_catalog(x, y, epoch, t, tph):
    t = np.ascontiguousarray(t, np.int64)
    n = int(x.numel() if hasattr(x, "numel") else len(x))
    return sas_catalog(n=n, x=_dev_ptr(x), y=_dev_ptr(y), epoch=_dev_ptr(epoch),
                       n_epochs=int(t.shape[0]), t=t.ctypes.data, ticks_per_hour=int(tph),
                       on_device=1), t


class Batch:
    """sas_batch_create / sas_batch_run / sas_batch_destroy.

    fields: list of (grid, x, y, epoch, t, ticks_per_hour, n_min) with x, y,
    epoch device arrays that stay alive (and keep their sizes) for the life of
    the batch.  opts: None or one sas_opts per field."""

    def __init__(self, fields, opts=None, stream=None):
        n = len(fields)
        self._keep = []
        cats = (sas_catalog * n)()
        grids = (_p * n)()
        nmin = (ctypes.c_uint32 * n)()
        for i, (g, x, y, e, t, tph, n_min) in enumerate(fields):
            c, tt = _device_catalog(x, y, e, t, tph)
            self._keep += [tt, g, x, y, e]
            cats[i] = c
            grids[i] = g.handle
            nmin[i] = int(n_min)
        op = None
        if opts is not None:
            arr = (sas_opts * n)(*opts)
            self._keep.append(arr)
            op = arr
        h = _p()
        _check(_lib.sas_batch_create(grids, cats, nmin, n, op, _stream_handle(stream), ctypes.byref(h)))
        self._h = h
        self.n_fields = n

    def run(self, stream=None):
        _check(_lib.sas_batch_run(self._h, _stream_handle(stream)))

    def field_info(self, f: int) -> dict:
        inf = sas_result_info()
        _check(_lib.sas_batch_field_info(self._h, int(f), ctypes.byref(inf)))
        return {k: getattr(inf, k) for k, _ in sas_result_info._fields_}

    def candidates(self, f: int):
        inf = self.field_info(f)
        nc_v, ni_v = inf["n_candidates"], inf["n_ids"]
        cands = np.zeros(nc_v, CANDIDATE_DTYPE)
        ids = np.zeros(ni_v, np.uint32)
        nc, ni = ctypes.c_uint64(), ctypes.c_uint64()
        _check(_lib.sas_batch_candidates(self._h, int(f), cands.ctypes.data if nc_v else None, nc_v,
                                         ctypes.byref(nc), ids.ctypes.data if ni_v else None, ni_v,
                                         ctypes.byref(ni), 0))
        return cands, ids

    def peaks(self, f: int, idx_dev, stream=None) -> int:
        n = ctypes.c_uint64()
        _check(_lib.sas_batch_peaks(self._h, int(f), _opt_ptr(idx_dev), ctypes.byref(n),
                                    _stream_handle(stream)))
        return n.value

    def owned(self, f: int, idx_dev, n_keep: int = 0, stream=None) -> int:
        n = ctypes.c_uint64()
        _check(_lib.sas_batch_owned(self._h, int(f), int(n_keep), _opt_ptr(idx_dev), ctypes.byref(n),
                                    _stream_handle(stream)))
        return n.value

    def vet(self, vetter, field_dev, cand_dev, logit_dev, cap: int, stream=None) -> int:
        """sas_batch_vet: (field, candidate, logit) of every kept candidate of
        every field into device arrays with room for cap items; returns the
        number of items."""
        n = ctypes.c_uint64()
        _check(_lib.sas_batch_vet(self._h, vetter._h, _dev_ptr(field_dev), _dev_ptr(cand_dev),
                                  _dev_ptr(logit_dev), int(cap), ctypes.byref(n), _stream_handle(stream)))
        return n.value

    def stamps(self, f: int, idx_dev, count: int, out_dev, stream=None):
        _check(_lib.sas_batch_stamps(self._h, int(f), _opt_ptr(idx_dev), int(count),
                                     _opt_ptr(out_dev) if count else None, _stream_handle(stream)))

    def stats(self):
        ms, fb = ctypes.c_float(), ctypes.c_uint64()
        rb = ctypes.c_uint64()
        _check(_lib.sas_batch_stats(self._h, ctypes.byref(ms), ctypes.byref(fb), ctypes.byref(rb)))
        self.rebuilds = rb.value
        return ms.value, fb.value

    def destroy(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.sas_batch_destroy(self._h)
            self._h = _p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def sas_autotune(grid: Grid, x, y, epoch, t, ticks_per_hour: int, n_min: int,
                 base: sas_opts | None = None, reps: int = 3, stream=None):
    """Fastest (superbin, velocity_block) options for this field and their
    median device time in ms (device arrays x, y, epoch)."""
    cat, tt = _device_catalog(x, y, epoch, t, ticks_per_hour)
    best, ms = sas_opts(), ctypes.c_float()
    _check(_lib.sas_autotune(grid.handle, ctypes.byref(cat), int(n_min),
                             ctypes.byref(base) if base is not None else None, int(reps),
                             _stream_handle(stream), ctypes.byref(best), ctypes.byref(ms)))
    return best, ms.value


# ---- stamps and the candidate vetter ------------------------------------------------

_lib.sas_stamps.argtypes = [_p, ctypes.c_uint64, ctypes.c_uint64, _p, _p]
_lib.sas_vet_num_params.restype = ctypes.c_uint64
_lib.sas_vet_create.argtypes = [ctypes.c_int, ctypes.c_uint32, ctypes.POINTER(_p)]
_lib.sas_vet_destroy.argtypes = [_p]
_lib.sas_vet_set_adam.argtypes = [_p, ctypes.c_float, ctypes.c_float, ctypes.c_float]
_lib.sas_vet_check.argtypes = [_p]
_lib.sas_vet_set_state.argtypes = [_p, _p, _p, _p, ctypes.c_uint64]
_lib.sas_vet_get_state.argtypes = [_p, _p, _p, _p, ctypes.POINTER(ctypes.c_uint64)]
_lib.sas_vet_get_bf16.argtypes = [_p, _p]
_lib.sas_vet_get_activations.argtypes = [_p, ctypes.c_uint32, ctypes.c_uint64, _p]
_lib.sas_vet_forward.argtypes = [_p, _p, _p, ctypes.c_uint64, _p, _p]
_lib.sas_vet_gradients.argtypes = [_p, _p, _p, _p, ctypes.c_uint32, _p, _p, _p]
_lib.sas_vet_apply_gradients.argtypes = [_p, _p, ctypes.c_float, _p]
_lib.sas_vet_train_step.argtypes = [_p, _p, _p, _p, ctypes.c_uint32, ctypes.c_float, _p, _p]
_lib.sas_stamps_indexed.argtypes = [_p, _p, ctypes.c_uint64, _p, _p]
_lib.sas_peaks.argtypes = [_p, _p, ctypes.POINTER(ctypes.c_uint64), _p]
_lib.sas_batch_peaks.argtypes = [_p, ctypes.c_uint32, _p, ctypes.POINTER(ctypes.c_uint64), _p]
_lib.sas_batch_stamps.argtypes = [_p, ctypes.c_uint32, _p, ctypes.c_uint64, _p, _p]
_lib.sas_owned.argtypes = [_p, ctypes.c_uint32, _p, ctypes.POINTER(ctypes.c_uint64), _p]
_lib.sas_batch_owned.argtypes = [_p, ctypes.c_uint32, ctypes.c_uint32, _p, ctypes.POINTER(ctypes.c_uint64), _p]
_lib.sas_peel.argtypes = [_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, _p, ctypes.POINTER(_p)]
_lib.sas_batch_vet.argtypes = [_p, _p, _p, _p, _p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64), _p]
EXPORTED += ["sas_stamps", "sas_vet_num_params", "sas_vet_create", "sas_vet_destroy",
             "sas_vet_set_adam", "sas_vet_set_state", "sas_vet_get_state", "sas_vet_get_bf16", "sas_vet_get_activations",
             "sas_vet_forward", "sas_vet_gradients", "sas_vet_apply_gradients",
             "sas_vet_train_step", "sas_vet_check", "sas_stamps_indexed", "sas_peaks", "sas_batch_peaks",
             "sas_batch_stamps", "sas_owned", "sas_batch_owned", "sas_batch_vet", "sas_peel"]

STAMP_SHAPE = (9, 15, 15)
VET_MAX_BATCH = 32768


def sas_stamps(result: Result, out_dev, first: int = 0, count: int | None = None, stream=None) -> int:
    """Stamps of candidates [first, first + count) into a device uint16 array
    of count x 9 x 15 x 15 (asynchronous on stream); returns count."""
    if count is None:
        count = result.info()["n_candidates"] - first
    _check(_lib.sas_stamps(result._h, int(first), int(count), _dev_ptr(out_dev) if count else None,
                           _stream_handle(stream)))
    return count


def sas_stamps_indexed(result: Result, idx_dev, count: int, out_dev, stream=None) -> int:
    """Stamps of candidates idx[0..count) (device uint32 indices)."""
    _check(_lib.sas_stamps_indexed(result._h, _dev_ptr(idx_dev) if count else None, int(count),
                                   _dev_ptr(out_dev) if count else None, _stream_handle(stream)))
    return count


def sas_peaks(result: Result, idx_dev, stream=None) -> int:
    """Local peaks: ascending candidate indices into idx_dev (device uint32 with
    room for n_candidates); returns their number (synchronizes)."""
    n = ctypes.c_uint64()
    _check(_lib.sas_peaks(result._h, _dev_ptr(idx_dev) if idx_dev is not None else None, ctypes.byref(n),
                          _stream_handle(stream)))
    return n.value


def sas_owned(result: Result, idx_dev, n_keep: int = 0, stream=None) -> int:
    """Ownership selection: ascending kept candidate indices into idx_dev
    (device uint32, room for n_candidates); returns their number (synchronizes).
    n_keep > 0 also keeps candidates that own at least n_keep detections."""
    n = ctypes.c_uint64()
    _check(_lib.sas_owned(result._h, int(n_keep), _dev_ptr(idx_dev) if idx_dev is not None else None,
                          ctypes.byref(n), _stream_handle(stream)))
    return n.value


PEEL_SEQUENTIAL = 1


def sas_peel(result: Result, n_min: int, max_clusters: int = 1000, stream=None, sequential: bool = False) -> Result:
    """Cluster finding (Sec. 2.1 step 3) over a search result: a new Result
    whose candidates are the clusters in the order found."""
    h = _p()
    flags = PEEL_SEQUENTIAL if sequential else 0
    _check(_lib.sas_peel(result._h, int(n_min), int(max_clusters), flags, _stream_handle(stream),
                         ctypes.byref(h)))
    return Result(h)


TRACK_DTYPE = np.dtype([("vx", "<f8"), ("vy", "<f8"), ("x0", "<f8"), ("y0", "<f8"), ("res_xx", "<f8"),
                        ("res_xy", "<f8"), ("res_yy", "<f8"), ("det", "<f8"), ("status", "<u4"),
                        ("iterations", "<u4"), ("h", "<u4"), ("n_points", "<u4"), ("id_off", "<u8"),
                        ("id_len", "<u4"), ("cluster", "<u4")])
assert TRACK_DTYPE.itemsize == 96
TRACK_CONVERGED, TRACK_MAX_ITER, TRACK_DEGENERATE, TRACK_TOO_MANY = 0, 1, 2, 3
REFINE_MAX_POINTS = 1024


class sas_refine_opts(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("n_starts", ctypes.c_uint32), ("n_best", ctypes.c_uint32),
                ("max_csteps", ctypes.c_uint32), ("max_iter", ctypes.c_uint32), ("radius", ctypes.c_int32),
                ("reserved", ctypes.c_uint32)]


_lib.sas_refine.argtypes = [_p, _p, ctypes.POINTER(sas_refine_opts), _p, ctypes.POINTER(_p)]
_lib.sas_tracks_get.argtypes = [_p, _p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64), _p, ctypes.c_uint64,
                                ctypes.POINTER(ctypes.c_uint64), ctypes.c_int]
_lib.sas_tracks_free.argtypes = [_p]
_lib.sas_tracks_free.restype = None
EXPORTED += ["sas_refine", "sas_tracks_get", "sas_tracks_free"]


class Tracks:
    """Refined trajectories (sas_tracks); owns device memory until freed."""

    def __init__(self, h):
        self._h = h

    def tracks(self):
        """(tracks: structured array of TRACK_DTYPE, ids: uint32 array)."""
        nt, ni = ctypes.c_uint64(), ctypes.c_uint64()
        _lib.sas_tracks_get(self._h, None, 0, ctypes.byref(nt), None, 0, ctypes.byref(ni), 0)
        tr = np.zeros(nt.value, TRACK_DTYPE)
        ids = np.zeros(ni.value, np.uint32)
        _check(_lib.sas_tracks_get(self._h, tr.ctypes.data if nt.value else None, nt.value, ctypes.byref(nt),
                                   ids.ctypes.data if ni.value else None, ni.value, ctypes.byref(ni), 0))
        return tr, ids

    def free(self):
        if self._h is not None and self._h.value:
            _lib.sas_tracks_free(self._h)
            self._h = _p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def sas_refine(search: Result, clusters: Result | None = None, seed: int = 0, n_starts: int = 0, n_best: int = 0,
               max_csteps: int = 0, max_iter: int = 0, radius: int = 0, stream=None) -> Tracks:
    """Refinement and gathering (Sec. 2.1 steps 4-6) of every cluster of
    `clusters` (default: the search's own candidates); zeros take the
    library's defaults."""
    o = sas_refine_opts(seed & ((1 << 64) - 1), n_starts, n_best, max_csteps, max_iter, radius, 0)
    h = _p()
    _check(_lib.sas_refine(search._h, (clusters or search)._h, ctypes.byref(o), _stream_handle(stream),
                           ctypes.byref(h)))
    return Tracks(h)


# ---- search parameters (Sec. 2.2): host functions of the library ----------
_D = ctypes.c_double
_PD = ctypes.POINTER(ctypes.c_double)
_lib.sas_param_velocity_count.argtypes = [_D] * 6 + [_PD]
_lib.sas_param_n_stacks.argtypes = [_D] * 3 + [_PD]
_lib.sas_param_peak_density.argtypes = [_D, _D, _PD]
_lib.sas_param_peaks_above.argtypes = [_D, _D, _PD]
_lib.sas_param_noise_rate.argtypes = [_D, _p, ctypes.c_uint32, _D, _PD]
_lib.sas_param_poisson_sf.argtypes = [ctypes.c_uint32, _D, _PD]
_lib.sas_param_choose_n_min.argtypes = [_D, _D, ctypes.POINTER(ctypes.c_uint32)]
_lib.sas_param_p_signal.argtypes = [_D] * 4 + [_PD]
_lib.sas_param_signal_tail.argtypes = [_p, ctypes.c_uint32, ctypes.c_uint32, _PD]
_lib.sas_param_dx_scan.argtypes = [_D, _D, _p, ctypes.c_uint32, _p, ctypes.c_uint32, _D, _D, _D, _D, _p, _p, _p]
EXPORTED += ["sas_param_velocity_count", "sas_param_n_stacks", "sas_param_peak_density", "sas_param_peaks_above",
             "sas_param_noise_rate", "sas_param_poisson_sf", "sas_param_choose_n_min", "sas_param_p_signal",
             "sas_param_signal_tail", "sas_param_dx_scan"]


def _d_call(fn, *args) -> float:
    out = ctypes.c_double()
    _check(fn(*args, ctypes.byref(out)))
    return out.value


class params:
    """sas_param_*: the parameter relations of Sec. 2.2 (host computation)."""

    @staticmethod
    def velocity_count(vmin_x, vmax_x, vmin_y, vmax_y, dx, dt) -> float:
        return _d_call(_lib.sas_param_velocity_count, vmin_x, vmax_x, vmin_y, vmax_y, dx, dt)

    @staticmethod
    def n_stacks(n_velocities, omega, dx) -> float:
        return _d_call(_lib.sas_param_n_stacks, n_velocities, omega, dx)

    @staticmethod
    def peak_density(z, a=1.0) -> float:
        return _d_call(_lib.sas_param_peak_density, z, a)

    @staticmethod
    def peaks_above(nu_th, a=1.0) -> float:
        return _d_call(_lib.sas_param_peaks_above, nu_th, a)

    @staticmethod
    def noise_rate(nu_th, a_list, dx) -> float:
        a = np.ascontiguousarray(a_list, np.float64)
        return _d_call(_lib.sas_param_noise_rate, nu_th, a.ctypes.data if len(a) else None, len(a), dx)

    @staticmethod
    def poisson_sf(k, lam) -> float:
        return _d_call(_lib.sas_param_poisson_sf, int(k), lam)

    @staticmethod
    def choose_n_min(lam, eps) -> int:
        out = ctypes.c_uint32()
        _check(_lib.sas_param_choose_n_min(lam, eps, ctypes.byref(out)))
        return out.value

    @staticmethod
    def p_signal(nu, nu_th, a, dx) -> float:
        return _d_call(_lib.sas_param_p_signal, nu, nu_th, a, dx)

    @staticmethod
    def signal_tail(p_list, k) -> float:
        p = np.ascontiguousarray(p_list, np.float64)
        return _d_call(_lib.sas_param_signal_tail, p.ctypes.data if len(p) else None, len(p), int(k))

    @staticmethod
    def dx_scan(nu, nu_th, a_list, dx_list, dv, dt, omega, n_false):
        a = np.ascontiguousarray(a_list, np.float64)
        dx = np.ascontiguousarray(dx_list, np.float64)
        es, en = np.zeros(len(dx)), np.zeros(len(dx))
        nm = np.zeros(len(dx), np.uint32)
        _check(_lib.sas_param_dx_scan(nu, nu_th, a.ctypes.data if len(a) else None, len(a),
                                      dx.ctypes.data if len(dx) else None, len(dx), dv, dt, omega, n_false,
                                      es.ctypes.data, en.ctypes.data, nm.ctypes.data))
        return [(float(d), float(s), float(n), int(m)) for d, s, n, m in zip(dx, es, en, nm)]


def _opt_ptr(a):
    return None if a is None else _dev_ptr(a)


def vet_num_params() -> int:
    return int(_lib.sas_vet_num_params())


class Vetter:
    """sas_vet_*: the candidate-vetting CNN on one device.  Device arrays are
    torch CUDA tensors (or __cuda_array_interface__ objects); host arrays are
    NumPy."""

    def __init__(self, device: int = 0, max_batch: int = 1024):
        h = _p()
        _check(_lib.sas_vet_create(int(device), int(max_batch), ctypes.byref(h)))
        self._h = h
        self.max_batch = int(max_batch)
        self.n_params = vet_num_params()

    def check(self):
        """Synchronize; raise if a tensor-core wait gave up since the last check."""
        _check(_lib.sas_vet_check(self._h))

    def set_adam(self, beta1=0.9, beta2=0.999, eps=1e-8):
        _check(_lib.sas_vet_set_adam(self._h, beta1, beta2, eps))

    def set_state(self, params, m=None, v=None, step: int = 0):
        p = np.ascontiguousarray(params, np.float32)
        assert p.shape == (self.n_params,)
        mm = None if m is None else np.ascontiguousarray(m, np.float32)
        vv = None if v is None else np.ascontiguousarray(v, np.float32)
        _check(_lib.sas_vet_set_state(self._h, p.ctypes.data, None if mm is None else mm.ctypes.data,
                                      None if vv is None else vv.ctypes.data, int(step)))

    def get_state(self):
        """(params, m, v, step) as float32 host arrays."""
        p = np.zeros(self.n_params, np.float32)
        m = np.zeros(self.n_params, np.float32)
        v = np.zeros(self.n_params, np.float32)
        st = ctypes.c_uint64()
        _check(_lib.sas_vet_get_state(self._h, p.ctypes.data, m.ctypes.data, v.ctypes.data,
                                      ctypes.byref(st)))
        return p, m, v, st.value

    def get_bf16(self) -> np.ndarray:
        """The BF16 working copy as float32 values."""
        raw = np.zeros(self.n_params, np.uint16)
        _check(_lib.sas_vet_get_bf16(self._h, raw.ctypes.data))
        return (raw.astype(np.uint32) << 16).view(np.float32)

    def activations(self, layer: int, n: int) -> np.ndarray:
        """The BF16 activations of layer 1..4 that the last batch stored (first n
        samples), as float32: [n, 32, h, h] for the convolutions, [n, 64] for fc1."""
        shape = {1: (32, 13, 13), 2: (32, 11, 11), 3: (32, 9, 9), 4: (64,)}[int(layer)]
        raw = np.zeros((int(n),) + shape, np.uint16)
        _check(_lib.sas_vet_get_activations(self._h, int(layer), int(n), raw.ctypes.data))
        return (raw.astype(np.uint32) << 16).view(np.float32)

    def forward(self, stamps_dev, n: int, logits_dev, index=None, stream=None):
        _check(_lib.sas_vet_forward(self._h, _dev_ptr(stamps_dev) if n else None,
                                    _opt_ptr(index) if n else None, int(n),
                                    _dev_ptr(logits_dev) if n else None, _stream_handle(stream)))

    def gradients(self, stamps_dev, labels_dev, n: int, grad_dev, loss_dev=None, index=None,
                  stream=None):
        _check(_lib.sas_vet_gradients(self._h, _dev_ptr(stamps_dev), _dev_ptr(labels_dev), _opt_ptr(index),
                                      int(n), _dev_ptr(grad_dev), _opt_ptr(loss_dev),
                                      _stream_handle(stream)))

    def apply_gradients(self, grad_dev, lr: float, stream=None):
        _check(_lib.sas_vet_apply_gradients(self._h, _dev_ptr(grad_dev), float(lr),
                                            _stream_handle(stream)))

    def train_step(self, stamps_dev, labels_dev, n: int, lr: float, loss_dev=None, index=None,
                   stream=None):
        _check(_lib.sas_vet_train_step(self._h, _dev_ptr(stamps_dev), _dev_ptr(labels_dev), _opt_ptr(index),
                                       int(n), float(lr), _opt_ptr(loss_dev), _stream_handle(stream)))

    def destroy(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.sas_vet_destroy(self._h)
            self._h = _p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass
