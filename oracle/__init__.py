"""CPU oracle for catalog shift-and-stack (Sec. 2.1 steps 1-3) -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the C-ABI library and
its binding) never touches it; the two share no code.

* ``sas_oracle.c``  the definition written out in plain C (int64, floor division);
                    loaded here through ctypes.
* ``brute.py``      a second, independent formulation in pure Python
                    (dict of epoch sets) for tiny inputs; pins the C oracle.
* ``vetter.py``     float64 NumPy forward/backward of the candidate-vetting CNN.
* ``peel.py``       cluster finding (Sec. 2.1 step 3), over the candidate list and
                    as the literal rerun-the-search loop.
* ``refine.py``     refinement and gathering (Sec. 2.1 steps 4-6): MCD regression
                    by FAST-MCD with counter-based draws, gathering, iteration.

Parity status: the stack oracle is pinned (brute force, hand-built movers,
invariants, noise statistics; see tests/test_oracle_*.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sas_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_sas.so")
_lock = threading.Lock()
_lib = None

CAND_DTYPE = np.dtype([("v_idx", "<i8"), ("bx", "<i4"), ("by", "<i4"), ("distinct", "<i4"),
                       ("raw", "<i4"), ("id_off", "<i8"), ("id_len", "<i8")])
assert CAND_DTYPE.itemsize == 40


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (plain C11, -O2, OpenMP for
    oracle_stack_mt's loop over velocity chunks; without OpenMP that loop runs
    on one thread)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC]
        try:
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


def bind(path: str):
    """Load a compiled oracle library and declare its signatures."""
    lib = ctypes.CDLL(path)
    i64, i32, p = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p
    lib.oracle_stack.restype = ctypes.c_int
    lib.oracle_stack.argtypes = [i64, p, p, p, i32, p, i64,
                                 i32, i32, i32, i32, i32, i32, i32, i32,
                                 i32, i32, i32, i32, i32,
                                 i32, i64, i64, i64,
                                 p, i64, p, p, i64, p, p]
    lib.oracle_cell.restype = ctypes.c_int
    lib.oracle_cell.argtypes = [i64, p, p, p, i32, p, i64,
                                i32, i32, i32, i32, i32,
                                i32, i32, i32, i32, i32,
                                i64, i32, i32, p, p, p, i64, p]
    lib.oracle_histogram.restype = ctypes.c_int
    lib.oracle_histogram.argtypes = [i64, p, p, p, i32, p, i64, i64, i64,
                                     i32, i32, i32, i32, i32, p, p]
    lib.oracle_t0.restype = ctypes.c_int64
    lib.oracle_t0.argtypes = [i64, p, p]
    lib.oracle_stack_mt.restype = ctypes.c_int
    lib.oracle_stack_mt.argtypes = lib.oracle_stack.argtypes + [i32]
    lib.oracle_threads.restype = ctypes.c_int32
    lib.oracle_threads.argtypes = []
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = bind(build())
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _cat_arrays(cat):
    x = np.ascontiguousarray(cat.x, np.int32)
    y = np.ascontiguousarray(cat.y, np.int32)
    e = np.ascontiguousarray(cat.epoch, np.uint16)
    t = np.ascontiguousarray(cat.t, np.int64)
    return x, y, e, t


class OracleResult:
    def __init__(self, cands: np.ndarray, ids: np.ndarray, n_pairs: int):
        self.cands = cands
        self.ids = ids
        self.n_pairs = n_pairs

    def id_lists(self):
        return [self.ids[c["id_off"]: c["id_off"] + c["id_len"]] for c in self.cands]


def threads() -> int:
    """Threads the OpenMP form uses by default (1 when built without OpenMP)."""
    return int(_load().oracle_threads())


def stack(cat, grid, n_min: int, v_begin: int = 0, v_end: int | None = None,
          max_candidates: int = 0, lib=None, threads: int = 1) -> OracleResult:
    """Run the oracle search over lattice indices [v_begin, v_end).  threads == 1:
    the single loop over velocities (oracle_stack); otherwise oracle_stack_mt,
    the same search over velocity chunks in an OpenMP loop (threads <= 0: all
    of OpenMP's default team), merged in the same total order."""
    lib = lib or _load()
    x, y, e, t = _cat_arrays(cat)
    if v_end is None:
        v_end = grid.nvx * grid.nvy
    cap, ids_cap = 1024, 1 << 16
    while True:
        cands = np.zeros(cap, CAND_DTYPE)
        ids = np.zeros(ids_cap, np.int32)
        nc, ni, npairs = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        args = (x.shape[0], _ptr(x), _ptr(y), _ptr(e), t.shape[0], _ptr(t),
                int(cat.ticks_per_hour),
                grid.vx0, grid.vy0, grid.dvx, grid.dvy, grid.nvx, grid.nvy,
                grid.speed_min, grid.speed_max,
                grid.x_min, grid.y_min, grid.nbx, grid.nby, grid.bin,
                int(n_min), int(v_begin), int(v_end), int(max_candidates),
                _ptr(cands), cap, ctypes.byref(nc), _ptr(ids), ids_cap,
                ctypes.byref(ni), ctypes.byref(npairs))
        if threads == 1:
            rc = lib.oracle_stack(*args)
        else:
            rc = lib.oracle_stack_mt(*args, int(threads))
        if rc == 3:
            cap, ids_cap = max(cap, nc.value), max(ids_cap, ni.value)
            continue
        if rc != 0:
            raise RuntimeError(f"oracle_stack failed with status {rc}")
        return OracleResult(cands[: nc.value].copy(), ids[: ni.value].copy(), npairs.value)


def cell(cat, grid, v_idx: int, bx: int, by: int):
    """(distinct, raw, ids) of one histogram cell, from the definition alone."""
    lib = _load()
    x, y, e, t = _cat_arrays(cat)
    cap = 4096
    while True:
        ids = np.zeros(cap, np.int32)
        d, r, k = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        rc = lib.oracle_cell(x.shape[0], _ptr(x), _ptr(y), _ptr(e), t.shape[0], _ptr(t),
                             int(cat.ticks_per_hour), grid.vx0, grid.vy0, grid.dvx, grid.dvy,
                             grid.nvx, grid.x_min, grid.y_min, grid.nbx, grid.nby, grid.bin,
                             int(v_idx), int(bx), int(by), ctypes.byref(d), ctypes.byref(r),
                             _ptr(ids), cap, ctypes.byref(k))
        if rc != 0:
            raise RuntimeError(f"oracle_cell failed with status {rc}")
        if k.value > cap:
            cap = k.value
            continue
        return d.value, r.value, ids[: k.value].copy()


def histogram(cat, grid, vx: int, vy: int):
    """Dense (distinct, raw) histograms [nby, nbx] of one velocity (steps 1-2)."""
    lib = _load()
    x, y, e, t = _cat_arrays(cat)
    dist = np.zeros(grid.nbx * grid.nby, np.int32)
    raw = np.zeros(grid.nbx * grid.nby, np.int32)
    rc = lib.oracle_histogram(x.shape[0], _ptr(x), _ptr(y), _ptr(e), t.shape[0], _ptr(t),
                              int(cat.ticks_per_hour), int(vx), int(vy), grid.x_min, grid.y_min,
                              grid.nbx, grid.nby, grid.bin, _ptr(dist), _ptr(raw))
    if rc != 0:
        raise RuntimeError(f"oracle_histogram failed with status {rc}")
    return dist.reshape(grid.nby, grid.nbx), raw.reshape(grid.nby, grid.nbx)


def t0(cat) -> int:
    lib = _load()
    x, y, e, t = _cat_arrays(cat)
    return int(lib.oracle_t0(e.shape[0], _ptr(e), _ptr(t)))
