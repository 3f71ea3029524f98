"""The C-ABI library loads without a GPU, exports every symbol the public
headers declare, and rejects bad arguments on the host before touching CUDA."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sas():
    from paper_2509_26279_gb300 import _build
    _build.build()
    from paper_2509_26279_gb300 import sas as mod
    return mod


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(sas_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sas_create_grid", "sas_stack", "sas_candidates", "sas_result_free"):
        assert required in names


def test_every_declared_symbol_is_exported(sas):
    lib = ctypes.CDLL(sas.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(sas.EXPORTED) <= set(declared_functions())


def test_struct_sizes_match_header(sas):
    assert ctypes.sizeof(sas.sas_grid_desc) == 13 * 4
    assert ctypes.sizeof(sas.sas_catalog) == 8 + 3 * 8 + 8 + 8 + 8 + 8
    assert ctypes.sizeof(sas.sas_opts) == 3 * 8 + 10 * 4   # 10 uint32 fields
    assert ctypes.sizeof(sas.sas_result_info) == 5 * 8 + 10 * 4 + 6 * 4
    assert sas.CANDIDATE_DTYPE.itemsize == 32


def test_version_and_abi(sas):
    assert "sm_103a" in sas.sas_version()
    assert sas.library().sas_abi_version() == 2


def test_grid_validation_on_host(sas):
    from paper_2509_26279_gb300 import workloads as W
    good = W.tiny().grid
    sas.Grid(good)
    bad = [dict(nvx=0), dict(bin=0), dict(nby=0), dict(speed_min=5, speed_max=1),
           dict(x_min=1 << 28), dict(nbx=1 << 20, bin=1000), dict(nvx=1 << 16, nvy=1 << 16),
           dict(vx0=2**31 - 10, dvx=100, nvx=3)]
    for kw in bad:
        with pytest.raises(sas.SasError) as ei:
            sas.Grid(good, **kw)
        assert ei.value.status in (sas.SAS_ERR_ARG, sas.SAS_ERR_RANGE), kw


def test_stack_argument_checks_before_any_device_work(sas):
    import numpy as np
    from paper_2509_26279_gb300 import workloads as W
    g = sas.Grid(W.tiny().grid)
    x = np.zeros(3, np.int32)
    e = np.zeros(3, np.uint16)
    cases = [
        dict(t=np.zeros(0, np.int64), n_min=1, status=sas.SAS_ERR_RANGE),          # E = 0
        dict(t=np.zeros(1025, np.int64), n_min=1, status=sas.SAS_ERR_RANGE),       # E > max
        dict(t=np.zeros(2, np.int64), n_min=0, status=sas.SAS_ERR_ARG),            # n_min = 0
        dict(t=np.array([0, 1 << 33], np.int64), n_min=1, status=sas.SAS_ERR_RANGE),  # span
    ]
    for c in cases:
        with pytest.raises(sas.SasError) as ei:
            sas.sas_stack(g, x, x, e, c["t"], 3600, c["n_min"])
        assert ei.value.status == c["status"]
    with pytest.raises(sas.SasError) as ei:
        sas.sas_stack(g, x, x, e, np.zeros(2, np.int64), 0, 1)     # ticks_per_hour = 0
    assert ei.value.status == sas.SAS_ERR_ARG
    with pytest.raises(sas.SasError) as ei:
        sas.sas_stack(g, x, x, e, np.zeros(2, np.int64), 3600, 1,
                      opts=sas.make_opts(v_begin=5, v_end=2))
    assert ei.value.status == sas.SAS_ERR_ARG
