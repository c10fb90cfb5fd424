"""CPU checks of the C ABI: the library builds and loads, exports every
function include/lmspdhg.h declares, and rejects invalid host arguments
before touching a device.  No compute call is made (no GPU here)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lmspdhg.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b((?:lm|lmspdhg)_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def L():
    from paper_2201_05497_gb300 import build
    path = build.build()
    from paper_2201_05497_gb300 import lm
    return lm.load_library(path)


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert len(names) >= 25
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_host_only_queries(L):
    from paper_2201_05497_gb300 import lm
    g = lm.lm_grid((C.c_int32 * 3)(200, 200, 96), (C.c_float * 3)(2.5, 2.5, 2.5), (C.c_float * 3)(0, 0, 0))
    assert L.lm_version() >= 100
    assert L.lm_tv_ndim(C.byref(g)) == 3
    V = 200 * 200 * 96
    assert L.lm_fwd_workspace_bytes(C.byref(g)) >= 4 * V
    assert L.lm_back_workspace_bytes(C.byref(g), 1) >= 16 * V
    assert L.lm_knorm_workspace_bytes(C.byref(g)) >= 16 * V
    sb = L.lmspdhg_state_bytes(C.byref(g), 10_000_000, 28, 0)
    # images (x in two layouts x2, z, zc, T, w x2 with 3 components, dz x2) and 4 B/event of y + scratch
    assert sb >= (4 + 3 + 6 + 2) * 4 * V + 8 * 10_000_000
    assert sb < 2 * ((4 + 3 + 6 + 2) * 4 * V + 8 * 10_000_000)
    sc = lm.lm_scanner(36, 672, None)
    assert L.lm_n_lor(C.byref(sc)) == 672 * 671 // 2 * 36 * 36
    assert L.lm_setup_workspace_bytes(10_000_000) >= 12 * 2 * 10_000_000


def test_invalid_arguments_rejected_on_host(L):
    from paper_2201_05497_gb300 import lm
    g_bad = lm.lm_grid((C.c_int32 * 3)(0, 4, 4), (C.c_float * 3)(1, 1, 1), (C.c_float * 3)(0, 0, 0))
    assert L.lmspdhg_state_bytes(C.byref(g_bad), 10, 2, 0) == 0
    tof = lm.lm_tof(25.0, 22.0, 3.0, 28)  # even bin count
    g = lm.lm_grid((C.c_int32 * 3)(4, 4, 1), (C.c_float * 3)(1, 1, 1), (C.c_float * 3)(0, 0, 0))
    sc = lm.lm_scanner(1, 16, C.c_void_p(16))  # never dereferenced: rejected before any launch
    ev = lm.lm_events(None, None, None, None, None, 5)
    rc = L.lm_fwd(C.byref(sc), C.byref(g), C.byref(tof), None, C.byref(ev), None, None, 0, None)
    assert rc == 1
    assert b"odd" in L.lm_last_error()
    rc = L.lm_fwd(C.byref(sc), None, C.byref(tof), None, C.byref(ev), None, None, 0, None)
    assert rc == 1
    rc = L.lm_tv_prox(C.byref(g), None, C.c_float(0.1), None)
    assert rc == 1
    rc = L.lm_knorm_fp64(C.byref(g), 10, None, 0, None, None)
    assert rc == 1
