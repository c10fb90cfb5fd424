"""CPU checks of the C ABI: the library builds and loads, exports every
function include/lmspdhg.h and the benchmark's include/lm_measure.h
declare, and rejects invalid host arguments
before touching a device.  No compute call is made (no GPU here)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lmspdhg.h")
MEASURE_HEADER = os.path.join(ROOT, "include", "lm_measure.h")


def _declared():
    src = open(HEADER).read() + open(MEASURE_HEADER).read()
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


def test_struct_layouts_match_the_binding(L):
    """The binding's ctypes descriptors have the sizes the library was built with
    (load_library checks the same and refuses a mismatch)."""
    from paper_2201_05497_gb300 import lm
    sizes = (C.c_size_t * 6)()
    assert L.lm_struct_sizes(sizes, 6) == 6
    assert list(sizes) == [C.sizeof(t) for t in (lm.lm_scanner, lm.lm_grid, lm.lm_tof, lm.lm_events, lm.lm_params,
                                                 lm.lm_server_config)]
    assert L.lm_struct_sizes(None, 0) == 6


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


class _FakeCudaTensor:
    """Stands in for a CUDA tensor (no GPU here): what the binding's
    pointer marshalling looks at."""

    is_cuda = True

    def __init__(self, dtype, n, contiguous=True):
        self.dtype, self._n, self._c = dtype, n, contiguous

    def is_contiguous(self):
        return self._c

    def numel(self):
        return self._n

    def data_ptr(self):
        return 4096


def test_binding_checks_tensors_before_calling():
    """Every device argument is checked (device, layout, dtype, size) in
    Python before the library sees its pointer."""
    torch = pytest.importorskip("torch")
    from paper_2201_05497_gb300 import lm
    f32 = torch.float32
    assert lm._f32(_FakeCudaTensor(f32, 10), 10, "x").value == 4096
    assert lm._f32(None, 10, "x") is None
    with pytest.raises(TypeError, match="x: expected torch.float32"):
        lm._f32(_FakeCudaTensor(torch.float64, 10), 10, "x")
    with pytest.raises(ValueError, match="x: 9 elements, at least 10 needed"):
        lm._f32(_FakeCudaTensor(f32, 9), 10, "x")
    with pytest.raises(ValueError, match="contiguous"):
        lm._f32(_FakeCudaTensor(f32, 10, contiguous=False), 10, "x")
    with pytest.raises(ValueError, match="CUDA"):
        lm._f32(torch.zeros(10), 10, "x")
    ev = lm.DeviceEvents(_FakeCudaTensor(torch.int32, 5), _FakeCudaTensor(torch.int64, 5), None, None, None)
    ev.det1.shape = (5,)
    with pytest.raises(TypeError, match="det2"):
        ev.desc()


def test_state_options_rejected_on_host(L):
    """lmspdhg_create refuses an unknown image kernel, a TMA kernel on a grid
    it cannot tile, and an invalid resolution model before touching a
    device (the pointers below are never dereferenced)."""
    from paper_2201_05497_gb300 import lm
    fake = C.c_void_p(4096)
    sc = lm.lm_scanner(1, 16, fake)
    tof = lm.lm_tof(25.0, 22.0, 3.0, 0)
    ev = lm.lm_events(fake, fake, None, fake, fake, 8)
    off = (C.c_int64 * 3)(0, 4, 8)

    def create(n, **kw):
        g = lm.lm_grid((C.c_int32 * 3)(*n), (C.c_float * 3)(2.5, 2.5, 2.5), (C.c_float * 3)(0, 0, 0))
        p = lm.lm_params(beta=0.1, rho=0.999, n_subsets=2, kahan=1, **kw)
        h = C.c_void_p()
        rc = L.lmspdhg_create(C.byref(h), C.byref(sc), C.byref(g), C.byref(tof), C.byref(ev), fake, off, fake, fake,
                              C.byref(p), fake, 1 << 40, None)
        return rc, L.lm_last_error().decode()

    rc, msg = create((48, 40, 8), image_kernel=4)
    assert rc == 1 and "image_kernel" in msg
    for kind in (2, 3):
        rc, msg = create((16, 16, 8), image_kernel=kind)  # nx < 40
        assert rc == 1 and "TMA" in msg
    rc, msg = create((48, 40, 8), res_fwhm=4.5, deterministic=1)
    assert rc == 1 and "float-atomic" in msg
    rc, msg = create((48, 40, 8), res_fwhm=float("nan"))
    assert rc == 1 and "res_fwhm" in msg
    rc, msg = create((48, 40, 8), res_fwhm=200.0)  # more taps per side than the kernels take
    assert rc == 1 and "too wide" in msg
