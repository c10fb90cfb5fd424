"""The workspace-free deterministic back-projection (for callers that cannot
allocate device memory, e.g. a plug-in whose host application owns all
device memory, or a real-time path that must not allocate after start-up).

It is called through the C ABI and compared with the deterministic
back-projection that takes a caller workspace, on two calls in a row (the
second call must not see the first call's leftovers in the shared scratch).
This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2201_05497_gb300 import synth as S
from tests import _helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lm():
    from paper_2201_05497_gb300 import build, lm as _lm
    build.build()
    L = _lm.load_library()
    fn = L.lm_back_deterministic_noalloc
    fn.argtypes = [C.POINTER(_lm.lm_scanner), C.POINTER(_lm.lm_grid), C.POINTER(_lm.lm_tof),
                   C.POINTER(_lm.lm_events), C.c_void_p, C.c_void_p, C.c_void_p]
    fn.restype = C.c_int
    return _lm


def _noalloc(lm, geo, ev, v, img):
    d = ev.desc()
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lm.load_library().lm_back_deterministic_noalloc(C.byref(geo.sc), C.byref(geo.g), C.byref(geo.tof),
                                                           C.byref(d), C.c_void_p(v.data_ptr()),
                                                           C.c_void_p(img.data_ptr()), s)


@pytest.mark.parametrize("name,n", [("3d_small", 30000), ("2d_small", 20000), ("3d_mid", 40000)])
def test_noalloc_matches_workspace_version_twice(lm, name, n):
    wl, lf, ev = H.workload_data(name, n)
    geo = lm.Geometry.from_workload(wl)
    geo_o = O.Geometry.from_workload(wl)
    dev = lm.DeviceEvents.from_numpy(ev)
    rng = np.random.default_rng(4)
    base_np = rng.uniform(0, 1, geo.V).astype(np.float32)
    base = torch.from_numpy(base_np).cuda()
    for call in range(2):
        v_np = rng.normal(size=ev.n).astype(np.float32)
        v = torch.from_numpy(v_np).cuda()
        ref = lm.back(geo, v, dev, img=base.clone(), deterministic=True)
        out = base.clone()
        rc = _noalloc(lm, geo, dev, v, out)
        assert rc == 0, lm.load_library().lm_last_error()
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert H.rel_l2(o, r) < H.REL_EVENT, f"call {call}"
        # the fixed-point sums are exact, so the two versions agree bit for bit
        np.testing.assert_array_equal(o, r)
        # and both are the adjoint of the listmode projector: the FP64 oracle's
        # (P^LM)^T v added to the starting image
        img_or = base_np.astype(np.float64) + O.back(geo_o, ev, v_np.astype(np.float64))
        assert H.rel_l2(o, img_or) < H.REL_EVENT, f"call {call} vs oracle"


def test_noalloc_rejects_grids_above_its_capacity(lm):
    sc = S.Scanner(4, 64, 200.0, 4.0)
    xtal = torch.from_numpy(sc.crystal_table()).cuda()
    geo = lm.Geometry(xtal, sc.n_rings, sc.n_xtal, (256, 256, 65), (1.0, 1.0, 1.0), (0.0, 0.0, 0.0), 25.0, 22.0,
                      3.0, 17)
    ev = S.uniform_events(sc, S.Tof(25.0, 22.0, 3.0, 17), 100, seed=1)
    dev = lm.DeviceEvents.from_numpy(ev)
    v = torch.ones(ev.n, device="cuda")
    img = torch.zeros(1, device="cuda")  # never touched: the size check comes first
    rc = _noalloc(lm, geo, dev, v, img)
    assert rc == 6
    assert b"at most" in lm.load_library().lm_last_error()
