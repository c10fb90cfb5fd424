"""GPU parity of listmode EM-TV (Alg. 3, the warm start x0) against the FP64
oracle: the subset EM step, the weighted TV denoiser, whole passes over the
subsets with and without the prior, empty subsets, and argument errors."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from tests import _helpers as H

pytestmark = pytest.mark.gpu

PDHG_ITERS = 20


@pytest.fixture(scope="module")
def lm():
    from paper_2201_05497_gb300 import build, lm as _lm
    build.build()
    _lm.load_library()
    return _lm


class Prob:
    """One seeded workload on both sides; the oracle gets the float32 sens the
    GPU uses."""

    def __init__(self, lm, name, n_events=None, n_subsets=None):
        wl, lf, ev = H.workload_data(name, n_events)
        self.wl, self.ev = wl, ev
        self.n_sub = wl.n_subsets if n_subsets is None else n_subsets
        self.geo_o = O.Geometry.from_workload(wl)
        self.geo_g = lm.Geometry.from_workload(wl)
        self.E = O.EventArrays.from_events(ev)
        s32 = O.sens(self.geo_o, lf).astype(np.float32)
        self.sens_o = s32.astype(np.float64)
        self.sens_g = torch.from_numpy(s32).cuda()
        kappa = 0.8 * ev.n / self.sens_o.sum()
        self.x0 = np.full(self.geo_o.V, np.float32(kappa), dtype=np.float32)
        self.knorm = H.knorm_closed(wl.grid.n)
        self.pe = lm.event_setup(self.geo_g, lm.DeviceEvents.from_numpy(ev), self.n_sub)

    def subset_events(self, lm, i):
        a, b = int(self.pe.sub_off[i]), int(self.pe.sub_off[i + 1])
        d = self.pe.events
        return lm.DeviceEvents(d.det1[a:b], d.det2[a:b], None if d.tof is None else d.tof[a:b],
                               d.corr[a:b], d.contam[a:b])


@pytest.mark.parametrize("name", ["2d_small", "3d_small", "3d_quad"])
def test_em_step_matches_oracle(lm, name):
    p = Prob(lm, name)
    rng = np.random.default_rng(5)
    x = (p.x0 * rng.uniform(0.5, 1.5, p.geo_o.V)).astype(np.float32)
    x[::7] = 0.0  # voxels at zero stay at zero
    i = 1
    em = O.EMTV(p.geo_o, p.E, p.n_sub, beta=0.0, knorm=p.knorm)
    want = em.em_step(x.astype(np.float64), p.sens_o, i)
    got = lm.emtv_em_step(p.geo_g, p.subset_events(lm, i), p.n_sub, p.sens_g, torch.from_numpy(x).cuda())
    got = got.cpu().numpy()
    assert np.all(got[::7] == 0.0)
    assert np.all(got[p.sens_o == 0] == 0.0)
    err = H.rel_l2(got, want)
    assert err < H.REL_EVENT, err


@pytest.mark.parametrize("name", ["2d_small", "3d_small"])
@pytest.mark.parametrize("iters", [0, 1, PDHG_ITERS, 200])
def test_denoise_matches_oracle(lm, name, iters):
    p = Prob(lm, name)
    V = p.geo_o.V
    rng = np.random.default_rng(3)
    z = rng.uniform(0.0, 2.0, V).astype(np.float32)
    w = rng.uniform(0.5, 4.0, V).astype(np.float32)
    w[rng.uniform(0, 1, V) < 0.1] = 0.0  # held voxels
    free = (w > 0).astype(np.uint8)
    want, _ = O.emtv_denoise(p.geo_o, z, w, free, iters, p.knorm)
    got = lm.emtv_denoise(p.geo_g, torch.from_numpy(z).cuda(), torch.from_numpy(w).cuda(), iters, p.knorm)
    got = got.cpu().numpy()
    assert np.all(got[free == 0] == 0.0) and got.min() >= 0.0
    if iters == 0:
        np.testing.assert_array_equal(got, np.where(free > 0, z, 0.0).astype(np.float32))
    err = H.rel_l2(got, want)
    assert err < H.REL_EVENT, err


@pytest.mark.parametrize("name", ["2d_small", "3d_small", "3d_quad"])
@pytest.mark.parametrize("prior", [True, False])
def test_epoch_matches_oracle(lm, name, prior):
    """One pass over the subsets (the warm start of the listmode runs)."""
    p = Prob(lm, name)
    beta = p.wl.beta if prior else 0.0
    em = O.EMTV(p.geo_o, p.E, p.n_sub, beta=beta, knorm=p.knorm)
    want = em.epoch(p.x0.astype(np.float64), p.sens_o, pdhg_iters=PDHG_ITERS)
    x = torch.from_numpy(p.x0).cuda()
    lm.emtv_epoch(p.geo_g, p.pe, p.sens_g, x, beta=beta, pdhg_iters=PDHG_ITERS, knorm=p.knorm)
    got = x.cpu().numpy()
    assert got.min() >= 0.0
    err = H.rel_l2(got, want)
    assert err < H.REL_L2_IMAGE, err


def test_epoch_with_empty_subsets(lm):
    """Fewer events than subsets: the empty subsets' EM steps give z = 0."""
    p = Prob(lm, "2d_small", n_events=3, n_subsets=5)
    em = O.EMTV(p.geo_o, p.E, p.n_sub, beta=p.wl.beta, knorm=p.knorm)
    want = em.epoch(p.x0.astype(np.float64), p.sens_o, pdhg_iters=5)
    x = torch.from_numpy(p.x0).cuda()
    lm.emtv_epoch(p.geo_g, p.pe, p.sens_g, x, beta=p.wl.beta, pdhg_iters=5, knorm=p.knorm)
    got = x.cpu().numpy()
    assert np.all(want == 0.0)
    np.testing.assert_array_equal(got, np.zeros_like(got))


def test_emtv_argument_errors(lm):
    p = Prob(lm, "2d_small", n_events=2000)
    L = lm.load_library()
    g = p.geo_g
    x = torch.from_numpy(p.x0).cuda()
    nb = int(L.lm_emtv_workspace_bytes(C.byref(g.g)))
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    off = np.ascontiguousarray(p.pe.sub_off, dtype=np.int64)
    d = p.pe.events.desc()

    def call(ws_bytes=nb, iters=5, beta=0.1, knorm=p.knorm, off_arr=off):
        return L.lm_emtv_epoch(C.byref(g.sc), C.byref(g.g), C.byref(g.tof), C.byref(d),
                               off_arr.ctypes.data_as(C.POINTER(C.c_int64)), int(off_arr.shape[0] - 1),
                               lm._ptr(p.sens_g), lm._ptr(x), float(beta), int(iters), float(knorm),
                               lm._ptr(ws), int(ws_bytes), None)

    before = x.clone()
    assert call(ws_bytes=nb - 1) == 6       # LM_ERR_NOMEM
    assert call(iters=10001) == 1           # LM_ERR_INVALID_ARG
    assert call(iters=-1) == 1
    assert call(beta=-1.0) == 1
    assert call(knorm=0.0) == 1
    bad = off.copy()
    bad[1], bad[2] = bad[2], bad[1]
    assert call(off_arr=bad) == 1
    bad = off.copy()
    bad[-1] -= 1
    assert call(off_arr=bad) == 1
    torch.cuda.synchronize()
    assert torch.equal(x, before)           # nothing was queued
    assert call() == 0
    torch.cuda.synchronize()
    assert not torch.equal(x, before)
