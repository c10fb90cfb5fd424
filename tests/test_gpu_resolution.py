"""GPU parity of the image-space resolution model (P = A G, Eq. (1)'s limited
spatial resolution) against the FP64 oracle: G itself, and LM-SPDHG (Alg. 2)
with P = A G for single updates and whole epochs (TMA-staged and plain image
passes); the modes that do not support it refuse it."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2201_05497_gb300 import synth as S
from tests import _helpers as H

pytestmark = pytest.mark.gpu

FWHM = 4.5  # mm


@pytest.fixture(scope="module")
def lm():
    from paper_2201_05497_gb300 import build, lm as _lm
    build.build()
    _lm.load_library()
    return _lm


class Case:
    def __init__(self, lm, name, fwhm=FWHM, n_events=None):
        wl, lf, ev = H.workload_data(name, n_events)
        self.wl, self.ev, self.fwhm = wl, ev, fwhm
        self.n_sub = wl.n_subsets
        self.geo_o = O.Geometry.from_workload(wl)
        self.geo_g = lm.Geometry.from_workload(wl)
        self.E = O.EventArrays.from_events(ev)
        # P^T 1 = G A^T 1
        self.sens_or = O.res_apply(self.geo_o, fwhm, O.sens(self.geo_o, lf))
        self.mu = O.event_counts(ev.det1, ev.det2, ev.tof)
        self.x0 = np.full(self.geo_o.V, np.float32(0.8 * ev.n / self.sens_or.sum()), dtype=np.float32)
        self.knorm = H.knorm_closed(wl.grid.n)
        self.gamma = float(np.float32(3.0 / self.x0.max()))
        self.lm = lm

    def oracle(self):
        o = O.LM(self.geo_o, self.E, self.mu, self.n_sub, beta=self.wl.beta, gamma=self.gamma, rho=0.999,
                 knorm=self.knorm, res_fwhm=self.fwhm)
        o.init(self.x0, self.sens_or)
        return o

    def gpu(self, **kw):
        lm = self.lm
        pe = lm.event_setup(self.geo_g, lm.DeviceEvents.from_numpy(self.ev), self.n_sub)
        sens = torch.from_numpy(self.sens_or.astype(np.float32)).cuda()
        args = dict(beta=self.wl.beta, n_subsets=self.n_sub, gamma=self.gamma, rho=0.999, knorm=self.knorm,
                    kahan=True, group=0, projector="direct", res_fwhm=self.fwhm)
        args.update(kw)
        return lm.LMSPDHG(self.geo_g, pe, sens, torch.from_numpy(self.x0).cuda(), **args)


# 2d_small: the fused x/y pass alone; 3d_small, 3d_quad: the fused x/y and z passes (equal and unequal
# radii); FWHM 40 mm: 10 taps per side, the per-axis passes
@pytest.mark.parametrize("name,fwhm", [("2d_small", 4.5), ("3d_small", 6.0), ("3d_quad", 9.0), ("3d_small", 40.0)])
def test_res_apply_matches_oracle(lm, name, fwhm):
    wl = S.workload(name)
    geo_o, geo_g = O.Geometry.from_workload(wl), lm.Geometry.from_workload(wl)
    x = np.random.default_rng(1).uniform(0.0, 2.0, geo_o.V).astype(np.float32)
    got = lm.res_apply(geo_g, fwhm, torch.from_numpy(x).cuda()).cpu().numpy()
    assert H.rel_l2(got, O.res_apply(geo_o, fwhm, x)) < 1e-6
    # in place, and fwhm 0 copies
    xt = torch.from_numpy(x).cuda()
    lm.res_apply(geo_g, fwhm, xt, out=xt)
    np.testing.assert_array_equal(xt.cpu().numpy(), got)
    np.testing.assert_array_equal(lm.res_apply(geo_g, 0.0, torch.from_numpy(x).cuda()).cpu().numpy(), x)


@pytest.mark.parametrize("name", ["2d_small", "3d_small", "3d_quad"])
@pytest.mark.parametrize("sel", ["data", "prior"])
def test_single_update_matches_oracle(lm, name, sel):
    c = Case(lm, name)
    o = c.oracle()
    g = c.gpu()
    seq = [2 if sel == "data" else c.n_sub, c.n_sub, 0]
    for i in seq:
        o.update(i)
    g.updates(seq)
    assert H.rel_l2(g.x().cpu().numpy(), o.x) < 1e-5
    assert H.rel_l2(g.z().cpu().numpy(), o.z) < 1e-5
    assert H.rel_l2(g.w().cpu().numpy(), o.w) < H.REL_L2_IMAGE
    assert g.tuning()["image_kernel"] == ("tma" if name == "3d_quad" else "plain")


@pytest.mark.parametrize("name,epochs,image_kernel", [("2d_small", 3, 0), ("3d_small", 2, 0), ("3d_quad", 2, 2),
                                                       ("3d_quad", 2, 1)])
def test_epochs_match_oracle(lm, name, epochs, image_kernel):
    c = Case(lm, name)
    o = c.oracle()
    g = c.gpu(image_kernel=image_kernel)
    seq = S.selection_sequence(c.n_sub, 2 * c.n_sub * epochs, seed=3)
    for k in range(epochs):
        s = seq[2 * c.n_sub * k:2 * c.n_sub * (k + 1)]
        g.epoch(s)
        o.run(s)
    err = H.rel_l2(g.x().cpu().numpy(), o.x)
    assert err < H.REL_L2_IMAGE, err
    f_g, f_o = g.objective(), o.objective()
    assert abs(f_g - f_o) <= 1e-5 * abs(f_o)


def test_unsupported_modes_refuse(lm):
    c = Case(lm, "3d_quad", n_events=3000)
    with pytest.raises(lm.LMError) as ei:
        c.gpu(deterministic=True)
    assert ei.value.code == 1
    g = c.gpu()
    b = lm.Batch(2, c.n_sub)
    with pytest.raises(lm.LMError) as ei:
        b.set(0, g)
    assert ei.value.code == 1
    b.close()
    g.close()
