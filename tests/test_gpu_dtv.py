"""GPU parity of the directional TV prior (Sec. "Numerical experiments") against
the FP64 oracle: the field of a structural image, K and K^T, and LM-SPDHG
(Alg. 2) with K = P grad for single updates and whole epochs; a zero field
reproduces the TV path bit for bit (deterministic mode); TMA-staged data
passes with plain prior passes equal all-plain passes bit for bit."""
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
    _lm.load_library()
    return _lm


def structural_image(wl):
    """The paper's DTV experiments use the image itself with flipped
    contrast as the structural image: max(activity) - activity."""
    act = wl.phantom.voxelised(wl.grid).astype(np.float64)
    return (act.max() - act).astype(np.float32)


def eta_of(v, n):
    """eta = 1 % of the largest gradient magnitude of v."""
    a = v.reshape(n[2], n[1], n[0]).astype(np.float64)
    g2 = np.zeros_like(a)
    for ax in range(3):
        if a.shape[ax] > 1:
            d = np.diff(a, axis=ax)
            pad = [(0, 0)] * 3
            pad[ax] = (0, 1)
            g2 += np.pad(d, pad) ** 2
    return float(np.float32(0.01 * np.sqrt(g2.max())))


class Case:
    def __init__(self, lm, name, n_events=None):
        wl, lf, ev = H.workload_data(name, n_events)
        self.wl, self.ev = wl, ev
        self.n_sub = wl.n_subsets
        self.beta = 0.1  # the paper's DTV runs use beta = 0.1
        self.geo_o = O.Geometry.from_workload(wl)
        self.geo_g = lm.Geometry.from_workload(wl)
        self.E = O.EventArrays.from_events(ev)
        self.sens_or = O.sens(self.geo_o, lf)
        self.mu = O.event_counts(ev.det1, ev.det2, ev.tof)
        self.x0 = np.full(self.geo_o.V, np.float32(0.8 * ev.n / self.sens_or.sum()), dtype=np.float32)
        self.knorm = H.knorm_closed(wl.grid.n)
        self.gamma = float(np.float32(3.0 / self.x0.max()))
        self.perm = O.subset_permutation(ev.n, self.n_sub)
        v = structural_image(wl)
        self.v = v
        self.eta = eta_of(v, wl.grid.n)
        self.xi_g = lm.dtv_field(self.geo_g, torch.from_numpy(v).cuda(), self.eta)
        self.xi64 = self.xi_g.cpu().numpy().astype(np.float64)  # the same field on both sides
        self.lm = lm

    def oracle(self, xi=True):
        o = O.LM(self.geo_o, self.E, self.mu, self.n_sub, beta=self.beta, gamma=self.gamma, rho=0.999,
                 knorm=self.knorm, xi=self.xi64 if xi else None)
        o.init(self.x0, self.sens_or)
        return o

    def gpu(self, xi=None, deterministic=False, image_kernel=0):
        lm = self.lm
        pe = lm.event_setup(self.geo_g, lm.DeviceEvents.from_numpy(self.ev), self.n_sub)
        sens = torch.from_numpy(self.sens_or.astype(np.float32)).cuda()
        return lm.LMSPDHG(self.geo_g, pe, sens, torch.from_numpy(self.x0).cuda(), beta=self.beta,
                          n_subsets=self.n_sub, gamma=self.gamma, rho=0.999, knorm=self.knorm,
                          deterministic=deterministic, kahan=True, image_kernel=image_kernel, group=0,
                          projector="direct", xi=xi)


@pytest.mark.parametrize("name", ["2d_small", "3d_small"])
def test_field_and_operators_match_oracle(lm, name):
    c = Case(lm, name, n_events=2000)
    geo_o, geo_g = c.geo_o, c.geo_g
    want = O.dtv_xi(geo_o, c.v.astype(np.float64), c.eta)
    assert H.rel_l2(c.xi64, want) < 1e-6
    rng = np.random.default_rng(5)
    x = rng.uniform(0.0, 2.0, geo_o.V).astype(np.float32)
    g = rng.normal(size=geo_o.ndim * geo_o.V).astype(np.float32)
    kx = lm.dtv_grad(geo_g, c.xi_g, torch.from_numpy(x).cuda()).cpu().numpy()
    assert H.rel_l2(kx, O.dtv_grad(geo_o, c.xi64, x)) < 1e-6
    d = lm.dtv_div(geo_g, c.xi_g, torch.from_numpy(g).cuda()).cpu().numpy()
    assert H.rel_l2(d, -O.dtv_adj(geo_o, c.xi64, g)) < 1e-6
    # the part of K x along the field is what P leaves of it: (f . g)(1 - |f|^2)
    kx3 = kx.reshape(geo_o.ndim, geo_o.V)
    f3 = c.xi64.reshape(geo_o.ndim, geo_o.V)
    g3 = O.tv_grad(geo_o, x).reshape(geo_o.ndim, geo_o.V)
    along = (f3 * g3).sum(0) * (1.0 - (f3 * f3).sum(0))
    assert np.abs((kx3 * f3).sum(0) - along).max() <= 1e-5 * np.abs(kx3).max()


@pytest.mark.parametrize("name", ["2d_small", "3d_small", "3d_quad"])
@pytest.mark.parametrize("sel", ["data", "prior"])
def test_single_update_matches_oracle(lm, name, sel):
    c = Case(lm, name)
    o = c.oracle()
    g = c.gpu(xi=c.xi_g)
    seq = [2 if sel == "data" else c.n_sub, c.n_sub, 0]
    for i in seq:
        o.update(i)
    g.updates(seq)
    assert H.rel_l2(g.x().cpu().numpy(), o.x) < 1e-5
    assert H.rel_l2(g.z().cpu().numpy(), o.z) < 1e-5
    assert H.rel_l2(g.w().cpu().numpy(), o.w) < H.REL_L2_IMAGE
    # grids the TMA pass takes (3d_quad) stage every pass (the prior's with D from the dual step)
    assert g.tuning()["image_kernel"] == ("tma" if name == "3d_quad" else "plain")


@pytest.mark.parametrize("name,epochs", [("2d_small", 3), ("3d_small", 2), ("3d_quad", 2)])
def test_epochs_match_oracle(lm, name, epochs):
    c = Case(lm, name)
    o = c.oracle()
    g = c.gpu(xi=c.xi_g)
    seq = S.selection_sequence(c.n_sub, 2 * c.n_sub * epochs, seed=3)
    for k in range(epochs):
        s = seq[2 * c.n_sub * k:2 * c.n_sub * (k + 1)]
        g.epoch(s)
        o.run(s)
    err = H.rel_l2(g.x().cpu().numpy(), o.x)
    assert err < H.REL_L2_IMAGE, err
    f_g, f_o = g.objective(), o.objective()
    assert abs(f_g - f_o) <= 1e-5 * abs(f_o)
    # DTV differs from TV: the TV run ends elsewhere
    o_tv = c.oracle(xi=False)
    o_tv.run(seq)
    assert H.rel_l2(o_tv.x, o.x) > 10 * err


def test_zero_field_is_tv_bit_for_bit(lm):
    """xi = 0 makes P the identity: the DTV code path gives the TV result
    exactly (deterministic mode, plain image passes on both)."""
    c = Case(lm, "3d_quad")
    seq = S.selection_sequence(c.n_sub, 4 * c.n_sub, seed=3)
    zero = torch.zeros_like(c.xi_g)
    a = c.gpu(xi=zero, deterministic=True)
    b = c.gpu(xi=None, deterministic=True, image_kernel=1)
    for k in range(2):
        s = seq[2 * c.n_sub * k:2 * c.n_sub * (k + 1)]
        a.epoch(s)
        b.epoch(s)
    np.testing.assert_array_equal(a.x().cpu().numpy(), b.x().cpu().numpy())
    np.testing.assert_array_equal(a.w().cpu().numpy(), b.w().cpu().numpy())
    assert a.objective() == b.objective()


def test_tma_passes_equal_plain_passes(lm):
    """TMA-staged passes (the prior's staging D = P(w+ - w) of the dual step)
    and TMA-staged data passes with plain prior passes equal all-plain passes
    bit for bit (deterministic)."""
    c = Case(lm, "3d_quad")
    seq = S.selection_sequence(c.n_sub, 4 * c.n_sub, seed=3)
    g = {k: c.gpu(xi=c.xi_g, deterministic=True, image_kernel=k) for k in (1, 2, 3)}
    assert [g[k].tuning()["image_kernel"] for k in (1, 2, 3)] == ["plain", "tma", "tma_data"]
    for k in range(2):
        s = seq[2 * c.n_sub * k:2 * c.n_sub * (k + 1)]
        for st in g.values():
            st.epoch(s)
    for k in (2, 3):
        np.testing.assert_array_equal(g[k].x().cpu().numpy(), g[1].x().cpu().numpy())
        np.testing.assert_array_equal(g[k].z().cpu().numpy(), g[1].z().cpu().numpy())
        np.testing.assert_array_equal(g[k].w().cpu().numpy(), g[1].w().cpu().numpy())
        assert g[k].objective() == g[1].objective()
