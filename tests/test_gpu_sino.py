"""GPU sinogram SPDHG (Alg. 1, the paper's comparison method) against the
FP64 oracle's Alg. 1 on the full TOF sinogram: the bin layout of
lm_sino_setup (view-based subsets), whole epochs with empty bins kept at
y = 1, the objective of Eq. (1), and the appendix's equivalence with
LM-SPDHG on the GPU (one subset, same selection sequence)."""
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


def view_subset_of_bins(sc, nb, n_subsets):
    """Subset of every canonical bin: view (c1 + c2) mod n_xtal of its LOR's
    transaxial pair, subset = view mod n."""
    l = np.arange(sc.n_lor, dtype=np.int64)
    q = l // (sc.n_rings * sc.n_rings)
    c1, c2 = S.pair_of_q(q, sc.n_xtal)
    sub_l = ((c1 + c2) % sc.n_xtal) % n_subsets
    return np.repeat(sub_l, nb).astype(np.int32)


class Case:
    def __init__(self, lm, name, n_subsets=None, n_events=None):
        wl, lf, ev = H.workload_data(name, n_events)
        self.wl, self.lf = wl, lf
        sc, tof = wl.scanner, wl.tof
        self.nb = max(tof.n_bins, 1)
        self.n_sub = wl.n_subsets if n_subsets is None else n_subsets
        self.geo_o = O.Geometry.from_workload(wl)
        self.geo_g = lm.Geometry.from_workload(wl)
        self.d = S.sinogram_counts(sc, tof, ev)
        self.NB = self.d.size
        # flat contamination: the events' expected s per bin
        self.s = np.full(self.NB, float(ev.contam[0]), dtype=np.float32)
        self.sub = view_subset_of_bins(sc, self.nb, self.n_sub)
        self.sens_or = O.sens(self.geo_o, lf)
        self.x0 = np.full(self.geo_o.V, np.float32(0.8 * ev.n / self.sens_or.sum()), dtype=np.float32)
        self.knorm = H.knorm_closed(wl.grid.n)
        self.gamma = float(np.float32(3.0 / self.x0.max()))
        self.lm = lm
        self.ev = ev

    def oracle(self):
        o = O.Sino(self.geo_o, self.lf, self.d.astype(np.float64), self.s.astype(np.float64), self.sub, self.n_sub,
                   beta=self.wl.beta, gamma=self.gamma, rho=0.999, knorm=self.knorm)
        o.init(self.x0, self.sens_or)
        return o

    def bins(self):
        lm = self.lm
        d = torch.from_numpy(self.d.view(np.int16)).cuda().view(torch.uint16)
        return lm.sino_setup(self.geo_g, d, torch.from_numpy(self.s).cuda(), self.n_sub,
                             torch.from_numpy(self.lf).cuda())

    def gpu(self, pe=None, **kw):
        lm = self.lm
        pe = self.bins() if pe is None else pe
        sens = torch.from_numpy(self.sens_or.astype(np.float32)).cuda()
        args = dict(beta=self.wl.beta, n_subsets=self.n_sub, gamma=self.gamma, rho=0.999, knorm=self.knorm,
                    kahan=True, group=0, projector="direct", sinogram=True)
        args.update(kw)
        return lm.LMSPDHG(self.geo_g, pe, sens, torch.from_numpy(self.x0).cuda(), **args), pe


def _canonical_index(c, pe):
    """Canonical bin index of every position of the GPU layout."""
    sc = c.wl.scanner
    d1 = pe.events.det1.cpu().numpy()
    d2 = pe.events.det2.cpu().numpy()
    tb = pe.events.tof.cpu().numpy()
    return S.sinogram_bins(sc, c.wl.tof, d1, d2, tb)


def test_bin_layout(lm):
    """Every canonical bin appears once, in its view-based subset, with its
    count, contamination and LOR factor; inside a subset in canonical order."""
    c = Case(lm, "2d_small", n_subsets=7)
    pe = c.bins()
    b = _canonical_index(c, pe)
    assert np.array_equal(np.sort(b), np.arange(c.NB))
    off = pe.sub_off
    assert off[0] == 0 and off[-1] == c.NB
    for k in range(c.n_sub):
        seg = b[off[k]:off[k + 1]]
        assert np.all(c.sub[seg] == k)
        assert np.all(np.diff(seg) > 0)
    np.testing.assert_array_equal(pe.mu.view(torch.int16).cpu().numpy().view(np.uint16), c.d[b])
    np.testing.assert_array_equal(pe.events.contam.cpu().numpy(), c.s[b])
    np.testing.assert_array_equal(pe.events.corr.cpu().numpy(), c.lf[b // c.nb])


@pytest.mark.parametrize("name,epochs", [("2d_small", 3), ("3d_small", 1)])
def test_epochs_match_oracle(lm, name, epochs):
    c = Case(lm, name)
    o = c.oracle()
    g, pe = c.gpu()
    seq = S.selection_sequence(c.n_sub, 2 * c.n_sub * epochs, seed=3)
    for k in range(epochs):
        s = seq[2 * c.n_sub * k:2 * c.n_sub * (k + 1)]
        g.epoch(s)
        for i in s:
            o.update(int(i))
    err = H.rel_l2(g.x().cpu().numpy(), o.x)
    assert err < H.REL_L2_IMAGE, err
    f_g, f_o = g.objective(), o.objective()
    assert abs(f_g - f_o) <= 1e-5 * abs(f_o)
    # empty bins keep y = 1 (exact in real arithmetic; (a + 1) - sqrt((a - 1)^2) rounds within a few
    # float32 ulps of 2); y of the others matches the oracle's
    b = _canonical_index(c, pe)
    y = g.y().cpu().numpy()
    empty = c.d[b] == 0
    assert empty.any() and np.abs(y[empty] - 1.0).max() <= 1e-6
    assert H.rel_l2(y[~empty], o.y[b[~empty]]) < H.REL_L2_IMAGE


def test_listmode_equals_sinogram_on_gpu(lm):
    """Appendix: with one subset and the same selections, LM-SPDHG on the
    events and SPDHG on their sinogram give the same iterates (float32
    rounding apart)."""
    c = Case(lm, "2d_small", n_subsets=1)
    g_sino, _ = c.gpu()
    pe_lm = lm.event_setup(c.geo_g, lm.DeviceEvents.from_numpy(c.ev), 1)
    # the events' corr and contam equal the sinogram's LOR factor and s
    np.testing.assert_allclose(c.ev.corr, c.lf[S.lor_of_events(c.wl.scanner, c.ev.det1, c.ev.det2)], rtol=1e-6)
    g_lm = lm.LMSPDHG(c.geo_g, pe_lm, torch.from_numpy(c.sens_or.astype(np.float32)).cuda(),
                      torch.from_numpy(c.x0).cuda(), beta=c.wl.beta, n_subsets=1, gamma=c.gamma, rho=0.999,
                      knorm=c.knorm, kahan=True, group=0, projector="direct")
    seq = S.selection_sequence(1, 40, seed=3)
    g_sino.updates(seq)
    g_lm.updates(seq)
    assert H.rel_l2(g_sino.x().cpu().numpy(), g_lm.x().cpu().numpy()) < 1e-4
    assert abs(g_sino.objective() - float(c.s.astype(np.float64).sum()) - g_lm.objective()) <= 1e-5 * abs(
        g_lm.objective())


@pytest.mark.parametrize("name", ["2d_small", "3d_small"])
def test_generated_layout_equals_stored(lm, name):
    """lm_sino_count gives the counts of the stored layout (same order), and a
    state that computes every bin's geometry from its index (sinogram = 2)
    reproduces the stored-list state bit for bit (deterministic mode)."""
    c = Case(lm, name)
    gen = lm.sino_count(c.geo_g, lm.DeviceEvents.from_numpy(c.ev), c.n_sub)
    pe = c.bins()
    np.testing.assert_array_equal(pe.sub_off, gen.sub_off)
    mu_st = pe.mu.view(torch.int16).cpu().numpy().view(np.uint16)
    mu_gen = gen.mu.view(torch.int16).cpu().numpy().view(np.uint16)[:c.NB]
    np.testing.assert_array_equal(mu_gen, mu_st)
    # one lane-group width for both (the width sets the order of each event's forward sum)
    a, _ = c.gpu(pe=pe, deterministic=True, group=32)
    sens = torch.from_numpy(c.sens_or.astype(np.float32)).cuda()
    b = lm.LMSPDHG(c.geo_g, gen, sens, torch.from_numpy(c.x0).cuda(), beta=c.wl.beta, n_subsets=c.n_sub,
                   gamma=c.gamma, rho=0.999, knorm=c.knorm, deterministic=True, kahan=True, group=32,
                   projector="direct", sinogram=2, sino_s=float(c.s[0]), sino_lorf=torch.from_numpy(c.lf).cuda())
    seq = S.selection_sequence(c.n_sub, 4 * c.n_sub, seed=3)
    for k in range(2):
        s = seq[2 * c.n_sub * k:2 * c.n_sub * (k + 1)]
        a.epoch(s)
        b.epoch(s)
    np.testing.assert_array_equal(a.x().cpu().numpy(), b.x().cpu().numpy())
    np.testing.assert_array_equal(a.y().cpu().numpy(), b.y().cpu().numpy()[:c.NB])
    assert a.objective() == b.objective()


def test_count_rejects_invalid_events(lm):
    c = Case(lm, "2d_small", n_events=500)
    ev = lm.DeviceEvents.from_numpy(c.ev)
    ev.det1[7] = c.wl.scanner.n_det + 3
    with pytest.raises(lm.LMError) as ei:
        lm.sino_count(c.geo_g, ev, c.n_sub)
    assert ei.value.code == 2
