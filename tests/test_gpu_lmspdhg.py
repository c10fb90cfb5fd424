"""GPU parity of LM-SPDHG (Alg. 2) against the FP64 oracle: the
initialisation (Eq. yinit, z init, step sizes), single updates of both kinds,
whole epochs (graph-replayed), the FP64 objective, and the deterministic
mode's bit-reproducibility."""
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


class Case:
    """One seeded problem prepared for both sides."""

    def __init__(self, lm, name, n_events=None, n_subsets=None, beta=None):
        wl, lf, ev = H.workload_data(name, n_events)
        self.wl, self.lf, self.ev = wl, lf, ev
        self.n_sub = wl.n_subsets if n_subsets is None else n_subsets
        self.beta = wl.beta if beta is None else beta
        self.geo_o = O.Geometry.from_workload(wl)
        self.geo_g = lm.Geometry.from_workload(wl)
        self.E = O.EventArrays.from_events(ev)
        self.sens_or = O.sens(self.geo_o, lf)
        self.mu = O.event_counts(ev.det1, ev.det2, ev.tof)
        kappa = 0.8 * ev.n / self.sens_or.sum()
        self.x0 = np.full(self.geo_o.V, np.float32(kappa), dtype=np.float32)
        self.knorm = H.knorm_closed(wl.grid.n)
        self.gamma = float(np.float32(3.0 / self.x0.max()))
        perm = O.subset_permutation(ev.n, self.n_sub)
        self.perm = perm
        self.lm = lm

    def oracle(self):
        o = O.LM(self.geo_o, self.E, self.mu, self.n_sub, beta=self.beta, gamma=self.gamma, rho=0.999,
                 knorm=self.knorm)
        o.init(self.x0, self.sens_or)
        return o

    def gpu(self, deterministic=False, kahan=True, sens=None, image_kernel=0, group=0, projector="auto"):
        lm = self.lm
        pe = lm.event_setup(self.geo_g, lm.DeviceEvents.from_numpy(self.ev), self.n_sub)
        if sens is None:
            sens = torch.from_numpy(self.sens_or.astype(np.float32)).cuda()
        return lm.LMSPDHG(self.geo_g, pe, sens, torch.from_numpy(self.x0).cuda(), beta=self.beta,
                          n_subsets=self.n_sub, gamma=self.gamma, rho=0.999, knorm=self.knorm,
                          deterministic=deterministic, kahan=kahan, image_kernel=image_kernel, group=group,
                          projector=projector)


@pytest.mark.parametrize("name", ["2d_small", "3d_small"])
@pytest.mark.parametrize("det", [False, True])
def test_init_matches_oracle(lm, name, det):
    c = Case(lm, name)
    o = c.oracle()
    g = c.gpu(deterministic=det)
    y = g.y().cpu().numpy()
    np.testing.assert_allclose(y[c.perm], o.y, rtol=2e-5, atol=2e-5 * np.abs(o.y).max())
    assert H.rel_l2(g.z().cpu().numpy(), o.z) < 1e-5
    assert H.rel_l2(g.x().cpu().numpy(), o.x) == 0.0  # x0 itself before any update
    info = g.info()
    assert info["n_updates"] == 0 and abs(info["gamma"] - c.gamma) < 1e-7 * c.gamma


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
    # w = proj(w + S Kx): differences of neighbouring float32 x values cancel,
    # so w carries the image tolerance rather than the per-event one
    assert H.rel_l2(g.w().cpu().numpy(), o.w) < H.REL_L2_IMAGE
    np.testing.assert_allclose(g.y().cpu().numpy()[c.perm], o.y, rtol=1e-4, atol=1e-4 * np.abs(o.y).max())


@pytest.mark.parametrize("name,epochs", [("2d_small", 3), ("3d_small", 2), ("3d_mid", 2), ("3d_quad", 2)])
def test_epochs_match_oracle(lm, name, epochs):
    """Images after N epochs within 1e-3 relative L2 of the FP64 oracle;
    epochs are replayed from the captured CUDA graph."""
    c = Case(lm, name)
    o = c.oracle()
    g = c.gpu()
    seq = S.selection_sequence(c.n_sub, 2 * c.n_sub * epochs, seed=3)
    for k in range(epochs):
        s = seq[2 * c.n_sub * k:2 * c.n_sub * (k + 1)]
        g.epoch(s)
        o.run(s)
    err = H.rel_l2(g.x().cpu().numpy(), o.x)
    assert err < H.REL_L2_IMAGE, err
    assert H.rel_l2(g.z().cpu().numpy(), o.z) < H.REL_L2_IMAGE
    f_g, f_o = g.objective(), o.objective()
    assert abs(f_g - f_o) <= 1e-5 * abs(f_o)


def test_2d_full_config_epochs(lm):
    """The 2D configuration (256 crystals, 128^2 image, 2e5 events, 28
    subsets, beta 0.03) for 3 epochs."""
    c = Case(lm, "2d")
    o = c.oracle()
    g = c.gpu()
    seq = S.selection_sequence(c.n_sub, 2 * c.n_sub * 3, seed=3)
    for k in range(3):
        s = seq[2 * c.n_sub * k:2 * c.n_sub * (k + 1)]
        g.epoch(s)
        o.run(s)
    assert H.rel_l2(g.x().cpu().numpy(), o.x) < H.REL_L2_IMAGE


def test_graph_and_direct_paths_agree_deterministic(lm):
    """In deterministic mode the graph-replayed epoch, the directly launched
    updates and a second run are bit-identical."""
    c = Case(lm, "3d_small")
    seq = S.selection_sequence(c.n_sub, 4 * c.n_sub, seed=3)
    a = c.gpu(deterministic=True)
    a.epoch(seq[:2 * c.n_sub])
    a.epoch(seq[2 * c.n_sub:])
    b = c.gpu(deterministic=True)
    b.updates(seq[:5])
    b.updates(seq[5:])
    xa, xb = a.x().cpu().numpy(), b.x().cpu().numpy()
    np.testing.assert_array_equal(xa, xb)
    np.testing.assert_array_equal(a.y().cpu().numpy(), b.y().cpu().numpy())
    np.testing.assert_array_equal(a.z().cpu().numpy(), b.z().cpu().numpy())
    c2 = c.gpu(deterministic=True)
    c2.epoch(seq[:2 * c.n_sub])
    c2.epoch(seq[2 * c.n_sub:])
    np.testing.assert_array_equal(xa, c2.x().cpu().numpy())


def test_deterministic_and_atomic_modes_agree(lm):
    c = Case(lm, "2d_small")
    seq = S.selection_sequence(c.n_sub, 4 * c.n_sub, seed=5)
    a = c.gpu(deterministic=True)
    b = c.gpu(deterministic=False)
    a.updates(seq)
    b.updates(seq)
    assert H.rel_l2(a.x().cpu().numpy(), b.x().cpu().numpy()) < 1e-5


def test_kahan_off_runs_and_agrees(lm):
    c = Case(lm, "2d_small")
    o = c.oracle()
    g = c.gpu(kahan=False)
    seq = S.selection_sequence(c.n_sub, 2 * c.n_sub, seed=3)
    g.epoch(seq)
    o.run(seq)
    assert H.rel_l2(g.x().cpu().numpy(), o.x) < H.REL_L2_IMAGE


def test_gpu_sens_drives_iteration(lm):
    """End to end on the device: sensitivity from lm_sens, then epochs."""
    c = Case(lm, "3d_small")
    sens = lm.sens(c.geo_g, torch.from_numpy(c.lf).cuda())
    g = c.gpu(sens=sens)
    o = c.oracle()
    seq = S.selection_sequence(c.n_sub, 2 * c.n_sub, seed=3)
    g.epoch(seq)
    o.run(seq)
    assert H.rel_l2(g.x().cpu().numpy(), o.x) < H.REL_L2_IMAGE


def test_knorm_and_gamma_resolved_on_device(lm):
    c = Case(lm, "3d_small")
    pe = lm.event_setup(c.geo_g, lm.DeviceEvents.from_numpy(c.ev), c.n_sub)
    g = lm.LMSPDHG(c.geo_g, pe, torch.from_numpy(c.sens_or.astype(np.float32)).cuda(),
                   torch.from_numpy(c.x0).cuda(), beta=c.beta, n_subsets=c.n_sub, knorm_iters=500)
    info = g.info()
    assert abs(info["gamma"] - 3.0 / float(c.x0.max())) < 1e-6 * info["gamma"]
    kn = H.knorm_closed(c.wl.grid.n)
    assert info["knorm"] <= kn and info["knorm"] > 0.99 * kn


def test_x0_negative_rejected(lm):
    c = Case(lm, "2d_small")
    pe = lm.event_setup(c.geo_g, lm.DeviceEvents.from_numpy(c.ev), c.n_sub)
    x0 = torch.from_numpy(c.x0).cuda()
    x0[17] = -1.0
    with pytest.raises(lm.LMError) as ei:
        lm.LMSPDHG(c.geo_g, pe, torch.from_numpy(c.sens_or.astype(np.float32)).cuda(), x0, beta=0.03,
                   n_subsets=c.n_sub)
    assert ei.value.code == 3


@pytest.mark.parametrize("name", ["3d_quad", "2d"])
@pytest.mark.parametrize("kahan", [True, False])
def test_tma_and_plain_image_passes_agree(lm, name, kahan):
    """The TMA-staged image pass (prior dual step fused in), TMA-staged data
    passes with plain prior passes, and the plain-load pass compute the same
    operations in the same order: in deterministic mode x, z, w and y agree
    bit for bit after two epochs."""
    c = Case(lm, name, n_events=30000 if name == "2d" else None)
    seq = S.selection_sequence(c.n_sub, 4 * c.n_sub, seed=5)
    out = {}
    for kind in (1, 2, 3):
        g = c.gpu(deterministic=True, kahan=kahan, image_kernel=kind, group=16)
        assert g.tuning()["image_kernel"] == {1: "plain", 2: "tma", 3: "tma_data"}[kind]
        g.epoch(seq[:2 * c.n_sub])
        g.epoch(seq[2 * c.n_sub:])
        out[kind] = [a.cpu().numpy() for a in (g.x(), g.z(), g.w(), g.y())]
        g.close()
    for kind in (2, 3):
        for a, b in zip(out[1], out[kind]):
            np.testing.assert_array_equal(a, b)


def test_image_kernel_choice(lm):
    assert Case(lm, "3d_quad").gpu().tuning()["image_kernel"] == "tma"
    assert Case(lm, "3d_small").gpu().tuning()["image_kernel"] == "plain"
    for kind in (2, 3, 4):
        with pytest.raises(lm.LMError):
            Case(lm, "3d_small").gpu(image_kernel=kind)


@pytest.mark.parametrize("name", ["2d_small", "3d_small", "3d_quad", "3d_mid"])
def test_tiled_projector_matches_direct_and_oracle(lm, name):
    """The tile-binned projector (per-frame segments per 32x32x8 tile, shared
    memory gathers and scatters) computes the direct kernel's per-sample
    terms in another order: its iterates agree with the direct kernel's to
    float32 rounding and with the oracle to the image tolerance; every
    sample of every event lands in exactly one segment."""
    c = Case(lm, name)
    seq = S.selection_sequence(c.n_sub, 4 * c.n_sub, seed=9)
    out = {}
    for proj in ("direct", "tiled"):
        g = c.gpu(projector=proj, group=16)
        t = g.tuning()
        assert t["projector"] == proj
        if proj == "tiled":
            assert c.ev.n <= t["tile_segments"] <= 6 * c.ev.n
        g.epoch(seq[:2 * c.n_sub])
        g.epoch(seq[2 * c.n_sub:])
        out[proj] = (g.x().cpu().numpy(), g.y().cpu().numpy(), g.z().cpu().numpy(), g.objective())
        g.close()
    assert H.rel_l2(out["tiled"][0], out["direct"][0]) < 1e-5
    assert H.rel_l2(out["tiled"][1], out["direct"][1]) < 1e-5
    assert H.rel_l2(out["tiled"][2], out["direct"][2]) < 1e-5
    o = c.oracle()
    o.run(seq[:2 * c.n_sub])
    o.run(seq[2 * c.n_sub:])
    assert H.rel_l2(out["tiled"][0], o.x) < H.REL_L2_IMAGE
    assert abs(out["tiled"][3] - o.objective()) <= 1e-5 * abs(o.objective())


def test_tiled_projector_reinit_rebins(lm):
    """reinit with another frame's events in the same buffers bins them anew."""
    c = Case(lm, "3d_quad")
    g = c.gpu(projector="tiled", group=16)
    pe2 = lm.event_setup(c.geo_g, lm.DeviceEvents.from_numpy(H.workload_data("3d_quad", seed=5)[2]), c.n_sub,
                         into=g.pe)
    g.reinit(torch.from_numpy(c.x0).cuda())
    seq = S.selection_sequence(c.n_sub, 2 * c.n_sub, seed=2)
    g.epoch(seq)
    x_t = g.x().cpu().numpy()
    g.close()
    h = lm.LMSPDHG(c.geo_g, pe2, torch.from_numpy(c.sens_or.astype(np.float32)).cuda(),
                   torch.from_numpy(c.x0).cuda(), beta=c.beta, n_subsets=c.n_sub, gamma=c.gamma, rho=0.999,
                   knorm=c.knorm, projector="direct", group=16)
    h.epoch(seq)
    assert H.rel_l2(x_t, h.x().cpu().numpy()) < 1e-5


@pytest.mark.parametrize("name", ["3d_small", "3d_quad", "3d_mid"])
@pytest.mark.parametrize("group", [8, 16, 32])
def test_table_projector_matches_direct_and_oracle(lm, name, group):
    """The traversal-table data update (stored traversals and (P^LM 1)_e,
    quad gathers, x-principal events before the others) evaluates the direct
    kernel's per-sample terms in the same order: after two epochs its
    iterates agree with the direct kernel's to float32 rounding ((P^LM 1)_e
    is summed in another order and the atomics' order differs) and with the
    oracle to the image tolerance."""
    c = Case(lm, name)
    seq = S.selection_sequence(c.n_sub, 4 * c.n_sub, seed=9)
    out = {}
    for proj in ("direct", "table"):
        g = c.gpu(projector=proj, group=group)
        assert g.tuning()["projector"] == proj and g.tuning()["group"] == group
        g.epoch(seq[:2 * c.n_sub])
        g.epoch(seq[2 * c.n_sub:])
        out[proj] = (g.x().cpu().numpy(), g.y().cpu().numpy(), g.z().cpu().numpy(), g.objective())
        g.close()
    for k in range(3):
        assert H.rel_l2(out["table"][k], out["direct"][k]) < 1e-5, k
    o = c.oracle()
    o.run(seq[:2 * c.n_sub])
    o.run(seq[2 * c.n_sub:])
    assert H.rel_l2(out["table"][0], o.x) < H.REL_L2_IMAGE
    assert H.rel_l2(out["table"][2], o.z) < H.REL_L2_IMAGE
    np.testing.assert_allclose(out["table"][1][c.perm], o.y, rtol=1e-3, atol=1e-3 * np.abs(o.y).max())
    assert abs(out["table"][3] - o.objective()) <= 1e-5 * abs(o.objective())


def test_table_single_data_update_matches_direct(lm):
    """One data update: the duals of every event agree with the direct
    kernel's to a few float32 ulps (same forward projections, S_e from a
    differently ordered (P^LM 1)_e)."""
    c = Case(lm, "3d_mid")
    ys = []
    for proj in ("direct", "table"):
        g = c.gpu(projector=proj, group=32)
        g.updates([1])
        ys.append(g.y().cpu().numpy())
        g.close()
    np.testing.assert_allclose(ys[1], ys[0], rtol=4e-6, atol=4e-6 * np.abs(ys[0]).max())


def test_table_reinit_rebuilds(lm):
    """reinit with another frame's events in the same buffers stores their
    traversals anew."""
    c = Case(lm, "3d_quad")
    g = c.gpu(projector="table", group=32)
    pe2 = lm.event_setup(c.geo_g, lm.DeviceEvents.from_numpy(H.workload_data("3d_quad", seed=5)[2]), c.n_sub,
                         into=g.pe)
    g.reinit(torch.from_numpy(c.x0).cuda())
    seq = S.selection_sequence(c.n_sub, 2 * c.n_sub, seed=2)
    g.epoch(seq)
    x_t = g.x().cpu().numpy()
    g.close()
    h = lm.LMSPDHG(c.geo_g, pe2, torch.from_numpy(c.sens_or.astype(np.float32)).cuda(),
                   torch.from_numpy(c.x0).cuda(), beta=c.beta, n_subsets=c.n_sub, gamma=c.gamma, rho=0.999,
                   knorm=c.knorm, projector="direct", group=32)
    h.epoch(seq)
    assert H.rel_l2(x_t, h.x().cpu().numpy()) < 1e-5


def test_table_autotuner_picks_width_and_projector(lm):
    """With the table allowed ("auto") and the width left to the autotuner,
    the state times the table's variants and the direct kernel's widths on
    subset 0 and keeps the faster projector; asked for the table, it keeps
    the table without timing the direct kernel."""
    g = Case(lm, "3d_mid").gpu(projector="auto")
    t = g.tuning()
    assert t["group"] in (8, 16, 32)
    assert min(t["ms_g8"], t["ms_g16"], t["ms_g32"]) > 0.0
    assert t["data_update_ms_table"] > 0.0 and t["data_update_ms_direct"] > 0.0
    faster = "table" if t["data_update_ms_table"] <= t["data_update_ms_direct"] else "direct"
    assert t["projector"] == faster
    g.close()
    g = Case(lm, "3d_mid").gpu(projector="table")
    t = g.tuning()
    assert t["projector"] == "table" and t["group"] in (8, 16, 32)
    assert t["data_update_ms_table"] > 0.0 and t["data_update_ms_direct"] == 0.0
    g.close()
