"""Oracle parity of the benchmarked path on the 3D short frame's full grid.

The 3D scanner (36 rings x 672 crystals), the 200 x 200 x 96 image, the
28-subset split and TV beta = 0.03 of the benchmark, with the first 2e6
Monte Carlo events of the frame's generator (the FP64 oracle runs two epochs
of these in about a minute).  The GPU runs the benchmark's own settings:
float mode with the compensated z, the paired accumulators, the TMA-staged
image passes chosen automatically, graph-replayed epochs, and the event
kernel's lane-group width forced to 8, 16 and 32 in turn, with both the
traversal-table data update (the benchmark's) and the direct event kernel.  After two epochs x and z must be within 1e-3 relative L2
of the oracle and the FP64 objectives within 1e-5.

The sensitivity image of the full scanner (P^T 1 over 2.9e8 LORs x 41 TOF
bins) is out of the oracle's reach, so both sides get the same host-made
stand-in: the oracle's FP64 back-projection of ones over the frame's events
plus a small floor, rounded to float32.  Nothing the oracle is given comes
from the GPU.

The precision study of the same frame (float32 with and without the
compensated z, and the deterministic fixed-point back-projection, each
against the FP64 oracle) is printed as one PRECISION_STUDY_3D_SHORT line."""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2201_05497_gb300 import synth as S
from tests import _helpers as H

pytestmark = pytest.mark.gpu

N_EVENTS = 2_000_000
EPOCHS = 2


@pytest.fixture(scope="module")
def lm():
    from paper_2201_05497_gb300 import build, lm as _lm
    build.build()
    _lm.load_library()
    return _lm


class Frame:
    """The first N_EVENTS events of the 3D short frame, on both sides."""

    def __init__(self, lm):
        wl = S.workload("3d_short")
        self.wl, self.lm = wl, lm
        att = S.lor_attenuation_torch(wl.scanner, wl.phantom, device="cuda")
        raw = S.monte_carlo_events_torch(wl.scanner, wl.phantom, wl.tof, N_EVENTS, seed=2, lor_att=att,
                                         device="cuda")
        del att
        self.raw = {k: getattr(raw, k).cpu().numpy() for k in ("det1", "det2", "tof", "corr", "contam")}
        self.n_sub = wl.n_subsets
        self.geo_o = O.Geometry.from_workload(wl)
        self.geo_g = lm.Geometry.from_workload(wl)
        self.E = O.EventArrays(*(self.raw[k] for k in ("det1", "det2", "tof", "corr", "contam")))
        self.mu = O.event_counts(self.E.det1, self.E.det2, self.E.tof)
        bp = O.back(self.geo_o, self.E, np.ones(self.E.n))
        self.sens = (bp + 1e-3 * bp.mean()).astype(np.float32)
        kappa = 0.8 * self.E.n / float(self.sens.astype(np.float64).sum())
        self.x0 = np.full(self.geo_o.V, np.float32(kappa), dtype=np.float32)
        self.gamma = float(np.float32(3.0 / self.x0.max()))
        self.knorm = H.knorm_closed(wl.grid.n)
        self.seq = S.selection_sequence(self.n_sub, 2 * self.n_sub * EPOCHS, seed=3)
        o = O.LM(self.geo_o, self.E, self.mu, self.n_sub, beta=wl.beta, gamma=self.gamma, rho=0.999,
                 knorm=self.knorm)
        o.init(self.x0, self.sens.astype(np.float64))
        o.run(self.seq)
        self.x_or, self.z_or, self.f_or = o.x.copy(), o.z.copy(), o.objective()

    def gpu(self, **kw):
        lm = self.lm
        dev = lm.DeviceEvents(*(torch.from_numpy(self.raw[k]).cuda()
                                for k in ("det1", "det2", "tof", "corr", "contam")))
        pe = lm.event_setup(self.geo_g, dev, self.n_sub)
        g = lm.LMSPDHG(self.geo_g, pe, torch.from_numpy(self.sens).cuda(), torch.from_numpy(self.x0).cuda(),
                       beta=self.wl.beta, n_subsets=self.n_sub, gamma=self.gamma, rho=0.999, knorm=self.knorm,
                       **kw)
        for k in range(EPOCHS):
            g.epoch(self.seq[2 * self.n_sub * k:2 * self.n_sub * (k + 1)])
        return g

    def compare(self, g):
        x, z = g.x().cpu().numpy(), g.z().cpu().numpy()
        f = g.objective()
        return {"x_rel_l2": H.rel_l2(x, self.x_or), "z_rel_l2": H.rel_l2(z, self.z_or),
                "objective_rel_gap": (f - self.f_or) / abs(self.f_or)}


@pytest.fixture(scope="module")
def frame(lm):
    return Frame(lm)


@pytest.mark.parametrize("projector,group", [("table", 8), ("table", 16), ("table", 32), ("direct", 8),
                                             ("direct", 16), ("direct", 32)])
def test_3d_short_grid_two_epochs_match_oracle(frame, projector, group):
    g = frame.gpu(group=group, kahan=True, projector=projector)
    t = g.tuning()
    assert t["group"] == group and t["image_kernel"] == "tma" and t["projector"] == projector, t
    r = frame.compare(g)
    g.close()
    print(f"FULLGRID_PARITY projector={projector} group={group} " + json.dumps(r))
    assert r["x_rel_l2"] < H.REL_L2_IMAGE, r
    assert r["z_rel_l2"] < H.REL_L2_IMAGE, r
    assert abs(r["objective_rel_gap"]) < 1e-5, r


def test_precision_study_3d_short_frame(frame):
    """Float32 projections with the compensated z (the default), without it,
    and with the deterministic back-projection, each against the FP64
    oracle after the same two epochs; the deterministic mode is also
    bit-identical when repeated."""
    res = {}
    runs = {}
    for name, kw in [("fp32+kahan", dict(kahan=True)), ("fp32", dict(kahan=False)),
                     ("fp32+kahan deterministic", dict(kahan=True, deterministic=True))]:
        g = frame.gpu(**kw)
        res[name] = frame.compare(g)
        runs[name] = g.x().cpu().numpy()
        g.close()
    g = frame.gpu(kahan=True, deterministic=True)
    res["fp32+kahan deterministic"]["bit_identical_repeat"] = bool(
        np.array_equal(g.x().cpu().numpy(), runs["fp32+kahan deterministic"]))
    g.close()
    print("PRECISION_STUDY_3D_SHORT " + json.dumps(res))
    for name, r in res.items():
        assert r["x_rel_l2"] < H.REL_L2_IMAGE, (name, r)
        assert r["z_rel_l2"] < H.REL_L2_IMAGE, (name, r)
        assert abs(r["objective_rel_gap"]) < 1e-5, (name, r)
    assert res["fp32+kahan deterministic"]["bit_identical_repeat"]
