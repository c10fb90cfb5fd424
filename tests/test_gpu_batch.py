"""Batched epochs: frames of different sizes advanced together in one graph
give the same results as each frame alone (bit-identical in deterministic
mode, within float32 rounding otherwise), including a frame that joins the
batch while others are in flight and a frame that leaves."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2201_05497_gb300 import synth as S
from tests import _helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lm():
    from paper_2201_05497_gb300 import build, lm as _lm
    build.build()
    _lm.load_library()
    return _lm


def _frames(lm, name, sizes, det):
    wl = S.workload(name)
    geo = lm.Geometry.from_workload(wl)
    lf = torch.from_numpy(S.lor_attenuation(wl.scanner, wl.phantom)).cuda()
    sens = lm.sens(geo, lf)
    out = []
    for k, n in enumerate(sizes):
        ev = S.monte_carlo_events(wl.scanner, wl.phantom, wl.tof, n, seed=100 + k,
                                  lor_att=lf.cpu().numpy())
        dev = lm.DeviceEvents.from_numpy(ev)
        x0 = torch.full((geo.V,), 0.8 * n / float(sens.double().sum()), device="cuda")
        out.append((dev, x0))
    return wl, geo, sens, out


def _state(lm, wl, geo, sens, dev, x0, det, projector="direct"):
    pe = lm.event_setup(geo, dev, wl.n_subsets)
    # a batch runs the projector its frames were created with: compare with the same projector alone
    return lm.LMSPDHG(geo, pe, sens, x0, beta=wl.beta, n_subsets=wl.n_subsets, knorm=H.knorm_closed(wl.grid.n),
                      deterministic=det, group=16, projector=projector)


@pytest.mark.parametrize("name,sizes,projector", [("3d_small", [40000, 7000, 23000], "direct"),
                                                  ("3d_quad", [30000, 9000, 15000], "direct"),
                                                  ("2d_small", [20000, 3000], "direct"),
                                                  ("3d_small", [40000, 7000, 23000], "table"),
                                                  ("3d_quad", [30000, 9000, 15000], "table")])
@pytest.mark.parametrize("det", [True, False])
def test_batch_equals_alone(lm, name, sizes, projector, det):
    if projector == "table" and det:
        pytest.skip("the traversal table serves float-atomic mode")
    wl, geo, sens, frames = _frames(lm, name, sizes, det)
    n = wl.n_subsets
    E = 3
    seqs = [S.selection_sequence(n, 2 * n * E, seed=3 + k) for k in range(len(frames))]
    alone = []
    for k, (dev, x0) in enumerate(frames):
        st = _state(lm, wl, geo, sens, dev, x0, det, projector)
        assert st.tuning()["projector"] == projector
        for e in range(E):
            st.epoch(seqs[k][2 * n * e:2 * n * (e + 1)])
        alone.append((st.x().cpu().numpy(), st.y().cpu().numpy(), st.z().cpu().numpy()))
        st.close()
    b = lm.Batch(4, n)
    states = [_state(lm, wl, geo, sens, dev, x0, det, projector) for dev, x0 in frames]
    # frame 1 joins at epoch 1 (it then runs epochs 0..E-1 of its own sequence), slot 3 stays empty
    for k in range(len(states)):
        if k != 1:
            b.set(k, states[k])
    done = {k: 0 for k in range(len(states))}
    for e in range(E + 1):
        if e == 1:
            b.set(1, states[1])
        active = {k: states_k for k, states_k in enumerate(states)
                  if (k != 1 or e >= 1) and done[k] < E}
        slots = {k: k for k in range(len(states))}
        q = {}
        for k in active:
            q[slots[k]] = seqs[k][2 * n * done[k]:2 * n * (done[k] + 1)]
        b.epoch(q)
        for k in active:
            done[k] += 1
            if done[k] == E:
                b.set(slots[k], None)   # the frame leaves the batch
    for k, st in enumerate(states):
        x, y, z = st.x().cpu().numpy(), st.y().cpu().numpy(), st.z().cpu().numpy()
        if det:
            np.testing.assert_array_equal(x, alone[k][0])
            np.testing.assert_array_equal(y, alone[k][1])
            np.testing.assert_array_equal(z, alone[k][2])
        else:
            assert H.rel_l2(x, alone[k][0]) < H.REL_EVENT
            assert H.rel_l2(z, alone[k][2]) < H.REL_EVENT
    b.close()


def test_batch_outlives_its_first_state(lm):
    """The first state set into a batch leaves, is destroyed and its memory
    overwritten; the batch keeps running the other frames unchanged (it owns
    its configuration and TOF table)."""
    wl, geo, sens, frames = _frames(lm, "3d_quad", [20000, 8000, 12000], True)
    n = wl.n_subsets
    E = 3
    seqs = [S.selection_sequence(n, 2 * n * E, seed=7 + k) for k in range(3)]
    alone = []
    for k in (1, 2):
        dev, x0 = frames[k]
        st = _state(lm, wl, geo, sens, dev, x0, True)
        for e in range(E):
            st.epoch(seqs[k][2 * n * e:2 * n * (e + 1)])
        alone.append(st.x().cpu().numpy())
        st.close()
    b = lm.Batch(3, n)
    states = [_state(lm, wl, geo, sens, dev, x0, True) for dev, x0 in frames]
    for k in range(3):
        b.set(k, states[k])
    b.epoch({k: seqs[k][:2 * n] for k in range(3)})
    b.set(0, None)
    states[0].close()
    states[0].buf.fill_(255)
    torch.cuda.synchronize()
    for e in range(1, E):
        b.epoch({k: seqs[k][2 * n * e:2 * n * (e + 1)] for k in (1, 2)})
    for i, k in enumerate((1, 2)):
        np.testing.assert_array_equal(states[k].x().cpu().numpy(), alone[i])
    b.close()


@pytest.mark.parametrize("mode", ["dtv", "dtv_plain", "sinogram"])
def test_batch_of_prior_and_algorithm_variants(lm, mode):
    """Frames with the directional TV prior, or sinogram SPDHG frames, run in a
    batch give each frame's lone result bit for bit (deterministic mode): the
    batch reads every per-frame option from the frame's own argument tables."""
    wl, geo, sens, frames = _frames(lm, "3d_quad", [12000, 5000], True)
    n = wl.n_subsets
    E = 2
    seqs = [S.selection_sequence(n, 2 * n * E, seed=7 + k) for k in range(len(frames))]
    kw = dict(beta=0.1, n_subsets=n, knorm=H.knorm_closed(wl.grid.n), deterministic=True, group=16,
              projector="direct")
    extra = []
    if mode.startswith("dtv"):
        act = torch.from_numpy(wl.phantom.voxelised(wl.grid, supersample=1)).cuda()
        xi = lm.dtv_field(geo, (act.max() - act).contiguous(), 0.01)
        # TMA-staged passes on this grid unless plain ones are asked for
        kw.update(xi=xi, image_kernel=1 if mode == "dtv_plain" else 0)
        extra.append(xi)

    def make(k):
        dev, x0 = frames[k]
        if mode == "sinogram":
            gen = lm.sino_count(geo, dev, n)
            lf = torch.from_numpy(S.lor_attenuation(wl.scanner, wl.phantom)).cuda()
            extra.append((gen, lf))
            return lm.LMSPDHG(geo, gen, sens, x0, sinogram=2, sino_s=float(dev.contam[0].item()), sino_lorf=lf,
                              image_kernel=1, **kw)
        pe = lm.event_setup(geo, dev, n)
        return lm.LMSPDHG(geo, pe, sens, x0, **kw)

    alone = []
    for k in range(len(frames)):
        st = make(k)
        for e in range(E):
            st.epoch(seqs[k][2 * n * e:2 * n * (e + 1)])
        alone.append(st.x().cpu().numpy())
        st.close()
    states = [make(k) for k in range(len(frames))]
    b = lm.Batch(2, n)
    for k in range(len(frames)):
        b.set(k, states[k])
    for e in range(E):
        b.epoch({k: seqs[k][2 * n * e:2 * n * (e + 1)] for k in range(len(frames))})
    for k in range(len(frames)):
        np.testing.assert_array_equal(states[k].x().cpu().numpy(), alone[k])
    b.close()
