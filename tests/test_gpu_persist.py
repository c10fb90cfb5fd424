"""The persistent epoch kernel (one cooperative launch per epoch, grid-wide
barriers with bounded waits) against the captured graph of per-update
launches and against the FP64 oracle, on 2D frames; and a barrier wait that
runs out: a gate flag that nothing sets makes the kernel give up, the host
reads LM_ERR_TIMEOUT, and the state works again after lmspdhg_reinit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2201_05497_gb300 import synth as S
from tests import _helpers as H
from tests.test_gpu_lmspdhg import Case

pytestmark = pytest.mark.gpu

LM_ERR_TIMEOUT = 5


@pytest.fixture(scope="module")
def lm():
    from paper_2201_05497_gb300 import build, lm as _lm
    build.build()
    _lm.load_library()
    return _lm


def _state(lm, c, epoch_kernel, group=16):
    pe = lm.event_setup(c.geo_g, lm.DeviceEvents.from_numpy(c.ev), c.n_sub)
    return lm.LMSPDHG(c.geo_g, pe, torch.from_numpy(c.sens_or.astype(np.float32)).cuda(),
                      torch.from_numpy(c.x0).cuda(), beta=c.beta, n_subsets=c.n_sub, gamma=c.gamma, rho=0.999,
                      knorm=c.knorm, group=group, epoch_kernel=epoch_kernel)


@pytest.mark.parametrize("name,epochs", [("2d_small", 3), ("2d", 3)])
@pytest.mark.parametrize("group", [16, 32])
def test_persistent_epochs_match_graph_and_oracle(lm, name, epochs, group):
    c = Case(lm, name)
    seq = S.selection_sequence(c.n_sub, 2 * c.n_sub * epochs, seed=3)
    out = {}
    for kind in (1, 2):
        g = _state(lm, c, kind, group)
        assert g.tuning()["epoch_kernel"] == {1: "graph", 2: "persistent"}[kind]
        for k in range(epochs):
            g.epoch(seq[2 * c.n_sub * k:2 * c.n_sub * (k + 1)])
        out[kind] = (g.x().cpu().numpy(), g.z().cpu().numpy(), g.y().cpu().numpy(), g.objective())
        g.close()
    for k in range(3):
        assert H.rel_l2(out[2][k], out[1][k]) < 1e-5, k
    o = c.oracle()
    o.run(seq)
    assert H.rel_l2(out[2][0], o.x) < H.REL_L2_IMAGE
    assert abs(out[2][3] - o.objective()) <= 1e-5 * abs(o.objective())


def test_epoch_kernel_choice(lm):
    """Auto keeps the graph (faster on the 2D frame); the persistent kernel
    is taken when asked for and refused where it does not apply."""
    c = Case(lm, "2d_small")
    assert _state(lm, c, 0).tuning()["epoch_kernel"] == "graph"
    assert _state(lm, c, 2).tuning()["epoch_kernel"] == "persistent"
    h = Case(lm, "3d_small")
    g3 = lm.LMSPDHG(h.geo_g, lm.event_setup(h.geo_g, lm.DeviceEvents.from_numpy(h.ev), h.n_sub),
                    torch.from_numpy(h.sens_or.astype(np.float32)).cuda(), torch.from_numpy(h.x0).cuda(),
                    beta=h.beta, n_subsets=h.n_sub, gamma=h.gamma, knorm=h.knorm)
    assert g3.tuning()["epoch_kernel"] == "graph"
    with pytest.raises(lm.LMError):
        lm.LMSPDHG(h.geo_g, lm.event_setup(h.geo_g, lm.DeviceEvents.from_numpy(h.ev), h.n_sub),
                   torch.from_numpy(h.sens_or.astype(np.float32)).cuda(), torch.from_numpy(h.x0).cuda(),
                   beta=h.beta, n_subsets=h.n_sub, gamma=h.gamma, knorm=h.knorm, epoch_kernel=2)


def test_barrier_wait_runs_out(lm):
    c = Case(lm, "2d_small")
    g = _state(lm, c, 2)
    seq = S.selection_sequence(c.n_sub, 2 * c.n_sub, seed=3)
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")  # nothing ever sets it
    g.set_gate(flag)
    g.epoch(seq)
    with pytest.raises(lm.LMError) as e:
        g.objective()
    assert e.value.code == LM_ERR_TIMEOUT
    # the context is usable: without the gate a fresh start runs to the oracle's result
    g.set_gate(None)
    g.reinit(torch.from_numpy(c.x0).cuda())
    g.epoch(seq)
    f = g.objective()
    o = c.oracle()
    o.run(seq)
    assert H.rel_l2(g.x().cpu().numpy(), o.x) < H.REL_L2_IMAGE
    assert abs(f - o.objective()) <= 1e-5 * abs(o.objective())
    # a gate that is set lets the epoch through
    flag.fill_(1)
    g.set_gate(flag)
    g.epoch(seq)
    g.objective()
