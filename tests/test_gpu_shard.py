"""Event sharding of one frame (lm_params.shard) on one GPU: two states each
hold one half of every subset's events (event counts taken over the whole
list), the exchange of their partial back-projections is a device add in
place of the all-reduce a multi-GPU run would use, and the iterates must
equal those of one state holding all the events (the data term of Alg. 2 is
a sum over events; the dual step of an event needs only its projection)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2201_05497_gb300 import synth as S
from tests import _helpers as H
from tests.test_gpu_lmspdhg import Case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lm():
    from paper_2201_05497_gb300 import build, lm as _lm
    build.build()
    _lm.load_library()
    return _lm


def _halves(lm, c):
    """The whole list's event set-up, then two states' slices: the first
    and second half of every subset."""
    pe = lm.event_setup(c.geo_g, lm.DeviceEvents.from_numpy(c.ev), c.n_sub)
    off = np.asarray(pe.sub_off, dtype=np.int64)
    parts = []
    for h in range(2):
        idx = np.concatenate([np.arange(off[k] + (off[k + 1] - off[k]) // 2 * h,
                                        off[k + 1] if h else off[k] + (off[k + 1] - off[k]) // 2)
                              for k in range(c.n_sub)])
        sizes = [(off[k + 1] - off[k]) - (off[k + 1] - off[k]) // 2 if h else (off[k + 1] - off[k]) // 2
                 for k in range(c.n_sub)]
        it = torch.from_numpy(idx).cuda()
        ev = lm.DeviceEvents(*(getattr(pe.events, f)[it].contiguous() for f in ("det1", "det2", "tof", "corr",
                                                                                 "contam")))
        # uint16 has no CUDA gather in every torch release: gather the same bits as int16
        mu = pe.mu.view(torch.int16)[it].contiguous().view(pe.mu.dtype)
        sub_off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        parts.append((lm.PermutedEvents(ev, mu, sub_off), idx))
    return pe, parts


def _state(lm, c, pe, **kw):
    return lm.LMSPDHG(c.geo_g, pe, torch.from_numpy(c.sens_or.astype(np.float32)).cuda(),
                      torch.from_numpy(c.x0).cuda(), beta=c.beta, n_subsets=c.n_sub, gamma=c.gamma, rho=0.999,
                      knorm=c.knorm, group=32, **kw)


def _exchange(states):
    bufs = [s.shard_buffer() for s in states]
    total = bufs[0] + bufs[1]
    for b in bufs:
        b.copy_(total)


@pytest.mark.parametrize("name,projector", [("3d_mid", "table"), ("3d_quad", "direct"), ("2d_small", "direct")])
def test_two_shards_equal_one_state(lm, name, projector):
    c = Case(lm, name)
    pe, parts = _halves(lm, c)
    whole = _state(lm, c, pe, projector=projector)
    shards = [_state(lm, c, p, projector=projector, shard=True) for p, _ in parts]
    _exchange(shards)
    for s in shards:
        s.shard_init_finish()
    seq = S.selection_sequence(c.n_sub, 4 * c.n_sub, seed=9)
    whole.updates(seq)
    for sel in seq:
        for s in shards:
            s.shard_begin(int(sel))
        if sel < c.n_sub:
            _exchange(shards)
        for s in shards:
            s.shard_finish()
    xw, zw, yw = whole.x().cpu().numpy(), whole.z().cpu().numpy(), whole.y().cpu().numpy()
    for s, (_, idx) in zip(shards, parts):
        assert H.rel_l2(s.x().cpu().numpy(), xw) < 1e-5
        assert H.rel_l2(s.z().cpu().numpy(), zw) < 1e-5
        np.testing.assert_allclose(s.y().cpu().numpy(), yw[idx], rtol=1e-4, atol=1e-4 * np.abs(yw).max())
    # the objective: image parts from any state, the event sums added over the states
    pa, pb = shards[0].objective_parts(), shards[1].objective_parts()
    f_sh = pa[0] - (pa[2] + pb[2]) + c.beta * pa[1]
    assert abs(f_sh - whole.objective()) <= 1e-6 * abs(whole.objective())
    # and the sharded run is Alg. 2: against the FP64 oracle
    o = c.oracle()
    o.run(seq)
    assert H.rel_l2(shards[0].x().cpu().numpy(), o.x) < H.REL_L2_IMAGE


def test_shard_protocol_is_enforced(lm):
    c = Case(lm, "3d_small")
    pe, parts = _halves(lm, c)
    s = _state(lm, c, parts[0][0], shard=True)
    with pytest.raises(lm.LMError):
        s.epoch(S.selection_sequence(c.n_sub, 2 * c.n_sub, seed=1))
    with pytest.raises(lm.LMError):
        s.shard_begin(0)  # the initialisation's exchange is pending
    s.shard_init_finish()
    with pytest.raises(lm.LMError):
        s.shard_finish()  # no update begun
    s.shard_begin(c.n_sub)
    with pytest.raises(lm.LMError):
        s.objective_parts()
    s.shard_finish()
    with pytest.raises(lm.LMError):
        _state(lm, c, parts[0][0], shard=True, deterministic=True)
