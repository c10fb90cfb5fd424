"""Reconstruction server (continuous batching): frames of very different
event counts submitted while others are on the GPU are admitted as slots and
pool memory free up, run together, and each result equals the frame run
alone (bit for bit in deterministic mode, within float32 rounding of the
atomic back-projection otherwise).  Also: admission by device memory,
bounded waits, and a bad frame that fails alone without disturbing the rest."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2201_05497_gb300 import synth as S
from tests import _helpers as H

pytestmark = pytest.mark.gpu

SIZES = [30000, 4000, 60000, 12000, 2000, 45000]
EPOCHS = 2


@pytest.fixture(scope="module")
def lm():
    from paper_2201_05497_gb300 import build, lm as _lm
    build.build()
    _lm.load_library()
    return _lm


@pytest.fixture(scope="module")
def problem(lm):
    wl = S.workload("3d_quad")
    geo = lm.Geometry.from_workload(wl)
    lf_np = S.lor_attenuation(wl.scanner, wl.phantom)
    sens = lm.sens(geo, torch.from_numpy(lf_np).cuda())
    ssum = float(sens.double().sum())
    frames = []
    for k, n in enumerate(SIZES):
        # dynamic frames of one study: the inner activity varies with the seed; the attenuating
        # cylinder (and so P^T 1) is the same for every frame
        ph = S.Phantom.seeded(100 + k, (80.0, 60.0, 18.0), (80.0, 60.0), 4)
        ev = S.monte_carlo_events(wl.scanner, ph, wl.tof, n, seed=100 + k, lor_att=lf_np)
        seqs = S.selection_sequence(wl.n_subsets, 2 * wl.n_subsets * EPOCHS, seed=3 + k)
        frames.append((ev, np.float32(0.8 * n / ssum), np.asarray(seqs, dtype=np.uint16).reshape(EPOCHS, -1)))
    return wl, geo, sens, frames


def _alone(lm, wl, geo, sens, ev, x0v, seqs, det):
    pe = lm.event_setup(geo, lm.DeviceEvents.from_numpy(ev), wl.n_subsets)
    x0 = torch.full((geo.V,), float(x0v), dtype=torch.float32, device="cuda")
    # the server's frames keep traversal tables where they apply (3D TOF, float mode) and run 32 lanes
    # per event: compare with the same projector alone
    st = lm.LMSPDHG(geo, pe, sens, x0, beta=wl.beta, n_subsets=wl.n_subsets, knorm=H.knorm_closed(wl.grid.n),
                    deterministic=det, kahan=True, group=32, projector="auto")
    for e in range(seqs.shape[0]):
        st.epoch(seqs[e])
    out = st.x().cpu().numpy(), st.objective()
    st.close()
    return out


def _server(lm, wl, geo, sens, det, max_slots=4, pool_frames=None, max_events=max(SIZES)):
    fb = lm.Server.frame_bytes(geo, max_events, wl.n_subsets, det)
    L = lm.load_library()
    head = int(L.lm_setup_workspace_bytes(max_events)) + int(L.lmspdhg_batch_bytes(max_slots, wl.n_subsets))
    pool = head + 4096 + int((pool_frames if pool_frames is not None else max_slots + 1) * fb)
    return lm.Server(geo, sens, beta=wl.beta, knorm=H.knorm_closed(wl.grid.n), n_subsets=wl.n_subsets,
                     epochs=EPOCHS, max_slots=max_slots, max_events=max_events, pool_bytes=pool,
                     deterministic=det, kahan=True, group=32)


def _submit(srv, frame):
    ev, x0v, seqs = frame
    return srv.submit(ev.det1, ev.det2, ev.tof, ev.corr, ev.contam, x0v, seqs)


@pytest.mark.parametrize("det", [True, False])
def test_server_mix_equals_alone(lm, problem, det):
    wl, geo, sens, frames = problem
    alone = [_alone(lm, wl, geo, sens, ev, x0v, seqs, det) for ev, x0v, seqs in frames]
    srv = _server(lm, wl, geo, sens, det)
    # three frames first; the rest arrive while those are on the GPU
    tickets = [_submit(srv, f) for f in frames[:3]]
    max_inflight = 0
    t0 = time.time()
    while srv.stats()["in_flight"] == 0 and time.time() - t0 < 30:
        time.sleep(0.001)
    tickets += [_submit(srv, f) for f in frames[3:]]
    results = {}
    while len(results) < len(tickets) and time.time() - t0 < 120:
        max_inflight = max(max_inflight, srv.stats()["in_flight"])
        for k, t in enumerate(tickets):
            if k in results:
                continue
            try:
                results[k] = srv.wait(t, timeout_ms=1)
            except lm.LMError as e:
                assert e.code == 5, e  # LM_ERR_TIMEOUT: not finished yet
    max_inflight = srv.stats()["max_in_flight"]
    srv.close()
    assert len(results) == len(frames)
    assert max_inflight >= 2, "frames never overlapped on the GPU"
    for k, (x, obj, lat) in results.items():
        assert lat > 0.0
        if det:
            np.testing.assert_array_equal(x, alone[k][0])
            assert obj == alone[k][1]
        else:
            assert H.rel_l2(x, alone[k][0]) < H.REL_EVENT
            assert abs(obj - alone[k][1]) <= 1e-5 * abs(alone[k][1])


def test_server_admits_by_memory(lm, problem):
    """A pool with room for one largest frame runs frames one at a time even
    with free slots; every frame still completes and matches."""
    wl, geo, sens, frames = problem
    big = [f for f in frames if f[0].n >= 30000][:3]
    srv = _server(lm, wl, geo, sens, True, max_slots=4, pool_frames=1.5, max_events=max(SIZES))
    tickets = [_submit(srv, f) for f in big]
    seen = 0
    done = 0
    t0 = time.time()
    while done < len(tickets) and time.time() - t0 < 120:
        st = srv.stats()
        seen = max(seen, st["in_flight"])
        done = st["completed"]
        time.sleep(0.0005)
    outs = [srv.wait(t, timeout_ms=60000) for t in tickets]
    seen = max(seen, srv.stats()["max_in_flight"])
    srv.close()
    assert seen == 1
    ev, x0v, seqs = big[0]
    x_alone, obj_alone = _alone(lm, wl, geo, sens, ev, x0v, seqs, True)
    np.testing.assert_array_equal(outs[0][0], x_alone)


def test_server_errors_are_per_frame(lm, problem):
    wl, geo, sens, frames = problem
    srv = _server(lm, wl, geo, sens, True, max_slots=1)
    ev, x0v, seqs = frames[1]
    # oversize frame: refused at submit
    with pytest.raises(lm.LMError) as ei:
        big = np.zeros(max(SIZES) + 1, dtype=np.int32)
        srv.submit(big, big + 1, np.zeros_like(big, dtype=np.int16), None, np.ones(big.size, np.float32), x0v, seqs)
    assert ei.value.code == 6
    # x0 must be positive
    with pytest.raises(lm.LMError) as ei:
        _submit(srv, (ev, np.float32(0.0), seqs))
    assert ei.value.code == 3
    # one slot: the largest frame occupies it for two epochs; the others queue behind it
    t_big = _submit(srv, frames[2])
    bad_det = ev.det1.copy()
    bad_det[17] = wl.scanner.n_det + 5
    t_bad = srv.submit(bad_det, ev.det2, ev.tof, ev.corr, ev.contam, x0v, seqs)
    t_good = _submit(srv, frames[1])
    # a wait that runs out reports LM_ERR_TIMEOUT and leaves the ticket valid
    # (unless the frame already finished, which a zero timeout cannot exclude)
    try:
        got = srv.wait(t_good, timeout_ms=0)
    except lm.LMError as e:
        assert e.code == 5
        got = None
    # the frame with a detector index out of range fails on its own
    with pytest.raises(lm.LMError) as ei:
        srv.wait(t_bad, timeout_ms=60000)
    assert ei.value.code == 2
    x, obj, lat = got if got is not None else srv.wait(t_good, timeout_ms=60000)
    xb, objb, latb = srv.wait(t_big, timeout_ms=60000)
    srv.close()
    assert latb < lat, (latb, lat)
    np.testing.assert_array_equal(x, _alone(lm, wl, geo, sens, ev, x0v, seqs, True)[0])
    e2, x02, s2 = frames[2]
    np.testing.assert_array_equal(xb, _alone(lm, wl, geo, sens, e2, x02, s2, True)[0])


def test_server_pool_too_small(lm, problem):
    wl, geo, sens, frames = problem
    with pytest.raises(lm.LMError) as ei:
        lm.Server(geo, sens, beta=wl.beta, knorm=H.knorm_closed(wl.grid.n), n_subsets=wl.n_subsets,
                  epochs=EPOCHS, max_slots=2, max_events=100000, pool_bytes=1 << 20)
    assert ei.value.code == 6
