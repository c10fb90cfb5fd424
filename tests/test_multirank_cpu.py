"""World-size-2 gloo tests (CPU) of the multi-rank logic: the benchmark's
independent replicas (whole-job value = all ranks' events / slowest rank's
time; only rank 0 prints), and the decomposition behind event sharding of
one frame (partial back-projections summed by an all-reduce) and the
binding's exchange protocol for shard states."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    events = 1000.0 * (rank + 1)
    seconds = 2.0 + rank
    v, t, ev = bench.aggregate(world, rank, events, seconds)
    q.put((rank, v, t, ev))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, v, t, ev in res:
        assert t == 3.0            # slowest rank
        assert ev == 3000.0        # all ranks' events
        assert abs(v - 1000.0) < 1e-12


def _data_update_dz(O, geo, E, mu, x32, y, idx, gamma_rho, ones):
    """Partial dz of one data update over the events idx (oracle primitives):
    S_e = gamma rho / (P^LM 1)_e, y+ = prox_{D*}(y + S_e (P^LM x + s), mu S_e),
    dz = (P^LM)^T ((y+ - y) / mu)."""
    Es = O.EventArrays(E.det1[idx], E.det2[idx], E.tof[idx], E.corr[idx], E.contam[idx])
    p1 = O.fwd(geo, Es, ones)
    px = O.fwd(geo, Es, x32)
    v = np.zeros(idx.size)
    for k, e in enumerate(idx):
        Se = gamma_rho / p1[k] if p1[k] > 0 else 0.0
        a = y[e] + Se * (px[k] + float(E.contam[e]))
        yp = O.prox_dstar(a, float(mu[e]) * Se, 1.0)
        v[k] = (yp - y[e]) / float(mu[e])
    return O.back(geo, Es, v)


def _shard_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as O
    from tests.test_oracle_lmspdhg import _geometry, _knorm, tiny_problem
    sc, g, tof, ev = tiny_problem(n_events=400, seed=13)
    geo = _geometry(O, sc, g, tof)
    E = O.EventArrays.from_events(ev)
    mu = O.event_counts(ev.det1, ev.det2, ev.tof)  # a count over the whole list, shared by every shard
    n_sub, i = 3, 1
    sens = O.sens(geo, np.ones(sc.n_lor, np.float32))
    x0 = np.full(geo.V, np.float32(1.0))
    gamma = 3.0
    lm = O.LM(geo, E, mu, n_sub, beta=0.1, gamma=gamma, rho=0.999, knorm=_knorm(g.n))
    lm.init(x0, sens)
    # the primal step that opens the update, then the subset's events split across the ranks
    x = np.maximum(0.0, lm.x - lm.T * lm.zbar)
    x32 = x.astype(np.float32)
    ones = np.ones(geo.V, np.float32)
    sub = np.arange(i, ev.n, n_sub)
    mine = sub[rank::world]
    dz = torch.from_numpy(_data_update_dz(O, geo, E, mu, x32, lm.y, mine, gamma * 0.999, ones))
    dist.all_reduce(dz, op=dist.ReduceOp.SUM)
    full = _data_update_dz(O, geo, E, mu, x32, lm.y, sub, gamma * 0.999, ones)
    z_before = lm.z.copy()
    lm.update(i)
    q.put((rank, mine.size, dz.numpy(), full, lm.z - z_before))
    dist.barrier()
    dist.destroy_process_group()


def test_event_sharded_data_update_two_ranks():
    """Event sharding of one frame (each rank holds half of every subset's
    events and a full image): the partial back-projections summed by an
    all-reduce equal the single-rank data update, and the oracle's own update
    of z, because the dual step is per event (with mu counted over the whole
    list) and dz is a sum over events."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sorted(r[1] > 0 for r in res) == [True, True]
    for rank, n_mine, dz, full, dz_oracle in res:
        scale = np.abs(full).max()
        np.testing.assert_allclose(dz, full, rtol=0, atol=1e-12 * scale)
        # the oracle projects the FP64 x, the primitives above its float32 copy
        np.testing.assert_allclose(dz, dz_oracle, rtol=0, atol=1e-6 * scale)


class _FakeShardState:
    """Stands in for a shard state of the library on CPU ranks (the library
    needs a GPU): shard_begin puts this rank's partial dz of a data update in
    the buffer, shard_finish records what the exchange left there."""

    def __init__(self, rank, n_subsets, V=8):
        self.rank, self.n_subsets = rank, n_subsets
        self.buf = torch.zeros(V)
        self.log = []
        self.pending = None

    def shard_buffer(self):
        return self.buf

    def shard_begin(self, sel, stream=None):
        assert self.pending is None
        self.pending = sel
        if sel < self.n_subsets:
            self.buf.copy_(torch.arange(self.buf.numel(), dtype=torch.float32) * (self.rank + 1) + sel)

    def shard_finish(self, stream=None):
        sel = self.pending
        self.pending = None
        self.log.append((sel, self.buf.clone() if sel < self.n_subsets else None))

    def shard_init_finish(self, stream=None):
        self.log.append(("init", self.buf.clone()))


def _protocol_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2201_05497_gb300.lm import LMSPDHG
    st = _FakeShardState(rank, n_subsets=3)
    st.buf.fill_(float(rank + 1))
    LMSPDHG.shard_init(st, dist.all_reduce)
    LMSPDHG.shard_updates(st, [0, 3, 2, 3, 1], dist.all_reduce)
    q.put((rank, [(s, None if b is None else b.numpy()) for s, b in st.log]))
    dist.barrier()
    dist.destroy_process_group()


def test_shard_protocol_two_ranks():
    """The binding's shard protocol over a real process group: every data
    update's buffer holds the sum of both ranks' partials when the update
    finishes, prior updates exchange nothing, and both ranks see the same
    values (they then apply identical image passes)."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_protocol_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ar = np.arange(8, dtype=np.float32)
    for rank in (0, 1):
        log = res[rank]
        assert log[0][0] == "init" and np.all(log[0][1] == 3.0)
        assert [s for s, _ in log[1:]] == [0, 3, 2, 3, 1]
        for sel, b in log[1:]:
            if sel == 3:
                assert b is None
            else:
                np.testing.assert_array_equal(b, ar * 3 + 2 * sel)
