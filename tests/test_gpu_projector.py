"""GPU parity of the projector calls (lm_fwd, lm_back, lm_sens) against the
FP64 oracle, on seeded Monte Carlo and uniform event lists spanning many
warps and ragged tails, plus the GPU-side adjoint and brute-force checks."""
import math

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
    assert torch.cuda.is_available()
    _lm.load_library()
    return _lm


def _setup(lm, name, n_events, uniform=False, seed=2):
    wl = S.workload(name)
    if uniform:
        ev = S.uniform_events(wl.scanner, wl.tof, n_events, seed)
        lf = None
    else:
        wl, lf, ev = H.workload_data(name, n_events, seed)
    geo_o = O.Geometry.from_workload(wl)
    geo_g = lm.Geometry.from_workload(wl)
    return wl, lf, ev, geo_o, geo_g


def _one_sample_bound(wl):
    # largest possible weight of one sample: step (<= 2 h) times the TOF weight at the cut
    t = wl.tof
    w_cut = 0.5 * (math.erf((t.n_sigma * t.sigma + t.bin / 2) / (math.sqrt(2) * t.sigma)) -
                   math.erf((t.n_sigma * t.sigma - t.bin / 2) / (math.sqrt(2) * t.sigma)))
    return 2.0 * max(wl.grid.h) * w_cut * 4.0


@pytest.mark.parametrize("name,n,uniform", [("2d_small", 20000, False), ("2d_small", 7777, True),
                                            ("3d_small", 40000, False), ("3d_small", 9001, True),
                                            ("3d_mid", 60000, False)])
@pytest.mark.parametrize("use_ws", [False, True])
def test_fwd_matches_oracle(lm, name, n, uniform, use_ws):
    wl, lf, ev, geo_o, geo_g = _setup(lm, name, n, uniform)
    x = wl.phantom.voxelised(wl.grid) + np.float32(0.1)
    E = O.EventArrays.from_events(ev)
    p_or = O.fwd(geo_o, E, x)
    edge = O.tof_edge_distance(geo_o, E)
    sens = O.fwd_position_sensitivity(geo_o, E, x)
    dev = lm.DeviceEvents.from_numpy(ev)
    p = lm.fwd(geo_g, torch.from_numpy(x).cuda(), dev, use_workspace=use_ws).cpu().numpy()
    n_chk, n_edge, worst = H.check_event_projections(p, p_or, edge, _one_sample_bound(wl) * x.max(), sens,
                                                     max(wl.grid.n))
    assert n_chk > 0.99 * n
    assert worst <= H.REL_EVENT


@pytest.mark.parametrize("name,n", [("2d_small", 20000), ("3d_small", 30000), ("3d_mid", 40000)])
@pytest.mark.parametrize("use_ws", [False, True])
def test_back_matches_oracle(lm, name, n, use_ws):
    wl, lf, ev, geo_o, geo_g = _setup(lm, name, n)
    rng = np.random.default_rng(1)
    v = rng.normal(size=ev.n).astype(np.float32)
    E = O.EventArrays.from_events(ev)
    img_or = O.back(geo_o, E, v.astype(np.float64))
    dev = lm.DeviceEvents.from_numpy(ev)
    img = lm.back(geo_g, torch.from_numpy(v).cuda(), dev, use_workspace=use_ws).cpu().numpy()
    assert H.rel_l2(img, img_or) < H.REL_EVENT
    assert np.max(np.abs(img - img_or)) <= 1e-5 * np.max(np.abs(img_or))


@pytest.mark.parametrize("name", ["2d_small", "3d_small"])
def test_back_deterministic_bit_identical(lm, name):
    """Fixed-point back-projection: bit-identical across runs and workspace
    layouts, and within float32 rounding of the atomic version."""
    wl, lf, ev, geo_o, geo_g = _setup(lm, name, 30000)
    rng = np.random.default_rng(2)
    v = torch.from_numpy(rng.normal(size=ev.n).astype(np.float32)).cuda()
    dev = lm.DeviceEvents.from_numpy(ev)
    a = lm.back(geo_g, v, dev, deterministic=True).cpu().numpy()
    b = lm.back(geo_g, v, dev, deterministic=True).cpu().numpy()
    np.testing.assert_array_equal(a, b)
    f = lm.back(geo_g, v, dev, deterministic=False).cpu().numpy()
    E = O.EventArrays.from_events(ev)
    img_or = O.back(geo_o, E, v.cpu().numpy().astype(np.float64))
    assert H.rel_l2(a, img_or) < H.REL_EVENT
    assert H.rel_l2(f, img_or) < H.REL_EVENT


@pytest.mark.parametrize("name", ["2d_small", "3d_small"])
def test_gpu_adjoint(lm, name):
    """<P x, v> = <x, P^T v> on the GPU (sums in FP64 on the host)."""
    wl, lf, ev, geo_o, geo_g = _setup(lm, name, 50000, uniform=True)
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, geo_g.V).astype(np.float32)
    v = rng.normal(size=ev.n).astype(np.float32)
    dev = lm.DeviceEvents.from_numpy(ev)
    p = lm.fwd(geo_g, torch.from_numpy(x).cuda(), dev).cpu().numpy().astype(np.float64)
    bt = lm.back(geo_g, torch.from_numpy(v).cuda(), dev).cpu().numpy().astype(np.float64)
    lhs, rhs = p.dot(v), x.astype(np.float64).dot(bt)
    assert abs(lhs - rhs) <= 1e-5 * np.abs(p).dot(np.abs(v))


def test_bruteforce_tiny_grid(lm):
    """Dense A of a 4x4 (and 3x3x3) problem built column by column from the
    oracle: the GPU forward equals A x and the GPU back-projection A^T v."""
    for n, rings in [((4, 4, 1), 1), ((3, 3, 3), 3)]:
        sc = S.Scanner(rings, 20, 25.0, 3.0)
        g = S.Grid(n, (4.0, 4.0, 3.0))
        tof = S.Tof(6.0, 5.0, 3.0, 9)
        ev = S.uniform_events(sc, tof, 700, seed=7)
        geo_o = O.Geometry(sc.crystal_table(), sc.n_rings, sc.n_xtal, g.n, g.h, g.origin,
                           (tof.sigma, tof.bin, tof.n_sigma, tof.n_bins))
        E = O.EventArrays.from_events(ev)
        V = g.n_vox
        A = np.zeros((ev.n, V))
        for j in range(V):
            e = np.zeros(V, np.float32)
            e[j] = 1
            A[:, j] = O.fwd(geo_o, E, e)
        xtal = torch.from_numpy(sc.crystal_table()).cuda()
        geo_g = lm.Geometry(xtal, sc.n_rings, sc.n_xtal, g.n, g.h, g.origin, tof.sigma, tof.bin, tof.n_sigma,
                            tof.n_bins)
        dev = lm.DeviceEvents.from_numpy(ev)
        rng = np.random.default_rng(0)
        x = rng.uniform(0, 1, V).astype(np.float32)
        v = rng.normal(size=ev.n).astype(np.float32)
        p = lm.fwd(geo_g, torch.from_numpy(x).cuda(), dev).cpu().numpy()
        np.testing.assert_allclose(p, A @ x, rtol=1e-5, atol=1e-5 * np.abs(A @ x).max())
        bt = lm.back(geo_g, torch.from_numpy(v).cuda(), dev).cpu().numpy()
        np.testing.assert_allclose(bt, A.T @ v, rtol=1e-5, atol=1e-5 * np.abs(A.T @ v).max())


@pytest.mark.parametrize("name", ["2d_small", "3d_small", "3d_mid", "2d"])
def test_sens_matches_oracle(lm, name):
    """P^T 1 (TOF bins summed in closed form on the GPU, bin by bin in the
    oracle) over every canonical LOR with the attenuation factors."""
    wl = S.workload(name)
    lf = S.lor_attenuation(wl.scanner, wl.phantom)
    geo_o = O.Geometry.from_workload(wl)
    geo_g = lm.Geometry.from_workload(wl)
    s_or = O.sens(geo_o, lf)
    for use_ws in (False, True):
        s = lm.sens(geo_g, torch.from_numpy(lf).cuda(), use_workspace=use_ws).cpu().numpy()
        assert H.rel_l2(s, s_or) < 1e-5
        assert np.max(np.abs(s - s_or)) <= 2e-5 * np.max(s_or)


def test_empty_and_invalid_events_are_inert(lm):
    """Zero events is a no-op; events with out-of-range ids or TOF bins are
    skipped by the kernels (never dereferenced) and project to 0."""
    wl = S.workload("2d_small")
    geo_g = lm.Geometry.from_workload(wl)
    x = torch.ones(geo_g.V, device="cuda")
    empty = lm.DeviceEvents(torch.zeros(0, dtype=torch.int32, device="cuda"),
                            torch.zeros(0, dtype=torch.int32, device="cuda"),
                            torch.zeros(0, dtype=torch.int16, device="cuda"), None, None)
    assert lm.fwd(geo_g, x, empty).numel() == 0
    nd = wl.scanner.n_det
    bad = lm.DeviceEvents(torch.tensor([0, -1, nd, 3, 5], dtype=torch.int32, device="cuda"),
                          torch.tensor([nd + 7, 4, 2, 3, 40], dtype=torch.int32, device="cuda"),
                          torch.tensor([0, 0, 0, 0, 999], dtype=torch.int16, device="cuda"), None, None)
    p = lm.fwd(geo_g, x, bad).cpu().numpy()
    np.testing.assert_array_equal(p, 0.0)


def test_binding_rejects_wrong_dtype_and_size(lm):
    """Wrong dtypes and short buffers raise in the binding before any launch."""
    wl = S.workload("2d_small")
    geo = lm.Geometry.from_workload(wl)
    x = torch.ones(geo.V, device="cuda")
    with pytest.raises(TypeError):
        lm.res_apply(geo, 4.5, x.double())
    with pytest.raises(ValueError):
        lm.tv_grad(geo, x[:-1])
    ev = lm.DeviceEvents(torch.zeros(3, dtype=torch.int64, device="cuda"), torch.zeros(3, dtype=torch.int32,
                                                                                       device="cuda"), None, None, None)
    with pytest.raises(TypeError):
        lm.fwd(geo, x, ev)
