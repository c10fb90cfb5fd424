"""GPU parity of the event set-up (event counts, subset split: bit-exact),
the TV operators and the FP64 power iteration."""
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


@pytest.mark.parametrize("name,n,n_sub", [("2d_small", 20000, 7), ("2d_small", 20000, 1), ("3d_small", 40000, 28),
                                          ("2d_small", 5, 8), ("3d_mid", 200_000, 14)])
def test_event_setup_bit_exact(lm, name, n, n_sub):
    wl, lf, ev = H.workload_data(name, n)
    geo_g = lm.Geometry.from_workload(wl)
    pe = lm.event_setup(geo_g, lm.DeviceEvents.from_numpy(ev), n_sub)
    perm = O.subset_permutation(ev.n, n_sub)
    inv = np.empty(ev.n, dtype=np.int64)
    inv[perm] = np.arange(ev.n)
    np.testing.assert_array_equal(pe.sub_off, O.subset_offsets(ev.n, n_sub))
    np.testing.assert_array_equal(pe.events.det1.cpu().numpy(), ev.det1[inv])
    np.testing.assert_array_equal(pe.events.det2.cpu().numpy(), ev.det2[inv])
    np.testing.assert_array_equal(pe.events.tof.cpu().numpy(), ev.tof[inv])
    np.testing.assert_array_equal(pe.events.corr.cpu().numpy(), ev.corr[inv])
    np.testing.assert_array_equal(pe.events.contam.cpu().numpy(), ev.contam[inv])
    mu_or = O.event_counts(ev.det1, ev.det2, ev.tof)
    np.testing.assert_array_equal(pe.mu.cpu().numpy().astype(np.int64), mu_or[inv].astype(np.int64))


def test_event_setup_rejects_invalid_events(lm):
    """Invalid data found on the device is reported on the host; nothing out
    of range is dereferenced."""
    wl, lf, ev = H.workload_data("2d_small", 20000)
    geo_g = lm.Geometry.from_workload(wl)
    nd = wl.scanner.n_det
    for field, val, code in [("det1", nd, 2), ("det2", -3, 2), ("tof", 99, 2), ("contam", 0.0, 3),
                             ("corr", -1.0, 3)]:
        arrs = {k: getattr(ev, k).copy() for k in ("det1", "det2", "tof", "corr", "contam")}
        arrs[field][1234] = val
        bad = S.Events(**arrs)
        with pytest.raises(lm.LMError) as ei:
            lm.event_setup(geo_g, lm.DeviceEvents.from_numpy(bad), 7)
        assert ei.value.code == code
        assert "1234" in str(ei.value)


@pytest.mark.parametrize("n", [(37, 33, 11), (128, 128, 1), (200, 200, 96), (5, 1, 1)])
def test_tv_operators(lm, n):
    xtal = torch.zeros(6, device="cuda")
    geo = lm.Geometry(xtal, 1, 2, n, (1.0, 1.0, 1.0), (0.0, 0.0, 0.0))
    geo_o = O.Geometry(np.zeros((2, 3), np.float32), 1, 2, n, (1.0, 1.0, 1.0), (0.0, 0.0, 0.0))
    rng = np.random.default_rng(1)
    x = rng.normal(size=geo.V).astype(np.float32)
    g = lm.tv_grad(geo, torch.from_numpy(x).cuda()).cpu().numpy()
    g_or = O.tv_grad(geo_o, x.astype(np.float64))
    np.testing.assert_allclose(g, g_or, rtol=0, atol=1e-6 * np.abs(x).max())
    q = rng.normal(size=geo.ndim * geo.V).astype(np.float32)
    d = lm.tv_div(geo, torch.from_numpy(q).cuda()).cpu().numpy()
    d_or = -O.tv_adj(geo_o, q.astype(np.float64))
    np.testing.assert_allclose(d, d_or, rtol=0, atol=1e-5 * np.abs(q).max())
    w = torch.from_numpy(q * 0.05).cuda()
    lm.tv_prox(geo, w, 0.07)
    w_or = O.tv_prox(geo_o, (q * 0.05).astype(np.float64), 0.07)
    np.testing.assert_allclose(w.cpu().numpy(), w_or, rtol=2e-7, atol=1e-8)


@pytest.mark.parametrize("n,iters", [(( 16, 12, 1), 300), ((37, 33, 11), 200), ((200, 200, 96), 20)])
def test_knorm_fp64(lm, n, iters):
    """Same power iteration as the oracle (same start, same count) in FP64:
    equal to ~1e-12; never above the closed form."""
    xtal = torch.zeros(6, device="cuda")
    geo = lm.Geometry(xtal, 1, 2, n, (1.0, 1.0, 1.0), (0.0, 0.0, 0.0))
    geo_o = O.Geometry(np.zeros((2, 3), np.float32), 1, 2, n, (1.0, 1.0, 1.0), (0.0, 0.0, 0.0))
    k = lm.knorm_fp64(geo, iters)
    k_or = O.knorm_power(geo_o, iters)
    # the oracle sums V products sequentially in FP64: relative error up to ~V * 2^-53
    assert abs(k - k_or) <= max(1e-12, 4.0 * geo.V * 2.0 ** -53) * k_or
    assert k <= H.knorm_closed(n) * (1 + 1e-14)
