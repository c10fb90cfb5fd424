"""Pins of the oracle's directional TV operator (the paper's second prior,
Sec. "Numerical experiments"): K x = P_j (grad x)_j with P_j = I - xi_j xi_j^T
and xi the normalised gradient field of a structural image.  Pinned by the
adjoint identity, the closed form of K applied to the structural image itself
(zero with eta = 0, also for flipped contrast; |grad v| eta^2/(|grad v|^2 + eta^2)
otherwise), orthogonality to xi, the norm bound ||K|| <= ||grad||, and (in
test_oracle_lmspdhg.py) LM-SPDHG with DTV reaching an independently computed
minimiser and equalling sinogram SPDHG with DTV."""
import math

import numpy as np
import pytest


def _grid_geo(O, n):
    return O.Geometry(np.zeros((2, 3), np.float32), 1, 2, n, (1.0, 1.0, 1.0), (0.0, 0.0, 0.0))


def _fwd_diff(u, n):
    """Forward differences with a Neumann boundary from their definition,
    one component per axis with n_d > 1: [ndim, V] (x fastest)."""
    a = u.reshape(n[2], n[1], n[0])
    out = []
    for ax_img, m in ((2, n[0]), (1, n[1]), (0, n[2])):
        if m > 1:
            d = np.zeros_like(a)
            lo = [slice(None)] * 3
            hi = [slice(None)] * 3
            lo[ax_img] = slice(0, m - 1)
            hi[ax_img] = slice(1, m)
            d[tuple(lo)] = a[tuple(hi)] - a[tuple(lo)]
            out.append(d.reshape(-1))
    return np.array(out)


def _knorm_tv(n):
    return math.sqrt(sum(4.0 * math.sin(math.pi * (m - 1) / (2.0 * m)) ** 2 for m in n if m > 1))


def _random_field(rng, nd, V, unit_frac=0.5):
    xi = rng.normal(size=(nd, V))
    nrm = np.sqrt((xi * xi).sum(0))
    scale = np.where(rng.uniform(size=V) < unit_frac, 1.0, rng.uniform(0.0, 1.0, V))
    return (xi / nrm * scale).reshape(-1)


@pytest.mark.parametrize("n", [(7, 5, 1), (4, 6, 3)])
def test_dtv_adjoint(oracle_mod, n):
    O = oracle_mod
    geo = _grid_geo(O, n)
    rng = np.random.default_rng(1)
    V, nd = geo.V, geo.ndim
    xi = _random_field(rng, nd, V)
    x = rng.normal(size=V)
    q = rng.normal(size=nd * V)
    lhs = float(np.dot(O.dtv_grad(geo, xi, x), q))
    rhs = float(np.dot(x, O.dtv_adj(geo, xi, q)))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


@pytest.mark.parametrize("n", [(9, 8, 1), (6, 5, 4)])
def test_dtv_of_structural_image(oracle_mod, n):
    """With eta = 0 the structural image and its flipped contrast have no DTV;
    with eta > 0, |(K v)_j| = |grad v_j| eta^2 / (|grad v_j|^2 + eta^2)."""
    O = oracle_mod
    geo = _grid_geo(O, n)
    rng = np.random.default_rng(2)
    V = geo.V
    v = rng.uniform(0.0, 3.0, V)
    g = _fwd_diff(v, n)
    gn = np.sqrt((g * g).sum(0))
    xi0 = O.dtv_xi(geo, v, 0.0)
    for img in (v, 5.0 - 2.0 * v):
        kv = O.dtv_grad(geo, xi0, img).reshape(geo.ndim, V)
        assert np.abs(kv).max() <= 1e-12 * np.abs(g).max()
    eta = 0.7
    xi = O.dtv_xi(geo, v, eta)
    np.testing.assert_allclose(xi.reshape(geo.ndim, V), g / np.sqrt(gn ** 2 + eta ** 2), rtol=1e-14, atol=1e-15)
    kv = O.dtv_grad(geo, xi, v).reshape(geo.ndim, V)
    np.testing.assert_allclose(np.sqrt((kv * kv).sum(0)), gn * eta ** 2 / (gn ** 2 + eta ** 2), rtol=1e-12,
                               atol=1e-14)


def test_dtv_perpendicular_to_field(oracle_mod):
    """(K x)_j has no component along a unit xi_j; where xi_j = 0, K = grad."""
    O = oracle_mod
    n = (6, 7, 3)
    geo = _grid_geo(O, n)
    rng = np.random.default_rng(3)
    V, nd = geo.V, geo.ndim
    xi = _random_field(rng, nd, V, unit_frac=1.0).reshape(nd, V)
    xi[:, ::5] = 0.0
    x = rng.normal(size=V)
    kx = O.dtv_grad(geo, xi.reshape(-1), x).reshape(nd, V)
    assert np.abs((kx * xi).sum(0)).max() <= 1e-12 * np.abs(kx).max()
    g = _fwd_diff(x, n)
    np.testing.assert_allclose(kx[:, ::5], g[:, ::5], rtol=0, atol=1e-14)
    # and the parallel part that was removed is (xi . grad x) xi
    np.testing.assert_allclose(g - kx, xi * (xi * g).sum(0), rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("n", [(5, 4, 1), (4, 3, 3)])
def test_dtv_norm_below_tv_norm(oracle_mod, n):
    O = oracle_mod
    geo = _grid_geo(O, n)
    rng = np.random.default_rng(4)
    V, nd = geo.V, geo.ndim
    xi = _random_field(rng, nd, V)
    K = np.zeros((nd * V, V))
    for j in range(V):
        e = np.zeros(V)
        e[j] = 1.0
        K[:, j] = O.dtv_grad(geo, xi, e)
    nrm = np.linalg.norm(K, 2)
    assert nrm <= _knorm_tv(n) * (1 + 1e-12)
    K0 = np.zeros((nd * V, V))
    for j in range(V):
        e = np.zeros(V)
        e[j] = 1.0
        K0[:, j] = O.dtv_grad(geo, None, e)
    assert abs(np.linalg.norm(K0, 2) - _knorm_tv(n)) <= 1e-12 * _knorm_tv(n)
