"""Pins of the oracle's image-space resolution model G (P = A G, Eq. (1)'s
limited spatial resolution): G equals scipy's Gaussian filter with mirrored
faces (the same taps, truncation and boundary), G is symmetric with rows
summing to 1 (so P^T = G A^T and P 1 = A 1), and (in test_oracle_lmspdhg.py
and below) LM-SPDHG and the EM step with G match computations on the dense
A G built here."""
import math

import numpy as np
import pytest
from scipy import ndimage

from paper_2201_05497_gb300 import synth as S


def _geo(O, n, h):
    return O.Geometry(np.zeros((2, 3), np.float32), 1, 2, n, h, (0.0, 0.0, 0.0))


def _sigma_vox(fwhm, h):
    return fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0))) / h


@pytest.mark.parametrize("n,h,fwhm", [((24, 20, 1), (2.0, 2.0, 2.0), 4.5), ((16, 14, 12), (2.5, 2.5, 2.0), 6.0),
                                      ((30, 9, 8), (1.0, 3.0, 2.5), 3.0), ((9, 7, 2), (2.0, 2.0, 6.0), 6.0)])
def test_res_equals_scipy_gaussian_filter(oracle_mod, n, h, fwhm):
    """Also on an axis of two voxels (one tap per side there)."""
    O = oracle_mod
    geo = _geo(O, n, h)
    rng = np.random.default_rng(1)
    x = rng.uniform(0.0, 2.0, geo.V)
    got = O.res_apply(geo, fwhm, x).reshape(n[2], n[1], n[0])
    sig = [(_sigma_vox(fwhm, h[d]) if n[d] > 1 else 0.0) for d in (2, 1, 0)]
    want = ndimage.gaussian_filter(x.reshape(n[2], n[1], n[0]), sigma=sig, mode="reflect", truncate=3.0)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)


@pytest.mark.parametrize("n,h,fwhm", [((5, 4, 3), (1.0, 1.0, 1.0), 3.5), ((6, 3, 1), (2.0, 2.0, 2.0), 9.0)])
def test_res_symmetric_rows_sum_to_one(oracle_mod, n, h, fwhm):
    """Also with taps clipped to n_d - 1 on short axes."""
    O = oracle_mod
    geo = _geo(O, n, h)
    V = geo.V
    G = np.zeros((V, V))
    for j in range(V):
        e = np.zeros(V)
        e[j] = 1.0
        G[:, j] = O.res_apply(geo, fwhm, e)
    np.testing.assert_allclose(G, G.T, rtol=0, atol=1e-15)
    np.testing.assert_allclose(G.sum(1), np.ones(V), rtol=0, atol=1e-14)
    assert np.all(G >= 0.0)
    # fwhm 0 is the identity
    x = np.random.default_rng(2).normal(size=V)
    np.testing.assert_array_equal(O.res_apply(geo, 0.0, x), x)


def test_em_step_with_resolution_is_gradient_step(oracle_mod):
    """z = x - (x n / g) grad L_i(x) with L_i built on the dense A G (finite
    differences of the forward model only)."""
    O = oracle_mod
    sc = S.Scanner(1, 24, 30.0, 1.0)
    g = S.Grid((6, 5, 1), (4.0, 4.0, 4.0))
    tof = S.Tof(8.0, 6.0, 3.0, 9)
    ev = S.uniform_events(sc, tof, 200, 12)
    geo = O.Geometry(sc.crystal_table(), sc.n_rings, sc.n_xtal, g.n, g.h, g.origin,
                     (tof.sigma, tof.bin, tof.n_sigma, tof.n_bins))
    E = O.EventArrays.from_events(ev)
    fwhm, n_sub, i = 7.0, 2, 1
    V = geo.V
    idx = np.arange(i, ev.n, n_sub)
    Es = O.EventArrays(E.det1[idx], E.det2[idx], E.tof[idx], E.corr[idx], E.contam[idx])
    A = np.zeros((idx.size, V))
    G = np.zeros((V, V))
    for j in range(V):
        e = np.zeros(V, np.float32)
        e[j] = 1.0
        A[:, j] = O.fwd(geo, Es, e)
        G[:, j] = O.res_apply(geo, fwhm, e.astype(np.float64))
    P = A @ G
    s = Es.contam.astype(np.float64)
    rng = np.random.default_rng(3)
    x = rng.uniform(0.5, 2.0, V)
    sens = rng.uniform(0.5, 3.0, V)

    def L(xx):
        return float(np.dot(sens / n_sub, xx) - np.sum(np.log(P @ xx + s)))

    grad = np.zeros(V)
    for j in range(V):
        hs = 1e-6 * x[j]
        xp, xm = x.copy(), x.copy()
        xp[j] += hs
        xm[j] -= hs
        grad[j] = (L(xp) - L(xm)) / (2 * hs)
    want = x - x * n_sub / sens * grad
    z = O.EMTV(geo, E, n_sub, beta=0.0, knorm=1.0, res_fwhm=fwhm).em_step(x, sens, i)
    np.testing.assert_allclose(z, want, rtol=1e-6, atol=1e-7 * np.abs(want).max())


@pytest.mark.parametrize("sig_vox", [1.0, 1.6])
def test_res_clipped_taps_equal_scipy_radius(oracle_mod, sig_vox):
    """On axes shorter than the kernel the taps stop at r = n_d - 1 (each
    image value reflected at most once): the same as scipy's mirrored
    Gaussian filter with that radius.  sigma 1 voxel: r = 3 on axes of 5, 3
    and 4 voxels (clipped on the axis of 3, where r = n); sigma 1.6: r = 5
    (clipped on every axis)."""
    pytest.importorskip("scipy", minversion="1.10")
    O = oracle_mod
    n, h = (5, 3, 4), (1.0, 1.0, 1.0)
    fwhm = sig_vox * 2.0 * math.sqrt(2.0 * math.log(2.0))
    geo = _geo(O, n, h)
    x = np.random.default_rng(4).uniform(0.0, 2.0, geo.V)
    got = O.res_apply(geo, fwhm, x).reshape(n[2], n[1], n[0])
    r = [min(int(math.floor(3.0 * sig_vox + 0.5)), n[d] - 1) for d in (2, 1, 0)]
    want = ndimage.gaussian_filter(x.reshape(n[2], n[1], n[0]), sigma=[sig_vox] * 3, mode="reflect", radius=r)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)
