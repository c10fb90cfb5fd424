"""Pins of the oracle's LM-SPDHG (Alg. 2) against mathematics that does not
use its own iteration: the gradient of the objective (sign of the z
initialisation), an independent convex solve of the tiny dense problem
(fixed point, step sizes, prox, update signs) and Alg. 1 on the full
sinogram (the appendix's equivalence: LM-SPDHG and SPDHG produce the same
iterates)."""
import math

import numpy as np
import pytest
from scipy import optimize

from paper_2201_05497_gb300 import synth as S


def tiny_problem(n_xtal=24, n=(6, 5, 1), h=4.0, n_bins=9, n_events=300, seed=1, dup_free=False):
    sc = S.Scanner(1, n_xtal, 30.0, 1.0)
    g = S.Grid(n, (h, h, h))
    tof = S.Tof(8.0, 6.0, 3.0, n_bins)
    ev = S.uniform_events(sc, tof, n_events * (3 if dup_free else 1), seed)
    if dup_free:
        key = np.where(ev.det1 < ev.det2, ev.det1.astype(np.int64) * 100000 + ev.det2 * 100 + ev.tof,
                       ev.det2.astype(np.int64) * 100000 + ev.det1 * 100 - ev.tof)
        _, first = np.unique(key, return_index=True)
        ev = ev.subset(np.sort(first)[:n_events])
    return sc, g, tof, ev


def _geometry(O, sc, g, tof):
    return O.Geometry(sc.crystal_table(), sc.n_rings, sc.n_xtal, g.n, g.h, g.origin,
                      (tof.sigma, tof.bin, tof.n_sigma, tof.n_bins))


def _knorm(n):
    return math.sqrt(sum(4.0 * math.sin(math.pi * (m - 1) / (2.0 * m)) ** 2 for m in n if m > 1))


def test_zinit_is_data_gradient(oracle_mod):
    """Reading of the z initialisation's sign: z0 = P^T 1 + (P^LM)^T((y0-1)/mu)
    must equal the gradient of <P^T 1, x> - sum_e log((P^LM x)_e + s_e) at x0
    (it is P^T applied to the sinogram y that is 1 on empty bins and
    Eq. (yinit) elsewhere).  Checked by central finite differences."""
    O = oracle_mod
    sc, g, tof, ev = tiny_problem(n_events=400, seed=3)
    geo = _geometry(O, sc, g, tof)
    E = O.EventArrays.from_events(ev)
    mu = O.event_counts(ev.det1, ev.det2, ev.tof)
    lf = np.ones(sc.n_lor, np.float32)
    sens = O.sens(geo, lf)
    lm = O.LM(geo, E, mu, 1, beta=0.0, gamma=1.0, rho=0.999, knorm=_knorm(g.n))
    rng = np.random.default_rng(0)
    x0 = rng.uniform(0.5, 2.0, geo.V).astype(np.float32)
    lm.init(x0, sens)
    # gradient by central differences of the oracle objective (beta = 0)
    xd = x0.astype(np.float64)
    grad = np.zeros(geo.V)
    for j in range(geo.V):
        hstep = 1e-5
        xp, xm = xd.copy(), xd.copy()
        xp[j] += hstep
        xm[j] -= hstep
        grad[j] = (lm.objective(xp) - lm.objective(xm)) / (2 * hstep)
    np.testing.assert_allclose(lm.z, grad, rtol=1e-6, atol=1e-6 * np.abs(grad).max())
    # and y0 is Eq. (yinit) with d -> mu
    p = O.fwd(geo, E, x0)
    np.testing.assert_allclose(lm.y, 1.0 - mu / (p + ev.contam), rtol=1e-14)


def _dense_lm_matrix(O, geo, E):
    A = np.zeros((E.n, geo.V))
    for j in range(geo.V):
        e = np.zeros(geo.V, np.float32)
        e[j] = 1.0
        A[:, j] = O.fwd(geo, E, e)
    return A


def _dtv_field(O, geo, n, seed=21, eta=0.3):
    """A structural image (smooth blob plus noise) and its DTV field."""
    rng = np.random.default_rng(seed)
    ix, iy, iz = np.meshgrid(np.arange(n[0]), np.arange(n[1]), np.arange(n[2]), indexing="ij")
    v = np.exp(-((ix - 1.5) ** 2 + (iy - 2.0) ** 2) / 3.0) + 0.1 * rng.uniform(size=ix.shape)
    v = np.transpose(v, (2, 1, 0)).reshape(-1)  # x fastest
    return O.dtv_xi(geo, v, eta)


@pytest.mark.parametrize("prior", ["tv", "dtv", "tv+res", "tv-3d"])
def test_lmpdhg_reaches_independent_minimiser(oracle_mod, prior):
    """Brute force on a tiny grid: the dense P^LM is built column by column;
    L-BFGS-B on Eq. (1) with a smoothed TV (eps = 1e-9) gives the minimiser
    independently of Alg. 2.  LM-SPDHG (n = 1) must approach it: the objective
    gap and the KKT residual of x >= 0 become small.  For DTV the dense K is
    the dense TV matrix with P_j = I - xi_j xi_j^T applied to each voxel's
    rows, written here from the definition; with the resolution model the
    dense forward model is A G (G from its columns) and P^T 1 = G A^T 1.
    tv-3d and tv+res: two slices either side of the ring's plane (each
    sample split half and half between them, TV and G across them)."""
    O = oracle_mod
    sc, g, tof, ev = tiny_problem(n=(4, 3, 2) if prior in ("tv-3d", "tv+res") else (5, 4, 1), n_events=250, seed=5)
    geo = _geometry(O, sc, g, tof)
    E = O.EventArrays.from_events(ev)
    mu = O.event_counts(ev.det1, ev.det2, ev.tof)
    sens = O.sens(geo, np.ones(sc.n_lor, np.float32))
    A = _dense_lm_matrix(O, geo, E)
    fwhm = 6.0 if prior == "tv+res" else 0.0
    if fwhm > 0:
        G = np.zeros((geo.V, geo.V))
        for j in range(geo.V):
            e = np.zeros(geo.V)
            e[j] = 1.0
            G[:, j] = O.res_apply(geo, fwhm, e)
        A = A @ G
        sens = G @ sens
    s = ev.contam.astype(np.float64)
    beta = 0.5
    V = geo.V
    # K dense
    Km = np.zeros((geo.ndim * V, V))
    for j in range(V):
        e = np.zeros(V)
        e[j] = 1
        Km[:, j] = O.tv_grad(geo, e)
    xi = None
    if prior == "dtv":
        xi = _dtv_field(O, geo, g.n)
        Kr = Km.reshape(geo.ndim, V, V)
        X = xi.reshape(geo.ndim, V)
        par = np.einsum("cj,cjk->jk", X, Kr)
        Km = (Kr - X[:, :, None] * par[None]).reshape(geo.ndim * V, V)
    eps = 1e-9

    def f(x):
        u = A @ x + s
        gk = (Km @ x).reshape(geo.ndim, V)
        nrm = np.sqrt((gk ** 2).sum(0) + eps * eps)
        val = sens @ x - np.log(u).sum() + beta * nrm.sum()
        grad = sens - A.T @ (1.0 / u) + beta * Km.T @ (gk / nrm).reshape(-1)
        return val, grad

    x_init = np.full(V, 1.0)
    res = optimize.minimize(f, x_init, jac=True, method="L-BFGS-B", bounds=[(0, None)] * V,
                            options=dict(maxiter=20000, ftol=1e-16, gtol=1e-12, maxcor=30))
    x_star = res.x
    f_star = f(x_star)[0]

    x0 = np.full(V, np.float32(1.0))
    knorm = _knorm(g.n)
    lm = O.LM(geo, E, mu, 1, beta=beta, gamma=3.0 / float(x0.max()), rho=0.999, knorm=knorm, xi=xi,
              res_fwhm=fwhm)
    lm.init(x0, sens)
    seq = S.selection_sequence(1, 60000, seed=3)
    lm.run(seq)
    f_lm = lm.objective()
    assert abs(f_lm - lm.objective(x_star)) < 1e-12 * abs(f_star) + abs(f(x_star)[0] - lm.objective(x_star)) + 1e-12
    gap = (f_lm - f_star) / abs(f_star)
    assert gap < 1e-7
    assert np.linalg.norm(lm.x - x_star) / np.linalg.norm(x_star) < 2e-3
    # KKT of the data term + TV dual: r = grad D(x) + K^T w, r = 0 on x > 0, r >= 0 on x = 0
    r = sens - A.T @ (1.0 / (A @ lm.x + s)) + Km.T @ lm.w
    pos = lm.x > 1e-6 * lm.x.max()
    assert np.max(np.abs(r[pos])) < 1e-3 * np.abs(sens).max()
    wn = np.sqrt((lm.w.reshape(geo.ndim, V) ** 2).sum(0))
    assert np.all(wn <= beta * (1 + 1e-12))


def _sino_setup(O, geo, sc, tof, ev, n_subsets, lm_subset_of_event):
    nb = max(tof.n_bins, 1)  # non-TOF: one bin per LOR
    M = (nb - 1) // 2
    l = S.lor_of_events(sc, ev.det1, ev.det2)
    # canonical orientation: the TOF bin is signed toward the canonical det2
    d1c = np.empty_like(ev.det1)
    for k in range(ev.n):
        d1c[k], _ = geo.lor_dets(int(l[k]))
    m = np.where(ev.det1 == d1c, ev.tof, -ev.tof).astype(np.int64)
    b = l * nb + (m + M)
    NB = geo.n_lor * nb
    d = np.bincount(b, minlength=NB).astype(np.float64)
    s = np.full(NB, float(ev.contam[0]))
    sub = np.zeros(NB, np.int32)
    sub[b] = lm_subset_of_event
    return d, s, sub, b


@pytest.mark.parametrize("n_subsets,dup_free,prior,n,n_bins", [
    (1, False, "tv", (6, 5, 1), 9), (3, True, "tv", (6, 5, 1), 9), (3, True, "dtv", (6, 5, 1), 9),
    (3, True, "tv", (4, 3, 2), 9), (2, True, "dtv", (4, 3, 2), 9), (1, False, "tv", (6, 5, 1), 0)])
def test_lm_spdhg_equals_sinogram_spdhg(oracle_mod, n_subsets, dup_free, prior, n, n_bins):
    """Appendix: LM-SPDHG is SPDHG on the listmode reformulation.  With the
    same selection sequence (n = 1 with duplicated events, or n = 3 on
    duplicate-free data with the sinogram subset of a bin = the listmode
    subset of its event), Alg. 1 on the full sinogram (empty bins included,
    y = 1 there, Eq. (yinit) elsewhere) and Alg. 2 give the same x, z, w, and
    y of an event equals y of its bin.  Empty bins keep y = 1 (Sec.
    "Memory-efficient SPDHG").  The objectives differ by sum_b s_b only.
    Also on two-slice grids and without TOF (one bin per LOR)."""
    O = oracle_mod
    sc, g, tof, ev = tiny_problem(n=n, n_bins=n_bins, n_events=350, seed=11, dup_free=dup_free)
    ev = S.Events(ev.det1, ev.det2, ev.tof, ev.corr, np.full(ev.n, np.float32(0.05)))
    geo = _geometry(O, sc, g, tof)
    lf = np.random.default_rng(2).uniform(0.4, 1.0, sc.n_lor).astype(np.float32)
    l_ev = S.lor_of_events(sc, ev.det1, ev.det2)
    ev = S.Events(ev.det1, ev.det2, ev.tof, lf[l_ev], ev.contam)
    E = O.EventArrays.from_events(ev)
    mu = O.event_counts(ev.det1, ev.det2, ev.tof)
    if dup_free:
        assert mu.max() == 1
    else:
        assert mu.max() > 1
    sens = O.sens(geo, lf)
    knorm = _knorm(g.n)
    x0 = np.random.default_rng(4).uniform(0.5, 1.5, geo.V).astype(np.float32)
    gamma = 3.0 / float(x0.max())
    xi = _dtv_field(O, geo, g.n) if prior == "dtv" else None
    lm = O.LM(geo, E, mu, n_subsets, beta=0.2, gamma=gamma, rho=0.999, knorm=knorm, xi=xi)
    lm.init(x0, sens)
    d, s, sub, b_of_e = _sino_setup(O, geo, sc, tof, ev, n_subsets, np.arange(ev.n) % n_subsets)
    sino = O.Sino(geo, lf, d, s, sub, n_subsets, beta=0.2, gamma=gamma, rho=0.999, knorm=knorm, xi=xi)
    sino.init(x0, sens)
    np.testing.assert_allclose(lm.z, sino.z, rtol=1e-12, atol=1e-12 * np.abs(sino.z).max())
    seq = S.selection_sequence(n_subsets, 120, seed=3)
    for t, i in enumerate(seq):
        lm.update(int(i))
        sino.update(int(i))
        scale = np.abs(sino.x).max()
        np.testing.assert_allclose(lm.x, sino.x, rtol=0, atol=1e-11 * scale)
    np.testing.assert_allclose(lm.z, sino.z, rtol=0, atol=1e-10 * np.abs(sino.z).max())
    np.testing.assert_allclose(lm.w, sino.w, rtol=0, atol=1e-11)
    np.testing.assert_allclose(lm.y, sino.y[b_of_e], rtol=0, atol=1e-10 * np.abs(sino.y).max())
    empty = d == 0
    # exact in real arithmetic; (a + 1) - |a - 1| rounds to within a few ulps of 2
    assert np.max(np.abs(sino.y[empty] - 1.0)) <= 1e-14
    assert abs((sino.objective() - s.sum()) - lm.objective()) <= 1e-10 * abs(lm.objective())


def _all_bins(O, geo, tof, lf):
    """Every (LOR, TOF bin) of the scanner as one event, LOR factor in corr."""
    d1, d2, m, c = [], [], [], []
    for l in range(geo.n_lor):
        a, b = geo.lor_dets(l)
        for k in range(-tof.half, tof.half + 1):
            d1.append(a)
            d2.append(b)
            m.append(k)
            c.append(lf[l])
    return O.EventArrays(np.array(d1), np.array(d2), np.array(m), np.array(c, np.float32))


@pytest.mark.parametrize("binding,n_sub", [("data", 1), ("data", 3), ("prior", 1), ("prior", 3), ("mixed", 2)])
def test_step_sizes_meet_the_spdhg_condition(oracle_mod, binding, n_sub):
    """Eq. (lm_stepsizes) is SPDHG's diagonally preconditioned choice for
    balanced subsets (column sums P_i^T 1 = P^T 1 / n).  Made exact here: the
    n subsets are n copies of every bin, so the list's sensitivity is n P^T 1.
    Then S_b = gamma rho / (P 1)_b and T = rho p_i n / (gamma n P^T 1) give
    ||S^1/2 P_i T^1/2||^2 = rho^2 p_i, p_i = 1/(2n): a nonnegative P has the
    positive singular pair (sqrt(P 1), sqrt(P^T 1)) with singular value 1 once
    scaled (Perron-Frobenius).  The prior's S_{n+1} = gamma rho / ||K|| and
    T = rho p_{n+1} / (gamma ||K||) give S_{n+1} T ||K||^2 = rho^2 p_{n+1},
    p_{n+1} = 1/2.  T is the smaller of the two, so where one term sets T its
    condition holds with equality and the other's as an inequality.  T comes
    from the oracle's initialisation; S_{n+1} is read back from one prior
    update whose projection is inactive (beta huge): w+ = S_{n+1} K x."""
    O = oracle_mod
    sc, g, tof, ev = tiny_problem(n=(6, 5, 1), n_bins=5, n_events=200, seed=8)
    geo = _geometry(O, sc, g, tof)
    V = geo.V
    kn = _knorm(g.n)
    gamma, rho = 0.7, 0.9
    lf = np.random.default_rng(3).uniform(0.5, 1.0, geo.n_lor).astype(np.float32)
    sens0 = O.sens(geo, lf)
    # scale the LOR factors so that the chosen term sets T (T_data < T_prior <=> n P^T 1 > ||K||)
    scale = {"data": 2.0, "prior": 0.5, "mixed": 1.0}[binding] * kn / n_sub
    scale /= {"data": sens0.min(), "prior": sens0.max(), "mixed": np.median(sens0)}[binding]
    lf = (lf * scale).astype(np.float32)
    sens1 = O.sens(geo, lf)
    assert sens1.min() > 0
    E = O.EventArrays.from_events(ev)
    mu = O.event_counts(ev.det1, ev.det2, ev.tof)
    lm = O.LM(geo, E, mu, n_sub, beta=1e30, gamma=gamma, rho=rho, knorm=kn)
    lm.init(np.full(V, 2.0, np.float32), n_sub * sens1)
    T = lm.T.copy()
    # Alg. 1's oracle takes the same primal step sizes
    NB = geo.n_lor * tof.n_bins
    sino = O.Sino(geo, lf, np.zeros(NB), np.ones(NB), np.zeros(NB, np.int32), n_sub, beta=1e30, gamma=gamma,
                  rho=rho, knorm=kn)
    sino.init(np.full(V, 2.0, np.float32), n_sub * sens1)
    np.testing.assert_array_equal(sino.T, T)
    # data term of one subset (one copy of every bin): the dense operator; its column sums are P^T 1
    A = _dense_lm_matrix(O, geo, _all_bins(O, geo, tof, lf))
    np.testing.assert_allclose(A.sum(0), sens1, rtol=1e-12)
    r = A.sum(1)
    A, r = A[r > 0], r[r > 0]
    c_data = np.linalg.norm(np.sqrt(gamma * rho / r)[:, None] * A * np.sqrt(T)[None, :], 2) ** 2
    # prior term: S_{n+1} from one prior update, K dense from its columns
    lm.update(n_sub)
    Kx = O.tv_grad(geo, lm.x)
    s_prior = float(lm.w @ Kx / (Kx @ Kx))
    np.testing.assert_allclose(lm.w, s_prior * Kx, rtol=0, atol=1e-12 * np.abs(lm.w).max())
    Km = np.zeros((geo.ndim * V, V))
    for j in range(V):
        e = np.zeros(V)
        e[j] = 1.0
        Km[:, j] = O.tv_grad(geo, e)
    np.testing.assert_allclose(np.linalg.norm(Km, 2), kn, rtol=1e-12)
    c_prior = np.linalg.norm(Km * np.sqrt(s_prior * T)[None, :], 2) ** 2
    lim_data, lim_prior = rho ** 2 / (2 * n_sub), rho ** 2 / 2
    if binding == "data":
        assert abs(c_data - lim_data) <= 1e-10 * lim_data
        assert c_prior <= lim_prior * (1 - 1e-3)
    elif binding == "prior":
        np.testing.assert_allclose(s_prior * T * kn ** 2, lim_prior, rtol=1e-12)
        assert abs(c_prior - lim_prior) <= 1e-10 * lim_prior
        assert c_data <= lim_data * (1 - 1e-3)
    else:
        assert (T < T.max()).any() and (T == T.max()).any()  # both terms set T somewhere
        assert c_data <= lim_data * (1 + 1e-12) and c_prior <= lim_prior * (1 + 1e-12)
