"""Pins of the oracle's listmode EM-TV (Alg. 3) against mathematics that does
not use its own steps:
  * the subset EM step is the scaled gradient step z = x - (x n / g) grad L_i(x)
    of the subset's Poisson negative log-likelihood
    L_i(x) = <g/n, x> - sum_{e in N_i} log((P^LM x)_e + s_e), the gradient taken by
    central differences of L_i built from the forward projector only;
  * the weighted TV denoising reaches the closed-form minimiser of the
    two-voxel problem, the optimum of an independent constrained solver
    (scipy SLSQP on the epigraph form) on a small grid, the optimality
    conditions of its own dual variable, and the limits w -> inf (u = z) and
    held voxels (u = 0);
  * the pass over the subsets: beta -> 0 reduces it to listmode OSEM (the
    beta = 0 branch), and it is the composition of the two steps over the
    subsets 0..n-1 in order with w = g / (beta x) on the free voxels."""
import math

import numpy as np
import pytest
from scipy import optimize

from paper_2201_05497_gb300 import synth as S


def tiny(n=(5, 4, 1), n_events=240, seed=4, n_bins=9):
    sc = S.Scanner(1, 24, 30.0, 1.0)
    g = S.Grid(n, (4.0, 4.0, 4.0))
    tof = S.Tof(8.0, 6.0, 3.0, n_bins)
    ev = S.uniform_events(sc, tof, n_events, seed)
    return sc, g, tof, ev


def geometry(O, sc, g, tof):
    return O.Geometry(sc.crystal_table(), sc.n_rings, sc.n_xtal, g.n, g.h, g.origin,
                      (tof.sigma, tof.bin, tof.n_sigma, tof.n_bins))


def knorm(n):
    return math.sqrt(sum(4.0 * math.sin(math.pi * (m - 1) / (2.0 * m)) ** 2 for m in n if m > 1))


def tv_terms(u, n):
    """Per-voxel forward differences with a Neumann boundary (last difference
    0), one component per axis with n_d > 1: shape [ndim, V] (x fastest)."""
    a = u.reshape(n[2], n[1], n[0])
    comps = []
    for ax_img, m in ((2, n[0]), (1, n[1]), (0, n[2])):
        if m > 1:
            d = np.zeros_like(a)
            sl_lo = [slice(None)] * 3
            sl_hi = [slice(None)] * 3
            sl_lo[ax_img] = slice(0, m - 1)
            sl_hi[ax_img] = slice(1, m)
            d[tuple(sl_lo)] = a[tuple(sl_hi)] - a[tuple(sl_lo)]
            comps.append(d.reshape(-1))
    return np.array(comps)


def tv_adjoint(Q, n):
    """K^T Q for Q of shape [ndim, V]: the adjoint of tv_terms (minus the
    divergence), from its definition."""
    out = np.zeros((n[2], n[1], n[0]))
    c = 0
    for ax_img, m in ((2, n[0]), (1, n[1]), (0, n[2])):
        if m > 1:
            comp = Q[c].reshape(n[2], n[1], n[0])
            lo = [slice(None)] * 3
            hi = [slice(None)] * 3
            lo[ax_img] = slice(0, m - 1)
            hi[ax_img] = slice(1, m)
            out[tuple(lo)] -= comp[tuple(lo)]
            out[tuple(hi)] += comp[tuple(lo)]
            c += 1
    return out.reshape(-1)


def denoise_objective(u, z, w, n):
    k = tv_terms(u, n)
    return float(np.sum(0.5 * w * (u - z) ** 2) + np.sum(np.sqrt(np.sum(k * k, axis=0))))


# --------------------------------------------------------------------------
# EM step
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n_sub,i", [(1, 0), (3, 1), (4, 3)])
def test_em_step_is_scaled_loglik_gradient_step(oracle_mod, n_sub, i):
    O = oracle_mod
    sc, g, tof, ev = tiny(seed=5 + n_sub)
    geo = geometry(O, sc, g, tof)
    E = O.EventArrays.from_events(ev)
    rng = np.random.default_rng(11)
    x = rng.uniform(0.5, 2.0, geo.V)
    sens = rng.uniform(0.5, 3.0, geo.V)
    sens[3] = 0.0  # z_j = 0 where g_j = 0
    idx = np.arange(i, ev.n, n_sub)
    Es = O.EventArrays(E.det1[idx], E.det2[idx], E.tof[idx], E.corr[idx], E.contam[idx])
    # the subset's system matrix, column by column, from the forward projector
    # applied to unit images (exact in float32)
    A = np.zeros((idx.size, geo.V))
    for j in range(geo.V):
        e_j = np.zeros(geo.V, np.float32)
        e_j[j] = 1.0
        A[:, j] = O.fwd(geo, Es, e_j)
    s = Es.contam.astype(np.float64)

    def L(xx):
        return float(np.dot(sens / n_sub, xx) - np.sum(np.log(A @ xx + s)))

    grad = np.zeros(geo.V)
    for j in range(geo.V):
        h = 1e-6 * x[j]
        xp, xm = x.copy(), x.copy()
        xp[j] += h
        xm[j] -= h
        grad[j] = (L(xp) - L(xm)) / (2 * h)
    want = np.where(sens > 0, x - x * n_sub / np.where(sens > 0, sens, 1.0) * grad, 0.0)
    em = O.EMTV(geo, E, n_sub, beta=0.0, knorm=knorm(g.n))
    z = em.em_step(x, sens, i)
    assert z[3] == 0.0
    np.testing.assert_allclose(z, want, rtol=1e-6, atol=1e-7 * np.abs(want).max())
    # the step keeps the counts: sum_j g_j z_j / n = sum_e (Ax)_e / ((Ax)_e + s_e) over the voxels with g > 0
    Ax = A @ np.where(sens > 0, x, 0.0)
    lhs = float(np.dot(sens, z)) / n_sub
    rhs = float(np.sum((A * np.where(sens > 0, x, 0.0)).sum(axis=1) / (A @ x + s)))
    assert abs(lhs - rhs) <= 1e-10 * abs(rhs)
    assert Ax.shape[0] == idx.size


# --------------------------------------------------------------------------
# weighted TV denoising
# --------------------------------------------------------------------------
def test_denoise_two_voxels_closed_form(oracle_mod):
    """min w1/2 (u1-z1)^2 + w2/2 (u2-z2)^2 + |u2 - u1|: the voxels merge at the
    weighted mean when |z2 - z1| <= 1/w1 + 1/w2, else each moves 1/w_j
    towards the other."""
    O = oracle_mod
    sc, g, tof, _ = tiny(n=(2, 1, 1))
    geo = geometry(O, sc, g, tof)
    kn = knorm(g.n)
    for z, w in [((3.0, 5.0), (2.0, 0.5)), ((4.0, 4.6), (2.0, 3.0)), ((9.0, 2.0), (1.5, 4.0))]:
        z = np.array(z)
        w = np.array(w)
        u, q = O.emtv_denoise(geo, z, w, np.ones(2, np.uint8), 30000, kn)
        d = z[1] - z[0]
        if abs(d) <= 1 / w[0] + 1 / w[1]:
            want = np.full(2, (w[0] * z[0] + w[1] * z[1]) / (w[0] + w[1]))
        else:
            sg = math.copysign(1.0, d)
            want = np.array([z[0] + sg / w[0], z[1] - sg / w[1]])
        # the accelerated method's iterates approach the minimiser as O(1/k)
        np.testing.assert_allclose(u, want, rtol=1e-5, atol=1e-5)


def test_denoise_matches_independent_solver(oracle_mod):
    """A 4 x 3 grid with uneven weights and a voxel pushed to the bound
    u >= 0.  The dual of min_{u >= 0} sum w/2 (u-z)^2 + ||Ku||_{2,1} is the
    smooth concave problem max_{|q_j| <= 1} D(q) with u(q) = max(0, z - K^T q / w)
    and D(q) = sum w/2 (u(q)-z)^2 + <K^T q, u(q)> (gradient K u(q)); scipy's
    SLSQP solves it with the ball constraints, and strong duality makes its
    value the primal optimum.  The oracle's primal objective must equal it
    and its u must equal u(q*)."""
    O = oracle_mod
    n = (4, 3, 1)
    sc, g, tof, _ = tiny(n=n)
    geo = geometry(O, sc, g, tof)
    rng = np.random.default_rng(2)
    V = geo.V
    z = rng.uniform(0.0, 4.0, V)
    z[5] = -1.5  # the minimiser sits on u_5 = 0
    w = rng.uniform(0.5, 3.0, V)
    u, q = O.emtv_denoise(geo, z, w, np.ones(V, np.uint8), 20000, knorm(n))
    nd = 2

    def u_of(qf):
        kt = tv_adjoint(qf.reshape(nd, V), n)
        return np.maximum(0.0, z - kt / w), kt

    def neg_dual(qf):
        uq, kt = u_of(qf)
        val = float(np.sum(0.5 * w * (uq - z) ** 2) + np.dot(kt, uq))
        return -val, -tv_terms(uq, n).reshape(-1)

    def ball(qf):
        Q = qf.reshape(nd, V)
        return 1.0 - np.sum(Q * Q, axis=0)

    def ball_jac(qf):
        Q = qf.reshape(nd, V)
        J = np.zeros((V, nd * V))
        for c in range(nd):
            J[np.arange(V), c * V + np.arange(V)] = -2.0 * Q[c]
        return J

    res = optimize.minimize(neg_dual, np.zeros(nd * V), jac=True, method="SLSQP",
                            constraints=[{"type": "ineq", "fun": ball, "jac": ball_jac}],
                            options={"maxiter": 1000, "ftol": 1e-15})
    assert res.success, res.message
    d_star = -res.fun
    f_or = denoise_objective(u, z, w, n)
    assert u.min() >= 0.0 and u[5] == 0.0
    assert f_or >= d_star - 1e-9 * abs(d_star)  # weak duality
    assert f_or - d_star <= 1e-6 * abs(d_star)
    np.testing.assert_allclose(u, u_of(res.x)[0], atol=1e-4 * np.abs(u).max())
    assert q.shape[0] == nd * V


def test_denoise_optimality_conditions(oracle_mod):
    """The returned dual q certifies the primal u: |q_j| <= 1 with
    q_j = (Ku)_j / |(Ku)_j| where (Ku)_j != 0, and on the free voxels
    w (u - z) + K^T q = 0 where u > 0, >= 0 where u = 0."""
    O = oracle_mod
    n = (6, 5, 3)
    sc, g, tof, _ = tiny(n=n)
    geo = geometry(O, sc, g, tof)
    rng = np.random.default_rng(8)
    V = geo.V
    z = rng.uniform(-0.5, 3.0, V)
    w = rng.uniform(0.3, 2.0, V)
    z[[4, 40, 77]] = -8.0  # voxels held by the bound u >= 0
    w[[4, 40, 77]] = 3.0
    u, q = O.emtv_denoise(geo, z, w, np.ones(V, np.uint8), 20000, knorm(n))
    Q = q.reshape(3, V)
    assert np.sqrt((Q * Q).sum(axis=0)).max() <= 1.0 + 1e-12
    k = tv_terms(u, n)
    nk = np.sqrt((k * k).sum(axis=0))
    big = nk > 1e-3
    np.testing.assert_allclose(Q[:, big], k[:, big] / nk[big], atol=1e-4)
    r = w * (u - z) + tv_adjoint(Q, n)
    pos = u > 1e-6
    assert 0 < np.count_nonzero(~pos) < V
    assert np.abs(r[pos]).max() <= 1e-4 * np.abs(w * z).max()
    assert r[~pos].min() >= -1e-4 * np.abs(w * z).max()


@pytest.mark.parametrize("n", [(4, 3, 1), (6, 5, 3)])
def test_denoise_rate_bound(oracle_mod, n):
    """Chambolle & Pock (2011), Theorem 2: with G uniformly convex of modulus
    gam and tau_0 sigma_0 L^2 < 1, the iterates of their Alg. 2 satisfy
    N^2 ||u_N - u*||^2 <= (1 + eps) (||u* - u_0||^2 / (gam tau_0)^2 + L^2 ||q* - q_0||^2 / gam^2)
    for large N.  Checked with eps = 1 from N = 10 on, u*, q* from a long run."""
    O = oracle_mod
    sc, g, tof, _ = tiny(n=n)
    geo = geometry(O, sc, g, tof)
    V = geo.V
    rng = np.random.default_rng(2)
    z = rng.uniform(0.0, 4.0, V)
    w = rng.uniform(0.5, 3.0, V)
    kn = knorm(n)
    free = np.ones(V, np.uint8)
    us, qs = O.emtv_denoise(geo, z, w, free, 100000, kn)
    gam, tau0 = w.min(), 0.99 / kn
    bound = 2.0 * (np.sum((us - z) ** 2) / (gam * tau0) ** 2 + kn ** 2 * np.sum(qs ** 2) / gam ** 2)
    for N in (10, 30, 100, 300):
        u, _ = O.emtv_denoise(geo, z, w, free, N, kn)
        assert N * N * np.sum((u - us) ** 2) <= bound, N


def _two_voxel_saddle(z, w):
    """Saddle point of min_u sum w/2 (u-z)^2 + |u2 - u1| (positive z): the
    primal of the closed form above and the dual q = w1 (u1 - z1), from
    w1 (u1 - z1) - q = 0 (the first voxel's optimality condition; K^T q =
    (-q, q))."""
    d = z[1] - z[0]
    if abs(d) <= 1 / w[0] + 1 / w[1]:
        u = np.full(2, (w[0] * z[0] + w[1] * z[1]) / (w[0] + w[1]))
    else:
        sg = math.copysign(1.0, d)
        u = np.array([z[0] + sg / w[0], z[1] - sg / w[1]])
    return u, w[0] * (u[0] - z[0])


@pytest.mark.parametrize("z,w", [((0.64, 0.27), (0.0101, 0.0107)), ((0.2, 0.9), (0.01, 0.01)),
                                 ((0.3, 0.8), (0.001, 0.001)), ((1.0, 3.0), (0.3, 0.2)),
                                 ((0.0, 10.0), (0.05, 0.05))])
def test_denoise_nonasymptotic_bound(oracle_mod, z, w):
    """The non-asymptotic inequality behind Chambolle & Pock (2011),
    Theorem 2, for their Alg. 2 with G uniformly convex of modulus gam,
    tau_0 sigma_0 L^2 <= 1 and theta_n = 1/sqrt(1 + 2 gam tau_n):
        ||u_N - u*||^2 <= tau_N^2 (||u* - u_0||^2 / tau_0^2 + ||q* - q_0||^2 / (sigma_0 tau_0))
    for every N >= 0 (summing the one-step inequality: the extrapolation
    makes the coupling terms telescope, and Young's inequality with
    sigma_n tau_n L^2 = sigma_0 tau_0 L^2 <= 1 absorbs the last one).  The
    saddle point (u*, q*) is the two-voxel closed form and tau_N follows the
    theorem's schedule, so nothing on the right comes from the oracle.
    On the first three (weakly weighted) problems the iterates without the
    extrapolation exceed the bound by 30 %, while the accelerated scheme
    stays far below it."""
    O = oracle_mod
    sc, g, tof, _ = tiny(n=(2, 1, 1))
    geo = geometry(O, sc, g, tof)
    z, w = np.array(z), np.array(w)
    u_star, q_star = _two_voxel_saddle(z, w)
    L = knorm(g.n)
    gam, tau, sigma = w.min(), 0.99 / L, 0.99 / L
    rhs = np.sum((u_star - z) ** 2) / tau ** 2 + q_star ** 2 / (sigma * tau)
    for N in range(1, 120):
        tau = tau / math.sqrt(1.0 + 2.0 * gam * tau)  # tau_N
        u, _ = O.emtv_denoise(geo, z, w, np.ones(2, np.uint8), N, L)
        assert np.sum((u - u_star) ** 2) <= tau ** 2 * rhs * (1.0 + 1e-9), N


@pytest.mark.parametrize("z,w", [((0.64, 0.27), (0.9, 1.3)), ((0.2, 0.9), (0.5, 4.0)), ((-0.5, 2.0), (2.0, 1.0)),
                                 ((1.0, 3.0), (0.3, 0.2))])
def test_denoise_first_iterates_exact(oracle_mod, z, w):
    """The iterate path at a fixed iteration count.  On two voxels K u =
    (u2 - u1, 0), so the dual is one scalar q in [-1, 1] (the unit ball of
    one component), K^T q = (-q, q), and Chambolle & Pock's Alg. 2 with
    u_0 = ubar_0 = z, q_0 = 0, tau_0 = sigma_0 = 0.99 / L reads, per
    iteration n:
        q <- clip(q + sigma_n (ubar_2 - ubar_1), -1, 1)
        u_1 <- max(0, (u_1 + tau_n q + tau_n w_1 z_1) / (1 + tau_n w_1))
        u_2 <- max(0, (u_2 - tau_n q + tau_n w_2 z_2) / (1 + tau_n w_2))
        theta_n = 1 / sqrt(1 + 2 gam tau_n),  ubar = u_new + theta_n (u_new - u_old)
        tau_{n+1} = theta_n tau_n,  sigma_{n+1} = sigma_n / theta_n.
    Evaluated here in 40-digit arithmetic for N = 1..10; the oracle's
    iterates (general grid code) must agree to 1e-12.  A wrong theta, a
    missing or altered extrapolation, one iteration too many or too few,
    or a wrong sign of K^T q changes them by far more."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    O = oracle_mod
    sc, g, tof, _ = tiny(n=(2, 1, 1))
    geo = geometry(O, sc, g, tof)
    L = mp.sqrt(2)  # 4 sin^2(pi/4)
    assert abs(float(L) - knorm(g.n)) < 1e-15
    zz = [mp.mpf(v) for v in z]
    ww = [mp.mpf(v) for v in w]
    gam = min(ww)
    u = list(zz)
    ub = list(zz)
    q = mp.mpf(0)
    tau = sigma = mp.mpf("0.99") / L
    for N in range(1, 11):
        q = min(mp.mpf(1), max(mp.mpf(-1), q + sigma * (ub[1] - ub[0])))
        un = [max(mp.mpf(0), (u[0] + tau * q + tau * ww[0] * zz[0]) / (1 + tau * ww[0])),
              max(mp.mpf(0), (u[1] - tau * q + tau * ww[1] * zz[1]) / (1 + tau * ww[1]))]
        theta = 1 / mp.sqrt(1 + 2 * gam * tau)
        ub = [un[k] + theta * (un[k] - u[k]) for k in range(2)]
        u = un
        tau, sigma = theta * tau, sigma / theta
        got_u, got_q = O.emtv_denoise(geo, np.array(z), np.array(w), np.ones(2, np.uint8), N, knorm(g.n))
        want = np.array([float(v) for v in u])
        np.testing.assert_allclose(got_u, want, rtol=1e-12, atol=1e-14, err_msg=f"N={N}")
        assert abs(got_q[0] - float(q)) <= 1e-12, N
        assert got_q[1] == 0.0


def test_denoise_limits(oracle_mod):
    """w -> inf keeps u = max(z, 0); held voxels stay 0."""
    O = oracle_mod
    n = (5, 4, 2)
    sc, g, tof, _ = tiny(n=n)
    geo = geometry(O, sc, g, tof)
    rng = np.random.default_rng(3)
    V = geo.V
    z = rng.uniform(0.2, 3.0, V)
    free = np.ones(V, np.uint8)
    free[[0, 7, 13]] = 0
    u, _ = O.emtv_denoise(geo, z, np.full(V, 1e9), free, 50, knorm(n))
    want = np.where(free > 0, z, 0.0)
    np.testing.assert_allclose(u, want, rtol=0, atol=1e-7 * z.max() * 50)
    assert np.all(u[free == 0] == 0.0)


# --------------------------------------------------------------------------
# the pass over the subsets
# --------------------------------------------------------------------------
def _problem(O, n_sub, seed=6, n=(6, 5, 1)):
    sc, g, tof, ev = tiny(n=n, n_events=300, seed=seed)
    geo = geometry(O, sc, g, tof)
    E = O.EventArrays.from_events(ev)
    sens = O.sens(geo, np.ones(sc.n_lor, np.float32))
    x0 = np.full(geo.V, 0.8 * ev.n / sens.sum())
    return g, geo, E, sens, x0


def test_epoch_small_beta_is_osem(oracle_mod):
    O = oracle_mod
    g, geo, E, sens, x0 = _problem(O, 3)
    osem = O.EMTV(geo, E, 3, beta=0.0, knorm=knorm(g.n)).epoch(x0, sens)
    near = O.EMTV(geo, E, 3, beta=1e-9, knorm=knorm(g.n)).epoch(x0, sens, pdhg_iters=30)
    assert np.linalg.norm(near - osem) <= 1e-6 * np.linalg.norm(osem)
    # and a real prior smooths: the TV of the result drops
    tv = O.EMTV(geo, E, 3, beta=5.0, knorm=knorm(g.n)).epoch(x0, sens, pdhg_iters=100)
    tv_of = lambda u: float(np.sum(np.sqrt(np.sum(tv_terms(u, g.n) ** 2, axis=0))))
    assert tv_of(tv) < 0.8 * tv_of(osem)


@pytest.mark.parametrize("n", [(6, 5, 1), (4, 3, 2)])
def test_epoch_is_composition_of_steps(oracle_mod, n):
    O = oracle_mod
    n_sub, beta, iters = 4, 0.2, 25
    g, geo, E, sens, x0 = _problem(O, n_sub, seed=9, n=n)
    sens[0] = 0.0  # a voxel outside the field of view is held at 0
    em = O.EMTV(geo, E, n_sub, beta=beta, knorm=knorm(g.n))
    x = x0.copy()
    for i in range(n_sub):
        z = em.em_step(x, sens, i)
        free = ((x > 0) & (sens > 0)).astype(np.uint8)
        w = np.where(free > 0, sens / (beta * np.where(x > 0, x, 1.0)), 0.0)
        x, _ = O.emtv_denoise(geo, z, w, free, iters, knorm(g.n))
    got = em.epoch(x0, sens, pdhg_iters=iters)
    np.testing.assert_allclose(got, x, rtol=1e-12, atol=1e-14)
    assert got[0] == 0.0
