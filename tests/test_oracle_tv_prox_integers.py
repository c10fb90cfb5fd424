"""Pins of the oracle's TV operator, proximal maps, event counts, subset
split and selection sequence (closed forms, brute force, published values)."""
import collections
import math
import os

import numpy as np
import pytest
from scipy import optimize

from paper_2201_05497_gb300 import synth as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _grid_geo(O, n):
    h = (1.0, 1.0, 1.0)
    return O.Geometry(np.zeros((2, 3), np.float32), 1, 2, n, h, (0.0, 0.0, 0.0))


def _knorm_closed(n):
    """||K||^2 = sum_d 4 sin^2(pi (n_d - 1) / (2 n_d)) for forward differences
    with a Neumann boundary (largest eigenvalue of the 1D Laplacian with
    reflecting ends, summed over axes)."""
    return math.sqrt(sum(4.0 * math.sin(math.pi * (m - 1) / (2.0 * m)) ** 2 for m in n if m > 1))


@pytest.mark.parametrize("n", [(7, 5, 1), (4, 6, 3), (9, 1, 1)])
def test_tv_adjoint(oracle_mod, n):
    O = oracle_mod
    geo = _grid_geo(O, n)
    rng = np.random.default_rng(1)
    x = rng.normal(size=geo.V)
    q = rng.normal(size=geo.ndim * geo.V)
    lhs = np.dot(O.tv_grad(geo, x), q)
    rhs = np.dot(x, O.tv_adj(geo, q))
    assert abs(lhs - rhs) <= 1e-13 * (np.abs(x).sum() * np.abs(q).sum() / geo.V + 1)


def test_tv_grad_of_ramps(oracle_mod):
    """K applied to the coordinate ramps: 1 in the ramp's own component except
    on the last index (Neumann boundary), 0 in the other components."""
    O = oracle_mod
    n = (5, 4, 3)
    geo = _grid_geo(O, n)
    Z, Y, X = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    for d, R in enumerate([X, Y, Z]):
        g = O.tv_grad(geo, R.reshape(-1).astype(float)).reshape(3, n[2], n[1], n[0])
        for c in range(3):
            expect = np.zeros_like(g[c])
            if c == d:
                expect = (R < n[d] - 1).astype(float)
            np.testing.assert_array_equal(g[c], expect)


@pytest.mark.parametrize("n", [(4, 5, 3), (6, 7, 1), (3, 3, 3)])
def test_knorm_dense_spectral_norm(oracle_mod, n):
    """Brute force: the dense matrix of K (built column by column) has the
    closed-form spectral norm."""
    O = oracle_mod
    geo = _grid_geo(O, n)
    Kmat = np.zeros((geo.ndim * geo.V, geo.V))
    for j in range(geo.V):
        e = np.zeros(geo.V)
        e[j] = 1.0
        Kmat[:, j] = O.tv_grad(geo, e)
    assert abs(np.linalg.norm(Kmat, 2) - _knorm_closed(n)) <= 1e-12


@pytest.mark.parametrize("n", [(16, 12, 1), (10, 9, 8), (128, 128, 1)])
def test_knorm_power_iteration(oracle_mod, n):
    """The power iteration's Rayleigh quotient never exceeds ||K||^2 and
    approaches it; the error after k iterations is O(1/(n sqrt(k)))."""
    O = oracle_mod
    geo = _grid_geo(O, n)
    exact = _knorm_closed(n)
    prev = 0.0
    for it in (10, 100, 1000):
        est = O.knorm_power(geo, it)
        assert est <= exact * (1 + 1e-14)
        assert est >= prev - 1e-12
        prev = est
    assert (exact - prev) / exact < 2e-3 / math.sqrt(1000) * 10


def test_prox_rstar(oracle_mod):
    """beta prox_{R^*}(w/beta) = w / max(1, |w|/beta): projection onto the
    ball of radius beta per voxel; idempotent; the identity inside."""
    O = oracle_mod
    geo = _grid_geo(O, (6, 5, 4))
    rng = np.random.default_rng(2)
    w = rng.normal(scale=0.1, size=geo.ndim * geo.V)
    beta = 0.07
    p = O.tv_prox(geo, w, beta)
    nrm = np.sqrt((p.reshape(geo.ndim, -1) ** 2).sum(0))
    assert np.all(nrm <= beta * (1 + 1e-14))
    np.testing.assert_allclose(O.tv_prox(geo, p, beta), p, rtol=1e-15, atol=1e-18)
    nin = np.sqrt((w.reshape(geo.ndim, -1) ** 2).sum(0)) <= beta
    W, P = w.reshape(geo.ndim, -1), p.reshape(geo.ndim, -1)
    np.testing.assert_array_equal(P[:, nin], W[:, nin])
    # outside: same direction, norm beta
    out = ~nin
    np.testing.assert_allclose(nrm[out], beta, rtol=1e-14)
    cos = (W[:, out] * P[:, out]).sum(0) / (np.sqrt((W[:, out] ** 2).sum(0)) * nrm[out])
    np.testing.assert_allclose(cos, 1.0, rtol=1e-14)
    assert np.all(O.tv_prox(geo, w, 0.0) == 0.0)


def _dstar(v, d):
    """Convex conjugate of the Poisson term D(u) = u - d log u (Sec. 1)."""
    if d > 0:
        return -d + d * math.log(d / (1.0 - v)) if v < 1 else math.inf
    return 0.0 if v <= 1 else math.inf


@pytest.mark.parametrize("a,S,d", [(0.3, 0.5, 1.0), (-4.0, 2.0, 3.0), (2.5, 0.01, 1.0),
                                   (0.99, 10.0, 2.0), (-100.0, 1e-3, 1.0), (5.0, 1.0, 0.0)])
def test_prox_dstar_against_minimisation(oracle_mod, a, S, d):
    """Eq. (proxD) against direct 1D minimisation of
    (v - a)^2 / (2 S) + D^*(v; d) (weighted prox definition, Sec. 1)."""
    O = oracle_mod
    got = O.prox_dstar(a, S, d)
    if d > 0:
        f = lambda v: (v - a) ** 2 / (2 * S) + _dstar(v, d)
        # the derivative (v - a)/S + d/(1 - v) is increasing on v < 1
        g = lambda v: (v - a) / S + d / (1.0 - v)
        lo = min(a, 0.0) - 10.0
        hi = 1.0 - 1e-15
        root = optimize.brentq(g, lo, hi, xtol=1e-15, rtol=1e-15, maxiter=500)
        assert abs(got - root) <= 1e-10 * max(1.0, abs(root))
        assert f(got) <= f(root) + 1e-12
    else:
        # d = 0: the prox is the projection onto v <= 1
        assert abs(got - min(a, 1.0)) <= 1e-15


def test_prox_dstar_fixed_point_with_counts(oracle_mod):
    """Reading of the listmode prox with duplicates (appendix: d^LM = 1 with
    step mu S): with u = (Px+s)_e and y = 1 - mu/u (Eq. yinit) the prox returns
    y unchanged.  The literal 4 S_e (without mu) fails this for mu > 1."""
    O = oracle_mod
    rng = np.random.default_rng(3)
    for _ in range(200):
        u = rng.uniform(0.01, 50.0)
        mu = int(rng.integers(1, 6))
        S = rng.uniform(1e-3, 10.0)
        y = 1.0 - mu / u
        assert abs(O.prox_dstar(y + S * u, mu * S, 1.0) - y) <= 1e-9 * max(1.0, abs(y))
        if mu > 1:
            assert abs(O.prox_dstar(y + S * u, S, 1.0) - y) > 1e-6


def test_event_counts_bruteforce(oracle_mod):
    """mu_e = number of events of the whole list in the same data bin
    (unordered detector pair and TOF bin; footnote of Sec. "Listmode SPDHG")."""
    O = oracle_mod
    wl = S.workload("2d_small")
    ev = S.monte_carlo_events(wl.scanner, wl.phantom, wl.tof, 5000, seed=4)
    key = []
    for a, b, t in zip(ev.det1.tolist(), ev.det2.tolist(), ev.tof.tolist()):
        key.append((a, b, t) if a < b else (b, a, -t))
    cnt = collections.Counter(key)
    expect = np.array([cnt[k] for k in key], dtype=np.int32)
    mu = O.event_counts(ev.det1, ev.det2, ev.tof)
    np.testing.assert_array_equal(mu, expect)
    assert mu.max() > 1


@pytest.mark.parametrize("N,n", [(100, 7), (7, 7), (5, 8), (1000, 28), (0, 3)])
def test_subset_permutation(oracle_mod, N, n):
    """Every n-th event of the list goes to the n-th sub list (Sec. "Listmode
    SPDHG"); in subset-contiguous order event e sits at offset(e mod n) + e div n."""
    O = oracle_mod
    lists = [list(range(k, N, n)) for k in range(n)]
    order = [e for l in lists for e in l]
    perm = O.subset_permutation(N, n)
    inv = np.empty(N, dtype=np.int64)
    inv[perm] = np.arange(N)
    np.testing.assert_array_equal(inv, np.array(order, dtype=np.int64))
    off = O.subset_offsets(N, n)
    np.testing.assert_array_equal(np.diff(off), [len(l) for l in lists])


def test_splitmix64_published_values():
    with open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) as f:
        vals = [int(l, 16) for l in f if l.strip() and not l.startswith("#")]
    got = [int(v) for v in S.splitmix64_stream(0, len(vals))]
    assert got == vals


def test_selection_sequence_distribution():
    n = 28
    seq = S.selection_sequence(n, 200_000, seed=3)
    assert seq.min() >= 0 and seq.max() <= n
    frac_prior = np.mean(seq == n)
    assert abs(frac_prior - 0.5) < 0.005
    counts = np.bincount(seq[seq < n], minlength=n)
    assert np.all(np.abs(counts / counts.sum() - 1.0 / n) < 0.003)
    np.testing.assert_array_equal(seq[:56], S.selection_sequence(n, 56, seed=3))
