"""Pins of the oracle's TOF Joseph projector against closed forms and
invariants (no implementation to compare against exists).

Each test pins a different part of J so that a plausible mistake fails at
least one: the adjoint (fwd/back consistency), the TOF-sum identity (kernel
normalisation and telescoping), all-ones and axis-aligned chords (plane count,
step length, index strides), a linear ramp (axis order of the interpolation),
a uniform disk (geometry of oblique lines), point-source localisation (sign of
the TOF coordinate) and detector-swap symmetry.
"""
import itertools
import math

import numpy as np
import pytest

from paper_2201_05497_gb300 import synth as S


def _geo(O, wl, tof=None):
    sc, g, t = wl.scanner, wl.grid, wl.tof if tof is None else tof
    return O.Geometry(sc.crystal_table(), sc.n_rings, sc.n_xtal, g.n, g.h, g.origin,
                      None if t is None else (t.sigma, t.bin, t.n_sigma, t.n_bins))


def _pair_geo(O, a_list, b_list, n, h, origin, tof=None):
    """A 'scanner' whose crystals are the given endpoints: event k joins
    crystal 2k and 2k+1."""
    tab = np.empty((2 * len(a_list), 3), dtype=np.float32)
    tab[0::2] = np.asarray(a_list, dtype=np.float32)
    tab[1::2] = np.asarray(b_list, dtype=np.float32)
    geo = O.Geometry(tab, 1, tab.shape[0], n, h, origin, tof)
    d1 = np.arange(0, tab.shape[0], 2, dtype=np.int32)
    d2 = d1 + 1
    return geo, d1, d2, tab.astype(np.float64)


@pytest.mark.parametrize("name", ["2d_small", "3d_small"])
def test_adjoint(oracle_mod, name):
    O = oracle_mod
    wl = S.workload(name)
    geo = _geo(O, wl)
    ev = S.uniform_events(wl.scanner, wl.tof, 3000, seed=5)
    E = O.EventArrays.from_events(ev)
    rng = np.random.default_rng(7)
    x = rng.uniform(0, 1, geo.V).astype(np.float32)
    v = rng.normal(size=E.n)
    lhs = np.dot(O.fwd(geo, E, x), v)
    rhs = np.dot(x.astype(np.float64), O.back(geo, E, v))
    assert abs(lhs - rhs) <= 1e-12 * np.abs(O.fwd(geo, E, x)).dot(np.abs(v))


@pytest.mark.parametrize("name", ["2d_small", "3d_small"])
def test_tof_sum_equals_nontof(oracle_mod, name):
    """sum_m J^(m) = J^nonTOF when the kernel is untruncated and the bins
    cover the LOR: the bin-integrated Gaussians telescope to 1."""
    O = oracle_mod
    wl = S.workload(name)
    t = wl.tof
    wide = S.Tof(t.sigma, t.bin, 1000.0, 61)  # 61 bins: +-688 mm, far beyond every LOR
    geo = _geo(O, wl, wide)
    geo_nt = _geo(O, wl, S.Tof(t.sigma, t.bin, 3.0, 0))
    rng = np.random.default_rng(3)
    x = rng.uniform(0.2, 1.0, geo.V)
    nl = geo.n_lor
    for l in rng.integers(0, nl, 40):
        d1, d2 = geo.lor_dets(int(l))
        tsum = O.lor_tofsum_fwd(geo, d1, d2, x)
        nt = O.fwd_nontof(geo_nt, [d1], [d2], x)[0]
        assert abs(tsum - nt) <= 1e-12 * max(1.0, abs(nt))


@pytest.mark.parametrize("name", ["2d_small", "3d_small"])
def test_tof_sum_truncation_deficit(oracle_mod, name):
    """With the n_sigma = 3 cut, the per-sample mass lost to excluded bins is
    at most erfc((n_sigma - bin/(2 sigma))/sqrt(2)); for x >= 0 the TOF sum
    therefore lies in [(1 - bound) J^nonTOF, J^nonTOF]."""
    O = oracle_mod
    wl = S.workload(name)
    t = wl.tof
    cut = S.Tof(t.sigma, t.bin, 3.0, 61)
    geo = _geo(O, wl, cut)
    geo_nt = _geo(O, wl, S.Tof(t.sigma, t.bin, 3.0, 0))
    bound = math.erfc((3.0 - t.bin / (2.0 * t.sigma)) / math.sqrt(2.0))
    assert 0.0103 < bound < 0.0105
    rng = np.random.default_rng(4)
    x = rng.uniform(0.2, 1.0, geo.V)
    for l in rng.integers(0, geo.n_lor, 40):
        d1, d2 = geo.lor_dets(int(l))
        tsum = O.lor_tofsum_fwd(geo, d1, d2, x)
        nt = O.fwd_nontof(geo_nt, [d1], [d2], x)[0]
        assert tsum <= nt * (1 + 1e-12) + 1e-12
        assert tsum >= nt * (1.0 - bound) - 1e-12


def _interior_lines(rng, n, h, origin, count, axis=0, margin=1.0):
    """Random lines mostly along `axis` whose secondary coordinates stay within
    [margin, n-1-margin] voxel units at every plane of the grid."""
    lo = [origin[d] + margin * h[d] for d in range(3)]
    hi = [origin[d] + (n[d] - 1 - margin) * h[d] for d in range(3)]
    a_list, b_list = [], []
    R = 10.0 * max(n[d] * h[d] for d in range(3))
    ak = origin[axis] - 0.37 * R
    bk = origin[axis] + (n[axis] - 1) * h[axis] + 0.41 * R
    while len(a_list) < count:
        a = np.zeros(3)
        b = np.zeros(3)
        a[axis], b[axis] = ak, bk
        for d in range(3):
            if d == axis:
                continue
            if n[d] == 1:
                a[d] = b[d] = origin[d]
                continue
            # endpoints of the in-grid part chosen inside, then extrapolated linearly
            e0 = rng.uniform(lo[d], hi[d])
            e1 = rng.uniform(lo[d], hi[d])
            k0 = origin[axis]
            k1 = origin[axis] + (n[axis] - 1) * h[axis]
            slope = (e1 - e0) / (k1 - k0)
            a[d] = e0 + slope * (ak - k0)
            b[d] = e0 + slope * (bk - k0)
        # float32 endpoints: recheck the interior condition in FP64 on the rounded values
        af = a.astype(np.float32).astype(np.float64)
        bf = b.astype(np.float32).astype(np.float64)
        ok = True
        for i in range(n[axis]):
            qk = origin[axis] + i * h[axis]
            lam = (qk - af[axis]) / (bf[axis] - af[axis])
            for d in range(3):
                if d == axis or n[d] == 1:
                    continue
                u = (af[d] + lam * (bf[d] - af[d]) - origin[d]) / h[d]
                if not (0.0 <= u <= n[d] - 1):
                    ok = False
        if ok:
            a_list.append(af)
            b_list.append(bf)
    return a_list, b_list


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_all_ones_chord(oracle_mod, axis):
    """Through an all-ones image, a line whose secondary coordinates stay
    within the voxel-centre range collects exactly n_k * step."""
    O = oracle_mod
    n, h = (9, 11, 7), (4.0, 3.0, 5.0)
    origin = tuple(-0.5 * (n[d] - 1) * h[d] for d in range(3))
    rng = np.random.default_rng(10 + axis)
    a_l, b_l = _interior_lines(rng, n, h, origin, 12, axis=axis, margin=0.0)
    geo, d1, d2, tab = _pair_geo(O, a_l, b_l, n, h, origin)
    got = O.fwd_nontof(geo, d1, d2, np.ones(geo.V))
    for k in range(len(a_l)):
        d = tab[2 * k + 1] - tab[2 * k]
        L = np.linalg.norm(d)
        expect = n[axis] * h[axis] * L / abs(d[axis])
        assert abs(got[k] - expect) <= 1e-12 * expect


def test_axis_aligned_row_sums(oracle_mod):
    """An axis-parallel line through voxel centres gives h_k times the sum of
    the voxel row it runs along (catches stride / index mistakes)."""
    O = oracle_mod
    n, h = (6, 5, 4), (4.0, 2.0, 8.0)
    origin = tuple(-0.5 * (n[d] - 1) * h[d] for d in range(3))
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 1, n[0] * n[1] * n[2])
    X = x.reshape(n[2], n[1], n[0])
    c = [origin[d] + h[d] * np.arange(n[d]) for d in range(3)]
    R = 100.0
    a_l, b_l, expect = [], [], []
    for j in range(n[1]):
        for k in range(n[2]):
            a_l.append([-R, c[1][j], c[2][k]])
            b_l.append([R, c[1][j], c[2][k]])
            expect.append(h[0] * X[k, j, :].sum())
    for i in range(n[0]):
        for k in range(n[2]):
            a_l.append([c[0][i], -R, c[2][k]])
            b_l.append([c[0][i], R, c[2][k]])
            expect.append(h[1] * X[k, :, i].sum())
    for i in range(n[0]):
        for j in range(n[1]):
            a_l.append([c[0][i], c[1][j], R])
            b_l.append([c[0][i], c[1][j], -R])
            expect.append(h[2] * X[:, j, i].sum())
    geo, d1, d2, _ = _pair_geo(O, a_l, b_l, n, h, origin)
    got = O.fwd_nontof(geo, d1, d2, x)
    np.testing.assert_allclose(got, expect, rtol=1e-13, atol=0)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_linear_ramp_closed_form(oracle_mod, axis):
    """Bilinear interpolation reproduces a linear image exactly, so for an
    interior line J(ramp) = step * sum_i ramp(p_i) with p_i = a + lambda_i d
    (an arithmetic series).  Distinct slopes per axis catch transposed axes."""
    O = oracle_mod
    n, h = (10, 8, 6), (3.0, 4.0, 5.0)
    # the grid is passed as float32: use the rounded origin on both sides
    origin = tuple(float(np.float32(-0.5 * (n[d] - 1) * h[d] + 1.3 * d)) for d in range(3))
    alpha = np.array([0.7, -1.9, 3.1])
    delta = 40.0
    cz, cy, cx = np.meshgrid(*[origin[d] + h[d] * np.arange(n[d]) for d in (2, 1, 0)], indexing="ij")
    ramp = (alpha[0] * cx + alpha[1] * cy + alpha[2] * cz + delta).reshape(-1)
    rng = np.random.default_rng(20 + axis)
    a_l, b_l = _interior_lines(rng, n, h, origin, 10, axis=axis, margin=0.0)
    geo, d1, d2, tab = _pair_geo(O, a_l, b_l, n, h, origin)
    got = O.fwd_nontof(geo, d1, d2, ramp)
    for k in range(len(a_l)):
        a, b = tab[2 * k], tab[2 * k + 1]
        d = b - a
        nk = n[axis]
        sum_lam = (nk * (origin[axis] - a[axis]) + h[axis] * nk * (nk - 1) / 2.0) / d[axis]
        sum_p = nk * a + sum_lam * d
        step = h[axis] * np.linalg.norm(d) / abs(d[axis])
        expect = step * (alpha.dot(sum_p) + nk * delta)
        assert abs(got[k] - expect) <= 1e-11 * abs(expect)


def test_uniform_disk_chords(oracle_mod):
    """A supersampled uniform disk of radius r: the line integral at distance
    d from its centre is 2 sqrt(r^2 - d^2) within 2h (discretisation)."""
    O = oracle_mod
    n, h = (96, 96, 1), (1.0, 1.0, 1.0)
    origin = (-47.5, -47.5, 0.0)
    r = 30.0
    cx, cy = 3.0, -2.0
    ss = (np.arange(8) + 0.5) / 8 - 0.5
    xs = origin[0] + np.arange(n[0])
    ys = origin[1] + np.arange(n[1])
    img = np.zeros((n[1], n[0]))
    for dy in ss:
        for dx in ss:
            Y, X = np.meshgrid(ys + dy, xs + dx, indexing="ij")
            img += ((X - cx) ** 2 + (Y - cy) ** 2 <= r * r)
    img = (img / 64.0).reshape(-1)
    rng = np.random.default_rng(2)
    R = 200.0
    a_l, b_l, dist = [], [], []
    for _ in range(60):
        th = rng.uniform(0, np.pi)
        dd = rng.uniform(-0.95 * r, 0.95 * r)
        u = np.array([np.cos(th), np.sin(th)])
        nrm = np.array([-u[1], u[0]])
        c0 = np.array([cx, cy]) + dd * nrm
        a_l.append([*(c0 - R * u), 0.0])
        b_l.append([*(c0 + R * u), 0.0])
        dist.append(dd)
    geo, d1, d2, _ = _pair_geo(O, a_l, b_l, n, h, origin)
    got = O.fwd_nontof(geo, d1, d2, img)
    expect = 2.0 * np.sqrt(r * r - np.asarray(dist) ** 2)
    assert np.max(np.abs(got - expect)) <= 2.0 * h[0]
    # and the discretisation error is unbiased on average
    assert abs(np.mean(got - expect)) < 0.2


def test_tof_localises_point_source(oracle_mod):
    """A point source at t_src along det1->det2 (measured from the LOR centre)
    is seen most strongly in bin round(t_src / bin); the signs agree."""
    O = oracle_mod
    wl = S.workload("2d_small")
    t = wl.tof
    n, h, origin = wl.grid.n, wl.grid.h, wl.grid.origin
    V = n[0] * n[1]
    rng = np.random.default_rng(8)
    a_l, b_l, src_t, x_list = [], [], [], []
    for _ in range(12):
        i, j = rng.integers(8, n[0] - 8), rng.integers(8, n[1] - 8)
        src = np.array([origin[0] + i * h[0], origin[1] + j * h[1], 0.0])
        th = rng.uniform(0, np.pi)
        u = np.array([np.cos(th), np.sin(th), 0.0])
        a = src - 140.0 * u + rng.uniform(-40, 40) * u
        b = a + 300.0 * u
        a_l.append(a)
        b_l.append(b)
        af, bf = a.astype(np.float32).astype(float), b.astype(np.float32).astype(float)
        L = np.linalg.norm(bf - af)
        src_t.append(np.dot(src - 0.5 * (af + bf), (bf - af) / L))
        img = np.zeros(V, np.float32)
        img[j * n[0] + i] = 1.0
        x_list.append(img)
    geo, d1, d2, _ = _pair_geo(O, a_l, b_l, n, h, origin, (t.sigma, t.bin, t.n_sigma, t.n_bins))
    M = t.half
    for k in range(len(a_l)):
        vals = []
        for m in range(-M, M + 1):
            E = O.EventArrays([d1[k]], [d2[k]], [m])
            vals.append(O.fwd(geo, E, x_list[k])[0])
        best = int(np.argmax(vals)) - M
        assert best == int(np.rint(src_t[k] / t.bin)) or abs(src_t[k] / t.bin - np.rint(src_t[k] / t.bin)) > 0.45


@pytest.mark.parametrize("name", ["2d_small", "3d_small"])
def test_detector_swap_symmetry(oracle_mod, name):
    """(det1, det2, m) and (det2, det1, -m) are the same data bin."""
    O = oracle_mod
    wl = S.workload(name)
    geo = _geo(O, wl)
    ev = S.uniform_events(wl.scanner, wl.tof, 500, seed=9)
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 1, geo.V).astype(np.float32)
    a = O.fwd(geo, O.EventArrays(ev.det1, ev.det2, ev.tof), x)
    b = O.fwd(geo, O.EventArrays(ev.det2, ev.det1, -ev.tof), x)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)


def test_canonical_lor_enumeration(oracle_mod):
    """The canonical LOR order covers every unordered transaxial pair exactly
    once for every ring pair; the oracle's decoder and the generator's
    encoder are inverse."""
    O = oracle_mod
    for n_x, n_r in [(12, 1), (11, 3), (16, 2)]:
        sc = S.Scanner(n_r, n_x, 100.0, 5.0)
        geo = O.Geometry(sc.crystal_table(), n_r, n_x, (4, 4, 1), (1, 1, 1), (0, 0, 0))
        assert geo.n_lor == n_x * (n_x - 1) // 2 * n_r * n_r
        seen = set()
        d1s, d2s = [], []
        for l in range(geo.n_lor):
            d1, d2 = geo.lor_dets(l)
            c1, c2 = d1 % n_x, d2 % n_x
            assert c1 != c2
            key = (min(c1, c2), max(c1, c2), d1 // n_x if c1 < c2 else d2 // n_x,
                   d2 // n_x if c1 < c2 else d1 // n_x)
            assert key not in seen
            seen.add(key)
            d1s.append(d1)
            d2s.append(d2)
        expect = {(a, b, ra, rb) for a, b in itertools.combinations(range(n_x), 2)
                  for ra in range(n_r) for rb in range(n_r)}
        assert seen == expect
        l_back = S.lor_of_events(sc, np.array(d1s), np.array(d2s))
        np.testing.assert_array_equal(l_back, np.arange(geo.n_lor))
        l_sw = S.lor_of_events(sc, np.array(d2s), np.array(d1s))
        np.testing.assert_array_equal(l_sw, np.arange(geo.n_lor))


def test_sensitivity_is_tof_summed_backprojection(oracle_mod):
    """<P^T 1, x> equals the sum over all canonical LORs of c_l times the TOF
    sum of the LOR's projections of x (each bin projected on its own)."""
    O = oracle_mod
    wl = S.workload("2d_small")
    geo = _geo(O, wl)
    lf = S.lor_attenuation(wl.scanner, wl.phantom)
    sens = O.sens(geo, lf)
    rng = np.random.default_rng(5)
    x = rng.uniform(0, 1, geo.V)
    total = 0.0
    for l in range(geo.n_lor):
        d1, d2 = geo.lor_dets(l)
        total += float(lf[l]) * O.lor_tofsum_fwd(geo, d1, d2, x)
    assert abs(np.dot(sens, x) - total) <= 1e-11 * abs(total)
    assert np.all(sens >= 0)
