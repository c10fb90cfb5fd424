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


# --------------------------------------------------------------------------
# The two tolerance helpers (they state how loose a GPU parity check may be,
# so they are pinned too): both are checked through the forward projector
# alone, under a change of the TOF cut or of the detector positions.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["2d_small", "3d_small"])
def test_tof_edge_distance_is_the_cut_margin(oracle_mod, name):
    """d_e = distance of the event's nearest in-grid sample from the TOF
    truncation edge.  The bin weight does not depend on the cut, only the
    inclusion test |t - c_m| <= W does, so moving the cut W by less than d_e
    leaves (P^LM 1)_e unchanged bit for bit, while moving it by a little more
    than d_e (inwards or outwards, whichever side the nearest sample is on)
    changes it.  The image is all ones so that every in-grid sample
    contributes; the change is checked for d_e < sigma / 2, where the
    crossing sample's bin weight is far from underflowing to 0 in FP64.
    Events without an in-grid sample have d_e = inf and project to 0."""
    O = oracle_mod
    wl = S.workload(name)
    t = S.Tof(8.0, 6.0, 3.0, 61)  # W = 24 mm: n_sigma's float32 resolution moves W by ~2e-6 mm
    ev = S.uniform_events(wl.scanner, t, 600, seed=13)
    E = O.EventArrays.from_events(ev)
    geo = _geo(O, wl, t)
    ones = np.ones(geo.V, np.float32)
    d = O.tof_edge_distance(geo, E)
    p0 = O.fwd(geo, E, ones)
    assert np.all(p0[~np.isfinite(d)] == 0.0)
    fin = np.isfinite(d) & (d > 1e-3)
    assert fin.sum() > 200
    W = t.n_sigma * t.sigma

    def p_with_cut(Wn):
        return O.fwd(_geo(O, wl, S.Tof(t.sigma, t.bin, Wn / t.sigma, t.n_bins)), E, ones)

    # one geometry per distinct cut would be slow: group events by a cut that
    # suits all of them (the margin scales with each event's own d_e)
    for f_in, f_out, must_change in ((0.99, 0.99, False), (1.01, 1.01, True)):
        idx = np.nonzero(fin)[0]
        lo = np.empty(idx.size)
        hi = np.empty(idx.size)
        for k, e in enumerate(idx):
            sub = O.EventArrays(E.det1[e:e + 1], E.det2[e:e + 1], E.tof[e:e + 1], E.corr[e:e + 1])
            lo[k] = O.fwd(_geo(O, wl, S.Tof(t.sigma, t.bin, (W - f_in * d[e]) / t.sigma, t.n_bins)), sub, ones)[0]
            hi[k] = O.fwd(_geo(O, wl, S.Tof(t.sigma, t.bin, (W + f_out * d[e]) / t.sigma, t.n_bins)), sub, ones)[0]
        same = (lo == p0[idx]) & (hi == p0[idx])
        if must_change:
            near = d[idx] < 0.5 * t.sigma
            assert near.sum() > 30
            assert not np.any(same[near])
        else:
            assert np.all(same)


@pytest.mark.parametrize("name", ["2d_small", "3d_small"])
def test_position_sensitivity_is_the_gradient_norm(oracle_mod, name):
    """G_e = corr_e sum_samples step w_tof (|d interp/d u_1| + |d interp/d u_2|),
    u_1, u_2 the secondary voxel coordinates (axes k+1, k+2 mod 3 of the
    principal axis k).  Translating every detector by delta along a
    secondary axis a moves every sample of the event by delta/h_a voxels
    along a and leaves the principal-axis planes and the TOF coordinates
    alone, so (p(delta) - p(0))/delta h_a is the signed sum of d interp/d u_a.
    For the ramp x = 1 + 3 i_x + 5 i_y + 7 i_z (bilinear interpolation of a
    linear function is exact) and events whose samples keep all their
    neighbours inside the grid, every sample's derivative along a is the
    ramp's slope, so |D_1| + |D_2| = G_e; different slopes per axis catch a
    wrong choice of axes.  For a random image, |D_1| + |D_2| <= G_e (triangle
    inequality) away from cell crossings.  An axis of one voxel (z of a 2D
    grid) has no position to round and no term."""
    O = oracle_mod
    wl = S.workload(name)
    sc, g, t = wl.scanner, wl.grid, wl.tof
    t = S.Tof(8.0, 6.0, 3.0, 61)  # a short TOF window: more events keep all samples inside the grid
    ev = S.uniform_events(sc, t, 3000, seed=17)
    E = O.EventArrays.from_events(ev)
    tab = sc.crystal_table().astype(np.float32)
    geo = _geo(O, wl, t)
    nx, ny, nz = g.n
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ramp = (1.0 + 3.0 * ix + 5.0 * iy + 7.0 * iz).astype(np.float32).reshape(-1)
    slope = (3.0, 5.0, 7.0)
    # interior events: enlarging the grid by two voxels on every side (same
    # voxel centres) does not change their projection of ones
    big_n = tuple(m + 4 if m > 1 else m for m in g.n)
    big_o = tuple(o - 2 * hh if m > 1 else o for o, hh, m in zip(g.origin, g.h, g.n))
    geo_big = O.Geometry(tab, sc.n_rings, sc.n_xtal, big_n, g.h, big_o, (t.sigma, t.bin, t.n_sigma, t.n_bins))
    p1 = O.fwd(geo, E, np.ones(geo.V, np.float32))
    p1b = O.fwd(geo_big, E, np.ones(int(np.prod(big_n)), np.float32))
    inner = (p1 > 0) & (np.abs(p1b - p1) <= 1e-13 * p1)
    assert inner.sum() > 40
    # principal axis of each event as the projector defines it (float32 differences)
    dd = (tab[ev.det2] - tab[ev.det1]).astype(np.float32)
    k = np.argmax(np.abs(dd), axis=1)
    delta = 2.0 ** -6  # mm; the shifted float32 coordinates stay exact to ~1e-6 mm

    def deriv(x, axis, sign):
        sh = tab.copy()
        sh[:, axis] += np.float32(sign * delta)
        step = (sh[:, axis].astype(np.float64) - tab[:, axis])  # the shift actually applied per crystal
        geo_s = O.Geometry(sh, sc.n_rings, sc.n_xtal, g.n, g.h, g.origin, (t.sigma, t.bin, t.n_sigma, t.n_bins))
        assert np.all(np.abs(step - sign * delta) <= 1e-6)
        return (O.fwd(geo_s, E, x) - O.fwd(geo, E, x)) / (sign * delta) * g.h[axis]

    ev_i = np.arange(E.n)
    s1, s2 = (k + 1) % 3, (k + 2) % 3
    for x, exact in ((ramp, True), (np.random.default_rng(5).uniform(0, 1, geo.V).astype(np.float32), False)):
        G = O.fwd_position_sensitivity(geo, E, x)
        Dp = np.array([deriv(x, a, +1.0) for a in range(3)])
        Dm = np.array([deriv(x, a, -1.0) for a in range(3)])
        # no sample crosses a cell face within +-delta (else the one-sided
        # derivatives differ, e.g. a sample exactly on the last slice)
        # (an axis of one voxel always has its face at the sample: there the
        # helper, like the forward difference, takes the derivative upwards)
        smooth = np.ones(E.n, bool)
        for s in (s1, s2):
            a, b = Dp[s, ev_i], Dm[s, ev_i]
            flat = np.array([g.n[v] == 1 for v in s])
            smooth &= flat | (np.abs(a - b) <= 1e-5 * (np.abs(a) + np.abs(b) + 1e-12 * G.max()))
        use1 = np.array([g.n[v] > 1 for v in s1])
        use2 = np.array([g.n[v] > 1 for v in s2])
        both = np.where(use1, np.abs(Dp[s1, ev_i]), 0.0) + np.where(use2, np.abs(Dp[s2, ev_i]), 0.0)
        if exact:
            sel = inner & smooth
            assert sel.sum() > 40
            np.testing.assert_allclose(both[sel], G[sel], rtol=1e-4)
            # per axis, the derivative is the ramp's slope times the event's summed weight
            for e in np.nonzero(sel)[0]:
                a1, a2 = s1[e], s2[e]
                if g.n[a1] > 1 and g.n[a2] > 1:
                    assert abs(Dp[a1, e] / Dp[a2, e] - slope[a1] / slope[a2]) <= 1e-3 * slope[a1] / slope[a2]
        else:
            assert smooth.mean() > 0.8
            sel = smooth & (G > 0)
            assert np.all(both[sel] <= G[sel] * (1 + 1e-4))
