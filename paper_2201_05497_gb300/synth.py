"""Seeded synthetic inputs for listmode TOF PET reconstruction.

This module builds the *inputs* of the reconstruction problem and nothing
else: scanner crystal tables, image grids, TOF parameters, phantoms, a Monte
Carlo listmode event stream, per-LOR attenuation factors and the random
update-selection sequence.  It contains none of the reconstruction method's
arithmetic (no projector, no proximal map, no step sizes): events are drawn
by a physical Monte Carlo of positron annihilations (emission point, photon
direction, detector hit, attenuation survival, Gaussian timing noise), which
is independent of the Joseph projector used by the method.  Both the FP64
oracle and the CUDA path consume these arrays unchanged.

Workload shapes follow the paper's experiments (Sec. "Numerical
Experiments"): 400 ps TOF FWHM, 27 TOF bins for the 2D system, a flat
contamination, 28 subsets; the phantom stands in for the brainweb / XCAT
phantoms, which are not available here.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Tuple

import numpy as np

# speed of light in mm/ps; 400 ps FWHM -> sigma = 400 * c/2 / 2.3548 mm
C_MM_PER_PS = 0.299792458
FWHM_TO_SIGMA = 1.0 / (2.0 * math.sqrt(2.0 * math.log(2.0)))


# --------------------------------------------------------------------------
# SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
# generators", OOPSLA 2014).  Used for the random subset selection of
# Alg. 2 (the paper does not name a generator).
# --------------------------------------------------------------------------
_M64 = (1 << 64) - 1


def splitmix64_stream(seed: int, count: int) -> np.ndarray:
    """Return `count` successive SplitMix64 outputs for `seed` (uint64)."""
    out = np.empty(count, dtype=np.uint64)
    s = seed & _M64
    for i in range(count):
        s = (s + 0x9E3779B97F4A7C15) & _M64
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        out[i] = z ^ (z >> 31)
    return out


def selection_sequence(n_subsets: int, n_updates: int, seed: int = 3) -> np.ndarray:
    """Update selection for LM-SPDHG (Alg. 2, "Select i randomly").

    Probabilities follow the paper's choice p_k = 1/(2n) for the n data
    subsets and p_{n+1} = 1/2 for the prior.  Each draw takes a uniform
    u = (r >> 11) * 2^-53 from SplitMix64; u < 1/2 selects the prior
    (encoded as the value n), otherwise subset floor((u - 1/2) * 2n).
    Returns uint16 values in [0, n].
    """
    if n_subsets < 1 or n_subsets > 65534:
        raise ValueError("n_subsets out of range")
    r = splitmix64_stream(seed, n_updates)
    seq = np.empty(n_updates, dtype=np.uint16)
    for t in range(n_updates):
        u = float(int(r[t]) >> 11) * (2.0 ** -53)
        if u < 0.5:
            seq[t] = n_subsets
        else:
            k = int(math.floor((u - 0.5) * 2 * n_subsets))
            seq[t] = min(k, n_subsets - 1)
    return seq


# --------------------------------------------------------------------------
# Geometry descriptions
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Scanner:
    n_rings: int
    n_xtal: int
    radius: float          # mm
    ring_pitch: float      # mm (ignored for one ring)

    @property
    def n_det(self) -> int:
        return self.n_rings * self.n_xtal

    def ring_z(self) -> np.ndarray:
        return (np.arange(self.n_rings) - 0.5 * (self.n_rings - 1)) * self.ring_pitch

    def crystal_table(self) -> np.ndarray:
        """[n_rings*n_xtal, 3] float32 crystal centres, id = ring*n_xtal + c."""
        phi = 2.0 * np.pi * np.arange(self.n_xtal) / self.n_xtal
        xt = self.radius * np.cos(phi)
        yt = self.radius * np.sin(phi)
        z = self.ring_z()
        tab = np.empty((self.n_rings, self.n_xtal, 3), dtype=np.float64)
        tab[:, :, 0] = xt[None, :]
        tab[:, :, 1] = yt[None, :]
        tab[:, :, 2] = z[:, None]
        return tab.reshape(-1, 3).astype(np.float32)

    @property
    def n_pairs(self) -> int:
        return self.n_xtal * (self.n_xtal - 1) // 2

    @property
    def n_lor(self) -> int:
        return self.n_pairs * self.n_rings * self.n_rings


@dataclasses.dataclass
class Grid:
    n: Tuple[int, int, int]        # (nx, ny, nz); x fastest in memory
    h: Tuple[float, float, float]  # voxel size, mm

    @property
    def origin(self) -> Tuple[float, float, float]:
        """Centre of voxel 0 for a grid centred on the scanner axis."""
        return tuple(float(-0.5 * (self.n[d] - 1) * self.h[d]) for d in range(3))

    @property
    def n_vox(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]

    def centres(self):
        o = self.origin
        return [o[d] + self.h[d] * np.arange(self.n[d]) for d in range(3)]


@dataclasses.dataclass
class Tof:
    sigma: float      # mm
    bin: float        # mm (TOF bin width along the LOR)
    n_sigma: float    # truncation of the kernel
    n_bins: int       # odd; 0 = non-TOF

    @property
    def half(self) -> int:
        return (self.n_bins - 1) // 2


def tof_400ps(n_bins: int, bin_mm: float) -> Tof:
    sigma = 400.0 * C_MM_PER_PS / 2.0 * FWHM_TO_SIGMA   # 25.46 mm
    return Tof(sigma=float(np.float32(sigma)), bin=float(np.float32(bin_mm)), n_sigma=3.0,
               n_bins=n_bins)


# --------------------------------------------------------------------------
# Canonical LOR enumeration.  Transaxial crystal pairs {c1, c2}, c1 != c2,
# are numbered by q; ring pairs (r1, r2) are ordered.  LOR index
#   l = q * n_rings^2 + r1 * n_rings + r2,  det1 = r1*n_xtal + c1,
#   det2 = r2*n_xtal + c2.
# For q < n*floor((n-1)/2): off = 1 + q // n, c1 = q % n, c2 = (c1+off) % n.
# Otherwise (even n only): r = q - n*floor((n-1)/2), c1 = r, c2 = r + n/2.
# The same enumeration is written out in the library header.
# --------------------------------------------------------------------------
def pair_of_q(q: np.ndarray, n: int) -> Tuple[np.ndarray, np.ndarray]:
    q = np.asarray(q, dtype=np.int64)
    base = n * ((n - 1) // 2)
    c1 = np.where(q < base, q % n, q - base)
    off = np.where(q < base, 1 + q // n, n // 2)
    c2 = (c1 + off) % n
    return c1, c2


def q_of_pair(c1: np.ndarray, c2: np.ndarray, n: int) -> Tuple[np.ndarray, np.ndarray]:
    """Inverse of pair_of_q.  Returns (q, swapped) where swapped tells that
    the canonical orientation is (c2, c1)."""
    c1 = np.asarray(c1, dtype=np.int64)
    c2 = np.asarray(c2, dtype=np.int64)
    off = (c2 - c1) % n
    half = (n - 1) // 2
    base = n * half
    # orientation (c1 -> c2) is canonical if off <= half, or off == n/2 and c1 < n/2
    direct = (off >= 1) & (off <= half)
    even_mid = (n % 2 == 0) & (off == n // 2)
    q = np.empty_like(c1)
    swapped = np.zeros(c1.shape, dtype=bool)
    # direct orientation
    m = direct
    q[m] = (off[m] - 1) * n + c1[m]
    # reversed orientation: off' = n - off in [1, half]
    m = ~direct & ~even_mid
    offr = (n - off[m])
    q[m] = (offr - 1) * n + c2[m]
    swapped[m] = True
    # diametral pairs (even n)
    m = even_mid
    lo = np.minimum(c1[m], c2[m])
    q[m] = base + lo
    swapped[m] = c1[m] > c2[m]
    return q, swapped


def lor_of_events(sc: Scanner, det1: np.ndarray, det2: np.ndarray) -> np.ndarray:
    r1, c1 = np.divmod(det1.astype(np.int64), sc.n_xtal)
    r2, c2 = np.divmod(det2.astype(np.int64), sc.n_xtal)
    q, sw = q_of_pair(c1, c2, sc.n_xtal)
    ra = np.where(sw, r2, r1)
    rb = np.where(sw, r1, r2)
    return (q * sc.n_rings + ra) * sc.n_rings + rb


# --------------------------------------------------------------------------
# Phantom: an attenuating elliptic body (ellipse in 2D, elliptic cylinder
# along z in 3D, mu = 0.0096/mm) holding an activity region with seeded
# hot/cold inner ellipsoids (activity 0..4).
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Phantom:
    body_axes: Tuple[float, float, float]     # activity region semi-axes (mm)
    att_axes: Tuple[float, float]             # attenuating cylinder semi-axes (mm)
    mu_att: float                             # 1/mm
    inner: List[Tuple[Tuple[float, float, float], Tuple[float, float, float], float]]
    # each inner: (centre, semi-axes, activity)

    @staticmethod
    def seeded(seed: int, body_axes, att_axes, n_inner: int, mu_att: float = 0.0096,
               is2d: bool = False) -> "Phantom":
        rng = np.random.default_rng(seed)
        inner = []
        for _ in range(n_inner):
            ax = [rng.uniform(0.12, 0.3) * body_axes[0], rng.uniform(0.12, 0.3) * body_axes[1],
                  rng.uniform(0.15, 0.35) * body_axes[2] if not is2d else 1.0]
            c = [rng.uniform(-0.5, 0.5) * body_axes[0], rng.uniform(-0.5, 0.5) * body_axes[1],
                 rng.uniform(-0.5, 0.5) * body_axes[2] if not is2d else 0.0]
            inner.append((tuple(c), tuple(ax), float(rng.uniform(0.0, 4.0))))
        return Phantom(tuple(body_axes), tuple(att_axes), mu_att, inner)

    def activity(self, p: np.ndarray, is2d: bool) -> np.ndarray:
        """Activity at points p [..., 3]."""
        bx, by, bz = self.body_axes
        r = (p[..., 0] / bx) ** 2 + (p[..., 1] / by) ** 2
        if not is2d:
            r = r + (p[..., 2] / bz) ** 2
        act = np.where(r <= 1.0, 1.0, 0.0)
        for (c, ax, a) in self.inner:
            ri = ((p[..., 0] - c[0]) / ax[0]) ** 2 + ((p[..., 1] - c[1]) / ax[1]) ** 2
            if not is2d:
                ri = ri + ((p[..., 2] - c[2]) / ax[2]) ** 2
            act = np.where((ri <= 1.0) & (r <= 1.0), a, act)
        return act

    def voxelised(self, grid: Grid, supersample: int = 4) -> np.ndarray:
        """Activity image (x fastest) by supersampled membership, float32."""
        is2d = grid.n[2] == 1
        cx, cy, cz = grid.centres()
        ss = (np.arange(supersample) + 0.5) / supersample - 0.5
        img = np.zeros((grid.n[2], grid.n[1], grid.n[0]), dtype=np.float64)
        zs = [0.0] if is2d else list(ss)
        for dz in zs:
            for dy in ss:
                for dx in ss:
                    Z, Y, X = np.meshgrid(cz + dz * grid.h[2], cy + dy * grid.h[1],
                                          cx + dx * grid.h[0], indexing="ij")
                    p = np.stack([X, Y, Z], axis=-1)
                    img += self.activity(p, is2d)
        img /= (len(zs) * supersample * supersample)
        return img.astype(np.float32).reshape(-1)

    def att_chord_param(self, a: np.ndarray, d: np.ndarray) -> np.ndarray:
        """Length (in units of the line parameter) of the part of the line
        a + t d inside the attenuating elliptic cylinder (infinite along z)."""
        A, B = self.att_axes
        al = (d[..., 0] / A) ** 2 + (d[..., 1] / B) ** 2
        be = 2.0 * (a[..., 0] * d[..., 0] / A ** 2 + a[..., 1] * d[..., 1] / B ** 2)
        ga = (a[..., 0] / A) ** 2 + (a[..., 1] / B) ** 2 - 1.0
        disc = be * be - 4.0 * al * ga
        with np.errstate(invalid="ignore", divide="ignore"):
            dt = np.where((disc > 0) & (al > 0), np.sqrt(np.maximum(disc, 0.0)) / np.where(al > 0, al, 1.0), 0.0)
        return dt


def lor_attenuation(sc: Scanner, ph: Phantom, chunk: int = 1 << 22) -> np.ndarray:
    """exp(-mu * chord) for every canonical LOR, float32 [n_lor].

    The chord through the elliptic cylinder only depends on the transaxial
    pair q and, through the 3D length, on the ring difference."""
    tab = sc.crystal_table().astype(np.float64)
    n = sc.n_xtal
    q = np.arange(sc.n_pairs, dtype=np.int64)
    c1, c2 = pair_of_q(q, n)
    a = tab[c1]          # ring 0 entries carry the transaxial coordinates
    b = tab[c2]
    d = b - a
    dt = ph.att_chord_param(a, d)                       # [n_pairs]
    lxy = np.sqrt(d[:, 0] ** 2 + d[:, 1] ** 2)
    z = sc.ring_z()
    dz = (z[None, :] - z[:, None]).reshape(-1)          # r1*n_rings + r2 -> z[r2]-z[r1]
    out = np.empty(sc.n_lor, dtype=np.float32)
    nr2 = sc.n_rings * sc.n_rings
    for s in range(0, sc.n_pairs, max(1, chunk // nr2)):
        e = min(sc.n_pairs, s + max(1, chunk // nr2))
        L3 = np.sqrt(lxy[s:e, None] ** 2 + dz[None, :] ** 2)
        out[s * nr2:e * nr2] = np.exp(-ph.mu_att * dt[s:e, None] * L3).reshape(-1).astype(np.float32)
    return out


# --------------------------------------------------------------------------
# Monte Carlo listmode events
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Events:
    det1: np.ndarray   # int32
    det2: np.ndarray   # int32
    tof: np.ndarray    # int16 (signed bin, measured from the LOR centre toward det2)
    corr: np.ndarray   # float32 multiplicative correction (attenuation) of the event's LOR
    contam: np.ndarray # float32 expected contamination of the event's bin

    @property
    def n(self) -> int:
        return int(self.det1.shape[0])

    def subset(self, idx) -> "Events":
        return Events(self.det1[idx], self.det2[idx], self.tof[idx], self.corr[idx], self.contam[idx])


def _sample_emissions(rng, ph: Phantom, n: int, is2d: bool) -> np.ndarray:
    bx, by, bz = ph.body_axes
    amax = max([1.0] + [a for (_, _, a) in ph.inner])
    pts = []
    got = 0
    while got < n:
        m = int((n - got) * 1.6 * amax) + 1024
        p = np.empty((m, 3))
        p[:, 0] = rng.uniform(-bx, bx, m)
        p[:, 1] = rng.uniform(-by, by, m)
        p[:, 2] = 0.0 if is2d else rng.uniform(-bz, bz, m)
        act = ph.activity(p, is2d)
        keep = rng.uniform(0.0, amax, m) < act
        p = p[keep]
        pts.append(p)
        got += p.shape[0]
    return np.concatenate(pts)[:n]


def monte_carlo_events(sc: Scanner, ph: Phantom, tof: Tof, n_events: int, seed: int,
                       contamination: float = 0.2, lor_att: np.ndarray | None = None) -> Events:
    """Listmode events of a phantom acquisition.

    Trues: emission point ~ activity, isotropic photon pair direction,
    detection by the crystals nearest to the two cylinder hits (both within
    the axial extent), survival with probability exp(-mu * chord), TOF bin
    round((t + N(0, sigma)) / bin) clipped to the bin range, with t the
    emission position along the crystal-to-crystal line measured from its
    centre toward det2.  A fraction `contamination` of the events is drawn
    uniformly over (LOR, TOF bin); the expected contamination per bin is
    therefore flat, s = n_contam / (n_lor * n_bins).  Event order is
    shuffled (stand-in for chronological order) and each event's detector
    order is random.
    """
    rng = np.random.default_rng(seed)
    is2d = sc.n_rings == 1
    tab64 = sc.crystal_table().astype(np.float64)
    zr = sc.ring_z()
    n_true = int(round((1.0 - contamination) * n_events))
    n_rand = n_events - n_true
    M = tof.half if tof.n_bins > 0 else 0
    zlo = zr[0] - 0.5 * sc.ring_pitch
    zhi = zr[-1] + 0.5 * sc.ring_pitch

    d1s, d2s, tfs = [], [], []
    got = 0
    while got < n_true:
        m = max(4096, int((n_true - got) * 2.5))
        p = _sample_emissions(rng, ph, m, is2d)
        if is2d:
            phi = rng.uniform(0.0, np.pi, m)
            u = np.stack([np.cos(phi), np.sin(phi), np.zeros(m)], axis=1)
        else:
            cz = rng.uniform(-1.0, 1.0, m)
            phi = rng.uniform(0.0, 2.0 * np.pi, m)
            st = np.sqrt(1.0 - cz * cz)
            u = np.stack([st * np.cos(phi), st * np.sin(phi), cz], axis=1)
        uu = u[:, 0] ** 2 + u[:, 1] ** 2
        pu = p[:, 0] * u[:, 0] + p[:, 1] * u[:, 1]
        pp = p[:, 0] ** 2 + p[:, 1] ** 2
        disc = pu * pu - uu * (pp - sc.radius ** 2)
        ok = (uu > 1e-12) & (disc > 0)
        sq = np.sqrt(np.maximum(disc, 0.0))
        with np.errstate(invalid="ignore", divide="ignore"):
            s_lo = (-pu - sq) / np.where(uu > 0, uu, 1.0)
            s_hi = (-pu + sq) / np.where(uu > 0, uu, 1.0)
        h_lo = p + s_lo[:, None] * u
        h_hi = p + s_hi[:, None] * u
        if not is2d:
            ok &= (h_lo[:, 2] >= zlo) & (h_lo[:, 2] < zhi) & (h_hi[:, 2] >= zlo) & (h_hi[:, 2] < zhi)
        # attenuation survival along the full photon-pair line
        dt = ph.att_chord_param(p, u)
        ok &= rng.uniform(0.0, 1.0, m) < np.exp(-ph.mu_att * dt * np.sqrt(np.sum(u * u, axis=1)))

        def det_of(hp):
            ang = np.mod(np.arctan2(hp[:, 1], hp[:, 0]), 2.0 * np.pi)
            c = np.rint(ang * sc.n_xtal / (2.0 * np.pi)).astype(np.int64) % sc.n_xtal
            if is2d:
                r = np.zeros_like(c)
            else:
                r = np.clip(np.floor((hp[:, 2] - zlo) / sc.ring_pitch).astype(np.int64), 0, sc.n_rings - 1)
            return r * sc.n_xtal + c

        da = det_of(h_lo)
        db = det_of(h_hi)
        ok &= (da % sc.n_xtal) != (db % sc.n_xtal)
        da, db, p = da[ok], db[ok], p[ok]
        A = tab64[da]
        B = tab64[db]
        dd = B - A
        Ld = np.sqrt(np.sum(dd * dd, axis=1))
        t_true = np.sum((p - 0.5 * (A + B)) * dd, axis=1) / Ld
        if tof.n_bins > 0:
            tb = np.rint((t_true + rng.normal(0.0, tof.sigma, t_true.shape[0])) / tof.bin)
            tb = np.clip(tb, -M, M).astype(np.int64)
        else:
            tb = np.zeros(t_true.shape[0], dtype=np.int64)
        d1s.append(da)
        d2s.append(db)
        tfs.append(tb)
        got += da.shape[0]
    det1 = np.concatenate(d1s)[:n_true]
    det2 = np.concatenate(d2s)[:n_true]
    tb = np.concatenate(tfs)[:n_true]

    # contamination: uniform over (LOR, TOF bin)
    q = rng.integers(0, sc.n_pairs, n_rand)
    c1, c2 = pair_of_q(q, sc.n_xtal)
    r1 = rng.integers(0, sc.n_rings, n_rand)
    r2 = rng.integers(0, sc.n_rings, n_rand)
    rd1 = r1 * sc.n_xtal + c1
    rd2 = r2 * sc.n_xtal + c2
    rtb = rng.integers(-M, M + 1, n_rand) if tof.n_bins > 0 else np.zeros(n_rand, dtype=np.int64)

    det1 = np.concatenate([det1, rd1])
    det2 = np.concatenate([det2, rd2])
    tb = np.concatenate([tb, rtb])
    # random detector order: swapping the detectors flips the sign of the TOF bin
    sw = rng.uniform(0.0, 1.0, n_events) < 0.5
    det1, det2 = np.where(sw, det2, det1), np.where(sw, det1, det2)
    tb = np.where(sw, -tb, tb)
    perm = rng.permutation(n_events)
    det1, det2, tb = det1[perm], det2[perm], tb[perm]

    n_bins_eff = max(tof.n_bins, 1)
    s_flat = np.float32(n_rand / (sc.n_lor * n_bins_eff)) if n_rand > 0 else np.float32(1e-3)
    if lor_att is None:
        corr = np.ones(n_events, dtype=np.float32)
    else:
        corr = lor_att[lor_of_events(sc, det1, det2)].astype(np.float32)
    return Events(det1.astype(np.int32), det2.astype(np.int32), tb.astype(np.int16), corr,
                  np.full(n_events, s_flat, dtype=np.float32))


def monte_carlo_events_torch(sc: Scanner, ph: Phantom, tof: Tof, n_events: int, seed: int,
                             contamination: float = 0.2, lor_att=None, device="cuda", batch: int = 0):
    """The Monte Carlo of `monte_carlo_events`, run with torch on `device`
    (for the large workloads: the 3D rejection rate is ~98%, which makes
    the numpy version slow).  Same physics and conventions; a different
    random stream, so the lists differ from the numpy version's.  Returns
    an Events of torch tensors on `device`.  lor_att: torch float32 [n_lor]
    on `device` or None."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    f64 = torch.float64
    if batch <= 0:
        # candidates per pass: the 3D acceptance is ~0.2 %, so large passes keep the launch count low
        batch = 1 << (26 if n_events >= 1_000_000 else 22)
    is2d = sc.n_rings == 1
    tab = torch.from_numpy(sc.crystal_table().astype(np.float64)).to(device)
    zr = sc.ring_z()
    zlo = float(zr[0] - 0.5 * sc.ring_pitch)
    zhi = float(zr[-1] + 0.5 * sc.ring_pitch)
    n_true = int(round((1.0 - contamination) * n_events))
    n_rand = n_events - n_true
    M = tof.half if tof.n_bins > 0 else 0
    bx, by, bz = ph.body_axes
    amax = max([1.0] + [a for (_, _, a) in ph.inner])
    A, B = ph.att_axes

    def U(m, lo=0.0, hi=1.0):
        return torch.rand(m, generator=g, device=device, dtype=f64) * (hi - lo) + lo

    def activity(p):
        r = (p[:, 0] / bx) ** 2 + (p[:, 1] / by) ** 2
        if not is2d:
            r = r + (p[:, 2] / bz) ** 2
        act = torch.where(r <= 1.0, 1.0, 0.0).to(f64)
        for (c, ax, a) in ph.inner:
            ri = ((p[:, 0] - c[0]) / ax[0]) ** 2 + ((p[:, 1] - c[1]) / ax[1]) ** 2
            if not is2d:
                ri = ri + ((p[:, 2] - c[2]) / ax[2]) ** 2
            act = torch.where((ri <= 1.0) & (r <= 1.0), torch.full_like(act, a), act)
        return act

    def chord_param(a, d):
        al = (d[:, 0] / A) ** 2 + (d[:, 1] / B) ** 2
        be = 2.0 * (a[:, 0] * d[:, 0] / A ** 2 + a[:, 1] * d[:, 1] / B ** 2)
        ga = (a[:, 0] / A) ** 2 + (a[:, 1] / B) ** 2 - 1.0
        disc = be * be - 4.0 * al * ga
        ok = (disc > 0) & (al > 0)
        return torch.where(ok, torch.sqrt(torch.clamp(disc, min=0.0)) / torch.where(al > 0, al, torch.ones_like(al)),
                           torch.zeros_like(al))

    def det_of(hp):
        ang = torch.remainder(torch.atan2(hp[:, 1], hp[:, 0]), 2.0 * np.pi)
        c = torch.remainder(torch.round(ang * sc.n_xtal / (2.0 * np.pi)).long(), sc.n_xtal)
        if is2d:
            r = torch.zeros_like(c)
        else:
            r = torch.clamp(torch.floor((hp[:, 2] - zlo) / sc.ring_pitch).long(), 0, sc.n_rings - 1)
        return r * sc.n_xtal + c

    rmax = max(bx, by)
    cz_max = 1.0
    if not is2d and rmax < sc.radius:
        chord_min = 2.0 * math.sqrt(sc.radius ** 2 - rmax ** 2)
        t = (zhi - zlo) / chord_min
        cz_max = min(1.0, 1.001 * t / math.sqrt(1.0 + t * t))
    d1s, d2s, tbs = [], [], []
    got = 0
    while got < n_true:
        m = batch
        p = torch.stack([U(m, -bx, bx), U(m, -by, by), torch.zeros(m, device=device, dtype=f64) if is2d
                         else U(m, -bz, bz)], dim=1)
        keep = U(m, 0.0, amax) < activity(p)
        if is2d:
            phi = U(m, 0.0, np.pi)
            u = torch.stack([torch.cos(phi), torch.sin(phi), torch.zeros_like(phi)], dim=1)
        else:
            # Directions are isotropic; only |cos theta| <= cz_max can put both cylinder hits inside the
            # axial extent (the in-plane chord through any emission point is at least chord_min), so
            # drawing cos theta uniformly on [-cz_max, cz_max] leaves the accepted events' distribution
            # unchanged and saves the candidates that would all be rejected.
            cz = U(m, -cz_max, cz_max)
            phi = U(m, 0.0, 2.0 * np.pi)
            st = torch.sqrt(1.0 - cz * cz)
            u = torch.stack([st * torch.cos(phi), st * torch.sin(phi), cz], dim=1)
        uu = u[:, 0] ** 2 + u[:, 1] ** 2
        pu = p[:, 0] * u[:, 0] + p[:, 1] * u[:, 1]
        pp = p[:, 0] ** 2 + p[:, 1] ** 2
        disc = pu * pu - uu * (pp - sc.radius ** 2)
        keep &= (uu > 1e-12) & (disc > 0)
        sq = torch.sqrt(torch.clamp(disc, min=0.0))
        den = torch.where(uu > 0, uu, torch.ones_like(uu))
        h_lo = p + ((-pu - sq) / den)[:, None] * u
        h_hi = p + ((-pu + sq) / den)[:, None] * u
        if not is2d:
            keep &= (h_lo[:, 2] >= zlo) & (h_lo[:, 2] < zhi) & (h_hi[:, 2] >= zlo) & (h_hi[:, 2] < zhi)
        keep &= U(m) < torch.exp(-ph.mu_att * chord_param(p, u) * torch.sqrt((u * u).sum(1)))
        p, h_lo, h_hi = p[keep], h_lo[keep], h_hi[keep]
        da, db = det_of(h_lo), det_of(h_hi)
        ok = torch.remainder(da, sc.n_xtal) != torch.remainder(db, sc.n_xtal)
        da, db, p = da[ok], db[ok], p[ok]
        Aa, Bb = tab[da], tab[db]
        dd = Bb - Aa
        Ld = torch.sqrt((dd * dd).sum(1))
        t_true = ((p - 0.5 * (Aa + Bb)) * dd).sum(1) / Ld
        if tof.n_bins > 0:
            noise = torch.randn(t_true.shape[0], generator=g, device=device, dtype=f64) * tof.sigma
            tb = torch.clamp(torch.round((t_true + noise) / tof.bin), -M, M).long()
        else:
            tb = torch.zeros_like(da)
        d1s.append(da)
        d2s.append(db)
        tbs.append(tb)
        got += int(da.shape[0])
    det1 = torch.cat(d1s)[:n_true]
    det2 = torch.cat(d2s)[:n_true]
    tb = torch.cat(tbs)[:n_true]
    q = torch.randint(0, sc.n_pairs, (n_rand,), generator=g, device=device)
    base = sc.n_xtal * ((sc.n_xtal - 1) // 2)
    c1 = torch.where(q < base, torch.remainder(q, sc.n_xtal), q - base)
    off = torch.where(q < base, 1 + torch.div(q, sc.n_xtal, rounding_mode="floor"),
                      torch.full_like(q, sc.n_xtal // 2))
    c2 = torch.remainder(c1 + off, sc.n_xtal)
    r1 = torch.randint(0, sc.n_rings, (n_rand,), generator=g, device=device)
    r2 = torch.randint(0, sc.n_rings, (n_rand,), generator=g, device=device)
    rtb = (torch.randint(-M, M + 1, (n_rand,), generator=g, device=device) if tof.n_bins > 0
           else torch.zeros(n_rand, dtype=torch.long, device=device))
    det1 = torch.cat([det1, r1 * sc.n_xtal + c1])
    det2 = torch.cat([det2, r2 * sc.n_xtal + c2])
    tb = torch.cat([tb, rtb])
    sw = U(n_events) < 0.5
    det1, det2 = torch.where(sw, det2, det1), torch.where(sw, det1, det2)
    tb = torch.where(sw, -tb, tb)
    perm = torch.randperm(n_events, generator=g, device=device)
    det1, det2, tb = det1[perm], det2[perm], tb[perm]
    n_bins_eff = max(tof.n_bins, 1)
    s_flat = float(np.float32(n_rand / (sc.n_lor * n_bins_eff))) if n_rand > 0 else 1e-3
    if lor_att is None:
        corr = torch.ones(n_events, dtype=torch.float32, device=device)
    else:
        corr = lor_att[lor_of_events_torch(sc, det1, det2)].to(torch.float32)
    return Events(det1.to(torch.int32), det2.to(torch.int32), tb.to(torch.int16), corr,
                  torch.full((n_events,), s_flat, dtype=torch.float32, device=device))


def sinogram_bins(sc: Scanner, tof: Tof, det1: np.ndarray, det2: np.ndarray, tb: np.ndarray) -> np.ndarray:
    """Canonical sinogram bin of each event: b = l * nb + (m + M) with l the
    canonical LOR and m the TOF bin signed toward the canonical det2
    (nb = max(n_bins, 1), M = (nb - 1) / 2)."""
    r1, c1 = np.divmod(det1.astype(np.int64), sc.n_xtal)
    r2, c2 = np.divmod(det2.astype(np.int64), sc.n_xtal)
    _, sw = q_of_pair(c1, c2, sc.n_xtal)
    nb = max(tof.n_bins, 1)
    m = np.where(sw, -tb.astype(np.int64), tb.astype(np.int64)) if tof.n_bins > 0 else np.zeros(det1.shape, np.int64)
    return lor_of_events(sc, det1, det2) * nb + m + (nb - 1) // 2


def sinogram_counts(sc: Scanner, tof: Tof, ev: "Events") -> np.ndarray:
    """Counts d_b of the events in every canonical sinogram bin (uint16)."""
    nb = max(tof.n_bins, 1)
    d = np.bincount(sinogram_bins(sc, tof, ev.det1, ev.det2, ev.tof), minlength=sc.n_lor * nb)
    if d.max(initial=0) > 65535:
        raise ValueError("a sinogram bin holds more than 65535 counts")
    return d.astype(np.uint16)


def lor_of_events_torch(sc: Scanner, det1, det2):
    """Canonical LOR index of events (torch tensors), as lor_of_events."""
    import torch
    n = sc.n_xtal
    d1 = det1.long()
    d2 = det2.long()
    r1, c1 = torch.div(d1, n, rounding_mode="floor"), torch.remainder(d1, n)
    r2, c2 = torch.div(d2, n, rounding_mode="floor"), torch.remainder(d2, n)
    off = torch.remainder(c2 - c1, n)
    half = (n - 1) // 2
    base = n * half
    direct = (off >= 1) & (off <= half)
    even_mid = (off == n // 2) & (n % 2 == 0)
    q = torch.where(direct, (off - 1) * n + c1, (n - off - 1) * n + c2)
    q = torch.where(even_mid, base + torch.minimum(c1, c2), q)
    sw = torch.where(even_mid, c1 > c2, ~direct)
    ra = torch.where(sw, r2, r1)
    rb = torch.where(sw, r1, r2)
    return (q * sc.n_rings + ra) * sc.n_rings + rb


def sinogram_bins_torch(sc: Scanner, tof: Tof, det1, det2, tb):
    """sinogram_bins for torch tensors (int64 canonical bin per event)."""
    import torch
    n = sc.n_xtal
    c1 = torch.remainder(det1.long(), n)
    c2 = torch.remainder(det2.long(), n)
    off = torch.remainder(c2 - c1, n)
    half = (n - 1) // 2
    direct = (off >= 1) & (off <= half)
    even_mid = (off == n // 2) & (n % 2 == 0)
    sw = torch.where(even_mid, c1 > c2, ~direct)
    nb = max(tof.n_bins, 1)
    m = torch.where(sw, -tb.long(), tb.long()) if tof.n_bins > 0 else torch.zeros_like(c1)
    return lor_of_events_torch(sc, det1, det2) * nb + m + (nb - 1) // 2


def lor_attenuation_torch(sc: Scanner, ph: Phantom, device="cuda"):
    """lor_attenuation computed with torch on `device` (float32 [n_lor])."""
    import torch
    tab = torch.from_numpy(sc.crystal_table().astype(np.float64)).to(device)
    n = sc.n_xtal
    q = torch.arange(sc.n_pairs, device=device)
    base = n * ((n - 1) // 2)
    c1 = torch.where(q < base, torch.remainder(q, n), q - base)
    off = torch.where(q < base, 1 + torch.div(q, n, rounding_mode="floor"), torch.full_like(q, n // 2))
    c2 = torch.remainder(c1 + off, n)
    a, b = tab[c1], tab[c2]
    d = b - a
    A, B = ph.att_axes
    al = (d[:, 0] / A) ** 2 + (d[:, 1] / B) ** 2
    be = 2.0 * (a[:, 0] * d[:, 0] / A ** 2 + a[:, 1] * d[:, 1] / B ** 2)
    ga = (a[:, 0] / A) ** 2 + (a[:, 1] / B) ** 2 - 1.0
    disc = be * be - 4.0 * al * ga
    dt = torch.where((disc > 0) & (al > 0), torch.sqrt(torch.clamp(disc, min=0.0)) / al, torch.zeros_like(al))
    lxy = torch.sqrt(d[:, 0] ** 2 + d[:, 1] ** 2)
    z = torch.from_numpy(sc.ring_z()).to(device)
    dz = (z[None, :] - z[:, None]).reshape(-1)
    out = torch.empty(sc.n_lor, dtype=torch.float32, device=device)
    nr2 = sc.n_rings * sc.n_rings
    step = max(1, (1 << 24) // nr2)
    for s in range(0, sc.n_pairs, step):
        e = min(sc.n_pairs, s + step)
        L3 = torch.sqrt(lxy[s:e, None] ** 2 + dz[None, :] ** 2)
        out[s * nr2:e * nr2] = torch.exp(-ph.mu_att * dt[s:e, None] * L3).reshape(-1).to(torch.float32)
    return out


def uniform_events(sc: Scanner, tof: Tof, n_events: int, seed: int) -> Events:
    """Events uniform over (LOR, TOF bin), for operator tests."""
    rng = np.random.default_rng(seed)
    q = rng.integers(0, sc.n_pairs, n_events)
    c1, c2 = pair_of_q(q, sc.n_xtal)
    r1 = rng.integers(0, sc.n_rings, n_events)
    r2 = rng.integers(0, sc.n_rings, n_events)
    M = tof.half if tof.n_bins > 0 else 0
    tb = rng.integers(-M, M + 1, n_events)
    d1 = r1 * sc.n_xtal + c1
    d2 = r2 * sc.n_xtal + c2
    sw = rng.uniform(0, 1, n_events) < 0.5
    d1, d2 = np.where(sw, d2, d1), np.where(sw, d1, d2)
    tb = np.where(sw, -tb, tb)
    corr = rng.uniform(0.3, 1.0, n_events).astype(np.float32)
    contam = rng.uniform(0.01, 0.2, n_events).astype(np.float32)
    return Events(d1.astype(np.int32), d2.astype(np.int32), tb.astype(np.int16), corr, contam)


# --------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    name: str
    scanner: Scanner
    grid: Grid
    tof: Tof
    phantom: Phantom
    n_events: int
    n_subsets: int
    beta: float
    epochs: int


def workload(name: str) -> Workload:
    """The workloads of the paper's experiments, at their sizes, plus
    reduced versions for tests (same structure, fewer crystals/voxels)."""
    tof_bin = 600.0 / 27.0   # 27 TOF bins over a 600 mm ring diameter
    if name == "2d":
        sc = Scanner(1, 256, 300.0, 1.0)
        g = Grid((128, 128, 1), (2.0, 2.0, 2.0))
        ph = Phantom.seeded(1, (110.0, 80.0, 1.0), (110.0, 80.0), 6, is2d=True)
        return Workload(name, sc, g, tof_400ps(27, tof_bin), ph, 200_000, 28, 0.03, 20)
    if name == "3d_short":
        sc = Scanner(36, 672, 410.0, 250.0 / 36.0)
        g = Grid((200, 200, 96), (2.5, 2.5, 2.5))
        ph = Phantom.seeded(1, (190.0, 130.0, 115.0), (190.0, 130.0), 8)
        return Workload(name, sc, g, tof_400ps(41, tof_bin), ph, 10_000_000, 28, 0.03, 10)
    if name == "3d_long":
        sc = Scanner(36, 672, 410.0, 250.0 / 36.0)
        g = Grid((200, 200, 96), (2.5, 2.5, 2.5))
        ph = Phantom.seeded(1, (190.0, 130.0, 115.0), (190.0, 130.0), 8)
        return Workload(name, sc, g, tof_400ps(41, tof_bin), ph, 500_000_000, 56, 0.01, 10)
    # reduced workloads for tests
    if name == "2d_small":
        sc = Scanner(1, 96, 150.0, 1.0)
        g = Grid((45, 37, 1), (4.0, 4.0, 4.0))
        ph = Phantom.seeded(11, (70.0, 50.0, 1.0), (70.0, 50.0), 4, is2d=True)
        return Workload(name, sc, g, tof_400ps(15, tof_bin), ph, 20_000, 7, 0.03, 3)
    if name == "3d_small":
        sc = Scanner(6, 112, 160.0, 8.0)
        g = Grid((37, 33, 11), (5.0, 5.0, 4.0))
        ph = Phantom.seeded(12, (80.0, 60.0, 20.0), (80.0, 60.0), 4)
        return Workload(name, sc, g, tof_400ps(17, tof_bin), ph, 40_000, 7, 0.03, 2)
    if name == "3d_mid":
        sc = Scanner(12, 224, 260.0, 8.0)
        g = Grid((70, 66, 24), (4.0, 4.0, 4.0))
        ph = Phantom.seeded(13, (120.0, 90.0, 40.0), (120.0, 90.0), 6)
        return Workload(name, sc, g, tof_400ps(27, tof_bin), ph, 200_000, 14, 0.03, 2)
    if name == "3d_quad":
        # row length a multiple of 4 (the image kernels' vector path), ragged 32-tiles in x and y
        sc = Scanner(6, 112, 160.0, 8.0)
        g = Grid((44, 36, 10), (5.0, 5.0, 4.0))
        ph = Phantom.seeded(14, (80.0, 60.0, 18.0), (80.0, 60.0), 4)
        return Workload(name, sc, g, tof_400ps(17, tof_bin), ph, 40_000, 7, 0.03, 2)
    raise KeyError(name)


def uniform_x0(grid: Grid, value: float) -> np.ndarray:
    return np.full(grid.n_vox, np.float32(value), dtype=np.float32)
