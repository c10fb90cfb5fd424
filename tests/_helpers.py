"""Shared fixtures for the GPU parity tests: seeded workloads, the oracle's
view of them and the tolerance rules.

Tolerances (written here once, used by every parity test):
  * per-event projections: |p_gpu - p_oracle| <= 1e-5 |p_oracle| (events with
    |p_oracle| < 1e-6 max|p|: 1e-5 max|p| absolute) plus the float32
    position term 4 ulp(n_max) * G_e, where G_e (from the oracle) is the
    sensitivity of p_e to a one-voxel shift of its sample positions and
    ulp(n_max) the float32 resolution of the largest voxel coordinate; at
    most 0.5 % of the events may need the position term.  Events whose
    nearest sample lies within 1e-3 mm of the TOF truncation edge may differ
    by one sample's weight (float32 and FP64 can decide the cut differently);
  * images after N epochs: relative L2 error <= 1e-3;
  * integer / index outputs: bit-exact.
"""
from __future__ import annotations

import functools
import math

import numpy as np

from paper_2201_05497_gb300 import synth as S

REL_EVENT = 1e-5
FLOOR = 1e-6
EDGE_MM = 1e-3
REL_L2_IMAGE = 1e-3


def knorm_closed(n) -> float:
    """||K|| of forward differences with a Neumann boundary, in closed form."""
    return math.sqrt(sum(4.0 * math.sin(math.pi * (m - 1) / (2.0 * m)) ** 2 for m in n if m > 1))


@functools.lru_cache(maxsize=None)
def workload_data(name: str, n_events: int | None = None, seed: int = 2):
    wl = S.workload(name)
    lf = S.lor_attenuation(wl.scanner, wl.phantom)
    n = wl.n_events if n_events is None else n_events
    ev = S.monte_carlo_events(wl.scanner, wl.phantom, wl.tof, n, seed, lor_att=lf)
    return wl, lf, ev


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def position_eps(n_max: int) -> float:
    """4 ulp of a float32 voxel coordinate of magnitude up to n_max."""
    return 4.0 * 2.0 ** (math.ceil(math.log2(max(n_max, 2))) - 23)


def check_event_projections(p_gpu, p_or, edge_dist, one_sample_bound, sens=None, n_max=256):
    """Apply the per-event tolerance rule; returns (n_checked, n_edge, worst
    relative error among events that meet the pure relative bound)."""
    p_gpu = np.asarray(p_gpu, dtype=np.float64)
    p_or = np.asarray(p_or, dtype=np.float64)
    pmax = np.max(np.abs(p_or)) if p_or.size else 0.0
    err = np.abs(p_gpu - p_or)
    edge = edge_dist < EDGE_MM
    big = np.abs(p_or) >= FLOOR * pmax
    tol_rel = np.where(big, REL_EVENT * np.abs(p_or), REL_EVENT * pmax)
    pos = 0.0 if sens is None else position_eps(n_max) * np.asarray(sens)
    tol = tol_rel + pos
    need_pos = (~edge) & (err > tol_rel)
    if need_pos.sum() > 0.005 * max(1, p_or.size):
        raise AssertionError(f"{need_pos.sum()} events need the float32 position term (> 0.5 %)")
    bad = (~edge) & (err > tol)
    if np.any(bad):
        i = np.flatnonzero(bad)[:5]
        raise AssertionError(f"{bad.sum()} events beyond tolerance; e.g. idx {i}: gpu {p_gpu[i]} oracle {p_or[i]}")
    bad_edge = edge & (err > one_sample_bound + tol)
    if np.any(bad_edge):
        raise AssertionError(f"{bad_edge.sum()} boundary events beyond the one-sample bound")
    rel = np.where(big, err / np.maximum(np.abs(p_or), 1e-300), err / max(pmax, 1e-300))
    ok = (~edge) & (~need_pos)
    worst = float(np.max(rel[ok])) if ok.any() else 0.0
    return int((~edge).sum()), int(edge.sum()), worst
