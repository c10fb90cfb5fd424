"""FP64 CPU oracle for the LM-SPDHG hot path (Python side).

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product
library never does, and this package never imports the product library.

The arithmetic lives in ``lmoracle.c`` (plain double precision C, built with
gcc on first use); this module only marshals numpy arrays.  Functions follow
the paper's notation: ``fwd`` is P^LM (Eq. lmop), ``back`` its adjoint,
``sens`` is P^T 1, ``lm_init``/``lm_update`` are Alg. 2, ``sino_*`` are
Alg. 1 on a full TOF sinogram, ``dtv_*`` the directional TV operator (the
paper's second prior; ``xi`` of ``LM``/``Sino``), ``EMTV``/``emtv_denoise`` are Alg. 3 (the
listmode EM-TV warm start).  Every function is pinned by the CPU tests,
including the denoiser's iterate path at a fixed iteration count and the two
tolerance helpers ``tof_edge_distance`` and ``fwd_position_sensitivity``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lmoracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_LIB_OMP_PATH = os.path.join(_HERE, "liboracle_omp.so")
_lock = threading.Lock()
_libs = {}
_threads = 1


def _compile(out: str, extra) -> None:
    if not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", *extra, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable C, no target-specific flags):
    liboracle.so, single-threaded (every parity test uses it), and
    liboracle_omp.so, the same source with OpenMP (event loops over
    thread-private FP64 images added in thread order, voxel loops split):
    used only to time the oracle on all host cores."""
    if force:
        for f in (_LIB_PATH, _LIB_OMP_PATH):
            if os.path.exists(f):
                os.remove(f)
    _compile(_LIB_PATH, [])
    try:
        _compile(_LIB_OMP_PATH, ["-fopenmp"])
    except (subprocess.CalledProcessError, OSError):
        pass  # no OpenMP in this compiler: the timing baseline stays single-threaded
    return _LIB_PATH


def use_threads(n: int) -> int:
    """Select the OpenMP build with n threads (n > 1) or the single-threaded
    build (n <= 1) for every later call; returns the threads in use.  Only
    the CPU timing baseline calls this."""
    global _threads
    build()
    if n > 1 and os.path.exists(_LIB_OMP_PATH):
        L = _load(_LIB_OMP_PATH)
        L.or_set_threads(int(n))
        _threads = int(L.or_threads())
    else:
        _threads = 1
    return _threads


class Scanner(C.Structure):
    _fields_ = [("n_rings", C.c_int32), ("n_xtal", C.c_int32), ("xtal", C.POINTER(C.c_float))]


class Grid(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("h", C.c_float * 3), ("origin", C.c_float * 3)]


class Tof(C.Structure):
    _fields_ = [("sigma", C.c_float), ("bin", C.c_float), ("n_sigma", C.c_float), ("n_bins", C.c_int32)]


class LmProblem(C.Structure):
    _fields_ = [("sc", C.POINTER(Scanner)), ("g", C.POINTER(Grid)), ("tof", C.POINTER(Tof)),
                ("det1", C.POINTER(C.c_int32)), ("det2", C.POINTER(C.c_int32)),
                ("tbin", C.POINTER(C.c_int16)), ("corr", C.POINTER(C.c_float)),
                ("contam", C.POINTER(C.c_float)), ("mu", C.POINTER(C.c_int32)),
                ("n_ev", C.c_int64), ("n_subsets", C.c_int32),
                ("beta", C.c_double), ("gamma", C.c_double), ("rho", C.c_double), ("knorm", C.c_double),
                ("xi", C.POINTER(C.c_double)), ("res_fwhm", C.c_double)]


class LmState(C.Structure):
    _fields_ = [("x", C.POINTER(C.c_double)), ("z", C.POINTER(C.c_double)),
                ("zbar", C.POINTER(C.c_double)), ("w", C.POINTER(C.c_double)),
                ("y", C.POINTER(C.c_double)), ("T", C.POINTER(C.c_double))]


class SinoProblem(C.Structure):
    _fields_ = [("sc", C.POINTER(Scanner)), ("g", C.POINTER(Grid)), ("tof", C.POINTER(Tof)),
                ("lor_factor", C.POINTER(C.c_float)), ("d", C.POINTER(C.c_double)),
                ("s", C.POINTER(C.c_double)), ("sub", C.POINTER(C.c_int32)),
                ("n_subsets", C.c_int32),
                ("beta", C.c_double), ("gamma", C.c_double), ("rho", C.c_double), ("knorm", C.c_double),
                ("xi", C.POINTER(C.c_double))]


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def lib():
    """The oracle library in use (single-threaded unless use_threads chose
    the OpenMP build)."""
    build()
    return _load(_LIB_OMP_PATH if _threads > 1 else _LIB_PATH)


def _load(path):
    with _lock:
        if path not in _libs:
            L = C.CDLL(path)
            P = C.POINTER
            L.or_fwd.argtypes = [P(Scanner), P(Grid), P(Tof), P(C.c_int32), P(C.c_int32), P(C.c_int16),
                                 P(C.c_float), C.c_int64, P(C.c_float), P(C.c_double)]
            L.or_back.argtypes = [P(Scanner), P(Grid), P(Tof), P(C.c_int32), P(C.c_int32), P(C.c_int16),
                                  P(C.c_float), C.c_int64, P(C.c_double), P(C.c_double)]
            L.or_fwd_nontof.argtypes = [P(Scanner), P(Grid), P(C.c_int32), P(C.c_int32), C.c_int64,
                                        P(C.c_double), P(C.c_double)]
            L.or_lor_tofsum_fwd.argtypes = [P(Scanner), P(Grid), P(Tof), C.c_int32, C.c_int32, P(C.c_double)]
            L.or_lor_tofsum_fwd.restype = C.c_double
            L.or_sens.argtypes = [P(Scanner), P(Grid), P(Tof), P(C.c_float), P(C.c_double)]
            L.or_n_lor.argtypes = [P(Scanner)]
            L.or_n_lor.restype = C.c_int64
            L.or_lor_dets.argtypes = [P(Scanner), C.c_int64, P(C.c_int32), P(C.c_int32)]
            L.or_event_counts.argtypes = [P(C.c_int32), P(C.c_int32), P(C.c_int16), C.c_int64, P(C.c_int32)]
            L.or_tv_ndim.argtypes = [P(Grid)]
            L.or_tv_grad.argtypes = [P(Grid), P(C.c_double), P(C.c_double)]
            L.or_tv_adj.argtypes = [P(Grid), P(C.c_double), P(C.c_double)]
            L.or_tv_prox.argtypes = [P(Grid), P(C.c_double), C.c_double]
            L.or_dtv_grad.argtypes = [P(Grid), P(C.c_double), P(C.c_double), P(C.c_double)]
            L.or_dtv_adj.argtypes = [P(Grid), P(C.c_double), P(C.c_double), P(C.c_double)]
            L.or_dtv_xi.argtypes = [P(Grid), P(C.c_double), C.c_double, P(C.c_double)]
            L.or_res_apply.argtypes = [P(Grid), C.c_double, P(C.c_double), P(C.c_double)]
            L.or_knorm_power.argtypes = [P(Grid), C.c_int]
            L.or_knorm_power.restype = C.c_double
            L.or_prox_dstar.argtypes = [C.c_double, C.c_double, C.c_double]
            L.or_prox_dstar.restype = C.c_double
            L.or_lm_init.argtypes = [P(LmProblem), P(C.c_float), P(C.c_double), P(LmState)]
            L.or_lm_update.argtypes = [P(LmProblem), P(LmState), C.c_int32, P(C.c_double), P(C.c_double)]
            L.or_lm_objective.argtypes = [P(LmProblem), P(C.c_double), P(C.c_double)]
            L.or_lm_objective.restype = C.c_double
            L.or_tof_edge_distance.argtypes = [P(Scanner), P(Grid), P(Tof), P(C.c_int32), P(C.c_int32),
                                               P(C.c_int16), C.c_int64, P(C.c_double)]
            L.or_fwd_position_sensitivity.argtypes = [P(Scanner), P(Grid), P(Tof), P(C.c_int32), P(C.c_int32),
                                                      P(C.c_int16), P(C.c_float), C.c_int64, P(C.c_float),
                                                      P(C.c_double)]
            L.or_sino_nbins.argtypes = [P(SinoProblem)]
            L.or_sino_nbins.restype = C.c_int64
            L.or_sino_init.argtypes = [P(SinoProblem), P(C.c_float), P(C.c_double), P(LmState)]
            L.or_sino_update.argtypes = [P(SinoProblem), P(LmState), C.c_int32, P(C.c_double), P(C.c_double)]
            L.or_sino_objective.argtypes = [P(SinoProblem), P(C.c_double)]
            L.or_sino_objective.restype = C.c_double
            L.or_emtv_em_step.argtypes = [P(LmProblem), P(C.c_double), P(C.c_double), C.c_int32, P(C.c_double)]
            L.or_emtv_denoise.argtypes = [P(Grid), P(C.c_double), P(C.c_double), P(C.c_uint8), C.c_int,
                                          C.c_double, P(C.c_double), P(C.c_double)]
            L.or_emtv_epoch.argtypes = [P(LmProblem), P(C.c_double), P(C.c_double), C.c_int]
            L.or_set_threads.argtypes = [C.c_int]
            L.or_threads.restype = C.c_int
            _libs[path] = L
    return _libs[path]


# --------------------------------------------------------------------------
# marshalling helpers (keep numpy arrays alive inside the wrapper objects)
# --------------------------------------------------------------------------
class Geometry:
    """Scanner table + grid + TOF as C structs."""

    def __init__(self, xtal: np.ndarray, n_rings: int, n_xtal: int, n, h, origin, tof=None):
        self.xtal = np.ascontiguousarray(xtal, dtype=np.float32).reshape(-1)
        self.sc = Scanner(n_rings, n_xtal, _p(self.xtal, C.c_float))
        self.g = Grid((C.c_int32 * 3)(*n), (C.c_float * 3)(*h), (C.c_float * 3)(*origin))
        if tof is None:
            self.tof = Tof(1.0, 1.0, 3.0, 0)
        else:
            self.tof = Tof(*tof)
        self.n = tuple(int(v) for v in n)
        self.V = int(n[0] * n[1] * n[2])

    @classmethod
    def from_workload(cls, wl):
        sc, g, t = wl.scanner, wl.grid, wl.tof
        return cls(sc.crystal_table(), sc.n_rings, sc.n_xtal, g.n, g.h, g.origin,
                   (t.sigma, t.bin, t.n_sigma, t.n_bins))

    @property
    def ndim(self) -> int:
        return int(lib().or_tv_ndim(C.byref(self.g)))

    @property
    def n_lor(self) -> int:
        return int(lib().or_n_lor(C.byref(self.sc)))

    def lor_dets(self, l: int):
        a = C.c_int32()
        b = C.c_int32()
        lib().or_lor_dets(C.byref(self.sc), int(l), C.byref(a), C.byref(b))
        return a.value, b.value


class EventArrays:
    def __init__(self, det1, det2, tof, corr=None, contam=None):
        self.det1 = np.ascontiguousarray(det1, dtype=np.int32)
        self.det2 = np.ascontiguousarray(det2, dtype=np.int32)
        self.tof = np.ascontiguousarray(tof, dtype=np.int16)
        n = self.det1.shape[0]
        self.corr = np.ascontiguousarray(np.ones(n, np.float32) if corr is None else corr, dtype=np.float32)
        self.contam = np.ascontiguousarray(np.zeros(n, np.float32) if contam is None else contam, dtype=np.float32)
        self.n = n

    @classmethod
    def from_events(cls, ev):
        return cls(ev.det1, ev.det2, ev.tof, ev.corr, ev.contam)


def fwd(geo: Geometry, ev: EventArrays, x: np.ndarray, use_corr: bool = True) -> np.ndarray:
    """(P^LM x)_e in FP64 for a float32 image x."""
    x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1)
    out = np.zeros(ev.n, dtype=np.float64)
    lib().or_fwd(C.byref(geo.sc), C.byref(geo.g), C.byref(geo.tof), _p(ev.det1, C.c_int32),
                 _p(ev.det2, C.c_int32), _p(ev.tof, C.c_int16),
                 _p(ev.corr, C.c_float) if use_corr else None, ev.n, _p(x, C.c_float), _p(out, C.c_double))
    return out


def tof_edge_distance(geo: Geometry, ev: EventArrays) -> np.ndarray:
    """Per event, distance (mm) of its nearest in-grid sample from the TOF
    truncation edge (inf for non-TOF or empty events)."""
    out = np.zeros(ev.n, dtype=np.float64)
    lib().or_tof_edge_distance(C.byref(geo.sc), C.byref(geo.g), C.byref(geo.tof), _p(ev.det1, C.c_int32),
                               _p(ev.det2, C.c_int32), _p(ev.tof, C.c_int16), ev.n, _p(out, C.c_double))
    return out


def fwd_position_sensitivity(geo: Geometry, ev: EventArrays, x: np.ndarray) -> np.ndarray:
    """Per event, |d (P^LM x)_e / d(sample position)| summed over samples, in
    image units per voxel of shift (see lmoracle.c)."""
    x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1)
    out = np.zeros(ev.n, dtype=np.float64)
    lib().or_fwd_position_sensitivity(C.byref(geo.sc), C.byref(geo.g), C.byref(geo.tof), _p(ev.det1, C.c_int32),
                                      _p(ev.det2, C.c_int32), _p(ev.tof, C.c_int16), _p(ev.corr, C.c_float), ev.n,
                                      _p(x, C.c_float), _p(out, C.c_double))
    return out


def back(geo: Geometry, ev: EventArrays, v: np.ndarray, use_corr: bool = True) -> np.ndarray:
    """(P^LM)^T v in FP64."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    img = np.zeros(geo.V, dtype=np.float64)
    lib().or_back(C.byref(geo.sc), C.byref(geo.g), C.byref(geo.tof), _p(ev.det1, C.c_int32),
                  _p(ev.det2, C.c_int32), _p(ev.tof, C.c_int16),
                  _p(ev.corr, C.c_float) if use_corr else None, ev.n, _p(v, C.c_double), _p(img, C.c_double))
    return img


def fwd_nontof(geo: Geometry, det1, det2, x: np.ndarray) -> np.ndarray:
    d1 = np.ascontiguousarray(det1, dtype=np.int32)
    d2 = np.ascontiguousarray(det2, dtype=np.int32)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
    out = np.zeros(d1.shape[0], dtype=np.float64)
    lib().or_fwd_nontof(C.byref(geo.sc), C.byref(geo.g), _p(d1, C.c_int32), _p(d2, C.c_int32), d1.shape[0],
                        _p(x, C.c_double), _p(out, C.c_double))
    return out


def lor_tofsum_fwd(geo: Geometry, det1: int, det2: int, x: np.ndarray) -> float:
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
    return float(lib().or_lor_tofsum_fwd(C.byref(geo.sc), C.byref(geo.g), C.byref(geo.tof), det1, det2,
                                         _p(x, C.c_double)))


def sens(geo: Geometry, lor_factor: np.ndarray | None = None) -> np.ndarray:
    img = np.zeros(geo.V, dtype=np.float64)
    lf = None if lor_factor is None else np.ascontiguousarray(lor_factor, dtype=np.float32)
    lib().or_sens(C.byref(geo.sc), C.byref(geo.g), C.byref(geo.tof),
                  None if lf is None else _p(lf, C.c_float), _p(img, C.c_double))
    return img


def event_counts(det1, det2, tof) -> np.ndarray:
    d1 = np.ascontiguousarray(det1, dtype=np.int32)
    d2 = np.ascontiguousarray(det2, dtype=np.int32)
    t = np.ascontiguousarray(tof, dtype=np.int16)
    mu = np.zeros(d1.shape[0], dtype=np.int32)
    lib().or_event_counts(_p(d1, C.c_int32), _p(d2, C.c_int32), _p(t, C.c_int16), d1.shape[0], _p(mu, C.c_int32))
    return mu


def subset_permutation(n_events: int, n_subsets: int) -> np.ndarray:
    """perm[e] = position of event e in the subset-contiguous order: subset
    e mod n, rank e div n inside it (Sec. "Listmode SPDHG")."""
    e = np.arange(n_events, dtype=np.int64)
    counts = np.array([len(range(k, n_events, n_subsets)) for k in range(n_subsets)], dtype=np.int64)
    off = np.concatenate([[0], np.cumsum(counts)])
    return off[e % n_subsets] + e // n_subsets


def subset_offsets(n_events: int, n_subsets: int) -> np.ndarray:
    counts = np.array([len(range(k, n_events, n_subsets)) for k in range(n_subsets)], dtype=np.int64)
    return np.concatenate([[0], np.cumsum(counts)])


def tv_grad(geo: Geometry, x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
    out = np.zeros(geo.ndim * geo.V, dtype=np.float64)
    lib().or_tv_grad(C.byref(geo.g), _p(x, C.c_double), _p(out, C.c_double))
    return out


def tv_adj(geo: Geometry, q: np.ndarray) -> np.ndarray:
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(-1)
    out = np.zeros(geo.V, dtype=np.float64)
    lib().or_tv_adj(C.byref(geo.g), _p(q, C.c_double), _p(out, C.c_double))
    return out


def _xi_ptr(xi):
    return None if xi is None else _p(xi, C.c_double)


def dtv_xi(geo: Geometry, v: np.ndarray, eta: float) -> np.ndarray:
    """Directional-TV field xi = grad v / sqrt(|grad v|^2 + eta^2), [ndim][V]."""
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1)
    out = np.zeros(geo.ndim * geo.V, dtype=np.float64)
    lib().or_dtv_xi(C.byref(geo.g), _p(v, C.c_double), float(eta), _p(out, C.c_double))
    return out


def dtv_grad(geo: Geometry, xi: np.ndarray | None, x: np.ndarray) -> np.ndarray:
    """K x = P grad x (DTV; xi None = TV)."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
    xi = None if xi is None else np.ascontiguousarray(xi, dtype=np.float64)
    out = np.zeros(geo.ndim * geo.V, dtype=np.float64)
    lib().or_dtv_grad(C.byref(geo.g), _xi_ptr(xi), _p(x, C.c_double), _p(out, C.c_double))
    return out


def dtv_adj(geo: Geometry, xi: np.ndarray | None, q: np.ndarray) -> np.ndarray:
    """K^T q = grad^T (P q)."""
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(-1)
    xi = None if xi is None else np.ascontiguousarray(xi, dtype=np.float64)
    out = np.zeros(geo.V, dtype=np.float64)
    lib().or_dtv_adj(C.byref(geo.g), _xi_ptr(xi), _p(q, C.c_double), _p(out, C.c_double))
    return out


def res_apply(geo: Geometry, fwhm: float, x: np.ndarray) -> np.ndarray:
    """G x: the separable Gaussian resolution model (mirrored faces)."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
    out = np.zeros(geo.V, dtype=np.float64)
    lib().or_res_apply(C.byref(geo.g), float(fwhm), _p(x, C.c_double), _p(out, C.c_double))
    return out


def tv_prox(geo: Geometry, w: np.ndarray, beta: float) -> np.ndarray:
    w = np.array(w, dtype=np.float64).reshape(-1)
    lib().or_tv_prox(C.byref(geo.g), _p(w, C.c_double), float(beta))
    return w


def knorm_power(geo: Geometry, iters: int) -> float:
    return float(lib().or_knorm_power(C.byref(geo.g), int(iters)))


def prox_dstar(a: float, S: float, d: float) -> float:
    return float(lib().or_prox_dstar(float(a), float(S), float(d)))


class LM:
    """Alg. 2 state in FP64: ``init`` then ``update(i)`` for each selection."""

    def __init__(self, geo: Geometry, ev: EventArrays, mu: np.ndarray, n_subsets: int,
                 beta: float, gamma: float, rho: float, knorm: float, xi: np.ndarray | None = None,
                 res_fwhm: float = 0.0):
        self.geo, self.ev = geo, ev
        self.mu = np.ascontiguousarray(mu, dtype=np.int32)
        self.xi = None if xi is None else np.ascontiguousarray(xi, dtype=np.float64)
        V, nd = geo.V, geo.ndim
        self.x = np.zeros(V)
        self.z = np.zeros(V)
        self.zbar = np.zeros(V)
        self.w = np.zeros(max(nd, 1) * V)
        self.y = np.zeros(ev.n)
        self.T = np.zeros(V)
        self._dz = np.zeros(V)
        self._gw = np.zeros(max(nd, 1) * V)
        self.prob = LmProblem(C.pointer(geo.sc), C.pointer(geo.g), C.pointer(geo.tof),
                              _p(ev.det1, C.c_int32), _p(ev.det2, C.c_int32), _p(ev.tof, C.c_int16),
                              _p(ev.corr, C.c_float), _p(ev.contam, C.c_float), _p(self.mu, C.c_int32),
                              ev.n, n_subsets, beta, gamma, rho, knorm, _xi_ptr(self.xi), float(res_fwhm))
        self.state = LmState(_p(self.x, C.c_double), _p(self.z, C.c_double), _p(self.zbar, C.c_double),
                             _p(self.w, C.c_double), _p(self.y, C.c_double), _p(self.T, C.c_double))

    def init(self, x0: np.ndarray, sens_img: np.ndarray):
        self._x0 = np.ascontiguousarray(x0, dtype=np.float32).reshape(-1)
        self._sens = np.ascontiguousarray(sens_img, dtype=np.float64)
        lib().or_lm_init(C.byref(self.prob), _p(self._x0, C.c_float), _p(self._sens, C.c_double),
                         C.byref(self.state))

    def update(self, i: int):
        lib().or_lm_update(C.byref(self.prob), C.byref(self.state), int(i), _p(self._dz, C.c_double),
                           _p(self._gw, C.c_double))

    def run(self, seq):
        for i in seq:
            self.update(int(i))

    def objective(self, x: np.ndarray | None = None) -> float:
        xx = np.ascontiguousarray(self.x if x is None else x, dtype=np.float64)
        return float(lib().or_lm_objective(C.byref(self.prob), _p(xx, C.c_double), _p(self._sens, C.c_double)))


class EMTV:
    """Listmode EM-TV (Alg. 3) in FP64: the subset EM step, the weighted TV
    denoising by accelerated PDHG, and one pass over the subsets."""

    def __init__(self, geo: Geometry, ev: EventArrays, n_subsets: int, beta: float, knorm: float,
                 res_fwhm: float = 0.0):
        self.geo, self.ev = geo, ev
        self._mu = np.ones(max(ev.n, 1), dtype=np.int32)
        self.prob = LmProblem(C.pointer(geo.sc), C.pointer(geo.g), C.pointer(geo.tof),
                              _p(ev.det1, C.c_int32), _p(ev.det2, C.c_int32), _p(ev.tof, C.c_int16),
                              _p(ev.corr, C.c_float), _p(ev.contam, C.c_float), _p(self._mu, C.c_int32),
                              ev.n, n_subsets, beta, 0.0, 0.0, knorm, None, float(res_fwhm))

    def em_step(self, x: np.ndarray, sens_img: np.ndarray, i: int) -> np.ndarray:
        xx = np.ascontiguousarray(x, dtype=np.float64)
        ss = np.ascontiguousarray(sens_img, dtype=np.float64)
        z = np.zeros(self.geo.V)
        lib().or_emtv_em_step(C.byref(self.prob), _p(ss, C.c_double), _p(xx, C.c_double), int(i),
                              _p(z, C.c_double))
        return z

    def epoch(self, x: np.ndarray, sens_img: np.ndarray, pdhg_iters: int = 20) -> np.ndarray:
        xx = np.array(x, dtype=np.float64)
        ss = np.ascontiguousarray(sens_img, dtype=np.float64)
        lib().or_emtv_epoch(C.byref(self.prob), _p(ss, C.c_double), _p(xx, C.c_double), int(pdhg_iters))
        return xx


def emtv_denoise(geo: Geometry, z: np.ndarray, w: np.ndarray, free: np.ndarray, iters: int, knorm: float):
    """argmin_{u>=0} sum w/2 (u-z)^2 + ||Ku||_{2,1} by accelerated PDHG;
    returns (u, q) with q the dual variable."""
    zz = np.ascontiguousarray(z, dtype=np.float64)
    ww = np.ascontiguousarray(w, dtype=np.float64)
    ff = np.ascontiguousarray(free, dtype=np.uint8)
    u = np.zeros(geo.V)
    q = np.zeros(max(geo.ndim, 1) * geo.V)
    lib().or_emtv_denoise(C.byref(geo.g), _p(zz, C.c_double), _p(ww, C.c_double), _p(ff, C.c_uint8), int(iters),
                          float(knorm), _p(u, C.c_double), _p(q, C.c_double))
    return u, q


class Sino:
    """Alg. 1 on the full TOF sinogram (every LOR and TOF bin)."""

    def __init__(self, geo: Geometry, lor_factor: np.ndarray, d: np.ndarray, s: np.ndarray,
                 sub: np.ndarray, n_subsets: int, beta: float, gamma: float, rho: float, knorm: float,
                 xi: np.ndarray | None = None):
        self.geo = geo
        self.xi = None if xi is None else np.ascontiguousarray(xi, dtype=np.float64)
        self.lf = np.ascontiguousarray(lor_factor, dtype=np.float32)
        self.d = np.ascontiguousarray(d, dtype=np.float64)
        self.s = np.ascontiguousarray(s, dtype=np.float64)
        self.sub = np.ascontiguousarray(sub, dtype=np.int32)
        V, nd = geo.V, geo.ndim
        self.x = np.zeros(V)
        self.z = np.zeros(V)
        self.zbar = np.zeros(V)
        self.w = np.zeros(max(nd, 1) * V)
        self.y = np.zeros(self.d.shape[0])
        self.T = np.zeros(V)
        self._dz = np.zeros(V)
        self._gw = np.zeros(max(nd, 1) * V)
        self.prob = SinoProblem(C.pointer(geo.sc), C.pointer(geo.g), C.pointer(geo.tof),
                                _p(self.lf, C.c_float), _p(self.d, C.c_double), _p(self.s, C.c_double),
                                _p(self.sub, C.c_int32), n_subsets, beta, gamma, rho, knorm, _xi_ptr(self.xi))
        self.state = LmState(_p(self.x, C.c_double), _p(self.z, C.c_double), _p(self.zbar, C.c_double),
                             _p(self.w, C.c_double), _p(self.y, C.c_double), _p(self.T, C.c_double))
        assert lib().or_sino_nbins(C.byref(self.prob)) == self.d.shape[0]

    def init(self, x0, sens_img):
        self._x0 = np.ascontiguousarray(x0, dtype=np.float32).reshape(-1)
        self._sens = np.ascontiguousarray(sens_img, dtype=np.float64)
        lib().or_sino_init(C.byref(self.prob), _p(self._x0, C.c_float), _p(self._sens, C.c_double),
                           C.byref(self.state))

    def update(self, i: int):
        lib().or_sino_update(C.byref(self.prob), C.byref(self.state), int(i), _p(self._dz, C.c_double),
                             _p(self._gw, C.c_double))

    def objective(self, x=None) -> float:
        xx = np.ascontiguousarray(self.x if x is None else x, dtype=np.float64)
        return float(lib().or_sino_objective(C.byref(self.prob), _p(xx, C.c_double)))
