"""Python binding of liblmspdhg.so (the C ABI in include/lmspdhg.h).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  Device buffers are torch CUDA tensors (used for memory and streams);
calls run on torch's current CUDA stream unless a stream is given.  There is
no CPU fallback: importing this module without the built library, or calling
it without a CUDA device, raises.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
from typing import Optional, Sequence

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblmspdhg.so")

LM_OK = 0
ERRORS = {1: "LM_ERR_INVALID_ARG", 2: "LM_ERR_OUT_OF_RANGE", 3: "LM_ERR_DOMAIN", 4: "LM_ERR_CUDA",
          5: "LM_ERR_TIMEOUT", 6: "LM_ERR_NOMEM"}


class LMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class lm_scanner(C.Structure):
    _fields_ = [("n_rings", C.c_int32), ("n_xtal", C.c_int32), ("xtal_xyz", C.c_void_p)]


class lm_grid(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("h", C.c_float * 3), ("origin", C.c_float * 3)]


class lm_tof(C.Structure):
    _fields_ = [("sigma_mm", C.c_float), ("bin_mm", C.c_float), ("n_sigma", C.c_float), ("n_bins", C.c_int32)]


class lm_events(C.Structure):
    _fields_ = [("det1", C.c_void_p), ("det2", C.c_void_p), ("tof", C.c_void_p), ("corr", C.c_void_p),
                ("contam", C.c_void_p), ("n", C.c_int64)]


class lm_params(C.Structure):
    _fields_ = [("beta", C.c_float), ("gamma", C.c_float), ("rho", C.c_float), ("knorm", C.c_double),
                ("knorm_iters", C.c_int32), ("n_subsets", C.c_int32), ("deterministic", C.c_int32),
                ("kahan", C.c_int32), ("group", C.c_int32), ("image_kernel", C.c_int32),
                ("tile_buf", C.c_void_p), ("tile_bytes", C.c_size_t), ("xi", C.c_void_p),
                ("res_fwhm", C.c_float), ("sinogram", C.c_int32), ("sino_q", C.c_void_p),
                ("sino_qoff", C.c_void_p), ("sino_lorf", C.c_void_p), ("sino_s", C.c_float),
                ("trav_buf", C.c_void_p), ("trav_bytes", C.c_size_t), ("shard", C.c_int32),
                ("epoch_kernel", C.c_int32), ("trav_keep", C.c_int32)]


_lib = None


class lm_server_config(C.Structure):
    _fields_ = [("beta", C.c_float), ("rho", C.c_float), ("knorm", C.c_double), ("n_subsets", C.c_int32),
                ("epochs", C.c_int32), ("max_slots", C.c_int32), ("deterministic", C.c_int32),
                ("kahan", C.c_int32), ("group", C.c_int32), ("max_events", C.c_int64)]


def load_library(path: str = LIB_PATH) -> C.CDLL:
    """Load liblmspdhg.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} not found: build it with `python -m paper_2201_05497_gb300.build`")
    L = C.CDLL(path)
    P, V, I32, I64, F, D, SZ = C.POINTER, C.c_void_p, C.c_int32, C.c_int64, C.c_float, C.c_double, C.c_size_t
    sig = {
        "lm_last_error": ([], C.c_char_p),
        "lm_version": ([], C.c_int),
        "lm_struct_sizes": ([P(SZ), C.c_int], C.c_int),
        "lm_fwd_workspace_bytes": ([P(lm_grid)], SZ),
        "lm_fwd": ([P(lm_scanner), P(lm_grid), P(lm_tof), V, P(lm_events), V, V, SZ, V], C.c_int),
        "lm_back_workspace_bytes": ([P(lm_grid), C.c_int], SZ),
        "lm_back": ([P(lm_scanner), P(lm_grid), P(lm_tof), P(lm_events), V, V, C.c_int, V, SZ, V], C.c_int),
        "lm_n_lor": ([P(lm_scanner)], I64),
        "lm_sens_workspace_bytes": ([P(lm_grid)], SZ),
        "lm_sens": ([P(lm_scanner), P(lm_grid), P(lm_tof), V, V, V, SZ, V], C.c_int),
        "lm_tv_ndim": ([P(lm_grid)], C.c_int),
        "lm_tv_grad": ([P(lm_grid), V, V, V], C.c_int),
        "lm_tv_div": ([P(lm_grid), V, V, V], C.c_int),
        "lm_tv_prox": ([P(lm_grid), V, F, V], C.c_int),
        "lm_dtv_field": ([P(lm_grid), V, F, V, V], C.c_int),
        "lm_res_workspace_bytes": ([P(lm_grid)], SZ),
        "lm_sino_n_bins": ([P(lm_scanner), P(lm_tof)], I64),
        "lm_sino_workspace_bytes": ([P(lm_scanner), I32], SZ),
        "lm_sino_setup": ([P(lm_scanner), P(lm_tof), I32, V, V, V, V, V, V, V, V, V, P(I64), V, SZ, V], C.c_int),
        "lm_sino_count": ([P(lm_scanner), P(lm_tof), I32, P(lm_events), V, V, V, P(I64), V, SZ, V], C.c_int),
        "lm_res_apply": ([P(lm_grid), F, V, V, V, SZ, V], C.c_int),
        "lm_dtv_grad": ([P(lm_grid), V, V, V, V], C.c_int),
        "lm_dtv_div": ([P(lm_grid), V, V, V, V], C.c_int),
        "lm_knorm_workspace_bytes": ([P(lm_grid)], SZ),
        "lm_knorm_fp64": ([P(lm_grid), I32, V, SZ, P(D), V], C.c_int),
        "lm_setup_workspace_bytes": ([I64], SZ),
        "lm_event_setup": ([P(lm_scanner), P(lm_tof), P(lm_events), I32, V, V, V, V, V, V, P(I64), V, SZ, V],
                           C.c_int),
        "lmspdhg_state_bytes": ([P(lm_grid), I64, I32, I32], SZ),
        "lmspdhg_state_bytes_ex": ([P(lm_grid), I64, I32, P(lm_params)], SZ),
        "lmspdhg_create": ([P(V), P(lm_scanner), P(lm_grid), P(lm_tof), P(lm_events), V, P(I64), V, V,
                            P(lm_params), V, SZ, V], C.c_int),
        "lmspdhg_updates": ([V, P(C.c_uint16), I32, V], C.c_int),
        "lmspdhg_epoch": ([V, P(C.c_uint16), V], C.c_int),
        "lmspdhg_get_x": ([V, V, V], C.c_int),
        "lmspdhg_get_y": ([V, V, V], C.c_int),
        "lmspdhg_get_z": ([V, V, V], C.c_int),
        "lmspdhg_get_w": ([V, V, V], C.c_int),
        "lmspdhg_objective_fp64": ([V, P(D), V], C.c_int),
        "lmspdhg_info": ([V, P(I64), P(D), P(D)], C.c_int),
        "lmspdhg_destroy": ([V], C.c_int),
        "lmspdhg_reinit": ([V, V, V], C.c_int),
        "lmspdhg_tuning": ([V, P(I32), P(D)], C.c_int),
        "lmspdhg_image_kernel": ([V, P(I32)], C.c_int),
        "lmspdhg_projector": ([V, P(I32), P(I64)], C.c_int),
        "lmspdhg_tile_bytes": ([P(lm_grid), I64, I32], SZ),
        "lmspdhg_trav_bytes": ([P(lm_grid), I64], SZ),
        "lmspdhg_shard_buffer": ([V, P(V)], C.c_int),
        "lmspdhg_shard_init_finish": ([V, V], C.c_int),
        "lmspdhg_shard_begin": ([V, C.c_uint16, V], C.c_int),
        "lmspdhg_shard_finish": ([V, V], C.c_int),
        "lmspdhg_objective_parts_fp64": ([V, P(D), V], C.c_int),
        "lmspdhg_set_gate": ([V, V], C.c_int),
        "lmspdhg_tuning_projectors": ([V, P(D), P(D)], C.c_int),
        "lmspdhg_epoch_kernel": ([V, P(I32)], C.c_int),
        "lmspdhg_profile": ([V, P(C.c_uint16), I32, P(D), P(I64), V], C.c_int),
        "lm_kernel_launches": ([], I64),
        "lm_traversal_stats": ([P(lm_scanner), P(lm_grid), P(lm_tof), P(lm_events), V, SZ, P(I64), P(I64), V],
                               C.c_int),
        "lm_probe_l2": ([V, SZ, I32, I32, P(D), V], C.c_int),
        "lmspdhg_batch_bytes": ([I32, I32], SZ),
        "lmspdhg_batch_create": ([P(V), I32, I32, V, SZ, V], C.c_int),
        "lmspdhg_batch_set": ([V, I32, V, V], C.c_int),
        "lmspdhg_batch_epoch": ([V, P(C.c_uint16), V], C.c_int),
        "lmspdhg_batch_destroy": ([V], C.c_int),
        "lm_server_frame_bytes": ([P(lm_grid), I64, I32, I32], SZ),
        "lm_server_create": ([P(V), P(lm_scanner), P(lm_grid), P(lm_tof), V, P(lm_server_config), V, SZ],
                             C.c_int),
        "lm_server_submit": ([V, V, V, V, V, V, I64, F, P(C.c_uint16), P(I64)], C.c_int),
        "lm_server_wait": ([V, I64, V, P(D), P(D), I32], C.c_int),
        "lm_server_stats": ([V, P(I64), P(I64), P(I64), P(SZ), P(I64)], C.c_int),
        "lm_server_destroy": ([V], C.c_int),
        "lm_emtv_workspace_bytes": ([P(lm_grid)], SZ),
        "lm_emtv_epoch": ([P(lm_scanner), P(lm_grid), P(lm_tof), P(lm_events), P(I64), I32, V, V, F, I32, D, V,
                           SZ, V], C.c_int),
        "lm_emtv_em_step": ([P(lm_scanner), P(lm_grid), P(lm_tof), P(lm_events), I32, V, V, V, V, SZ, V],
                            C.c_int),
        "lm_emtv_denoise": ([P(lm_grid), V, V, V, I32, D, V, SZ, V], C.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    # the descriptor structs above must match the library's layout
    sizes = (C.c_size_t * 6)()
    L.lm_struct_sizes(sizes, 6)
    mine = [C.sizeof(t) for t in (lm_scanner, lm_grid, lm_tof, lm_events, lm_params, lm_server_config)]
    if list(sizes) != mine:
        raise RuntimeError(f"struct layouts differ from the library's: binding {mine}, library {list(sizes)}")
    _lib = L
    return L


def _check(rc: int):
    if rc != LM_OK:
        raise LMError(rc, load_library().lm_last_error().decode())


def _ptr(t: Optional[torch.Tensor], dtype: Optional[torch.dtype] = None, numel: Optional[int] = None,
         name: str = "tensor"):
    """Device pointer of t (None passes through).  Raises before any call into
    the library if t is not a contiguous CUDA tensor, or (when given) has
    another dtype or fewer than numel elements."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name}: expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name}: expected {dtype}, got {t.dtype}")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name}: {t.numel()} elements, at least {numel} needed")
    return C.c_void_p(t.data_ptr())


def _f32(t: Optional[torch.Tensor], numel: int, name: str):
    return _ptr(t, torch.float32, numel, name)


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


# --------------------------------------------------------------------------
# descriptors
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Geometry:
    """Scanner (crystal table on the device), image grid and TOF kernel."""
    xtal: torch.Tensor          # float32 [n_det, 3] on the device
    n_rings: int
    n_xtal: int
    n: Sequence[int]
    h: Sequence[float]
    origin: Sequence[float]
    tof_sigma: float = 1.0
    tof_bin: float = 1.0
    tof_nsigma: float = 3.0
    tof_nbins: int = 0

    def __post_init__(self):
        self.sc = lm_scanner(self.n_rings, self.n_xtal, C.c_void_p(self.xtal.data_ptr()))
        self.g = lm_grid((C.c_int32 * 3)(*[int(v) for v in self.n]), (C.c_float * 3)(*self.h),
                         (C.c_float * 3)(*self.origin))
        self.tof = lm_tof(self.tof_sigma, self.tof_bin, self.tof_nsigma, self.tof_nbins)

    @classmethod
    def from_workload(cls, wl, device="cuda"):
        sc, g, t = wl.scanner, wl.grid, wl.tof
        xtal = torch.from_numpy(sc.crystal_table()).to(device)
        return cls(xtal, sc.n_rings, sc.n_xtal, g.n, g.h, g.origin, t.sigma, t.bin, t.n_sigma, t.n_bins)

    @property
    def V(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])

    @property
    def ndim(self) -> int:
        return int(load_library().lm_tv_ndim(C.byref(self.g)))

    @property
    def n_lor(self) -> int:
        return int(load_library().lm_n_lor(C.byref(self.sc)))


@dataclasses.dataclass
class DeviceEvents:
    det1: torch.Tensor
    det2: torch.Tensor
    tof: Optional[torch.Tensor]
    corr: Optional[torch.Tensor]
    contam: Optional[torch.Tensor]

    @property
    def n(self) -> int:
        return int(self.det1.shape[0])

    def desc(self) -> lm_events:
        n = self.n
        return lm_events(_ptr(self.det1, torch.int32, n, "det1"), _ptr(self.det2, torch.int32, n, "det2"),
                         _ptr(self.tof, torch.int16, n, "tof"), _ptr(self.corr, torch.float32, n, "corr"),
                         _ptr(self.contam, torch.float32, n, "contam"), n)

    @classmethod
    def from_numpy(cls, ev, device="cuda"):
        t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(device)
        return cls(t(ev.det1), t(ev.det2), t(ev.tof), t(ev.corr), t(ev.contam))


def _ws(nbytes: int, device) -> Optional[torch.Tensor]:
    if nbytes <= 0:
        return None
    return torch.empty(int(nbytes), dtype=torch.uint8, device=device)


# --------------------------------------------------------------------------
# operators
# --------------------------------------------------------------------------
def fwd(geo: Geometry, x: torch.Tensor, ev: DeviceEvents, out: Optional[torch.Tensor] = None,
        use_workspace: bool = True, stream=None) -> torch.Tensor:
    """(P^LM x)_e (Eq. lmop)."""
    L = load_library()
    if out is None:
        out = torch.empty(ev.n, dtype=torch.float32, device=x.device)
    ws = _ws(L.lm_fwd_workspace_bytes(C.byref(geo.g)), x.device) if use_workspace else None
    d = ev.desc()
    _check(L.lm_fwd(C.byref(geo.sc), C.byref(geo.g), C.byref(geo.tof), _f32(x, geo.V, "x"), C.byref(d),
                    _f32(out, ev.n, "out"),
                    _ptr(ws), 0 if ws is None else ws.numel(), _stream(stream)))
    return out


def back(geo: Geometry, v: torch.Tensor, ev: DeviceEvents, img: Optional[torch.Tensor] = None,
         deterministic: bool = False, use_workspace: bool = True, stream=None) -> torch.Tensor:
    """img += (P^LM)^T v."""
    L = load_library()
    if img is None:
        img = torch.zeros(geo.V, dtype=torch.float32, device=v.device)
    nb = L.lm_back_workspace_bytes(C.byref(geo.g), int(deterministic))
    ws = _ws(nb, v.device) if (use_workspace or deterministic) else None
    d = ev.desc()
    _check(L.lm_back(C.byref(geo.sc), C.byref(geo.g), C.byref(geo.tof), C.byref(d), _f32(v, ev.n, "v"),
                     _f32(img, geo.V, "img"),
                     int(deterministic), _ptr(ws), 0 if ws is None else ws.numel(), _stream(stream)))
    return img


def sens(geo: Geometry, lor_factor: Optional[torch.Tensor] = None, out: Optional[torch.Tensor] = None,
         use_workspace: bool = True, stream=None) -> torch.Tensor:
    """P^T 1 over every canonical LOR and TOF bin."""
    L = load_library()
    dev = geo.xtal.device
    if out is None:
        out = torch.empty(geo.V, dtype=torch.float32, device=dev)
    ws = _ws(L.lm_sens_workspace_bytes(C.byref(geo.g)), dev) if use_workspace else None
    _check(L.lm_sens(C.byref(geo.sc), C.byref(geo.g), C.byref(geo.tof), _f32(lor_factor, geo.n_lor, "lor_factor"),
                     _f32(out, geo.V, "out"), _ptr(ws),
                     0 if ws is None else ws.numel(), _stream(stream)))
    return out


def tv_grad(geo: Geometry, x: torch.Tensor, out=None, stream=None) -> torch.Tensor:
    L = load_library()
    if out is None:
        out = torch.empty(geo.ndim * geo.V, dtype=torch.float32, device=x.device)
    _check(L.lm_tv_grad(C.byref(geo.g), _f32(x, geo.V, "x"), _f32(out, geo.ndim * geo.V, "out"), _stream(stream)))
    return out


def tv_div(geo: Geometry, g: torch.Tensor, out=None, stream=None) -> torch.Tensor:
    L = load_library()
    if out is None:
        out = torch.empty(geo.V, dtype=torch.float32, device=g.device)
    _check(L.lm_tv_div(C.byref(geo.g), _f32(g, geo.ndim * geo.V, "g"), _f32(out, geo.V, "out"), _stream(stream)))
    return out


def tv_prox(geo: Geometry, w: torch.Tensor, beta: float, stream=None) -> torch.Tensor:
    L = load_library()
    _check(L.lm_tv_prox(C.byref(geo.g), _f32(w, geo.ndim * geo.V, "w"), float(beta), _stream(stream)))
    return w


def res_apply(geo: Geometry, fwhm: float, x: torch.Tensor, out=None, stream=None,
              ws: Optional[torch.Tensor] = None) -> torch.Tensor:
    """G x: the image-space resolution model (separable Gaussian, mirrored faces).
    `ws`: a workspace of at least lm_res_workspace_bytes bytes (else allocated)."""
    L = load_library()
    if out is None:
        out = torch.empty(geo.V, dtype=torch.float32, device=x.device)
    if ws is None or ws.numel() < int(L.lm_res_workspace_bytes(C.byref(geo.g))):
        ws = _ws(L.lm_res_workspace_bytes(C.byref(geo.g)), x.device)
    _check(L.lm_res_apply(C.byref(geo.g), float(fwhm), _f32(x, geo.V, "x"), _f32(out, geo.V, "out"), _ptr(ws),
                          ws.numel(), _stream(stream)))
    return out


def dtv_field(geo: Geometry, v: torch.Tensor, eta: float, out=None, stream=None) -> torch.Tensor:
    """Directional-TV field of the structural image v: [ndim * V]."""
    L = load_library()
    if out is None:
        out = torch.empty(geo.ndim * geo.V, dtype=torch.float32, device=v.device)
    _check(L.lm_dtv_field(C.byref(geo.g), _f32(v, geo.V, "v"), float(eta), _f32(out, geo.ndim * geo.V, "out"),
                          _stream(stream)))
    return out


def dtv_grad(geo: Geometry, xi: torch.Tensor, x: torch.Tensor, out=None, stream=None) -> torch.Tensor:
    L = load_library()
    if out is None:
        out = torch.empty(geo.ndim * geo.V, dtype=torch.float32, device=x.device)
    nv = geo.ndim * geo.V
    _check(L.lm_dtv_grad(C.byref(geo.g), _f32(xi, nv, "xi"), _f32(x, geo.V, "x"), _f32(out, nv, "out"),
                         _stream(stream)))
    return out


def dtv_div(geo: Geometry, xi: torch.Tensor, g: torch.Tensor, out=None, stream=None) -> torch.Tensor:
    """-K^T g for the directional TV."""
    L = load_library()
    if out is None:
        out = torch.empty(geo.V, dtype=torch.float32, device=g.device)
    nv = geo.ndim * geo.V
    _check(L.lm_dtv_div(C.byref(geo.g), _f32(xi, nv, "xi"), _f32(g, nv, "g"), _f32(out, geo.V, "out"),
                        _stream(stream)))
    return out


def knorm_fp64(geo: Geometry, iters: int, stream=None) -> float:
    L = load_library()
    ws = _ws(L.lm_knorm_workspace_bytes(C.byref(geo.g)), geo.xtal.device)
    out = C.c_double()
    _check(L.lm_knorm_fp64(C.byref(geo.g), int(iters), _ptr(ws), ws.numel(), C.byref(out), _stream(stream)))
    return float(out.value)


def kernel_launches() -> int:
    return int(load_library().lm_kernel_launches())


def traversal_stats(geo: Geometry, ev: DeviceEvents, stream=None):
    """(samples, neighbour touches) of the events' traversals.  A measurement
    utility of the benchmark (include/lm_measure.h), not part of Alg. 2."""
    L = load_library()
    ws = torch.empty(16, dtype=torch.uint8, device=ev.det1.device)
    ns, nt = C.c_int64(), C.c_int64()
    d = ev.desc()
    _check(L.lm_traversal_stats(C.byref(geo.sc), C.byref(geo.g), C.byref(geo.tof), C.byref(d), _ptr(ws), 16,
                                C.byref(ns), C.byref(nt), _stream(stream)))
    return ns.value, nt.value


def probe_l2(nbytes: int, mode: int, iters: int = 20, device="cuda", stream=None) -> float:
    """L2 throughput (GB/s) of the library's probe kernel on a buffer of nbytes.
    A measurement utility of the benchmark (include/lm_measure.h)."""
    buf = torch.empty(int(nbytes), dtype=torch.uint8, device=device)
    out = C.c_double()
    _check(load_library().lm_probe_l2(_ptr(buf), buf.numel(), int(mode), int(iters), C.byref(out), _stream(stream)))
    return float(out.value)


@dataclasses.dataclass
class PermutedEvents:
    events: DeviceEvents        # subset-contiguous order
    mu: torch.Tensor            # uint16 event counts (same order)
    sub_off: np.ndarray         # int64 [n_subsets + 1]


def event_setup(geo: Geometry, ev: DeviceEvents, n_subsets: int, stream=None, into: "PermutedEvents" = None,
                ws: Optional[torch.Tensor] = None) -> PermutedEvents:
    """Validation, event counts mu and the subset-contiguous split.  `into`
    reuses the buffers of an earlier result (same size); `ws` a workspace of
    at least lm_setup_workspace_bytes(n) bytes."""
    L = load_library()
    dev = ev.det1.device
    n = ev.n
    if into is not None:
        if into.events.n != n or into.sub_off.shape[0] != n_subsets + 1:
            raise ValueError("buffers of a different size")
        out, mu, off = into.events, into.mu, into.sub_off
    else:
        out = DeviceEvents(torch.empty(n, dtype=torch.int32, device=dev),
                           torch.empty(n, dtype=torch.int32, device=dev),
                           torch.empty(n, dtype=torch.int16, device=dev),
                           torch.empty(n, dtype=torch.float32, device=dev),
                           torch.empty(n, dtype=torch.float32, device=dev))
        mu = torch.empty(n, dtype=torch.uint16, device=dev)
        off = np.zeros(n_subsets + 1, dtype=np.int64)
    if ws is None:
        ws = _ws(L.lm_setup_workspace_bytes(n), dev)
    d = ev.desc()
    _check(L.lm_event_setup(C.byref(geo.sc), C.byref(geo.tof), C.byref(d), int(n_subsets), _ptr(out.det1),
                            _ptr(out.det2), _ptr(out.tof), _ptr(out.corr), _ptr(out.contam), _ptr(mu),
                            off.ctypes.data_as(C.POINTER(C.c_int64)), _ptr(ws), ws.numel(), _stream(stream)))
    return PermutedEvents(out, mu, off)


# --------------------------------------------------------------------------
# listmode EM-TV warm start (Alg. 3)
# --------------------------------------------------------------------------
def _emtv_ws(geo: Geometry, ws, dev):
    nb = int(load_library().lm_emtv_workspace_bytes(C.byref(geo.g)))
    if ws is None or ws.numel() < nb:
        ws = _ws(nb, dev)
    return ws


def emtv_epoch(geo: Geometry, pe: PermutedEvents, sens_img: torch.Tensor, x: torch.Tensor, *, beta: float,
               pdhg_iters: int, knorm: float, ws: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """One listmode EM-TV pass over the subsets (Alg. 3), x updated in place."""
    L = load_library()
    ws = _emtv_ws(geo, ws, x.device)
    d = pe.events.desc()
    off = np.ascontiguousarray(pe.sub_off, dtype=np.int64)
    _check(L.lm_emtv_epoch(C.byref(geo.sc), C.byref(geo.g), C.byref(geo.tof), C.byref(d),
                           off.ctypes.data_as(C.POINTER(C.c_int64)), int(off.shape[0] - 1),
                           _f32(sens_img, geo.V, "sens_img"), _f32(x, geo.V, "x"),
                           float(beta), int(pdhg_iters), float(knorm), _ptr(ws), ws.numel(), _stream(stream)))
    return x


def emtv_em_step(geo: Geometry, ev: DeviceEvents, n_subsets: int, sens_img: torch.Tensor, x: torch.Tensor,
                 out: Optional[torch.Tensor] = None, ws: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """z = x n / g * (P^LM)^T (1 / (P^LM x + s)) over the events of ev."""
    L = load_library()
    ws = _emtv_ws(geo, ws, x.device)
    if out is None:
        out = torch.empty(geo.V, dtype=torch.float32, device=x.device)
    d = ev.desc()
    _check(L.lm_emtv_em_step(C.byref(geo.sc), C.byref(geo.g), C.byref(geo.tof), C.byref(d), int(n_subsets),
                             _f32(sens_img, geo.V, "sens_img"), _f32(x, geo.V, "x"), _f32(out, geo.V, "out"),
                             _ptr(ws), ws.numel(), _stream(stream)))
    return out


def emtv_denoise(geo: Geometry, z: torch.Tensor, w: torch.Tensor, iters: int, knorm: float,
                 out: Optional[torch.Tensor] = None, ws: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """argmin_{u >= 0} sum w/2 (u - z)^2 + ||K u||_{2,1} by `iters` accelerated
    primal-dual iterations; voxels with w <= 0 held at 0."""
    L = load_library()
    ws = _emtv_ws(geo, ws, z.device)
    if out is None:
        out = torch.empty(geo.V, dtype=torch.float32, device=z.device)
    _check(L.lm_emtv_denoise(C.byref(geo.g), _f32(z, geo.V, "z"), _f32(w, geo.V, "w"), _f32(out, geo.V, "out"),
                             int(iters), float(knorm), _ptr(ws),
                             ws.numel(), _stream(stream)))
    return out


def sino_setup(geo: Geometry, d: torch.Tensor, s: torch.Tensor, n_subsets: int,
               lor_factor: Optional[torch.Tensor] = None, stream=None) -> PermutedEvents:
    """The bins of a TOF sinogram (counts d uint16, contamination s float32, both
    in canonical bin order) as an event list for sinogram SPDHG (Alg. 1):
    view-based subsets; ``mu`` holds the counts."""
    L = load_library()
    dev = d.device
    nb = int(L.lm_sino_n_bins(C.byref(geo.sc), C.byref(geo.tof)))
    if d.numel() != nb or s.numel() != nb:
        raise ValueError(f"the sinogram has {nb} bins")
    ev = DeviceEvents(torch.empty(nb, dtype=torch.int32, device=dev), torch.empty(nb, dtype=torch.int32, device=dev),
                      torch.empty(nb, dtype=torch.int16, device=dev), torch.empty(nb, dtype=torch.float32, device=dev),
                      torch.empty(nb, dtype=torch.float32, device=dev))
    mu = torch.empty(nb, dtype=torch.uint16, device=dev)
    off = np.zeros(n_subsets + 1, dtype=np.int64)
    ws = _ws(L.lm_sino_workspace_bytes(C.byref(geo.sc), int(n_subsets)), dev)
    _check(L.lm_sino_setup(C.byref(geo.sc), C.byref(geo.tof), int(n_subsets), _ptr(d, torch.uint16, nb, "d"),
                           _f32(s, nb, "s"), _f32(lor_factor, geo.n_lor, "lor_factor"),
                           _ptr(ev.det1), _ptr(ev.det2), _ptr(ev.tof), _ptr(ev.corr), _ptr(ev.contam), _ptr(mu),
                           off.ctypes.data_as(C.POINTER(C.c_int64)), _ptr(ws), ws.numel(), _stream(stream)))
    return PermutedEvents(ev, mu, off)


@dataclasses.dataclass
class _CountOnly:
    """Event-list descriptor of a generated sinogram: only the bin count."""
    n: int

    def desc(self) -> lm_events:
        return lm_events(None, None, None, None, None, self.n)


@dataclasses.dataclass
class GeneratedSinogram:
    events: _CountOnly
    mu: torch.Tensor          # counts d_b (uint16), subset order
    sub_off: np.ndarray       # int64 [n_subsets + 1] bin offsets
    q: torch.Tensor           # int32 transaxial pairs of the subsets
    qoff: torch.Tensor        # int64 [n_subsets + 1]


def sino_count(geo: Geometry, ev: DeviceEvents, n_subsets: int, stream=None) -> GeneratedSinogram:
    """Histogram of the events over every sinogram bin for the generated
    sinogram layout (lm_params.sinogram = 2)."""
    L = load_library()
    dev = ev.det1.device
    nb = int(L.lm_sino_n_bins(C.byref(geo.sc), C.byref(geo.tof)))
    mu = torch.empty((nb + 1) // 2 * 2, dtype=torch.uint16, device=dev)
    n_pairs = geo.sc.n_xtal * (geo.sc.n_xtal - 1) // 2
    q = torch.empty(n_pairs, dtype=torch.int32, device=dev)
    qoff = torch.empty(n_subsets + 1, dtype=torch.int64, device=dev)
    off = np.zeros(n_subsets + 1, dtype=np.int64)
    ws = _ws(L.lm_sino_workspace_bytes(C.byref(geo.sc), int(n_subsets)), dev)
    d = ev.desc()
    _check(L.lm_sino_count(C.byref(geo.sc), C.byref(geo.tof), int(n_subsets), C.byref(d), _ptr(mu), _ptr(q),
                           _ptr(qoff), off.ctypes.data_as(C.POINTER(C.c_int64)), _ptr(ws), ws.numel(),
                           _stream(stream)))
    return GeneratedSinogram(_CountOnly(nb), mu, off, q, qoff)


class LMSPDHG:
    """Alg. 2 on the device.  Holds the state buffer and the library handle."""

    def __init__(self, geo: Geometry, pe: PermutedEvents, sens_img: torch.Tensor, x0: torch.Tensor, *,
                 beta: float, n_subsets: int, gamma: float = 0.0, rho: float = 0.999, knorm: float = 0.0,
                 knorm_iters: int = 0, deterministic: bool = False, kahan: bool = True, group: int = 0,
                 image_kernel: int = 0, projector: str = "auto", xi: Optional[torch.Tensor] = None,
                 res_fwhm: float = 0.0, sinogram: int = 0, sino_s: float = 0.0,
                 sino_lorf: Optional[torch.Tensor] = None, shard: bool = False, epoch_kernel: int = 0,
                 stream=None):
        L = load_library()
        self.geo, self.pe, self.sens = geo, pe, sens_img
        self.shard = bool(shard)
        self.xi = xi  # directional TV field (referenced by the state), None = TV
        self.n_subsets = n_subsets
        # projector of the data updates: "table" (stored traversals, 40 B per
        # event; 3D TOF data in float-atomic mode without the resolution model
        # or sinogram bins), "direct" (the event kernel), "tiled" (the
        # tile-binned projector, TOF data in float-atomic mode); "auto" takes the
        # table where it applies and the direct kernel elsewhere
        self.tile = None
        self.trav = None
        if projector not in ("auto", "table", "direct", "tiled"):
            raise ValueError("projector must be 'auto', 'table', 'direct' or 'tiled'")
        if projector == "tiled" and geo.tof_nbins > 0 and not deterministic:
            tb = int(L.lmspdhg_tile_bytes(C.byref(geo.g), pe.events.n, int(n_subsets)))
            self.tile = torch.empty(tb, dtype=torch.uint8, device=x0.device)
        table_ok = (geo.tof_nbins > 0 and not deterministic and res_fwhm == 0.0 and sinogram == 0)
        if projector == "table" and not table_ok:
            raise ValueError("the traversal table needs TOF data in float-atomic mode, without the "
                             "resolution model or sinogram bins")
        if projector in ("auto", "table") and table_ok:
            nb = int(L.lmspdhg_trav_bytes(C.byref(geo.g), pe.events.n))
            if nb == 0 and projector == "table":
                raise ValueError("the traversal table needs a 3D grid (n_y, n_z > 1)")
            if nb > 0:
                self.trav = torch.empty(nb, dtype=torch.uint8, device=x0.device)
        self.params = lm_params(beta, gamma, rho, knorm, knorm_iters, n_subsets, int(deterministic), int(kahan),
                                int(group), int(image_kernel), None if self.tile is None else self.tile.data_ptr(),
                                0 if self.tile is None else self.tile.numel(),
                                _f32(xi, geo.ndim * geo.V, "xi"), float(res_fwhm),
                                int(sinogram), _ptr(getattr(pe, "q", None)), _ptr(getattr(pe, "qoff", None)),
                                _f32(sino_lorf, geo.n_lor, "sino_lorf"), float(sino_s),
                                None if self.trav is None else self.trav.data_ptr(),
                                0 if self.trav is None else self.trav.numel(), int(self.shard),
                                int(epoch_kernel), int(projector == "table"))
        self._keep = (sino_lorf,)
        nbytes = L.lmspdhg_state_bytes_ex(C.byref(geo.g), pe.events.n, int(n_subsets), C.byref(self.params))
        if nbytes == 0:
            raise LMError(1, "invalid state size")
        self.buf = torch.empty(int(nbytes), dtype=torch.uint8, device=x0.device)
        self._ev = pe.events.desc()
        self._off = np.ascontiguousarray(pe.sub_off, dtype=np.int64)
        h = C.c_void_p()
        _check(L.lmspdhg_create(C.byref(h), C.byref(geo.sc), C.byref(geo.g), C.byref(geo.tof), C.byref(self._ev),
                                _ptr(pe.mu), self._off.ctypes.data_as(C.POINTER(C.c_int64)),
                                _f32(sens_img, geo.V, "sens_img"), _f32(x0, geo.V, "x0"), C.byref(self.params),
                                _ptr(self.buf), self.buf.numel(), _stream(stream)))
        self.h = h

    def _seq(self, seq):
        a = np.ascontiguousarray(np.asarray(seq, dtype=np.uint16))
        return a, a.ctypes.data_as(C.POINTER(C.c_uint16))

    def updates(self, seq, stream=None):
        a, p = self._seq(seq)
        _check(load_library().lmspdhg_updates(self.h, p, int(a.shape[0]), _stream(stream)))

    def epoch(self, seq, stream=None):
        a, p = self._seq(seq)
        if a.shape[0] != 2 * self.n_subsets:
            raise ValueError("an epoch is 2n updates")
        _check(load_library().lmspdhg_epoch(self.h, p, _stream(stream)))

    def x(self, stream=None) -> torch.Tensor:
        out = torch.empty(self.geo.V, dtype=torch.float32, device=self.buf.device)
        _check(load_library().lmspdhg_get_x(self.h, _ptr(out), _stream(stream)))
        return out

    def y(self, stream=None) -> torch.Tensor:
        out = torch.empty(max(1, self.pe.events.n), dtype=torch.float32, device=self.buf.device)
        _check(load_library().lmspdhg_get_y(self.h, _ptr(out), _stream(stream)))
        return out[:self.pe.events.n]

    def z(self, stream=None) -> torch.Tensor:
        out = torch.empty(self.geo.V, dtype=torch.float32, device=self.buf.device)
        _check(load_library().lmspdhg_get_z(self.h, _ptr(out), _stream(stream)))
        return out

    def w(self, stream=None) -> torch.Tensor:
        out = torch.empty(max(1, self.geo.ndim) * self.geo.V, dtype=torch.float32, device=self.buf.device)
        _check(load_library().lmspdhg_get_w(self.h, _ptr(out), _stream(stream)))
        return out

    def reinit(self, x0: torch.Tensor, stream=None):
        _check(load_library().lmspdhg_reinit(self.h, _f32(x0, self.geo.V, "x0"), _stream(stream)))

    def profile(self, seq, stream=None):
        """Per-kernel timing of `seq` (direct launches with CUDA events)."""
        a, p = self._seq(seq)
        ms = (C.c_double * 4)()
        n = (C.c_int64 * 4)()
        _check(load_library().lmspdhg_profile(self.h, p, int(a.shape[0]), ms, n, _stream(stream)))
        keys = ["data_events", "prior_dual", "image_after_data", "image_after_prior"]
        return {k: (ms[i], n[i]) for i, k in enumerate(keys)}

    def objective(self, stream=None) -> float:
        v = C.c_double()
        _check(load_library().lmspdhg_objective_fp64(self.h, C.byref(v), _stream(stream)))
        return float(v.value)

    # ---- event sharding of one frame (shard=True): see lmspdhg_shard_* ----
    def shard_buffer(self) -> torch.Tensor:
        """The state's exchange buffer (V floats inside the state buffer): the
        partial back-projection of this state's events between shard_begin and
        shard_finish, which the caller sums over the states in place."""
        p = C.c_void_p()
        _check(load_library().lmspdhg_shard_buffer(self.h, C.byref(p)))
        off = p.value - self.buf.data_ptr()
        return self.buf[off:off + 4 * self.geo.V].view(torch.float32)

    def shard_init_finish(self, stream=None):
        _check(load_library().lmspdhg_shard_init_finish(self.h, _stream(stream)))

    def shard_begin(self, sel: int, stream=None):
        _check(load_library().lmspdhg_shard_begin(self.h, int(sel), _stream(stream)))

    def shard_finish(self, stream=None):
        _check(load_library().lmspdhg_shard_finish(self.h, _stream(stream)))

    def shard_init(self, exchange, stream=None):
        """Completes a shard state's initialisation: exchange(buf) must sum the
        states' buffers in place on every rank (e.g. torch.distributed.all_reduce
        over the ranks that share the frame)."""
        exchange(self.shard_buffer())
        self.shard_init_finish(stream)

    def shard_updates(self, seq, exchange, stream=None):
        """The updates of `seq` on a shard state, with exchange(buf) between the
        event kernels and the image pass of every data update (a prior update
        needs none: every rank holds the same x and w)."""
        for sel in np.asarray(seq, dtype=np.int64):
            self.shard_begin(int(sel), stream)
            if sel < self.n_subsets:
                exchange(self.shard_buffer())
            self.shard_finish(stream)

    def objective_parts(self, stream=None):
        out = (C.c_double * 4)()
        _check(load_library().lmspdhg_objective_parts_fp64(self.h, out, _stream(stream)))
        return list(out)

    def info(self):
        n = C.c_int64()
        g = C.c_double()
        k = C.c_double()
        _check(load_library().lmspdhg_info(self.h, C.byref(n), C.byref(g), C.byref(k)))
        return dict(n_updates=n.value, gamma=g.value, knorm=k.value)

    def set_gate(self, flag: Optional[torch.Tensor]):
        """Failure injection for the persistent epoch kernel: its first block
        waits (at most one second) for the device int32 `flag` to become non-zero
        before the first update; None removes the gate."""
        self._gate = flag
        _check(load_library().lmspdhg_set_gate(self.h, None if flag is None else _ptr(flag)))

    def tuning(self):
        g = C.c_int32()
        ms = (C.c_double * 3)()
        _check(load_library().lmspdhg_tuning(self.h, C.byref(g), ms))
        kind = C.c_int32()
        _check(load_library().lmspdhg_image_kernel(self.h, C.byref(kind)))
        pk, nseg = C.c_int32(), C.c_int64()
        _check(load_library().lmspdhg_projector(self.h, C.byref(pk), C.byref(nseg)))
        ek = C.c_int32()
        _check(load_library().lmspdhg_epoch_kernel(self.h, C.byref(ek)))
        tms, dms = C.c_double(), C.c_double()
        _check(load_library().lmspdhg_tuning_projectors(self.h, C.byref(tms), C.byref(dms)))
        return dict(group=g.value, ms_g8=ms[0], ms_g16=ms[1], ms_g32=ms[2],
                    epoch_kernel={1: "graph", 2: "persistent"}[ek.value],
                    data_update_ms_table=tms.value, data_update_ms_direct=dms.value,
                    image_kernel={1: "plain", 2: "tma", 3: "tma_data"}[kind.value],
                    projector={1: "direct", 2: "tiled", 3: "table"}[pk.value], tile_segments=nseg.value)

    def close(self):
        if getattr(self, "h", None):
            load_library().lmspdhg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several LMSPDHG states advanced together, one graph per epoch."""

    def __init__(self, capacity: int, n_subsets: int, device="cuda", stream=None):
        L = load_library()
        self.capacity, self.n_subsets = int(capacity), int(n_subsets)
        nbytes = L.lmspdhg_batch_bytes(self.capacity, self.n_subsets)
        if nbytes == 0:
            raise LMError(1, "invalid batch size")
        self.buf = torch.empty(int(nbytes), dtype=torch.uint8, device=device)
        h = C.c_void_p()
        _check(L.lmspdhg_batch_create(C.byref(h), self.capacity, self.n_subsets, _ptr(self.buf), self.buf.numel(),
                                      _stream(stream)))
        self.h = h
        self.states = [None] * self.capacity

    def set(self, slot: int, state: Optional["LMSPDHG"], stream=None):
        _check(load_library().lmspdhg_batch_set(self.h, int(slot), None if state is None else state.h,
                                                _stream(stream)))
        self.states[slot] = state

    def epoch(self, seqs, stream=None):
        """seqs: dict slot -> sequence (2n) or an array [capacity, 2n]."""
        a = np.zeros((self.capacity, 2 * self.n_subsets), dtype=np.uint16)
        if isinstance(seqs, dict):
            for k, v in seqs.items():
                a[k] = np.asarray(v, dtype=np.uint16)
        else:
            a[:] = np.asarray(seqs, dtype=np.uint16)
        a = np.ascontiguousarray(a)
        _check(load_library().lmspdhg_batch_epoch(self.h, a.ctypes.data_as(C.POINTER(C.c_uint16)),
                                                  _stream(stream)))

    def close(self):
        if getattr(self, "h", None):
            load_library().lmspdhg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching reconstruction server (lm_server_*): frames are
    submitted from host arrays and reconstructed by the library's worker
    thread, several at a time, inside a caller-owned device pool."""

    def __init__(self, geo: "Geometry", sens: torch.Tensor, *, beta: float, knorm: float, n_subsets: int,
                 epochs: int, max_slots: int, max_events: int, pool_bytes: int, rho: float = 0.999,
                 deterministic: bool = False, kahan: bool = True, group: int = 32):
        L = load_library()
        self.geo = geo
        self.sens = sens
        self.n_subsets, self.epochs = int(n_subsets), int(epochs)
        self.cfg = lm_server_config(float(beta), float(rho), float(knorm), self.n_subsets, self.epochs,
                                    int(max_slots), int(deterministic), int(kahan), int(group), int(max_events))
        self.pool = torch.empty(int(pool_bytes), dtype=torch.uint8, device=sens.device)
        h = C.c_void_p()
        _check(L.lm_server_create(C.byref(h), C.byref(geo.sc), C.byref(geo.g), C.byref(geo.tof),
                                  _f32(sens, geo.V, "sens"),
                                  C.byref(self.cfg), _ptr(self.pool), self.pool.numel()))
        self.h = h

    @staticmethod
    def frame_bytes(geo: "Geometry", n_events: int, n_subsets: int, deterministic: bool = False) -> int:
        return int(load_library().lm_server_frame_bytes(C.byref(geo.g), int(n_events), int(n_subsets),
                                                        int(deterministic)))

    def submit(self, det1, det2, tof, corr, contam, x0_value: float, seqs) -> int:
        """Host arrays (numpy); seqs: uint16 [epochs, 2n].  Returns a ticket."""
        d1 = np.ascontiguousarray(det1, dtype=np.int32)
        d2 = np.ascontiguousarray(det2, dtype=np.int32)
        tb = None if tof is None else np.ascontiguousarray(tof, dtype=np.int16)
        cr = None if corr is None else np.ascontiguousarray(corr, dtype=np.float32)
        ct = np.ascontiguousarray(contam, dtype=np.float32)
        sq = np.ascontiguousarray(seqs, dtype=np.uint16).reshape(-1)
        if sq.size != self.epochs * 2 * self.n_subsets:
            raise ValueError("seqs must hold epochs * 2 * n_subsets selections")
        t = C.c_int64()
        hp = lambda a: None if a is None else a.ctypes.data_as(C.c_void_p)
        _check(load_library().lm_server_submit(self.h, hp(d1), hp(d2), hp(tb), hp(cr), hp(ct), int(d1.size),
                                               float(x0_value), sq.ctypes.data_as(C.POINTER(C.c_uint16)),
                                               C.byref(t)))
        return int(t.value)

    def wait(self, ticket: int, timeout_ms: int = 60000, want_x: bool = True):
        """Returns (x or None, objective, latency_ms); raises LMError on
        timeout (code LM_ERR_TIMEOUT, the ticket stays valid) or failure."""
        x = np.empty(self.geo.V, dtype=np.float32) if want_x else None
        obj, lat = C.c_double(), C.c_double()
        _check(load_library().lm_server_wait(self.h, int(ticket), None if x is None else x.ctypes.data_as(C.c_void_p),
                                             C.byref(obj), C.byref(lat), int(timeout_ms)))
        return x, obj.value, lat.value

    def stats(self):
        c, f, q, u, m = C.c_int64(), C.c_int64(), C.c_int64(), C.c_size_t(), C.c_int64()
        _check(load_library().lm_server_stats(self.h, C.byref(c), C.byref(f), C.byref(q), C.byref(u), C.byref(m)))
        return {"completed": c.value, "in_flight": f.value, "queued": q.value, "pool_used": u.value,
                "max_in_flight": m.value}

    def close(self):
        if getattr(self, "h", None):
            load_library().lm_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
