"""Thin Python binding of the C ABI in include/comet_scan.h.

Argument marshalling only: every function takes torch CUDA tensors, checks their dtype, device and
contiguity, and passes raw device pointers to the library function of the same name, on the current
torch stream.  There is no CPU path: if the shared library is missing the import-time loader raises.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import threading
from typing import Optional

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libcomet_scan.so")

COMET_OK = 0
COMET_F32 = 0
COMET_F64 = 1
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "NO_MEMORY", 5: "UNSUPPORTED"}


class CometError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class _Field(C.Structure):
    _fields_ = [("kind", C.c_int32), ("b", C.c_double * 3), ("table", C.c_void_p),
                ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("origin", C.c_double * 3), ("spacing", C.c_double)]


class _Params(C.Structure):
    _fields_ = [("h", C.c_double), ("n_steps", C.c_int32), ("stride", C.c_int32),
                ("lam", C.c_double), ("tol", C.c_double), ("max_iter", C.c_int32),
                ("zmin", C.c_double), ("zmax", C.c_double), ("rmax", C.c_double)]


class _Lattice(C.Structure):
    _fields_ = [("vx", C.c_double), ("vy", C.c_double), ("centre", C.c_double * 4),
                ("half_width", C.c_double * 4), ("counts", C.c_int32 * 4), ("charge", C.c_int32)]


class BatchCaps(C.Structure):
    """Mirror of comet_batch_caps."""
    _fields_ = [("max_events", C.c_int32), ("max_seeds", C.c_int64), ("max_total_seeds", C.c_int64),
                ("max_wires", C.c_int32), ("max_total_wires", C.c_int32), ("dca_ctas_per_sm", C.c_int32),
                ("dca_item_groups", C.c_int32)]


class BatchEvent(C.Structure):
    """Mirror of comet_batch_event (pointers are device addresses)."""
    _fields_ = [("active", C.c_int32), ("lattice", _Lattice), ("n_steps", C.c_int32),
                ("seeds", C.c_void_p), ("charge", C.c_void_p), ("points", C.c_void_p),
                ("n_valid", C.c_void_p), ("bounds", C.c_void_p), ("wires", C.c_void_p),
                ("W", C.c_int32), ("ldw", C.c_int32), ("hit_offsets", C.c_void_p),
                ("drift", C.c_void_p), ("hit_mask", C.c_void_p), ("rss", C.c_void_p),
                ("n_in", C.c_void_p), ("best_idx", C.c_void_p), ("best_rss", C.c_void_p),
                ("hit_class", C.c_void_p), ("n_unconverged", C.c_void_p)]


_lib = None
_lock = threading.Lock()

# (name, argtypes) of every exported entry point
_vp, _i32, _i64 = C.c_void_p, C.c_int32, C.c_int64
SIGNATURES = {
    "comet_ctx_create": [C.c_int, C.POINTER(C.c_void_p)],
    "comet_ctx_destroy": [_vp],
    "comet_ctx_status": [_vp, C.POINTER(C.c_int32)],
    "comet_ctx_set_copy_wait": [_vp, _i64],
    "comet_ctx_set_dca_ctas_per_sm": [_vp, _i32],
    "comet_ctx_set_dca_chunk_wires": [_vp, _i32],
    "comet_ctx_set_record_blocks": [_vp, _i32],
    "comet_kernel_arch": [C.POINTER(C.c_int32)],
    "comet_last_error": [],
    "comet_scan_lattice": [_vp, C.c_int, C.POINTER(_Lattice), _vp, _vp, _i64, _vp],
    "comet_scan_propagate": [_vp, C.c_int, C.POINTER(_Field), C.POINTER(_Params), _vp, _vp, _i64,
                             _vp, _vp, _vp, _vp],
    "comet_scan_dca": [_vp, C.c_int, C.POINTER(_Field), C.POINTER(_Params), _vp, _vp, _vp, _i64,
                       _vp, _vp, _i32, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "comet_scan_select": [_vp, C.c_int, _vp, _i64, _i32, _vp, _vp, _vp],
    "comet_scan_select_noalloc": [C.c_int, _vp, _i64, _i32, _vp, _vp, _vp],
    "comet_scan_refine_refs": [_vp, C.c_int, _vp, _i64, _vp, _i32, C.POINTER(C.c_double), _i32, _vp,
                               _vp, _vp],
    "comet_scan_lattice_refined": [_vp, C.c_int, C.POINTER(_Lattice), _vp, _vp, _i32, _vp, _vp, _i64,
                                   _vp],
    "comet_scan_jacobian": [_vp, C.c_int, C.POINTER(_Field), C.POINTER(_Params), _vp, _i64, C.c_double,
                            C.c_double, _i32, _vp, _i32, _i32, _vp, _vp, _vp, C.c_double, _vp, _vp,
                            _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "comet_scan_gn_step": [_vp, _vp, _i64, _vp, _vp, C.c_double, _vp],
    "comet_scan_lm_step": [_vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, C.c_double,
                           C.c_double, _i32, _vp],
    "comet_scan_batch_update": [_vp, C.c_int, C.POINTER(_Field), C.POINTER(_Params),
                                C.POINTER(BatchCaps), C.POINTER(BatchEvent), _i32],
    "comet_scan_batch": [_vp, C.c_int, C.POINTER(_Field), C.POINTER(_Params), C.POINTER(BatchCaps),
                         C.POINTER(BatchEvent), _i32, _vp],
    "comet_scan_classify": [_vp, C.c_int, C.POINTER(_Field), C.POINTER(_Params), _vp, _vp, _vp,
                            _i64, _vp, _vp, _i32, _i32, _vp, _vp, _vp, _vp, _vp, _i32, _vp],
}


def lib():
    """The loaded library (built by ``paper_1911_09340_gb300.build``).  Raises if it is absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing: build it with "
                                  "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = C.CDLL(LIB_PATH)
            for name, args in SIGNATURES.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = None if name == "comet_ctx_destroy" else (
                    C.c_char_p if name == "comet_last_error" else C.c_int)
            _lib = L
    return _lib


def _check(status: int):
    if status != COMET_OK:
        raise CometError(status, lib().comet_last_error().decode())


_DTYPE = {torch.float32: 0, torch.float64: 1}


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return COMET_F32
    if t.dtype == torch.float64:
        return COMET_F64
    raise TypeError(f"expected float32 or float64, got {t.dtype}")


def _ptr(t: Optional[torch.Tensor], dtype=None) -> Optional[int]:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


@dataclasses.dataclass
class ScanParams:
    """Mirror of comet_scan_params (see include/comet_scan.h)."""
    h: float = 1e-3
    n_steps: int = 2200
    stride: int = 1
    lam: float = 1e-2
    tol: float = 1e-12
    max_iter: int = 16
    zmin: float = -0.80
    zmax: float = 0.80
    rmax: float = 0.90

    @property
    def n_rec(self) -> int:
        return self.n_steps // self.stride + 1

    def c(self) -> _Params:
        return _Params(self.h, self.n_steps, self.stride, self.lam, self.tol, self.max_iter,
                       self.zmin, self.zmax, self.rmax)


class DeviceField:
    """Mirror of comet_field.  ``table`` [3][nz][ny][nx] (if given) is copied to the device as
    float32, component-major (kind 1) or, with ``interleaved``, as [nz][ny][nx][4] (kind 2: one
    16-byte load per grid node; identical results)."""

    def __init__(self, kind: int = 0, b=(0.0, 0.0, 1.0), table=None, origin=(0.0, 0.0, 0.0),
                 spacing: float = 0.0, device="cuda", interleaved: bool = False):
        self.kind = kind
        self.b = tuple(float(x) for x in b)
        self.table = None
        self.origin = tuple(float(x) for x in origin)
        self.spacing = float(spacing)
        if kind in (1, 2):
            t = torch.as_tensor(table).to(dtype=torch.float32)
            self.shape = tuple(t.shape[1:])          # (nz, ny, nx)
            if interleaved or kind == 2:
                self.kind = 2
                t4 = torch.zeros(self.shape + (4,), dtype=torch.float32)
                t4[..., :3] = t.permute(1, 2, 3, 0)
                t = t4
            self.table = t.to(device=device).contiguous()

    @classmethod
    def from_synth(cls, f, device="cuda", interleaved: bool = False):
        return cls(f.kind, f.b, f.table, f.origin, f.spacing, device, interleaved)

    def c(self) -> _Field:
        if self.kind == 0:
            return _Field(0, (C.c_double * 3)(*self.b), None, 0, 0, 0, (C.c_double * 3)(0, 0, 0), 0.0)
        nz, ny, nx = self.shape
        return _Field(self.kind, (C.c_double * 3)(*self.b), self.table.data_ptr(), nx, ny, nz,
                      (C.c_double * 3)(*self.origin), self.spacing)


class Context:
    """Owns a comet_ctx bound to one CUDA device."""

    def __init__(self, device: int = 0):
        h = C.c_void_p()
        _check(lib().comet_ctx_create(int(device), C.byref(h)))
        self.handle = h
        self.device = device
        self.record_blocks = 1

    def status(self) -> int:
        v = C.c_int32(0)
        _check(lib().comet_ctx_status(self.handle, C.byref(v)))
        return v.value

    def set_copy_wait(self, ns: int):
        """Limit (ns) of a kernel's wait for a staging bulk copy; 0 forces the plain-load path."""
        _check(lib().comet_ctx_set_copy_wait(self.handle, int(ns)))

    def set_dca_chunk_wires(self, wires: int):
        """Wires per chunk of the DCA's per-seed sums (0: automatic)."""
        _check(lib().comet_ctx_set_dca_chunk_wires(self.handle, int(wires)))

    def set_record_blocks(self, on: int):
        """1 (default): FP64 axial-field recording of few seeds one super-segment per warp; 0: one
        warp per 32 seeds always (bit-identical to the batched recording)."""
        _check(lib().comet_ctx_set_record_blocks(self.handle, int(on)))
        self.record_blocks = int(on)

    def set_dca_ctas_per_sm(self, n: int):
        """Cap of the persistent DCA launch's resident CTAs per SM (0: as many as fit)."""
        _check(lib().comet_ctx_set_dca_ctas_per_sm(self.handle, int(n)))

    def close(self):
        if self.handle:
            lib().comet_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lattice_struct(spec) -> _Lattice:
    return _Lattice(float(spec.vxy[0]), float(spec.vxy[1]), (C.c_double * 4)(*spec.centre),
                    (C.c_double * 4)(*spec.half_width), (C.c_int32 * 4)(*spec.counts),
                    int(spec.charge))


def comet_scan_lattice(ctx: Context, spec, seeds: torch.Tensor, charge: Optional[torch.Tensor] = None,
                       stream=None):
    lat = lattice_struct(spec)
    _check(lib().comet_scan_lattice(ctx.handle, _dtype_code(seeds), C.byref(lat), _ptr(seeds),
                                    _ptr(charge, torch.int8), seeds.shape[-1], _stream(stream)))


BOUNDS_PER_GROUP = 200     # float4 bounding spheres per 32-seed group (8 + 8 * 24)


def bounds_shape(S: int):
    """Shape of the optional search-bounds tensor (float32) for S seeds."""
    return ((S + 31) // 32, BOUNDS_PER_GROUP, 4)


def comet_scan_propagate(ctx: Context, field: DeviceField, params: ScanParams, seeds, charge,
                         points, n_valid, bounds=None, stream=None):
    dt = _dtype_code(seeds)
    S = seeds.shape[-1]
    f, p = field.c(), params.c()
    _check(lib().comet_scan_propagate(ctx.handle, dt, C.byref(f), C.byref(p), _ptr(seeds),
                                      _ptr(charge, torch.int8), S, _ptr(points, seeds.dtype),
                                      _ptr(n_valid, torch.int32), _ptr(bounds, torch.float32),
                                      _stream(stream)))


def comet_scan_dca(ctx: Context, field: DeviceField, params: ScanParams, points, n_valid, charge,
                   wires, hit_offsets, drift, hit_mask, rss, n_in, dca_out=None, n_unconverged=None,
                   n_wires: Optional[int] = None, bounds=None, stream=None, best_idx=None,
                   best_rss=None):
    """``wires`` is [6][ldw]; the first ``n_wires`` columns (default: all) are the wires.
    ``best_idx`` ([1] int64) / ``best_rss`` ([1]): the seed of lowest RSS selected in the launch."""
    dt = _dtype_code(points)
    S = n_valid.shape[0]
    ldw = wires.shape[-1]
    W = ldw if n_wires is None else int(n_wires)
    f, p = field.c(), params.c()
    _check(lib().comet_scan_dca(ctx.handle, dt, C.byref(f), C.byref(p), _ptr(points),
                                _ptr(n_valid, torch.int32), _ptr(charge, torch.int8), S,
                                _ptr(bounds, torch.float32), _ptr(wires, points.dtype), W, ldw, _ptr(hit_offsets, torch.int32),
                                _ptr(drift, points.dtype), _ptr(hit_mask, torch.uint8),
                                _ptr(rss, points.dtype), _ptr(n_in, torch.int32),
                                _ptr(dca_out, points.dtype), _ptr(n_unconverged, torch.int32),
                                _ptr(best_idx, torch.int64), _ptr(best_rss, points.dtype),
                                _stream(stream)))


def comet_scan_select(ctx: Context, rss, k: int, idx_out, rss_out=None, stream=None):
    _check(lib().comet_scan_select(ctx.handle, _dtype_code(rss), _ptr(rss), rss.shape[0], int(k),
                                   _ptr(idx_out, torch.int64), _ptr(rss_out, rss.dtype),
                                   _stream(stream)))


def comet_scan_select_noalloc(rss, k: int, idx_out, rss_out=None, stream=None):
    """comet_scan_select without a context and without device allocation (static scratch on the
    device that holds ``rss``; see include/comet_scan.h for its size limit and sharing rules).  Runs
    with that device current, on its current stream unless ``stream`` is given."""
    for t in (idx_out, rss_out):
        if t is not None and t.device != rss.device:
            raise ValueError("rss, idx_out and rss_out must be on one device")
    with torch.cuda.device(rss.device):
        st = stream if stream is not None else torch.cuda.current_stream(rss.device)
        _check(lib().comet_scan_select_noalloc(_dtype_code(rss), _ptr(rss), rss.shape[0], int(k),
                                               _ptr(idx_out, torch.int64), _ptr(rss_out, rss.dtype),
                                               st.cuda_stream))


def kernel_arch() -> int:
    """SM version of the library's device code (major * 10 + minor) on the current device."""
    v = C.c_int32(0)
    _check(lib().comet_kernel_arch(C.byref(v)))
    return v.value


def comet_scan_refine_refs(ctx: Context, seeds, idx, half_width, K: int, refs_out, n_refs_out,
                           stream=None):
    """Sparse reference points for a finer scan: ``refs_out`` [K, 4] float64 (z0, phi, pz, pT),
    ``n_refs_out`` [1] int32, both on the device."""
    hw = (C.c_double * 4)(*[float(v) for v in half_width])
    _check(lib().comet_scan_refine_refs(ctx.handle, _dtype_code(seeds), _ptr(seeds), seeds.shape[-1],
                                        _ptr(idx, torch.int64), idx.shape[0], hw, int(K),
                                        _ptr(refs_out, torch.float64), _ptr(n_refs_out, torch.int32),
                                        _stream(stream)))


def comet_scan_lattice_refined(ctx: Context, shape_spec, refs, n_refs, K: int, seeds,
                               charge: Optional[torch.Tensor] = None, stream=None):
    """K lattices of ``shape_spec``'s half-widths and counts around the references (centre ignored)."""
    lat = lattice_struct(shape_spec)
    _check(lib().comet_scan_lattice_refined(ctx.handle, _dtype_code(seeds), C.byref(lat),
                                            _ptr(refs, torch.float64), _ptr(n_refs, torch.int32),
                                            int(K), _ptr(seeds), _ptr(charge, torch.int8),
                                            seeds.shape[-1], _stream(stream)))


JAC_WORK_PER_PAIR = 11   # doubles of comet_scan_jacobian scratch per (seed, wire)


def comet_scan_jacobian(ctx: Context, field: DeviceField, params: ScanParams, theta, vx: float,
                        vy: float, charge: int, wires, hit_offsets, drift, hit_mask, tau: float, work,
                        srss, grad, jtj, jtr, dca_out=None, jac_out=None, n_unconverged=None,
                        n_wires: Optional[int] = None, stream=None, grad6=None):
    """Smoothed RSS, its gradient and the Gauss-Newton normal equations of seeds theta [S, 4]
    (float64 device; z0, phi, pz, pT); see include/comet_scan.h."""
    f64 = torch.float64
    ldw = wires.shape[-1]
    W = ldw if n_wires is None else int(n_wires)
    f, p = field.c(), params.c()
    _check(lib().comet_scan_jacobian(ctx.handle, COMET_F64, C.byref(f), C.byref(p), _ptr(theta, f64),
                                     theta.shape[0], float(vx), float(vy), int(charge),
                                     _ptr(wires, f64), W, ldw, _ptr(hit_offsets, torch.int32),
                                     _ptr(drift, f64), _ptr(hit_mask, torch.uint8), float(tau),
                                     _ptr(work, f64), _ptr(srss, f64), _ptr(grad, f64), _ptr(jtj, f64),
                                     _ptr(jtr, f64), _ptr(dca_out, f64), _ptr(jac_out, f64),
                                     _ptr(grad6, f64), _ptr(n_unconverged, torch.int32),
                                     _stream(stream)))


def comet_scan_gn_step(ctx: Context, theta, jtj, jtr, mu: float = 0.0, stream=None):
    f64 = torch.float64
    _check(lib().comet_scan_gn_step(ctx.handle, _ptr(theta, f64), theta.shape[0], _ptr(jtj, f64),
                                    _ptr(jtr, f64), float(mu), _stream(stream)))


def comet_scan_lm_step(ctx: Context, theta, srss, jtj, jtr, theta_try, srss_try, jtj_try, jtr_try, mu,
                       up: float = 3.0, down: float = 1.0 / 3.0, first: bool = False, stream=None):
    """Levenberg-Marquardt accept/reject of the trial seeds and the next trial (see
    include/comet_scan.h); every array float64 on the device, the trial's may be None when first."""
    f64 = torch.float64
    _check(lib().comet_scan_lm_step(ctx.handle, theta.shape[0], _ptr(theta, f64), _ptr(srss, f64),
                                    _ptr(jtj, f64), _ptr(jtr, f64), _ptr(theta_try, f64),
                                    _ptr(srss_try, f64), _ptr(jtj_try, f64), _ptr(jtr_try, f64),
                                    _ptr(mu, f64), float(up), float(down), int(bool(first)),
                                    _stream(stream)))


def comet_scan_batch_update(ctx: Context, dtype, field: DeviceField, params: ScanParams, caps: BatchCaps,
                            events, B: int):
    """Packs B comet_batch_event descriptors (a ctypes array) into the context's staging buffer."""
    f, p = field.c(), params.c()
    _check(lib().comet_scan_batch_update(ctx.handle, _DTYPE[dtype], C.byref(f), C.byref(p),
                                         C.byref(caps), events, int(B)))


def comet_scan_batch(ctx: Context, dtype, field: DeviceField, params: ScanParams, caps: BatchCaps,
                     events=None, B: int = 0, stream=None):
    """Enqueues the last packed batch (after packing ``events`` when given)."""
    f, p = field.c(), params.c()
    _check(lib().comet_scan_batch(ctx.handle, _DTYPE[dtype], C.byref(f), C.byref(p), C.byref(caps),
                                  events, int(B), _stream(stream)))


def comet_scan_classify(ctx: Context, field: DeviceField, params: ScanParams, points, n_valid,
                        charge, seed_index, wires, hit_offsets, drift, hit_mask, hit_class,
                        dca_wire=None, update_mask: bool = False, n_wires: Optional[int] = None,
                        stream=None):
    dt = _dtype_code(points)
    S = n_valid.shape[0]
    ldw = wires.shape[-1]
    W = ldw if n_wires is None else int(n_wires)
    f, p = field.c(), params.c()
    _check(lib().comet_scan_classify(ctx.handle, dt, C.byref(f), C.byref(p), _ptr(points),
                                     _ptr(n_valid, torch.int32), _ptr(charge, torch.int8), S,
                                     _ptr(seed_index, torch.int64), _ptr(wires, points.dtype), W,
                                     ldw, _ptr(hit_offsets, torch.int32), _ptr(drift, points.dtype),
                                     _ptr(hit_mask, torch.uint8), _ptr(hit_class, torch.uint8),
                                     _ptr(dca_wire, points.dtype), int(bool(update_mask)),
                                     _stream(stream)))
