"""Thin Python binding of the C ABI in include/mt.h (libmagtile.so).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Functions carry the ABI's names; handles are wrapped in small
owner objects that release them.  Device buffers are torch CUDA tensors
(torch provides memory and streams, nothing else).  If the library has not
been built, importing this module raises: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import sys

import numpy as np

from . import build as _build

MT_OK, MT_EINVAL, MT_ENOMEM, MT_EOVERLAP, MT_ENOCONV, MT_ETIMEOUT, MT_ENONFINITE, MT_ECUDA, MT_EBUSY = range(9)
MT_F64, MT_F32, MT_BF16_SCALED, MT_BF16_SPLIT = range(4)
MT_FORM_GILBERT, MT_FORM_LL = 0, 1
(MT_LAYOUT_STREAM, MT_LAYOUT_DENSE, MT_LAYOUT_SPARSE, MT_LAYOUT_STREAM6, MT_LAYOUT_STREAM_FULL,
 MT_LAYOUT_STREAM_HALF) = 0, 1, 2, 3, 4, 5
MT_PATH_GRAPH, MT_PATH_PERSISTENT = 1, 2
PREC_NAMES = {"f64": MT_F64, "f32": MT_F32, "bf16": MT_BF16_SCALED, "bf16_scaled": MT_BF16_SCALED,
              "split": MT_BF16_SPLIT, "bf16_split": MT_BF16_SPLIT}


class MtError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__("%s failed with status %d: %s" % (where, status, message))
        self.status = status


class LlgParams(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("alpha", ctypes.c_void_p), ("Ha", ctypes.c_void_p),
                ("form", ctypes.c_int), ("precess", ctypes.c_int), ("exch_scale", ctypes.c_void_p)]


class OdeOpts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("atol", ctypes.c_double), ("h0", ctypes.c_double),
                ("hmax", ctypes.c_double), ("max_steps", ctypes.c_int64), ("fixed_h", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("n_accept", ctypes.c_int64), ("n_reject", ctypes.c_int64), ("n_rhs", ctypes.c_int64),
                ("t", ctypes.c_double), ("h", ctypes.c_double), ("tau", ctypes.c_double),
                ("status", ctypes.c_int32), ("pad", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


class TensorInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("prec", ctypes.c_int32), ("rows_per_panel", ctypes.c_int32),
                ("cols_per_chunk", ctypes.c_int32), ("layout", ctypes.c_int32), ("planes", ctypes.c_int32),
                ("bytes", ctypes.c_int64), ("near_blocks", ctypes.c_int64), ("half", ctypes.c_int32),
                ("row_warps", ctypes.c_int32)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_batch", ctypes.c_int32), ("prec", ctypes.c_int32),
                ("layout", ctypes.c_int32), ("form", ctypes.c_int32), ("gamma", ctypes.c_double),
                ("ode", OdeOpts), ("replays_per_poll", ctypes.c_int32), ("max_running", ctypes.c_int32)]


MT_JOB_RELAX, MT_JOB_SWEEP = 0, 1


class Job(ctypes.Structure):
    _fields_ = [("geometry", ctypes.c_int32), ("kind", ctypes.c_int32), ("alpha", ctypes.c_double),
                ("Ha", ctypes.c_double * 3), ("m0", ctypes.c_void_p), ("tol", ctypes.c_double),
                ("t_max", ctypes.c_double), ("n_fields", ctypes.c_int64), ("fields", ctypes.c_void_p)]


class JobResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("geometry", ctypes.c_int32), ("t_submit", ctypes.c_double),
                ("t_start", ctypes.c_double), ("t_done", ctypes.c_double), ("n_accept", ctypes.c_int64),
                ("n_reject", ctypes.c_int64), ("n_rhs", ctypes.c_int64), ("t_sim", ctypes.c_double),
                ("tau", ctypes.c_double), ("values_done", ctypes.c_int64), ("values_converged", ctypes.c_int64)]

    def as_dict(self):
        return {k: (list(v) if hasattr(v, "__len__") else v) for k, v in
                ((k, getattr(self, k)) for k, _ in self._fields_)}


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("evictions", ctypes.c_int64), ("assemblies", ctypes.c_int64), ("resident", ctypes.c_int64),
                ("bytes_in_use", ctypes.c_size_t), ("budget", ctypes.c_size_t)]


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_D = ctypes.c_double
_I = ctypes.c_int
_PP = ctypes.POINTER(ctypes.c_void_p)

# name -> (restype, argtypes); mirrors include/mt.h
_SIGS = {
    "mt_version": (ctypes.c_char_p, []),
    "mt_last_error": (ctypes.c_char_p, []),
    "mt_ctx_create": (_I, [_I, ctypes.c_size_t, _PP]),
    "mt_ctx_destroy": (None, [_P]),
    "mt_ctx_bytes_in_use": (ctypes.c_size_t, [_P]),
    "mt_selftest_wait_timeout": (_I, [_P, _D]),
    "mt_tiles_create": (_I, [_P, _I64, _P, _P, _P, _P, _P, _P, _P, _PP]),
    "mt_tiles_create_tetra": (_I, [_P, _I64, _P, _I64, _P, _P, _P, _P, _P, _PP]),
    "mt_tiles_destroy": (None, [_P]),
    "mt_demag_assemble": (_I, [_P, _I, _PP]),
    "mt_demag_assemble_ex": (_I, [_P, _I, _I, _PP]),
    "mt_tensor_destroy": (None, [_P]),
    "mt_tensor_threshold": (_I, [_P, _D, _PP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]),
    "mt_tensor_get_info": (_I, [_P, ctypes.POINTER(TensorInfo)]),
    "mt_tensor_read_rows": (_I, [_P, _I64, _I64, _P]),
    "mt_demag_blocks": (_I, [_P, _I64, _P, _P]),
    "mt_demag_field": (_I, [_P, _P, _I, _P, _P]),
    "mt_demag_field_f64": (_I, [_P, _P, _I, _P, _P]),
    "mt_demag_field_noalloc": (_I, [_P, _P, _I, _P, _P]),
    "mt_llg_rhs": (_I, [_P, ctypes.POINTER(LlgParams), _P, _I, _P, _P, _P]),
    "mt_energy": (_I, [_P, ctypes.POINTER(LlgParams), _P, _I, _P, _P]),
    "mt_integrator_create": (_I, [_P, ctypes.POINTER(LlgParams), ctypes.POINTER(OdeOpts), _I, _P, _PP]),
    "mt_integrator_destroy": (None, [_P]),
    "mt_integrator_set_state": (_I, [_P, _P, _I, _D]),
    "mt_integrator_get_state": (_I, [_P, _P, _I]),
    "mt_integrator_set_params": (_I, [_P, ctypes.POINTER(LlgParams)]),
    "mt_integrator_stream": (_P, [_P]),
    "mt_integrator_step": (_I, [_P, _I64]),
    "mt_integrator_run": (_I, [_P, _D, _I64, _P, _P]),
    "mt_integrator_relax": (_I, [_P, _D, _D, _P]),
    "mt_integrator_hysteresis": (_I, [_P, _P, _P, _I64, _D, _D, _P, _P, _P, _P, _P]),
    "mt_integrator_crossover": (_I, [_P, _P, _I, _P, _P, _D, _D, _P, _P, _P, _P, _P]),
    "mt_integrator_stats": (_I, [_P, _P]),
    "mt_integrator_checkpoint_bytes": (_I, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    "mt_integrator_checkpoint": (_I, [_P, _P, ctypes.c_size_t]),
    "mt_integrator_restore": (_I, [_P, _P, ctypes.c_size_t]),
    "mt_integrator_set_path": (_I, [_P, _I]),
    "mt_selftest_grid_barrier_timeout": (_I, [_P]),
    "mt_integrator_get_path": (_I, [_P]),
    "mt_integrate": (_I, [_P, ctypes.POINTER(LlgParams), ctypes.POINTER(OdeOpts), _P, _I, _D, _D, _I64, _P, _P,
                          _P]),
    "mt_relax": (_I, [_P, ctypes.POINTER(LlgParams), ctypes.POINTER(OdeOpts), _D, _D, _P, _I, _P, _P]),
    "mt_server_create": (_I, [_P, ctypes.POINTER(ServerOpts), _PP]),
    "mt_server_add_geometry": (_I, [_P, _I64, _P, _P, _P, _P, _P, _P, _P, ctypes.POINTER(ctypes.c_int32)]),
    "mt_server_submit": (_I, [_P, ctypes.POINTER(Job), ctypes.POINTER(ctypes.c_uint64)]),
    "mt_server_wait": (_I, [_P, ctypes.c_uint64, _D, ctypes.POINTER(JobResult), _P, _P]),
    "mt_server_get_stats": (_I, [_P, ctypes.POINTER(ServerStats)]),
    "mt_server_destroy": (None, [_P]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libmagtile.so; raises if it was not built (no fallback)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise ImportError("libmagtile.so is not built (%s); run paper_2107_05364_gb300.build.build() "
                              "or __graft_entry__.build()" % path)
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols() -> list[str]:
    return sorted(_SIGS)


def _check(status: int, where: str):
    if status != MT_OK:
        raise MtError(status, where, lib().mt_last_error().decode())


def _ptr(x):
    """Raw pointer of a numpy array or torch tensor (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return ctypes.c_void_p(x.ctypes.data)
    return ctypes.c_void_p(x.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _device_vector(x, count: int, dtype_name: str, device: int, where: str, what: str):
    """Refuse anything but a contiguous torch CUDA tensor of `count`
    elements of the given dtype on the library context's device: the kernels
    read and write exactly that many elements through the raw pointer, so a
    host array, a short tensor, a strided view or another device's memory
    would become an out-of-bounds device access."""
    import torch
    dt = getattr(torch, dtype_name)
    if not isinstance(x, torch.Tensor):
        raise ValueError("%s: %s must be a torch CUDA tensor, got %s" % (where, what, type(x).__name__))
    if not x.is_cuda:
        raise ValueError("%s: %s is in host memory; a CUDA tensor is required" % (where, what))
    if x.dtype != dt:
        raise ValueError("%s: %s has dtype %s, %s is required" % (where, what, x.dtype, dt))
    if not x.is_contiguous():
        raise ValueError("%s: %s must be contiguous" % (where, what))
    if x.numel() != count:
        raise ValueError("%s: %s has %d elements, %d (B * 3n) are required" % (where, what, x.numel(), count))
    if x.device.index != device:
        raise ValueError("%s: %s is on cuda:%s, the context is on cuda:%d" % (where, what, x.device.index, device))


def _tensor_device(T) -> int:
    return int(T.tiles.ctx.device)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a if shape is None else a.reshape(shape)


# ---------------------------------------------------------------------------
# handle owners
# ---------------------------------------------------------------------------
class Ctx:
    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        h = ctypes.c_void_p()
        _check(lib().mt_ctx_create(device, hbm_budget_bytes, ctypes.byref(h)), "mt_ctx_create")
        self.h = h
        self.device = device

    def bytes_in_use(self) -> int:
        return int(lib().mt_ctx_bytes_in_use(self.h))

    def close(self):
        if self.h:
            lib().mt_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        # at interpreter exit the CUDA runtime may already be gone: leave the
        # memory to the process teardown
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


class TilesH:
    def __init__(self, ctx: Ctx, tiles=None, tetra=None):
        """tiles: cuboid tile set (centre, edge, Ms, Aex, Ku, axis, nbr);
        tetra: (vertices (nv, 3), tets (n, 4), Ms, Aex, Ku, axis)."""
        self.ctx = ctx
        if tetra is not None:
            verts, tets, Ms, Aex, Ku, axis = tetra
            verts = _f64(verts)
            tets = np.ascontiguousarray(tets, np.int32)
            n = tets.shape[0]
            self.n = n
            arrs = [_f64(np.broadcast_to(np.asarray(Ms, np.float64), (n,))),
                    _f64(np.broadcast_to(np.asarray(Aex, np.float64), (n,))),
                    _f64(np.broadcast_to(np.asarray(Ku, np.float64), (n,))),
                    _f64(np.broadcast_to(np.asarray(axis, np.float64).reshape(-1, 3), (n, 3)))]
            h = ctypes.c_void_p()
            _check(lib().mt_tiles_create_tetra(ctx.h, verts.size // 3, _ptr(verts), n, _ptr(tets),
                                               *[_ptr(a) for a in arrs], ctypes.byref(h)), "mt_tiles_create_tetra")
            self.h = h
            return
        self.n = int(tiles.centre.shape[0])
        arrs = [_f64(tiles.centre), _f64(tiles.edge), _f64(tiles.Ms), _f64(tiles.Aex), _f64(tiles.Ku),
                _f64(tiles.axis)]
        nbr = None if tiles.nbr is None else np.ascontiguousarray(tiles.nbr, np.int32)
        h = ctypes.c_void_p()
        _check(lib().mt_tiles_create(ctx.h, self.n, *[_ptr(a) for a in arrs], _ptr(nbr), ctypes.byref(h)),
               "mt_tiles_create")
        self.h = h

    def close(self):
        if self.h:
            lib().mt_tiles_destroy(self.h)
            self.h = None

    def __del__(self):
        # at interpreter exit the CUDA runtime may already be gone: leave the
        # memory to the process teardown
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


class TensorH:
    def __init__(self, tiles: TilesH, prec, layout: int = MT_LAYOUT_STREAM):
        prec = PREC_NAMES[prec] if isinstance(prec, str) else int(prec)
        h = ctypes.c_void_p()
        _check(lib().mt_demag_assemble_ex(tiles.h, prec, int(layout), ctypes.byref(h)), "mt_demag_assemble_ex")
        self.layout = int(layout)
        self.h = h
        self.tiles = tiles
        self.n = tiles.n
        self.prec = prec

    def info(self) -> dict:
        inf = TensorInfo()
        _check(lib().mt_tensor_get_info(self.h, ctypes.byref(inf)), "mt_tensor_get_info")
        return {k: getattr(inf, k) for k, _ in inf._fields_}

    def close(self):
        if self.h:
            lib().mt_tensor_destroy(self.h)
            self.h = None

    def __del__(self):
        # at interpreter exit the CUDA runtime may already be gone: leave the
        # memory to the process teardown
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


def llg_params(B: int, gamma=2.211e5, alpha=0.02, Ha=(0.0, 0.0, 0.0), form=MT_FORM_GILBERT, precess=1,
               exch_scale=None):
    """Returns (LlgParams, keep-alive arrays)."""
    a = np.ascontiguousarray(np.broadcast_to(np.asarray(alpha, np.float64), (B,)))
    h = np.ascontiguousarray(np.broadcast_to(np.asarray(Ha, np.float64).reshape(-1, 3), (B, 3)))
    x = None if exch_scale is None else np.ascontiguousarray(
        np.broadcast_to(np.asarray(exch_scale, np.float64), (B,)))
    p = LlgParams(float(gamma), a.ctypes.data, h.ctypes.data, int(form), int(precess),
                  None if x is None else x.ctypes.data)
    return p, (a, h, x)


def ode_opts(rtol=1e-6, atol=1e-6, h0=1e-14, hmax=1e-11, max_steps=10_000_000, fixed_h=0.0):
    return OdeOpts(float(rtol), float(atol), float(h0), float(hmax), int(max_steps), float(fixed_h))


# ---------------------------------------------------------------------------
# ABI functions (same names)
# ---------------------------------------------------------------------------
def mt_version() -> str:
    return lib().mt_version().decode()


def mt_ctx_create(device: int = 0, hbm_budget_bytes: int = 0) -> Ctx:
    return Ctx(device, hbm_budget_bytes)


def mt_selftest_wait_timeout(ctx: Ctx, limit_s: float = 0.2) -> int:
    """Status of the bounded-wait self-test (MT_ETIMEOUT = works as designed)."""
    return int(lib().mt_selftest_wait_timeout(ctx.h, float(limit_s)))


def mt_selftest_grid_barrier_timeout(ctx: Ctx) -> int:
    """Status of the grid-barrier self-test (MT_ETIMEOUT = works as designed)."""
    return int(lib().mt_selftest_grid_barrier_timeout(ctx.h))


def mt_tiles_create(ctx: Ctx, tiles) -> TilesH:
    return TilesH(ctx, tiles)


def mt_tiles_create_tetra(ctx: Ctx, vertices, tets, Ms, Aex, Ku, axis=(0.0, 0.0, 1.0)) -> TilesH:
    return TilesH(ctx, tetra=(vertices, tets, Ms, Aex, Ku, axis))


def mt_demag_assemble(tiles: TilesH, prec="f32") -> TensorH:
    return TensorH(tiles, prec)


def mt_demag_assemble_ex(tiles: TilesH, prec="bf16", layout: int = MT_LAYOUT_DENSE) -> TensorH:
    return TensorH(tiles, prec, layout)


class _Wrapped(TensorH):
    """A tensor handle made by a library call other than assembly."""

    def __init__(self, h, tiles, prec, layout):  # noqa: D401 - plain holder
        self.h = h
        self.tiles = tiles
        self.n = tiles.n
        self.prec = prec
        self.layout = layout


def mt_tensor_threshold(T: TensorH, fraction: float):
    """Sec. 4.3.1 thresholded copy: returns (tensor, cut value t, kept elements)."""
    h = ctypes.c_void_p()
    thr = ctypes.c_double()
    kept = ctypes.c_int64()
    _check(lib().mt_tensor_threshold(T.h, float(fraction), ctypes.byref(h), ctypes.byref(thr), ctypes.byref(kept)),
           "mt_tensor_threshold")
    return _Wrapped(h, T.tiles, MT_F32, MT_LAYOUT_SPARSE), thr.value, kept.value


def mt_tensor_read_rows(T: TensorH, i0: int, i1: int) -> np.ndarray:
    out = np.empty((i1 - i0, T.n, 6))
    _check(lib().mt_tensor_read_rows(T.h, i0, i1, _ptr(out)), "mt_tensor_read_rows")
    return out


def mt_demag_blocks(tiles: TilesH, pairs) -> np.ndarray:
    pr = np.ascontiguousarray(pairs, np.int64).reshape(-1, 2)
    out = np.empty((pr.shape[0], 6))
    _check(lib().mt_demag_blocks(tiles.h, pr.shape[0], _ptr(pr), _ptr(out)), "mt_demag_blocks")
    return out


def _field_args(T, m, H, B, dtype_name, where):
    if int(B) < 1:
        raise ValueError("%s: B must be >= 1" % where)
    dev = _tensor_device(T)
    _device_vector(m, 3 * T.n * int(B), dtype_name, dev, where, "m")
    _device_vector(H, 3 * T.n * int(B), dtype_name, dev, where, "H")


def mt_demag_field(T: TensorH, m, H, B: int = 1, stream=None):
    """m, H: torch CUDA float32 tensors of B*3n elements."""
    _field_args(T, m, H, B, "float32", "mt_demag_field")
    _check(lib().mt_demag_field(T.h, _ptr(m), B, _ptr(H), _stream(stream)), "mt_demag_field")


def mt_demag_field_f64(T: TensorH, m, H, B: int = 1, stream=None):
    """m, H: torch CUDA float64 tensors of B*3n elements."""
    _field_args(T, m, H, B, "float64", "mt_demag_field_f64")
    _check(lib().mt_demag_field_f64(T.h, _ptr(m), B, _ptr(H), _stream(stream)), "mt_demag_field_f64")


def mt_demag_field_noalloc(T: TensorH, m, H, B: int = 1, stream=None):
    """mt_demag_field without any device allocation by the library: work
    areas come from a fixed per-GPU array (see include/mt.h).  Calls that
    overlap on the GPU race; the first call on a device should precede any
    stream capture."""
    _field_args(T, m, H, B, "float32", "mt_demag_field_noalloc")
    _check(lib().mt_demag_field_noalloc(T.h, _ptr(m), B, _ptr(H), _stream(stream)), "mt_demag_field_noalloc")


def mt_llg_rhs(T: TensorH, params: LlgParams, m, dmdt, tau=None, B: int = 1, stream=None):
    """m, dmdt: torch CUDA float32 tensors of B*3n elements; tau: None or B floats."""
    _field_args(T, m, dmdt, B, "float32", "mt_llg_rhs")
    if tau is not None:
        _device_vector(tau, int(B), "float32", _tensor_device(T), "mt_llg_rhs", "tau")
    _check(lib().mt_llg_rhs(T.h, ctypes.byref(params), _ptr(m), B, _ptr(dmdt), _ptr(tau), _stream(stream)),
           "mt_llg_rhs")


def mt_energy(T: TensorH, params: LlgParams, m, B: int = 1, stream=None) -> np.ndarray:
    """Energies (J) of B states: (B, 5) = total, Zeeman, demag, exchange, anisotropy."""
    if int(B) < 1:
        raise ValueError("mt_energy: B must be >= 1")
    _device_vector(m, 3 * T.n * int(B), "float32", _tensor_device(T), "mt_energy", "m")
    E = np.zeros((B, 5))
    _check(lib().mt_energy(T.h, ctypes.byref(params), _ptr(m), B, _ptr(E), _stream(stream)), "mt_energy")
    return E


def mt_integrate(T: TensorH, params: LlgParams, opts: OdeOpts, m, t0: float, t1: float, n_out: int = 1, B: int = 1,
                 stream=None, check: bool = True):
    """One-call integration of the DEVICE state m (torch CUDA float32, B*3n,
    in/out) from t0 to t1; returns (status, mavg (n_out, B, 3), stats)."""
    if int(B) < 1:
        raise ValueError("mt_integrate: B must be >= 1")
    _device_vector(m, 3 * T.n * int(B), "float32", _tensor_device(T), "mt_integrate", "m")
    mavg = np.zeros((int(n_out), int(B), 3))
    st = (Stats * int(B))()
    s = lib().mt_integrate(T.h, ctypes.byref(params), ctypes.byref(opts), _ptr(m), int(B), float(t0), float(t1),
                           int(n_out), _ptr(mavg), st, _stream(stream))
    if check:
        _check(s, "mt_integrate")
    return s, mavg, [x.as_dict() for x in st]


def mt_relax(T: TensorH, params: LlgParams, opts: OdeOpts, m, tol: float, t_max: float, B: int = 1, stream=None,
             check: bool = True):
    """One-call relaxation (Eq. 2) of the DEVICE state m (torch CUDA
    float32, B*3n, in/out); returns (status, stats)."""
    if int(B) < 1:
        raise ValueError("mt_relax: B must be >= 1")
    _device_vector(m, 3 * T.n * int(B), "float32", _tensor_device(T), "mt_relax", "m")
    st = (Stats * int(B))()
    s = lib().mt_relax(T.h, ctypes.byref(params), ctypes.byref(opts), float(tol), float(t_max), _ptr(m), int(B), st,
                       _stream(stream))
    if check:
        _check(s, "mt_relax")
    return s, [x.as_dict() for x in st]


class Integrator:
    """Owner of an mt_integrator handle (Dormand-Prince state of B sims)."""

    def __init__(self, T: TensorH, params: LlgParams, opts: OdeOpts, B: int = 1, stream=None):
        h = ctypes.c_void_p()
        self._stream = _stream(stream)
        _check(lib().mt_integrator_create(T.h, ctypes.byref(params), ctypes.byref(opts), B, self._stream,
                                          ctypes.byref(h)), "mt_integrator_create")
        self.h = h
        self.T = T
        self.B = B
        self.n = T.n

    def set_state(self, m, t0: float = 0.0):
        """m: numpy float32 (host) or torch CUDA float32, B*3n elements."""
        is_host = isinstance(m, np.ndarray)
        if is_host:
            m = np.ascontiguousarray(m, np.float32)
            if m.size != self.B * 3 * self.n:
                raise ValueError("set_state: %d elements, %d (B * 3n) are required" % (m.size, self.B * 3 * self.n))
            self._host_keep = m
        else:
            _device_vector(m, self.B * 3 * self.n, "float32", _tensor_device(self.T), "set_state", "m")
        _check(lib().mt_integrator_set_state(self.h, _ptr(m), int(is_host), float(t0)), "mt_integrator_set_state")

    def get_state(self, out=None):
        if out is None:
            out = np.empty((self.B, self.n, 3), np.float32)
        is_host = isinstance(out, np.ndarray)
        if is_host:
            if out.dtype != np.float32 or not out.flags.c_contiguous or out.size != self.B * 3 * self.n:
                raise ValueError("get_state: a contiguous float32 array of B * 3n elements is required")
        else:
            _device_vector(out, self.B * 3 * self.n, "float32", _tensor_device(self.T), "get_state", "out")
        _check(lib().mt_integrator_get_state(self.h, _ptr(out), int(is_host)), "mt_integrator_get_state")
        return out

    def set_params(self, params: LlgParams):
        _check(lib().mt_integrator_set_params(self.h, ctypes.byref(params)), "mt_integrator_set_params")

    def path(self) -> int:
        """MT_PATH_GRAPH or MT_PATH_PERSISTENT: how the steps execute."""
        return int(lib().mt_integrator_get_path(self.h))

    def set_path(self, path: int):
        _check(lib().mt_integrator_set_path(self.h, int(path)), "mt_integrator_set_path")

    def checkpoint(self) -> bytes:
        """Byte image of the dynamic state (times, step sizes, counters, m,
        the next step's starting derivative); see mt_integrator_checkpoint."""
        nb = ctypes.c_size_t()
        _check(lib().mt_integrator_checkpoint_bytes(self.h, ctypes.byref(nb)), "mt_integrator_checkpoint_bytes")
        buf = ctypes.create_string_buffer(nb.value)
        _check(lib().mt_integrator_checkpoint(self.h, buf, nb.value), "mt_integrator_checkpoint")
        return buf.raw

    def restore(self, image: bytes):
        """Load a checkpoint image (same n and B)."""
        image = bytes(image)
        _check(lib().mt_integrator_restore(self.h, ctypes.c_char_p(image), len(image)), "mt_integrator_restore")

    def stream_handle(self) -> int:
        """cudaStream_t of the integrator's launches (for timing)."""
        return int(lib().mt_integrator_stream(self.h) or 0)

    def step(self, nsteps: int):
        _check(lib().mt_integrator_step(self.h, int(nsteps)), "mt_integrator_step")

    def run(self, t1: float, n_out: int = 1, check: bool = True):
        mavg = np.zeros((n_out, self.B, 3))
        st = (Stats * self.B)()
        s = lib().mt_integrator_run(self.h, float(t1), int(n_out), _ptr(mavg), st)
        if check:
            _check(s, "mt_integrator_run")
        return s, mavg, [x.as_dict() for x in st]

    def relax(self, tol: float, t_max: float, check: bool = True):
        st = (Stats * self.B)()
        s = lib().mt_integrator_relax(self.h, float(tol), float(t_max), st)
        if check:
            _check(s, "mt_integrator_relax")
        return s, [x.as_dict() for x in st]

    def hysteresis(self, direction, H, t_step: float, tol: float = 0.0):
        """Field schedule H[s] * direction_b (A/m), relaxed at each value;
        returns (mavg (S, B, 3), tau (S, B), hc (B,), mr (B, 3), stats)."""
        d = np.ascontiguousarray(np.broadcast_to(np.asarray(direction, np.float64).reshape(-1, 3), (self.B, 3)))
        H = np.ascontiguousarray(H, np.float64).ravel()
        S = H.size
        mavg = np.zeros((S, self.B, 3))
        tau = np.zeros((S, self.B))
        hc = np.zeros(self.B)
        mr = np.zeros((self.B, 3))
        st = (Stats * self.B)()
        _check(lib().mt_integrator_hysteresis(self.h, _ptr(d), _ptr(H), S, float(t_step), float(tol), _ptr(mavg),
                                              _ptr(tau), _ptr(hc), _ptr(mr), st), "mt_integrator_hysteresis")
        return mavg, tau, hc, mr, [x.as_dict() for x in st]

    def crossover(self, lam, mA, mB, tol: float, t_max: float, states: bool = False):
        """Relax families A and B at sizes lam (B = 2K); returns (eA, eB
        (J/m^3), lam_cross, relaxed states (B, n, 3) or None, stats)."""
        lam = np.ascontiguousarray(lam, np.float64).ravel()
        K = lam.size
        mA = np.ascontiguousarray(mA, np.float32).ravel()
        mB = np.ascontiguousarray(mB, np.float32).ravel()
        eA, eB = np.zeros(K), np.zeros(K)
        lc = ctypes.c_double(0.0)
        mo = np.empty((self.B, self.n, 3), np.float32) if states else None
        st = (Stats * self.B)()
        _check(lib().mt_integrator_crossover(self.h, _ptr(lam), K, _ptr(mA), _ptr(mB), float(tol), float(t_max),
                                             _ptr(eA), _ptr(eB), ctypes.byref(lc), _ptr(mo), st),
               "mt_integrator_crossover")
        return eA, eB, lc.value, mo, [x.as_dict() for x in st]

    def stats(self):
        st = (Stats * self.B)()
        _check(lib().mt_integrator_stats(self.h, st), "mt_integrator_stats")
        return [x.as_dict() for x in st]

    def close(self):
        if self.h:
            lib().mt_integrator_destroy(self.h)
            self.h = None

    def __del__(self):
        # at interpreter exit the CUDA runtime may already be gone: leave the
        # memory to the process teardown
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


def mt_integrator_create(T: TensorH, params: LlgParams, opts: OdeOpts, B: int = 1, stream=None) -> Integrator:
    return Integrator(T, params, opts, B, stream)


class Server:
    """Owner of an mt_server handle: relax jobs on many geometries,
    continuously batched on the device (see include/mt.h)."""

    def __init__(self, ctx: Ctx, max_batch: int = 16, prec="f32", layout: int = MT_LAYOUT_STREAM,
                 hbm_budget_bytes: int = 0, gamma: float = 2.211e5, form: int = MT_FORM_GILBERT,
                 opts: OdeOpts | None = None, replays_per_poll: int = 0, max_running: int = 0):
        prec = PREC_NAMES[prec] if isinstance(prec, str) else int(prec)
        o = ServerOpts(int(hbm_budget_bytes), int(max_batch), prec, int(layout), int(form), float(gamma),
                       opts or ode_opts(rtol=1e-5, atol=1e-5), int(replays_per_poll), int(max_running))
        h = ctypes.c_void_p()
        _check(lib().mt_server_create(ctx.h, ctypes.byref(o), ctypes.byref(h)), "mt_server_create")
        self.h = h
        self.ctx = ctx
        self.n = {}
        self._sweeps = {}

    def add_geometry(self, tiles) -> int:
        arrs = [_f64(tiles.centre), _f64(tiles.edge), _f64(tiles.Ms), _f64(tiles.Aex), _f64(tiles.Ku),
                _f64(tiles.axis)]
        nbr = None if tiles.nbr is None else np.ascontiguousarray(tiles.nbr, np.int32)
        gid = ctypes.c_int32()
        n = int(arrs[0].size // 3)
        _check(lib().mt_server_add_geometry(self.h, n, *[_ptr(a) for a in arrs], _ptr(nbr), ctypes.byref(gid)),
               "mt_server_add_geometry")
        self.n[gid.value] = n
        return gid.value

    def submit(self, geometry: int, m0, alpha: float = 0.5, Ha=(0.0, 0.0, 0.0), tol: float = 1e-4,
               t_max: float = 1e-9, fields=None) -> int:
        """A relax job (fields None: relax at Ha) or a sweep job (fields:
        (S, 3) applied fields in A/m, relaxed at in turn, t_max per value)."""
        m0 = np.ascontiguousarray(m0, np.float32).ravel()
        if m0.size != 3 * self.n[int(geometry)]:
            raise ValueError("submit: m0 has %d values, %d (3n) are required" % (m0.size, 3 * self.n[int(geometry)]))
        f = None if fields is None else np.ascontiguousarray(fields, np.float64).reshape(-1, 3)
        j = Job(int(geometry), MT_JOB_RELAX if f is None else MT_JOB_SWEEP, float(alpha),
                (ctypes.c_double * 3)(*[float(x) for x in Ha]), m0.ctypes.data, float(tol), float(t_max),
                0 if f is None else f.shape[0], None if f is None else f.ctypes.data)
        jid = ctypes.c_uint64()
        _check(lib().mt_server_submit(self.h, ctypes.byref(j), ctypes.byref(jid)), "mt_server_submit")
        if f is not None:
            self._sweeps[jid.value] = f.shape[0]
        return jid.value

    def wait(self, job_id: int, timeout_s: float = 60.0, geometry: int | None = None):
        """Returns (status, result dict, final m (n,3) or None); a sweep
        job's result dict also holds "sweep": (S, 4) = <m>, torque per value."""
        res = JobResult()
        m = None
        if geometry is not None:
            m = np.empty((self.n[geometry], 3), np.float32)
        nf = self._sweeps.get(job_id)
        sw = None if nf is None else np.full((nf, 4), np.nan)
        s = lib().mt_server_wait(self.h, ctypes.c_uint64(job_id), float(timeout_s), ctypes.byref(res), _ptr(m),
                                 _ptr(sw))
        d = res.as_dict()
        if s == MT_OK and nf is not None:
            d["sweep"] = sw
            del self._sweeps[job_id]
        return s, d, m

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().mt_server_get_stats(self.h, ctypes.byref(st)), "mt_server_get_stats")
        return {k: getattr(st, k) for k, _ in st._fields_}

    def close(self):
        if self.h:
            lib().mt_server_destroy(self.h)
            self.h = None

    def __del__(self):
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


def mt_server_create(ctx: Ctx, **kw) -> Server:
    return Server(ctx, **kw)
