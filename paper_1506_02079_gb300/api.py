"""Thin Python binding of libemfuse.so (argument marshalling only).

Every function has the name of the C entry point it calls (``include/emfuse.h``).  Tensors
are PyTorch tensors used purely as device (or pinned host) memory; all arithmetic runs in the
library's CUDA kernels on the current PyTorch stream.  A missing library raises
``EmfuseUnavailable``; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

from . import build as _build

__all__ = [
    "EmfuseError", "EmfuseUnavailable", "SolveOpts", "SliceStats", "lib", "library_path",
    "default_opts", "emfuse_smooth_z", "emfuse_smooth_z_robust", "emfuse_smooth_z_noalloc",
    "emfuse_screened_poisson",
    "emfuse_autotune_result", "TuneEntry", "emfuse_fuse_color", "emfuse_screened_poisson_dct",
    "emfuse_smooth_gradient_domain", "emfuse_smooth_gradient_domain_mg", "emfuse_correct_stack",
    "emfuse_backward", "emfuse_version", "emfuse_release_cache", "emfuse_kernel_binary_version",
    "emfuse_probe_fp64_fma_rate", "PendingStats", "EMFUSE_U8", "EMFUSE_F32", "PREC_FP32", "PREC_MIXED",
    "PREC_FP64", "EXPORTED_SYMBOLS",
]

EMFUSE_U8, EMFUSE_F32 = 0, 1
PREC_FP32, PREC_MIXED, PREC_FP64 = 0, 1, 2
STATUS = {0: "EMFUSE_OK", 1: "EMFUSE_EINVAL", 2: "EMFUSE_ECUDA", 3: "EMFUSE_ENOMEM",
          4: "EMFUSE_ENOCONV", 5: "EMFUSE_ETIMEOUT"}
EXPORTED_SYMBOLS = ["emfuse_default_opts", "emfuse_smooth_z", "emfuse_screened_poisson",
                    "emfuse_correct_stack", "emfuse_backward", "emfuse_last_error",
                    "emfuse_version", "emfuse_kernel_launches", "emfuse_profile_begin",
                    "emfuse_profile_end", "emfuse_release_cache", "emfuse_smooth_z_noalloc",
                    "emfuse_selftest_fpconv", "emfuse_autotune_result", "emfuse_smooth_z_robust",
                    "emfuse_fuse_color", "emfuse_screened_poisson_dct", "emfuse_smooth_gradient_domain",
                    "emfuse_smooth_gradient_domain_mg",
                    "emfuse_selftest_wait_timeout", "emfuse_kernel_binary_version",
                    "emfuse_probe_fp64_fma_rate"]


class EmfuseError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class EmfuseUnavailable(RuntimeError):
    pass


class SolveOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_vcycles", ctypes.c_int), ("nu_pre", ctypes.c_int),
                ("nu_post", ctypes.c_int), ("precision", ctypes.c_int), ("fused", ctypes.c_int),
                ("first_vcycles", ctypes.c_int), ("tile_rows", ctypes.c_int), ("autotune", ctypes.c_int),
                ("no_graphs", ctypes.c_int), ("robust_kappa", ctypes.c_float), ("host_pipeline", ctypes.c_int),
                ("verify_residual", ctypes.c_int), ("async_solve", ctypes.c_int), ("host_chunk", ctypes.c_int)]


class TuneEntry(ctypes.Structure):
    _fields_ = [("nu_pre", ctypes.c_int), ("nu_post", ctypes.c_int), ("tile_rows", ctypes.c_int),
                ("vcycles", ctypes.c_int), ("ms", ctypes.c_double)]


class SliceStats(ctypes.Structure):
    _fields_ = [("vcycles", ctypes.c_int), ("converged", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("b_norm", ctypes.c_double),
                ("rel_residual_check", ctypes.c_double)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB_PATH


def lib() -> ctypes.CDLL:
    """The loaded libemfuse.so (loaded once; raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise EmfuseUnavailable(
                    f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
            L = ctypes.CDLL(path)
            i64, vp, fl, db, ci = ctypes.c_int64, ctypes.c_void_p, ctypes.c_float, ctypes.c_double, ctypes.c_int
            L.emfuse_default_opts.argtypes = [ctypes.POINTER(SolveOpts)]
            L.emfuse_default_opts.restype = None
            L.emfuse_smooth_z.argtypes = [vp, ci, vp, i64, i64, i64, i64, i64, i64, fl, fl, vp]
            L.emfuse_smooth_z_robust.argtypes = [vp, ci, vp, i64, i64, i64, i64, i64, i64, fl, fl, fl, vp]
            L.emfuse_fuse_color.argtypes = [vp, vp, vp, i64, i64, i64, db, ctypes.POINTER(SolveOpts), vp, vp]
            L.emfuse_screened_poisson_dct.argtypes = [vp, vp, vp, i64, i64, i64, db, ci, vp]
            L.emfuse_smooth_gradient_domain.argtypes = [vp, ci, vp, i64, i64, i64, db, ci, vp]
            L.emfuse_smooth_gradient_domain_mg.argtypes = [vp, ci, vp, i64, i64, i64, db,
                                                           ctypes.POINTER(SolveOpts), vp, vp]
            L.emfuse_selftest_wait_timeout.argtypes = [ci, vp]
            L.emfuse_selftest_wait_timeout.restype = ci
            L.emfuse_smooth_z_noalloc.argtypes = [vp, ci, vp, i64, i64, i64, i64, i64, i64, fl, fl, vp]
            L.emfuse_selftest_fpconv.argtypes = [vp, vp]
            L.emfuse_kernel_binary_version.argtypes = [vp]
            L.emfuse_kernel_binary_version.restype = ci
            L.emfuse_probe_fp64_fma_rate.argtypes = [vp, vp]
            L.emfuse_probe_fp64_fma_rate.restype = ci
            L.emfuse_autotune_result.argtypes = [vp, ci]
            L.emfuse_autotune_result.restype = ci
            L.emfuse_selftest_fpconv.restype = ci
            L.emfuse_screened_poisson.argtypes = [vp, vp, vp, i64, vp, vp, vp, db,
                                                  ctypes.POINTER(SolveOpts), vp, vp]
            L.emfuse_correct_stack.argtypes = [vp, ci, ci, vp, i64, i64, i64, fl, fl, db,
                                               ctypes.POINTER(SolveOpts), vp, vp]
            L.emfuse_backward.argtypes = [vp, vp, vp, vp, ci, i64, i64, i64, fl, fl, db, vp, vp, vp,
                                          vp, vp, ctypes.POINTER(SolveOpts), vp]
            for name in ("emfuse_smooth_z", "emfuse_screened_poisson", "emfuse_correct_stack",
                         "emfuse_backward", "emfuse_smooth_z_noalloc", "emfuse_smooth_z_robust",
                         "emfuse_fuse_color", "emfuse_screened_poisson_dct", "emfuse_smooth_gradient_domain"):
                getattr(L, name).restype = ci
            L.emfuse_last_error.restype = ctypes.c_char_p
            L.emfuse_last_error.argtypes = []
            L.emfuse_version.restype = ctypes.c_char_p
            L.emfuse_version.argtypes = []
            L.emfuse_kernel_launches.restype = ctypes.c_uint64
            L.emfuse_kernel_launches.argtypes = []
            L.emfuse_release_cache.restype = None
            L.emfuse_release_cache.argtypes = []
            _lib = L
        return _lib


def emfuse_version() -> str:
    return lib().emfuse_version().decode()


def emfuse_kernel_binary_version() -> int:
    """Binary version (major * 10 + minor) of the library's device code on the current device."""
    v = ctypes.c_int(0)
    _check(lib().emfuse_kernel_binary_version(ctypes.byref(v)))
    return v.value


def emfuse_probe_fp64_fma_rate(device: torch.device | None = None) -> float:
    """Measured FP64 FMA throughput of the current device in TFLOP/s (CUDA events)."""
    dev = device or torch.device("cuda", torch.cuda.current_device())
    v = ctypes.c_double(0.0)
    _check(lib().emfuse_probe_fp64_fma_rate(ctypes.byref(v), ctypes.c_void_p(_stream_ptr(dev))))
    return v.value


def emfuse_release_cache() -> None:
    """Free the solver plans and workspaces kept between calls."""
    lib().emfuse_release_cache()


def default_opts(**kw) -> SolveOpts:
    o = SolveOpts()
    lib().emfuse_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _check(code: int, allow_noconv: bool = False):
    if code == 0 or (allow_noconv and code == 4):
        return code
    raise EmfuseError(code, lib().emfuse_last_error().decode())


def _stream_ptr(device: torch.device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.uint8:
        return EMFUSE_U8
    if t.dtype == torch.float32:
        return EMFUSE_F32
    raise TypeError(f"unsupported dtype {t.dtype}: use uint8 or float32")


def _require_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise ValueError("expected a CUDA tensor")
        if t is not None and not t.is_contiguous():
            raise ValueError("expected a contiguous tensor")


class PendingStats:
    """Per-slice results of an asynchronous solve (opts.async_solve = 1).  The library writes
    them from a stream callback; ``result()`` waits for the stream to pass the solve and returns
    them.  Holds the array the callback writes into until then."""

    def __init__(self, arr, stream_ptr: int, device: torch.device):
        self._arr = arr
        # an event recorded right after the call on the stream it was queued on (the current
        # PyTorch stream, the default stream included) completes after the stream callback
        self._done = torch.cuda.Event()
        self._done.record(torch.cuda.current_stream(device))

    def result(self) -> list[dict]:
        self._done.synchronize()
        return _stats_list(self._arr)


def _is_async(opts) -> bool:
    return opts is not None and bool(getattr(opts, "async_solve", 0))


def _stats_list(arr) -> list[dict]:
    return [{"vcycles": s.vcycles, "converged": bool(s.converged), "rel_residual": s.rel_residual,
             "b_norm": s.b_norm, "rel_residual_check": s.rel_residual_check} for s in arr]


def emfuse_smooth_z(stack: torch.Tensor, sigma_xy: float = 1.0, sigma_z: float = 3.0,
                    out: torch.Tensor | None = None, z0: int = 0, z1: int | None = None) -> torch.Tensor:
    """Phase 1 (Sec. 3 "Anisotropic Smoothing"): I1 = I0 * G.  ``stack`` is [z][y][x] on CUDA."""
    _require_cuda(stack)
    nz, ny, nx = stack.shape
    z1 = nz if z1 is None else z1
    if out is None:
        out = torch.empty((z1 - z0, ny, nx), device=stack.device, dtype=torch.float32)
    _require_cuda(out)
    _check(lib().emfuse_smooth_z(stack.data_ptr(), _dtype_code(stack), out.data_ptr(), nx, ny, nz,
                                 nx, z0, z1, float(sigma_xy), float(sigma_z), _stream_ptr(stack.device)))
    return out


def emfuse_smooth_z_robust(stack: torch.Tensor, sigma_xy: float = 1.0, sigma_z: float = 3.0, kappa: float = 2.0,
                           out: torch.Tensor | None = None, z0: int = 0, z1: int | None = None) -> torch.Tensor:
    """Phase 1 with robust averaging across slices (values beyond kappa weighted standard
    deviations of each z-window's weighted mean are left out; Sec. 3, the outlier example)."""
    _require_cuda(stack)
    nz, ny, nx = stack.shape
    z1 = nz if z1 is None else z1
    if out is None:
        out = torch.empty((z1 - z0, ny, nx), device=stack.device, dtype=torch.float32)
    _require_cuda(out)
    _check(lib().emfuse_smooth_z_robust(stack.data_ptr(), _dtype_code(stack), out.data_ptr(), nx, ny, nz,
                                        nx, z0, z1, float(sigma_xy), float(sigma_z), float(kappa),
                                        _stream_ptr(stack.device)))
    return out


def emfuse_smooth_z_noalloc(stack: torch.Tensor, sigma_xy: float, sigma_z: float, out: torch.Tensor,
                            z0: int = 0, z1: int | None = None) -> torch.Tensor:
    """Allocation-free variant of :func:`emfuse_smooth_z` (the library allocates no device
    memory; ``out`` is the caller's).  Calls that overlap on the GPU race on its shared scratch."""
    _require_cuda(stack)
    _require_cuda(out)
    nz, ny, nx = stack.shape
    z1 = nz if z1 is None else z1
    _check(lib().emfuse_smooth_z_noalloc(stack.data_ptr(), _dtype_code(stack), out.data_ptr(), nx, ny,
                                         nz, nx, z0, z1, float(sigma_xy), float(sigma_z),
                                         _stream_ptr(stack.device)))
    return out


def emfuse_selftest_fpconv() -> tuple[int, int]:
    """Mismatch counts (widening, rounding) of the library's integer-pipe float/double
    conversions against the hardware conversions on the current CUDA device."""
    a, b = ctypes.c_int64(-1), ctypes.c_int64(-1)
    _check(lib().emfuse_selftest_fpconv(ctypes.byref(a), ctypes.byref(b)))
    return int(a.value), int(b.value)


def emfuse_autotune_result() -> list[dict]:
    """Candidates timed by the last autotuning solve on this thread, the chosen one first."""
    n = lib().emfuse_autotune_result(None, 0)
    buf = (TuneEntry * max(n, 1))()
    n = lib().emfuse_autotune_result(ctypes.addressof(buf), n)
    return [{"nu_pre": e.nu_pre, "nu_post": e.nu_post, "tile_rows": e.tile_rows, "vcycles": e.vcycles,
             "ms": e.ms} for e in buf[:n]]


def _pack_slices(s, o):
    """Accept 3-D stacks (uniform batch) or lists of 2-D slices (ragged batch)."""
    if isinstance(s, torch.Tensor) and s.dim() == 3:
        nz, ny, nx = s.shape
        nxs = np.full(nz, nx, dtype=np.int64)
        nys = np.full(nz, ny, dtype=np.int64)
        offs = np.arange(nz, dtype=np.int64) * nx * ny
        return s.contiguous(), o.contiguous(), nxs, nys, offs, None
    if isinstance(s, torch.Tensor) and s.dim() == 2:
        return _pack_slices(s[None], o[None])
    shapes = [tuple(t.shape) for t in s]
    nys = np.array([a for a, _ in shapes], dtype=np.int64)
    nxs = np.array([b for _, b in shapes], dtype=np.int64)
    offs = np.zeros(len(shapes), dtype=np.int64)
    offs[1:] = np.cumsum(nys * nxs)[:-1]
    sp = torch.cat([t.reshape(-1) for t in s])
    op = torch.cat([t.reshape(-1) for t in o])
    return sp, op, nxs, nys, offs, shapes


def emfuse_screened_poisson(s, o, alpha: float, opts: SolveOpts | None = None, *, nx=None, ny=None,
                            offsets=None, out: torch.Tensor | None = None, return_stats: bool = False,
                            allow_noconv: bool = False):
    """Phase 2 (Eq. (1)): (alpha I + L) f = alpha s + L o for every slice.

    ``s``/``o``: CUDA float32 stacks [z][y][x], single slices [y][x], lists of slices, or packed
    1-D buffers together with ``nx``, ``ny``, ``offsets`` (host int64 arrays).
    """
    if nx is not None:
        sp, op = s, o
        nxs, nys, offs = (np.ascontiguousarray(a, dtype=np.int64) for a in (nx, ny, offsets))
        shapes = "packed"
    else:
        sp, op, nxs, nys, offs, shapes = _pack_slices(s, o)
    _require_cuda(sp, op)
    if sp.dtype != torch.float32 or op.dtype != torch.float32:
        raise TypeError("s and o must be float32")
    f = torch.empty_like(sp) if out is None else out
    _require_cuda(f)
    n = len(nxs)
    stats = (SliceStats * n)()
    asynchronous = _is_async(opts)
    # an asynchronous solve writes stats later, from a stream callback: only when they are
    # returned (PendingStats keeps the array alive until then)
    want_stats = return_stats or not asynchronous
    code = lib().emfuse_screened_poisson(
        sp.data_ptr(), op.data_ptr(), f.data_ptr(), n, nxs.ctypes.data, nys.ctypes.data,
        offs.ctypes.data, float(alpha), ctypes.byref(opts) if opts is not None else None,
        ctypes.addressof(stats) if want_stats else None, _stream_ptr(sp.device))
    _check(code, allow_noconv)
    if shapes not in (None, "packed"):
        f = [f[int(a):int(a) + h * w].view(h, w) for a, (h, w) in zip(offs, shapes)]
    elif isinstance(s, torch.Tensor) and s.dim() == 2 and nx is None:
        f = f[0]
    if not return_stats:
        return f
    return (f, PendingStats(stats, _stream_ptr(sp.device), sp.device)) if asynchronous else (f, _stats_list(stats))


def emfuse_screened_poisson_dct(s: torch.Tensor, o: torch.Tensor, alpha: float, precision: int = PREC_FP64,
                                out: torch.Tensor | None = None) -> torch.Tensor:
    """Direct solve of Eq. (1) by fast transforms (cuFFT on the mirror-extended slices) for a
    uniform batch: ``s``, ``o`` CUDA float32 [z][y][x] or [y][x]; precision PREC_FP32 / PREC_FP64."""
    _require_cuda(s, o)
    s3 = s[None] if s.dim() == 2 else s
    o3 = o[None] if o.dim() == 2 else o
    if s3.shape != o3.shape or s3.dtype != torch.float32 or o3.dtype != torch.float32:
        raise ValueError("s and o must be float32 with the same shape")
    n, ny, nx = s3.shape
    f = torch.empty_like(s3) if out is None else out.view(n, ny, nx)
    _check(lib().emfuse_screened_poisson_dct(s3.data_ptr(), o3.data_ptr(), f.data_ptr(), n, nx, ny, float(alpha),
                                             int(precision), _stream_ptr(s3.device)))
    return f[0] if s.dim() == 2 else f


def emfuse_smooth_gradient_domain(stack: torch.Tensor, alpha: float, precision: int = PREC_FP32,
                                  out: torch.Tensor | None = None) -> torch.Tensor:
    """Phase 1 as the 3-D gradient-domain problem of the earlier method (Sec. 3 "Alternate
    Solutions": target gradients with their z-components zeroed, screened by alpha), solved
    exactly: a DCT along z (GEMM) splits it into slice problems solved by the batched
    mirror-extension FFT.  ``stack`` CUDA uint8 or float32
    [z][y][x]; precision PREC_FP32 / PREC_FP64.  Returns float32 of the same shape."""
    _require_cuda(stack)
    if stack.dim() != 3 or not stack.is_contiguous():
        raise ValueError("stack must be a contiguous [z][y][x] tensor")
    nz, ny, nx = stack.shape
    if out is None:
        out = torch.empty((nz, ny, nx), device=stack.device, dtype=torch.float32)
    _require_cuda(out)
    _check(lib().emfuse_smooth_gradient_domain(stack.data_ptr(), _dtype_code(stack), out.data_ptr(), nx, ny, nz,
                                               float(alpha), int(precision), _stream_ptr(stack.device)))
    return out


def emfuse_smooth_gradient_domain_mg(stack: torch.Tensor, alpha: float, opts: SolveOpts | None = None,
                                     out: torch.Tensor | None = None, return_stats: bool = False,
                                     allow_noconv: bool = False):
    """The 3-D gradient-domain smoothing by multigrid on the stack (Sec. 3 "Alternate Solutions"):
    FP32 V-cycles on the 7-point operator with FP64 defect correction to opts.tol.  ``stack``
    CUDA uint8 or float32 [z][y][x].  Returns float32 of the same shape (and with return_stats
    one dict for the whole stack)."""
    _require_cuda(stack)
    if stack.dim() != 3 or not stack.is_contiguous():
        raise ValueError("stack must be a contiguous [z][y][x] tensor")
    nz, ny, nx = stack.shape
    if out is None:
        out = torch.empty((nz, ny, nx), device=stack.device, dtype=torch.float32)
    _require_cuda(out)
    opts = opts if opts is not None else default_opts()
    stats = (SliceStats * 1)()
    code = lib().emfuse_smooth_gradient_domain_mg(stack.data_ptr(), _dtype_code(stack), out.data_ptr(), nx, ny, nz,
                                                  float(alpha), ctypes.byref(opts), ctypes.addressof(stats),
                                                  _stream_ptr(stack.device))
    _check(code, allow_noconv)
    return (out, _stats_list(stats)[0]) if return_stats else out


def emfuse_fuse_color(s_rgb: torch.Tensor, o_grey: torch.Tensor, alpha: float, opts: SolveOpts | None = None,
                      return_stats: bool = False, allow_noconv: bool = False):
    """Colour / monochrome fusion (Sec. 3): ``s_rgb`` [n][3][ny][nx] or [3][ny][nx] colour
    images (value constraints), ``o_grey`` [n][ny][nx] or [ny][nx] monochrome images (gradient
    constraints of every channel); CUDA float32.  Returns f with the shape of ``s_rgb``."""
    _require_cuda(s_rgb, o_grey)
    single = s_rgb.dim() == 3
    s4 = s_rgb[None] if single else s_rgb
    o3 = o_grey[None] if single else o_grey
    n, c, ny, nx = s4.shape
    if c != 3 or tuple(o3.shape) != (n, ny, nx):
        raise ValueError("expected s_rgb [n][3][ny][nx] and o_grey [n][ny][nx]")
    if s4.dtype != torch.float32 or o3.dtype != torch.float32:
        raise TypeError("s_rgb and o_grey must be float32")
    f = torch.empty_like(s4)
    stats = (SliceStats * (3 * n))()
    asynchronous = _is_async(opts)
    want_stats = return_stats or not asynchronous
    _check(lib().emfuse_fuse_color(s4.data_ptr(), o3.data_ptr(), f.data_ptr(), n, nx, ny, float(alpha),
                                   ctypes.byref(opts) if opts is not None else None,
                                   ctypes.addressof(stats) if want_stats else None,
                                   _stream_ptr(s4.device)), allow_noconv)
    f = f[0] if single else f
    if not return_stats:
        return f
    return (f, PendingStats(stats, _stream_ptr(s4.device), s4.device)) if asynchronous else (f, _stats_list(stats))


def emfuse_correct_stack(stack: torch.Tensor, sigma_xy: float = 1.0, sigma_z: float = 3.0,
                         alpha: float = 1e-3, opts: SolveOpts | None = None,
                         out: torch.Tensor | None = None, return_stats: bool = False,
                         allow_noconv: bool = False, device: int | None = None):
    """Both phases.  A CUDA ``stack`` is processed in place on the device; a CPU ``stack``
    (pinned memory recommended) is streamed through the device in z-chunks and the result is
    written to a CPU ``out``."""
    if not stack.is_contiguous():
        raise ValueError("expected a contiguous stack")
    nz, ny, nx = stack.shape
    on_host = not stack.is_cuda
    if out is None:
        out = torch.empty((nz, ny, nx), dtype=torch.float32, device=stack.device,
                          pin_memory=bool(on_host and stack.is_pinned()))
    if out.is_cuda == on_host:
        raise ValueError("out must live where the stack lives")
    dev = stack.device if stack.is_cuda else torch.device("cuda", torch.cuda.current_device() if device is None else device)
    stats = (SliceStats * nz)()
    asynchronous = _is_async(opts) and not on_host  # host buffers: the call always completes
    want_stats = return_stats or not asynchronous
    code = lib().emfuse_correct_stack(
        stack.data_ptr(), _dtype_code(stack), int(on_host), out.data_ptr(), nx, ny, nz,
        float(sigma_xy), float(sigma_z), float(alpha),
        ctypes.byref(opts) if opts is not None else None, ctypes.addressof(stats) if want_stats else None,
        _stream_ptr(dev))
    _check(code, allow_noconv)
    if not return_stats:
        return out
    return (out, PendingStats(stats, _stream_ptr(dev), dev)) if asynchronous else (out, _stats_list(stats))


def emfuse_backward(grad_f: torch.Tensor, f: torch.Tensor | None, s: torch.Tensor | None,
                    o: torch.Tensor | None, sigma_xy: float, sigma_z: float, alpha: float,
                    want=("s", "o", "in0", "alpha", "sigma_z"), opts: SolveOpts | None = None):
    """Adjoint of the correction (see include/emfuse.h).  Returns a dict of the requested
    gradients: 's', 'o', 'in0' (CUDA float32 tensors), 'alpha', 'sigma_z' (floats)."""
    _require_cuda(grad_f, f, s, o)
    g3 = grad_f if grad_f.dim() == 3 else grad_f[None]
    nz, ny, nx = g3.shape
    out = {}
    ptr = lambda t: t.data_ptr() if t is not None else None
    gs = torch.empty_like(g3) if "s" in want else None
    go = torch.empty_like(g3) if "o" in want else None
    gi = torch.empty_like(g3) if "in0" in want else None
    ga = ctypes.c_double(0.0)
    gz = ctypes.c_double(0.0)
    dt = _dtype_code(o) if o is not None else EMFUSE_F32
    code = lib().emfuse_backward(
        g3.data_ptr(), ptr(f), ptr(s), ptr(o), dt, nx, ny, nz, float(sigma_xy), float(sigma_z),
        float(alpha), ptr(gs), ptr(go), ptr(gi),
        ctypes.addressof(ga) if "alpha" in want else None,
        ctypes.addressof(gz) if "sigma_z" in want else None,
        ctypes.byref(opts) if opts is not None else None, _stream_ptr(g3.device))
    _check(code, allow_noconv=True)
    shape = grad_f.shape
    if gs is not None: out["s"] = gs.view(shape)
    if go is not None: out["o"] = go.view(shape)
    if gi is not None: out["in0"] = gi.view(shape)
    if "alpha" in want: out["alpha"] = ga.value
    if "sigma_z" in want: out["sigma_z"] = gz.value
    return out
