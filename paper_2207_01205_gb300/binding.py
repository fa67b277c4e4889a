"""Thin ctypes binding of the C ABI in ``include/fofse.h`` (same names).

Argument marshalling only: every step of the extrapolation runs in the CUDA
kernels of ``libfofse.so``.  Device buffers are torch tensors (PyTorch is used
for device memory and streams).  There is no CPU fallback: if the library
cannot be built or loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

from . import build as _build

OK, E_ARG, E_UNSUPPORTED, E_NOMEM, E_CUDA, E_TIMEOUT, E_STATE = range(7)
SUPPORT_FULL, SUPPORT_CAUSAL_L = 0, 1
FP32, FP64_VALIDATE, FP32_FULLFF = 0, 1, 3
BLK_OK, BLK_NO_SUPPORT, BLK_NONFINITE, BLK_TIMEOUT = 0, 1, 2, 3
COMP_CONSTANT, COMP_OFSE = 0, 1
BASIS_DFT, BASIS_DCT = 0, 1
PRECISIONS = {"fp32": FP32, "fp64": FP64_VALIDATE, "fp32_fullff": FP32_FULLFF}

INCLUDE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
HEADER = os.path.join(INCLUDE, "fofse.h")
PROBES_HEADER = os.path.join(INCLUDE, "fofse_probes.h")

_lock = threading.Lock()
_lib = None
_probes = None


class FofseError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib.fofse_status_string(status).decode() if _lib is not None else str(status)
        if _lib is not None and status == E_CUDA:
            msg += f" [{_lib.fofse_last_cuda_error_string().decode()}]"
        super().__init__(f"{where}: {msg} (status {status})")


class TraceEntry(ctypes.Structure):
    _fields_ = [("u1", ctypes.c_int16), ("u2", ctypes.c_int16), ("dc_re", ctypes.c_float),
                ("dc_im", ctypes.c_float)]


_vp = ctypes.c_void_p
_i = ctypes.c_int


def header_functions(header: str = HEADER) -> list[str]:
    """Names of the functions declared in a header (default include/fofse.h)."""
    txt = open(header).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(fofse_\w+)\s*\(", txt)))


def _declare(L):
    L.fofse_status_string.argtypes = [_i]
    L.fofse_status_string.restype = ctypes.c_char_p
    L.fofse_version.restype = _i
    L.fofse_plan_create.argtypes = [_i, _i, _i, ctypes.c_float, ctypes.c_float, _i,
                                    ctypes.POINTER(_vp)]
    L.fofse_plan_create.restype = _i
    L.fofse_plan_set_support.argtypes = [_vp, _i]
    L.fofse_plan_set_support.restype = _i
    L.fofse_plan_set_precision.argtypes = [_vp, _i]
    L.fofse_plan_set_precision.restype = _i
    L.fofse_plan_set_compensation.argtypes = [_vp, _i]
    L.fofse_plan_set_compensation.restype = _i
    L.fofse_plan_set_basis.argtypes = [_vp, _i]
    L.fofse_plan_set_basis.restype = _i
    L.fofse_plan_variant_count.argtypes = [_vp]
    L.fofse_plan_variant_count.restype = _i
    L.fofse_plan_set_variant.argtypes = [_vp, _i]
    L.fofse_plan_set_variant.restype = _i
    L.fofse_plan_destroy.argtypes = [_vp]
    L.fofse_plan_destroy.restype = None
    _ip = ctypes.POINTER(_i)
    L.fofse_plan_get_shape.argtypes = [_vp, _ip, _ip, _ip, _ip]
    L.fofse_plan_get_shape.restype = _i
    L.fofse_workspace_bytes.argtypes = [ctypes.POINTER(_vp), _i, _i]
    L.fofse_workspace_bytes.restype = ctypes.c_size_t
    L.fofse_extrapolate_batch.argtypes = [ctypes.POINTER(_vp), _i, _vp, _i, _vp, _vp, _i, _i, _i,
                                          _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
    L.fofse_extrapolate_batch.restype = _i
    L.fofse_extrapolate_batch_gamma.argtypes = [ctypes.POINTER(_vp), _i, _vp, _i, _vp, _vp, _i, _i,
                                                _i, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
    L.fofse_extrapolate_batch_gamma.restype = _i
    L.fofse_extrapolate_batch_noalloc.argtypes = [ctypes.POINTER(_vp), _i, _vp, _i, _vp, _vp, _i, _i,
                                                  _i, _vp, _vp, _vp, _vp, _vp, _vp]
    L.fofse_extrapolate_batch_noalloc.restype = _i
    L.fofse_backward.argtypes = [ctypes.POINTER(_vp), _i, _vp, _i, _vp, _vp, _i, _i, _i, _vp, _vp,
                                 _vp, _vp, _vp, _vp, _vp, _vp]
    L.fofse_backward.restype = _i
    L.fofse_error_curve.argtypes = [ctypes.POINTER(_vp), _i, _vp, _i, _vp, _vp, _i, _i, _i, _vp, _vp]
    L.fofse_error_curve.restype = _i
    L.fofse_volume_plan_create.argtypes = [_i, _i, _i, _i, _i, ctypes.c_float, ctypes.c_float, _i,
                                           ctypes.POINTER(_vp)]
    L.fofse_volume_plan_create.restype = _i
    L.fofse_volume_plan_destroy.argtypes = [_vp]
    L.fofse_volume_plan_destroy.restype = None
    L.fofse_volume_plan_set_precision.argtypes = [_vp, _i]
    L.fofse_volume_plan_set_precision.restype = _i
    L.fofse_volume_workspace_bytes.argtypes = [_vp, _i]
    L.fofse_volume_workspace_bytes.restype = ctypes.c_size_t
    L.fofse_volume_plan_variant_count.argtypes = [_vp]
    L.fofse_volume_plan_variant_count.restype = _i
    L.fofse_volume_plan_set_variant.argtypes = [_vp, _i]
    L.fofse_volume_plan_set_variant.restype = _i
    L.fofse_extrapolate_volume_batch.argtypes = [_vp, _vp, _i, _vp, _vp, _i, _i, _i, _i, _vp, _vp,
                                                 _vp, _vp, _vp, _vp, _vp]
    L.fofse_extrapolate_volume_batch.restype = _i
    L.fofse_volume_backward.argtypes = [_vp, _vp, _i, _vp, _vp, _i, _i, _i, _i, _vp, _vp, _vp, _vp,
                                        _vp, _vp, _vp, _vp, _vp]
    L.fofse_volume_backward.restype = _i
    L.fofse_volume_backward_workspace_bytes.argtypes = [_vp, _i]
    L.fofse_volume_backward_workspace_bytes.restype = ctypes.c_size_t
    L.fofse_check.argtypes = [_vp]
    L.fofse_check.restype = _i
    L.fofse_last_cuda_error.restype = _i
    L.fofse_last_cuda_error_string.restype = ctypes.c_char_p


def load(build: bool = True):
    """Load ``libfofse.so`` (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"libfofse.so not built ({path})")
            L = ctypes.CDLL(path)
            _declare(L)
            _lib = L
    return _lib


def load_probes():
    """Load ``libfofse_probes.so``, the measurement probes of
    include/fofse_probes.h (built with the product library)."""
    global _probes
    load()
    with _lock:
        if _probes is None:
            path = _build.PROBES_LIB
            if not os.path.exists(path):
                raise RuntimeError(f"libfofse_probes.so not built ({path})")
            L = ctypes.CDLL(path)
            for name in ("fofse_probe_smem", "fofse_probe_fma", "fofse_probe_dfma"):
                fn = getattr(L, name)
                fn.argtypes = [_i, _i, _vp, ctypes.POINTER(ctypes.c_double), _vp]
                fn.restype = _i
            _probes = L
    return _probes


def library_path() -> str:
    return _build.LIB


def _check(st, where):
    if st != OK:
        raise FofseError(st, where)


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(getattr(stream, "cuda_stream", stream))


# ----------------------------------------------------------------------------
# the C ABI, one Python function per entry point
# ----------------------------------------------------------------------------

def fofse_status_string(status: int) -> str:
    return load().fofse_status_string(status).decode()


def fofse_version() -> int:
    return load().fofse_version()


def fofse_plan_create(block, border, fft_size, rho, gamma, iters) -> int:
    h = ctypes.c_void_p()
    _check(load().fofse_plan_create(int(block), int(border), int(fft_size), float(rho),
                                    float(gamma), int(iters), ctypes.byref(h)), "fofse_plan_create")
    return h.value


def fofse_plan_set_support(plan, shape):
    _check(load().fofse_plan_set_support(ctypes.c_void_p(plan), int(shape)), "fofse_plan_set_support")


def fofse_plan_set_precision(plan, precision):
    _check(load().fofse_plan_set_precision(ctypes.c_void_p(plan), int(precision)),
           "fofse_plan_set_precision")


def fofse_plan_set_compensation(plan, compensation):
    _check(load().fofse_plan_set_compensation(ctypes.c_void_p(plan), int(compensation)),
           "fofse_plan_set_compensation")


def fofse_plan_set_basis(plan, basis):
    _check(load().fofse_plan_set_basis(ctypes.c_void_p(plan), int(basis)), "fofse_plan_set_basis")


def fofse_plan_variant_count(plan) -> int:
    return load().fofse_plan_variant_count(ctypes.c_void_p(plan))


def fofse_plan_set_variant(plan, variant):
    _check(load().fofse_plan_set_variant(ctypes.c_void_p(plan), int(variant)), "fofse_plan_set_variant")


def fofse_plan_get_shape(plan) -> tuple[int, int, int, int]:
    """(block, border, fft_size, iters) of a plan."""
    v = [ctypes.c_int() for _ in range(4)]
    _check(load().fofse_plan_get_shape(ctypes.c_void_p(plan), *[ctypes.byref(x) for x in v]),
           "fofse_plan_get_shape")
    return tuple(x.value for x in v)


def fofse_plan_destroy(plan):
    if plan:
        load().fofse_plan_destroy(ctypes.c_void_p(plan))


def _plan_array(plans):
    arr = (ctypes.c_void_p * len(plans))()
    for i, p in enumerate(plans):
        arr[i] = p
    return arr


def fofse_workspace_bytes(plans, n_blocks) -> int:
    return load().fofse_workspace_bytes(_plan_array(plans), len(plans), int(n_blocks))


def _require(t, name, dtype, shape=None, optional=False):
    """Host-side check of a tensor handed to the C ABI as a device pointer:
    the given dtype, a CUDA tensor (and leading shape), its last dimension
    contiguous.  Raises ValueError, so that a host tensor or a wrong dtype
    never reaches a kernel."""
    if t is None:
        if optional:
            return
        raise ValueError(f"{name} is required")
    if getattr(t, "dtype", None) != dtype:
        raise ValueError(f"{name} must be {dtype}, got {getattr(t, 'dtype', type(t))}")
    if not getattr(t, "is_cuda", False):
        raise ValueError(f"{name} must be a CUDA tensor")
    if shape is not None and tuple(t.shape[:len(shape)]) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}..., got {tuple(t.shape)}")
    if t.dim() and t.numel() and t.stride(-1) != 1:
        raise ValueError(f"{name} must be contiguous in its last dimension")


def _require_buffer(t, name, dtype, min_numel, optional=True):
    """A contiguous CUDA buffer of ``dtype`` with at least ``min_numel`` elements."""
    _require(t, name, dtype, optional=optional)
    if t is None:
        return
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.numel() < min_numel:
        raise ValueError(f"{name} holds {t.numel()} elements, the call writes {min_numel}")


def _check_frame_args(blocks, frame, avail, out_frame=None, name_out="out_frame"):
    """The block list and the frame / mask pair of a 2-D batch call; returns
    (n, H, W, pitch)."""
    import torch
    # dtypes first, so that each argument's own error shows before any device check
    for t, nm, dt in ((blocks, "blocks", torch.int32), (frame, "frame", torch.float32),
                      (avail, "avail", torch.uint8), (out_frame, name_out, torch.float32)):
        if t is not None and getattr(t, "dtype", None) != dt:
            raise ValueError(f"{nm} must be {dt}, got {getattr(t, 'dtype', type(t))}")
    if blocks.dim() != 2 or blocks.shape[1] != 3:
        raise ValueError(f"blocks must be an (n, 3) int32 tensor, got shape {tuple(blocks.shape)}")
    n = int(blocks.shape[0])
    _require(blocks, "blocks", torch.int32, (n, 3))
    if not blocks.is_contiguous():
        raise ValueError("blocks must be contiguous")
    _require(frame, "frame", torch.float32)
    _require(avail, "avail", torch.uint8)
    if frame.dim() != 2:
        raise ValueError(f"frame must be (height, width), got {tuple(frame.shape)}")
    if tuple(avail.shape) != tuple(frame.shape) or tuple(avail.stride()) != tuple(frame.stride()):
        raise ValueError("avail must have the frame's shape and strides")
    for t, nm in ((out_frame, name_out),):
        _require(t, nm, torch.float32, optional=True)
        if t is not None and (tuple(t.shape) != tuple(frame.shape)
                              or tuple(t.stride()) != tuple(frame.stride())):
            raise ValueError(f"{nm} must have the frame's shape and strides")
    dev = frame.device
    for t, nm in ((blocks, "blocks"), (avail, "avail"), (out_frame, name_out)):
        if t is not None and t.device != dev:
            raise ValueError(f"{nm} is on {t.device}, the frame on {dev}")
    if dev.index != torch.cuda.current_device():
        raise ValueError(f"the tensors are on {dev}, the current device is "
                         f"cuda:{torch.cuda.current_device()} (plans belong to one device)")
    H, W = frame.shape
    return n, H, W, frame.stride(0)


def _dims(plans):
    """(bmax, imax) over the plans of a call: the output tile side and the
    trace length per block."""
    shapes = [fofse_plan_get_shape(p) for p in plans]
    return max(s[0] for s in shapes), max(s[3] for s in shapes)


def _check_on(dev, *named):
    for t, nm in named:
        if t is not None and t.device != dev:
            raise ValueError(f"{nm} is on {t.device}, the frame on {dev}")


def _check_batch_outputs(plans, n, dev, out_blocks, trace, w0, status, gamma=None, rho_gamma=None,
                         workspace=None):
    import torch
    if not plans:
        raise ValueError("at least one plan is required")
    bmax, imax = _dims(plans)
    _require_buffer(out_blocks, "out_blocks", torch.float32, n * bmax * bmax)
    _require_buffer(trace, "trace", torch.int32, n * imax * 3)
    _require_buffer(w0, "w0", torch.float32, n)
    _require_buffer(status, "status", torch.int32, n)
    _require_buffer(gamma, "gamma", torch.float32, n * imax * 2)
    _require_buffer(rho_gamma, "rho_gamma", torch.float32, 2 * len(plans))
    _require_buffer(workspace, "workspace", torch.uint8, fofse_workspace_bytes(plans, n))
    _check_on(dev, (out_blocks, "out_blocks"), (trace, "trace"), (w0, "w0"), (status, "status"),
              (gamma, "gamma"), (rho_gamma, "rho_gamma"), (workspace, "workspace"))
    return bmax, imax


def fofse_extrapolate_batch(plans, blocks, frame, avail, *, out_frame=None, out_blocks=None,
                            trace=None, w0=None, status=None, workspace=None, rho_gamma=None,
                            stream=None):
    """blocks: (n, 3) int32 device tensor; frame float32 and avail uint8 device
    tensors of shape (H, W) (row pitch = stride(0)); out_blocks (n, bmax, bmax)
    float32, trace (n, max_iters, 3) int32, w0 (n,) float32, status (n,) int32,
    workspace uint8 of fofse_workspace_bytes(plans, n) bytes, rho_gamma
    (n_plans, 2) float32.  Every tensor is checked (CUDA, dtype, size, device)
    before the call."""
    n, H, W, pitch = _check_frame_args(blocks, frame, avail, out_frame)
    _check_batch_outputs(plans, n, frame.device, out_blocks, trace, w0, status,
                         rho_gamma=rho_gamma, workspace=workspace)
    _check(load().fofse_extrapolate_batch(
        _plan_array(plans), len(plans), _ptr(blocks), int(blocks.shape[0]), _ptr(frame),
        _ptr(avail), H, W, pitch, _ptr(rho_gamma), _ptr(out_frame), _ptr(out_blocks), _ptr(trace),
        _ptr(w0), _ptr(status), _ptr(workspace), _stream(stream)), "fofse_extrapolate_batch")


def fofse_extrapolate_batch_gamma(plans, blocks, frame, avail, *, out_frame=None, out_blocks=None,
                                  trace=None, w0=None, status=None, gamma=None, workspace=None,
                                  rho_gamma=None, stream=None):
    """fofse_extrapolate_batch that also writes the compensation factor of
    every iteration into ``gamma`` ((n, max_iters, 2) float32 device tensor)."""
    n, H, W, pitch = _check_frame_args(blocks, frame, avail, out_frame)
    _check_batch_outputs(plans, n, frame.device, out_blocks, trace, w0, status, gamma=gamma,
                         rho_gamma=rho_gamma, workspace=workspace)
    _check(load().fofse_extrapolate_batch_gamma(
        _plan_array(plans), len(plans), _ptr(blocks), int(blocks.shape[0]), _ptr(frame),
        _ptr(avail), H, W, pitch, _ptr(rho_gamma), _ptr(out_frame), _ptr(out_blocks), _ptr(trace),
        _ptr(w0), _ptr(status), _ptr(gamma), _ptr(workspace), _stream(stream)),
        "fofse_extrapolate_batch_gamma")


def fofse_extrapolate_batch_noalloc(plans, blocks, frame, avail, *, out_frame=None, out_blocks=None,
                                    trace=None, w0=None, status=None, stream=None):
    """The forward batch call for callers that cannot allocate device memory:
    no workspace argument; the library's fixed 256-byte counter array is used
    instead (fft_size 32/64 only; calls that overlap on the GPU must be
    serialised).  Tensors are checked as in fofse_extrapolate_batch."""
    n, H, W, pitch = _check_frame_args(blocks, frame, avail, out_frame)
    _check_batch_outputs(plans, n, frame.device, out_blocks, trace, w0, status)
    _check(load().fofse_extrapolate_batch_noalloc(
        _plan_array(plans), len(plans), _ptr(blocks), int(blocks.shape[0]), _ptr(frame),
        _ptr(avail), H, W, pitch, _ptr(out_frame), _ptr(out_blocks), _ptr(trace), _ptr(w0),
        _ptr(status), _stream(stream)), "fofse_extrapolate_batch_noalloc")


def fofse_backward(plans, blocks, frame, avail, trace, w0, grad_blocks, *, grad_frame=None,
                   grad_rho_gamma=None, workspace=None, rho_gamma=None, stream=None):
    """Frozen-path adjoint: trace and w0 from the forward call, grad_blocks
    (n, bmax, bmax) float32 dloss/dB_hat; grad_frame (frame's shape and
    strides) and grad_rho_gamma (n_plans, 2) float32 are accumulated.  Every
    tensor is checked (CUDA, dtype, size, device) before the call."""
    import torch
    n, H, W, pitch = _check_frame_args(blocks, frame, avail, grad_frame, "grad_frame")
    if trace is None or w0 is None or grad_blocks is None:
        raise ValueError("trace, w0 and grad_blocks are required")
    bmax, imax = _check_batch_outputs(plans, n, frame.device, None, trace, w0, None,
                                      rho_gamma=rho_gamma, workspace=workspace)
    _require_buffer(grad_blocks, "grad_blocks", torch.float32, n * bmax * bmax, optional=False)
    _require_buffer(grad_rho_gamma, "grad_rho_gamma", torch.float32, 2 * len(plans))
    _check_on(frame.device, (grad_blocks, "grad_blocks"), (grad_rho_gamma, "grad_rho_gamma"))
    _check(load().fofse_backward(
        _plan_array(plans), len(plans), _ptr(blocks), int(blocks.shape[0]), _ptr(frame),
        _ptr(avail), H, W, pitch, _ptr(rho_gamma), _ptr(trace), _ptr(w0), _ptr(grad_blocks),
        _ptr(grad_frame), _ptr(grad_rho_gamma), _ptr(workspace), _stream(stream)), "fofse_backward")


def fofse_error_curve(plans, blocks, trace, truth, sse, *, stream=None):
    """Squared error over B after every iteration count into ``sse``
    ((n, max_iters) float32 device tensor); ``truth`` (H, W) float32."""
    H, W = truth.shape
    pitch = truth.stride(0)
    assert truth.stride(1) == 1
    _check(load().fofse_error_curve(
        _plan_array(plans), len(plans), _ptr(blocks), int(blocks.shape[0]), _ptr(trace),
        _ptr(truth), H, W, pitch, _ptr(sse), _stream(stream)), "fofse_error_curve")


def fofse_probe_smem(ctas, rounds, sink, *, stream=None) -> float:
    """Queues the shared-memory load probe; returns the bytes it loads."""
    out = ctypes.c_double()
    _check(load_probes().fofse_probe_smem(int(ctas), int(rounds), _ptr(sink), ctypes.byref(out),
                                   _stream(stream)), "fofse_probe_smem")
    return out.value


def fofse_probe_fma(ctas, rounds, sink, *, stream=None) -> float:
    """Queues the FP32 FMA probe; returns the lane FMAs it issues."""
    out = ctypes.c_double()
    _check(load_probes().fofse_probe_fma(int(ctas), int(rounds), _ptr(sink), ctypes.byref(out),
                                  _stream(stream)), "fofse_probe_fma")
    return out.value


def fofse_probe_dfma(ctas, rounds, sink, *, stream=None) -> float:
    """Queues the FP64 FMA probe (sink: ctas x 1024 float64); returns the lane
    FMAs it issues."""
    out = ctypes.c_double()
    _check(load_probes().fofse_probe_dfma(int(ctas), int(rounds), _ptr(sink), ctypes.byref(out),
                                   _stream(stream)), "fofse_probe_dfma")
    return out.value


def fofse_last_cuda_error() -> int:
    return load().fofse_last_cuda_error()


def fofse_last_cuda_error_string() -> str:
    return load().fofse_last_cuda_error_string().decode()


def fofse_check(stream=None):
    _check(load().fofse_check(_stream(stream)), "fofse_check")


def fofse_volume_plan_create(block, border, depth, fft_size, fft_time, rho, gamma, iters) -> int:
    h = ctypes.c_void_p()
    _check(load().fofse_volume_plan_create(int(block), int(border), int(depth), int(fft_size),
                                           int(fft_time), float(rho), float(gamma), int(iters),
                                           ctypes.byref(h)), "fofse_volume_plan_create")
    return h.value


def fofse_volume_plan_set_precision(plan, precision):
    _check(load().fofse_volume_plan_set_precision(ctypes.c_void_p(plan), int(precision)),
           "fofse_volume_plan_set_precision")


def fofse_volume_workspace_bytes(plan, n_blocks) -> int:
    return load().fofse_volume_workspace_bytes(ctypes.c_void_p(plan), int(n_blocks))


def fofse_volume_plan_variant_count(plan) -> int:
    return load().fofse_volume_plan_variant_count(ctypes.c_void_p(plan))


def fofse_volume_plan_set_variant(plan, variant):
    _check(load().fofse_volume_plan_set_variant(ctypes.c_void_p(plan), int(variant)),
           "fofse_volume_plan_set_variant")


def fofse_volume_plan_destroy(plan):
    load().fofse_volume_plan_destroy(ctypes.c_void_p(plan) if plan else None)


def fofse_extrapolate_volume_batch(plan, blocks, video, avail, *, out_blocks, path=None, coef=None,
                                   w0=None, status=None, workspace=None, stream=None):
    """blocks: (n, 3) int32 device tensor (t, y, x); video float32 and avail
    uint8 device tensors of shape (F, H, W) with row pitch stride(1) and frame
    stride H * pitch; out_blocks (n, b, b) float32; path (n, iters, 3) int32,
    coef (n, iters, 2) float64, w0 (n,) float64, status (n,) int32; workspace
    uint8 of fofse_volume_workspace_bytes(plan, n) bytes (FP32 plans)."""
    import torch
    n = int(blocks.shape[0])
    _require(blocks, "blocks", torch.int32, (n, 3))
    if not blocks.is_contiguous():
        raise ValueError("blocks must be contiguous")
    _require(video, "video", torch.float32)
    _require(avail, "avail", torch.uint8)
    if video.dim() != 3:
        raise ValueError(f"video must be (frames, height, width), got {tuple(video.shape)}")
    _require(out_blocks, "out_blocks", torch.float32, (n,))
    if not out_blocks.is_contiguous():
        raise ValueError("out_blocks must be contiguous")
    for t, name, dt in ((path, "path", torch.int32), (coef, "coef", torch.float64),
                        (w0, "w0", torch.float64), (status, "status", torch.int32)):
        _require(t, name, dt, (n,), optional=True)
        if t is not None and not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    F, H, W = video.shape
    pitch = video.stride(1)
    if video.stride(0) != H * pitch:
        raise ValueError("video frames must be back to back (frame stride = height * row pitch)")
    if tuple(avail.shape) != tuple(video.shape) or tuple(avail.stride()) != tuple(video.stride()):
        raise ValueError("avail must have the video's shape and strides")
    _require_buffer(workspace, "workspace", torch.uint8, fofse_volume_workspace_bytes(plan, n))
    for t, nm in ((blocks, "blocks"), (avail, "avail"), (out_blocks, "out_blocks"), (path, "path"),
                  (coef, "coef"), (w0, "w0"), (status, "status"), (workspace, "workspace")):
        if t is not None and t.device != video.device:
            raise ValueError(f"{nm} is on {t.device}, the video on {video.device}")
    _check(load().fofse_extrapolate_volume_batch(
        ctypes.c_void_p(plan), _ptr(blocks), int(blocks.shape[0]), _ptr(video), _ptr(avail), F, H, W,
        pitch, _ptr(out_blocks), _ptr(path), _ptr(coef), _ptr(w0), _ptr(status), _ptr(workspace),
        _stream(stream)), "fofse_extrapolate_volume_batch")


def fofse_volume_backward_workspace_bytes(plan, n_blocks) -> int:
    return load().fofse_volume_backward_workspace_bytes(ctypes.c_void_p(plan), int(n_blocks))


def fofse_volume_backward(plan, blocks, video, avail, path, coef, w0, grad_blocks, *, status=None,
                          grad_video=None, grad_rho_gamma=None, workspace=None, stream=None):
    """Gradients of a loss on the volume batch's B_hat along the frozen path:
    path (n, iters, 3) int32, coef (n, iters, 2) float64, w0 (n,) float64 and
    status (n,) int32 from the forward call; grad_blocks (n, b, b) float32;
    grad_video (F, H, W) float32 with the video's strides and grad_rho_gamma
    (2,) float32 are accumulated into; workspace uint8 of
    fofse_volume_backward_workspace_bytes(plan, n) bytes."""
    import torch
    n = int(blocks.shape[0])
    # dtypes first, so that each argument's own error shows before any device check
    for t, name, dt in ((video, "video", torch.float32), (avail, "avail", torch.uint8),
                        (blocks, "blocks", torch.int32), (path, "path", torch.int32),
                        (coef, "coef", torch.float64), (w0, "w0", torch.float64),
                        (grad_blocks, "grad_blocks", torch.float32)):
        if getattr(t, "dtype", None) != dt:
            raise ValueError(f"{name} must be {dt}, got {getattr(t, 'dtype', type(t))}")
    _require(video, "video", torch.float32)
    _require(avail, "avail", torch.uint8)
    if video.dim() != 3:
        raise ValueError(f"video must be (frames, height, width), got {tuple(video.shape)}")
    for t, name, dt in ((blocks, "blocks", torch.int32), (path, "path", torch.int32),
                        (coef, "coef", torch.float64), (w0, "w0", torch.float64),
                        (grad_blocks, "grad_blocks", torch.float32)):
        _require(t, name, dt, (n,))
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    _require(status, "status", torch.int32, (n,), optional=True)
    F, H, W = video.shape
    pitch = video.stride(1)
    if video.stride(0) != H * pitch:
        raise ValueError("video frames must be back to back (frame stride = height * row pitch)")
    if tuple(avail.shape) != tuple(video.shape) or tuple(avail.stride()) != tuple(video.stride()):
        raise ValueError("avail must have the video's shape and strides")
    if grad_video is not None:
        _require(grad_video, "grad_video", torch.float32)
        if tuple(grad_video.shape) != tuple(video.shape) or tuple(grad_video.stride()) != tuple(video.stride()):
            raise ValueError("grad_video must have the video's shape and strides")
    _require_buffer(grad_rho_gamma, "grad_rho_gamma", torch.float32, 2)
    _require_buffer(workspace, "workspace", torch.uint8, fofse_volume_backward_workspace_bytes(plan, n))
    for t, nm in ((blocks, "blocks"), (avail, "avail"), (path, "path"), (coef, "coef"), (w0, "w0"),
                  (grad_blocks, "grad_blocks"), (status, "status"), (grad_video, "grad_video"),
                  (grad_rho_gamma, "grad_rho_gamma"), (workspace, "workspace")):
        if t is not None and t.device != video.device:
            raise ValueError(f"{nm} is on {t.device}, the video on {video.device}")
    _check(load().fofse_volume_backward(
        ctypes.c_void_p(plan), _ptr(blocks), n, _ptr(video), _ptr(avail), F, H, W, pitch, _ptr(path),
        _ptr(coef), _ptr(w0), _ptr(status), _ptr(grad_blocks), _ptr(grad_video), _ptr(grad_rho_gamma),
        _ptr(workspace), _stream(stream)), "fofse_volume_backward")
