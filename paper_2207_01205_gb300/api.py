"""Python-level API over the C ABI: plans as objects and batch calls that
allocate their outputs with torch on the frame's device."""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import binding as B

TRACE_DTYPE = np.dtype([("u1", "<i2"), ("u2", "<i2"), ("re", "<f4"), ("im", "<f4")])

# Plans released while a CUDA graph is being captured (for example by the
# garbage collector, inside the capture) are destroyed later: destroying a
# plan synchronises the device and frees memory, which would invalidate the
# capture.
_deferred = []


def _capturing() -> bool:
    try:
        return bool(torch.cuda.is_available() and torch.cuda.is_current_stream_capturing())
    except Exception:
        return False


def _destroy_deferred():
    while _deferred:
        destroy, h = _deferred.pop()
        destroy(h)


def _release(handle, destroy=None):
    destroy = destroy or B.fofse_plan_destroy
    if _capturing():
        _deferred.append((destroy, handle))
        return
    _destroy_deferred()
    destroy(handle)


class Plan:
    """One block class: b x b lost blocks, support border, T x T FFT, rho_hat,
    gamma and the number of iterations (paper Sec. 4 notation); compensation
    0 = the constant gamma of Eq. 14 (FOFSE), 1 = OFSE's (Eq. 10-13); basis
    0 = 2-D DFT, 1 = 2-D DCT-II."""

    def __init__(self, block, border, fft_size, rho, gamma, iters, support=0, precision="fp32",
                 compensation=0, basis=0):
        self.block, self.border, self.fft_size = int(block), int(border), int(fft_size)
        self.rho, self.gamma, self.iters = float(rho), float(gamma), int(iters)
        self.support = int(support)
        self.precision = precision
        self.compensation = int(compensation)
        self.basis = int(basis)
        if not _capturing():
            _destroy_deferred()
        h = B.fofse_plan_create(block, border, fft_size, rho, gamma, iters)
        try:
            B.fofse_plan_set_support(h, self.support)
            B.fofse_plan_set_precision(h, B.PRECISIONS[precision])
            B.fofse_plan_set_compensation(h, self.compensation)
            B.fofse_plan_set_basis(h, self.basis)
        except Exception:
            B.fofse_plan_destroy(h)   # the handle is never published: __del__ finds none
            raise
        self.handle = h

    @classmethod
    def from_spec(cls, spec, precision="fp32"):
        return cls(spec.block, spec.border, spec.fft_size, spec.rho, spec.gamma, spec.iters,
                   getattr(spec, "support", 0), precision, getattr(spec, "compensation", 0),
                   getattr(spec, "basis", 0))

    def close(self):
        h = getattr(self, "handle", None)
        if h:
            self.handle = None
            _release(h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclasses.dataclass
class Result:
    blocks: torch.Tensor       # (n, bmax, bmax) float32
    trace: torch.Tensor        # (n, imax, 3) int32 storage of fofse_trace_entry
    w0: torch.Tensor           # (n,) float32
    status: torch.Tensor       # (n,) int32
    out_frame: torch.Tensor | None = None
    gamma: torch.Tensor | None = None  # (n, imax, 2) float32: compensation factor per iteration

    def trace_numpy(self):
        return self.trace.cpu().numpy().view(TRACE_DTYPE).reshape(self.trace.shape[:2])

    def path(self):
        t = self.trace_numpy()
        return np.stack([t["u1"], t["u2"]], axis=-1).astype(np.int32)

    def dc(self):
        t = self.trace_numpy()
        return t["re"].astype(np.float64) + 1j * t["im"].astype(np.float64)


def alloc_outputs(plans, n, device, with_trace=True):
    bmax = max(p.block for p in plans)
    imax = max(p.iters for p in plans)
    blocks = torch.empty((n, bmax, bmax), dtype=torch.float32, device=device)
    trace = torch.empty((n, imax, 3), dtype=torch.int32, device=device) if with_trace else None
    w0 = torch.empty((n,), dtype=torch.float32, device=device)
    status = torch.empty((n,), dtype=torch.int32, device=device)
    return blocks, trace, w0, status


def workspace(plans, n_blocks, device):
    """Device scratch for a batch call with these plans (work-queue counters
    and, for fft_size 128, per-SM FFT buffers)."""
    nbytes = B.fofse_workspace_bytes([p.handle for p in plans], n_blocks)
    return torch.empty((max(nbytes, 1),), dtype=torch.uint8, device=device)


def extrapolate(plans, blocks, frame, avail, *, out_frame=None, with_trace=True, stream=None,
                ws=None, with_gamma=False, rho_gamma=None) -> Result:
    """Run the forward pass of every block.  ``blocks``: (n, 3) int32 tensor on
    the device (y, x, plan index); ``frame`` float32 and ``avail`` uint8 (H, W)
    tensors on the same device.  ``with_gamma`` also returns the compensation
    factor of every iteration (FOFSE_FP32 plans).  ``rho_gamma``: optional
    (n_plans, 2) float32 device tensor of (rho, gamma) per plan for this call
    (read on the device; no host round trip)."""
    plans = list(plans)
    n = int(blocks.shape[0])
    ob, tr, w0, st = alloc_outputs(plans, n, frame.device, with_trace)
    if ws is None:
        ws = workspace(plans, n, frame.device)
    handles = [p.handle for p in plans]
    if with_gamma:
        imax = max(p.iters for p in plans)
        gm = torch.empty((n, imax, 2), dtype=torch.float32, device=frame.device)
        B.fofse_extrapolate_batch_gamma(handles, blocks, frame, avail, out_frame=out_frame,
                                        out_blocks=ob, trace=tr, w0=w0, status=st, gamma=gm,
                                        workspace=ws, rho_gamma=rho_gamma, stream=stream)
        return Result(ob, tr, w0, st, out_frame, gm)
    B.fofse_extrapolate_batch(handles, blocks, frame, avail, out_frame=out_frame,
                              out_blocks=ob, trace=tr, w0=w0, status=st, workspace=ws,
                              rho_gamma=rho_gamma, stream=stream)
    return Result(ob, tr, w0, st, out_frame)


# ----------------------------------------------------------------------------
# video volumes
# ----------------------------------------------------------------------------

class VolumePlan:
    """Extrapolation over video volumes: b x b lost block, spatial border,
    ``depth`` frames on each side of the block's frame, T x T x Tt DFT grid
    (T = fft_size, Tt = fft_time), rho_hat, gamma, iterations; precision
    "fp32" (the product: FP32 spectrum, exact decisions) or "fp64"
    (validation)."""

    def __init__(self, block, border, depth, fft_size, fft_time, rho, gamma, iters, precision="fp32"):
        self.block, self.border, self.depth = int(block), int(border), int(depth)
        self.fft_size, self.fft_time = int(fft_size), int(fft_time)
        self.rho, self.gamma, self.iters = float(rho), float(gamma), int(iters)
        self.precision = precision
        if not _capturing():
            _destroy_deferred()
        h = B.fofse_volume_plan_create(block, border, depth, fft_size, fft_time, rho, gamma, iters)
        try:
            B.fofse_volume_plan_set_precision(h, B.PRECISIONS[precision])
        except Exception:
            B.fofse_volume_plan_destroy(h)   # the handle is never published: __del__ finds none
            raise
        self.handle = h

    @classmethod
    def from_spec(cls, spec, precision="fp32"):
        return cls(spec.block, spec.border, spec.depth, spec.fft_size, spec.fft_time, spec.rho,
                   spec.gamma, spec.iters, precision)

    def close(self):
        h = getattr(self, "handle", None)
        if h:
            self.handle = None
            _release(h, B.fofse_volume_plan_destroy)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclasses.dataclass
class VolumeResult:
    blocks: torch.Tensor               # (n, b, b) float32
    w0: torch.Tensor                   # (n,) float64
    status: torch.Tensor               # (n,) int32
    path: torch.Tensor | None = None   # (n, iters, 3) int32
    coef: torch.Tensor | None = None   # (n, iters, 2) float64


def volume_workspace(plan, n_blocks, device):
    """Device scratch for a volume batch call (empty for FP64 plans)."""
    nbytes = B.fofse_volume_workspace_bytes(plan.handle, n_blocks)
    return torch.empty((nbytes,), dtype=torch.uint8, device=device) if nbytes else None


def extrapolate_volume(plan, blocks, video, avail, *, with_path=True, stream=None,
                       ws=None) -> VolumeResult:
    """Extrapolate every block ((n, 3) int32 device tensor: t, y, x) of a video
    ((F, H, W) float32 device tensor, availability uint8 of the same layout)."""
    n = int(blocks.shape[0])
    dev = video.device
    out = torch.empty((n, plan.block, plan.block), dtype=torch.float32, device=dev)
    w0 = torch.empty((n,), dtype=torch.float64, device=dev)
    status = torch.empty((n,), dtype=torch.int32, device=dev)
    path = torch.empty((n, plan.iters, 3), dtype=torch.int32, device=dev) if with_path else None
    coef = torch.empty((n, plan.iters, 2), dtype=torch.float64, device=dev) if with_path else None
    if ws is None:
        ws = volume_workspace(plan, n, dev)
    B.fofse_extrapolate_volume_batch(plan.handle, blocks, video, avail, out_blocks=out, path=path,
                                     coef=coef, w0=w0, status=status, workspace=ws, stream=stream)
    return VolumeResult(out, w0, status, path, coef)


def volume_backward(plan, blocks, video, avail, res: VolumeResult, grad_blocks, *, stream=None):
    """Gradients of a loss on ``res.blocks`` (its gradient ``grad_blocks``,
    (n, b, b) float32) along the forward's frozen selection path: returns
    (dl/dvideo with the video's layout, (dl/drho, dl/dgamma))."""
    if res.path is None or res.coef is None:
        raise ValueError("the forward result must carry its path and coefficients")
    gv = torch.zeros_like(video)
    grg = torch.zeros((2,), dtype=torch.float32, device=video.device)
    n = int(blocks.shape[0])
    ws = torch.empty((B.fofse_volume_backward_workspace_bytes(plan.handle, n),), dtype=torch.uint8,
                     device=video.device)
    B.fofse_volume_backward(plan.handle, blocks, video, avail, res.path, res.coef, res.w0,
                            grad_blocks.contiguous(), status=res.status, grad_video=gv,
                            grad_rho_gamma=grg, workspace=ws, stream=stream)
    return gv, grg
