"""torch.autograd.Function over the C ABI: forward = fofse_extrapolate_batch,
backward = fofse_backward (selection path frozen; the saved trace holds the
path and coefficients, so no spectra are stored).  rho and gamma reach the
kernels as a device tensor (the ABI's device-side (rho, gamma)), so a tuning
loop over them makes no host round trip and creates no plans after the first
call."""
from __future__ import annotations

import threading

import torch

from . import api
from . import binding as B

_plans = {}
_plans_lock = threading.Lock()


def _plans_for(specs, precision, device):
    """Plans of these block classes, created once per (classes, precision,
    device); their own rho / gamma are placeholders (every call passes the
    values on the device)."""
    key = (tuple((s.block, s.border, s.fft_size, s.iters, getattr(s, "support", 0),
                  getattr(s, "basis", 0)) for s in specs), precision, str(device))
    with _plans_lock:
        plans = _plans.get(key)
        if plans is None:
            plans = [api.Plan(s.block, s.border, s.fft_size, 0.5, 0.5, s.iters,
                              getattr(s, "support", 0), precision, 0, getattr(s, "basis", 0))
                     for s in specs]
            _plans[key] = plans
        return plans


class FOFSEFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, frame, rho, gamma, avail, blocks, specs, precision):
        plans = _plans_for(specs, precision, frame.device)
        rg = torch.stack([rho.detach().reshape(-1), gamma.detach().reshape(-1)], dim=1)
        rg = rg.to(device=frame.device, dtype=torch.float32).contiguous()
        frame_c = frame.detach().contiguous()
        ws = api.workspace(plans, int(blocks.shape[0]), frame.device)
        res = api.extrapolate(plans, blocks, frame_c, avail, ws=ws, rho_gamma=rg)
        ctx.save_for_backward(frame_c, avail, blocks, res.trace, res.w0, rg)
        ctx.plans = plans
        ctx.ws = ws
        ctx.rho_shape, ctx.gamma_shape = rho.shape, gamma.shape
        ctx.mark_non_differentiable(res.status)
        return res.blocks, res.status

    @staticmethod
    def backward(ctx, grad_blocks, _grad_status):
        frame, avail, blocks, trace, w0, rg = ctx.saved_tensors
        need_f, need_r, need_g = ctx.needs_input_grad[0], ctx.needs_input_grad[1], ctx.needs_input_grad[2]
        gf = torch.zeros_like(frame) if need_f else None
        grg = torch.zeros((len(ctx.plans), 2), dtype=torch.float32, device=frame.device)
        B.fofse_backward([p.handle for p in ctx.plans], blocks, frame, avail, trace, w0,
                         grad_blocks.contiguous(), grad_frame=gf,
                         grad_rho_gamma=grg if (need_r or need_g) else None, workspace=ctx.ws,
                         rho_gamma=rg)
        gr = grg[:, 0].reshape(ctx.rho_shape) if need_r else None
        gg = grg[:, 1].reshape(ctx.gamma_shape) if need_g else None
        return gf, gr, gg, None, None, None, None


def extrapolate(frame, avail, blocks, specs, rho, gamma, precision: str = "fp32"):
    """Differentiable batch extrapolation.

    frame: (H, W) float32 CUDA tensor (may require grad); avail: (H, W) uint8;
    blocks: (n, 3) int32 (y, x, plan index); specs: per-plan objects with
    block, border, fft_size, iters (and optional support); rho, gamma: float
    tensors with one entry per plan (may require grad; device tensors keep
    the call free of host round trips).
    Returns (B_hat (n, bmax, bmax), status (n,))."""
    specs = list(specs)
    rho = torch.as_tensor(rho, dtype=torch.float32).reshape(len(specs))
    gamma = torch.as_tensor(gamma, dtype=torch.float32).reshape(len(specs))
    return FOFSEFunction.apply(frame, rho, gamma, avail, blocks, specs, precision)
