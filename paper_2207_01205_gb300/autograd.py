"""torch.autograd.Function over the C ABI: forward = fofse_extrapolate_batch,
backward = fofse_backward (selection path frozen; the saved trace holds the
path and coefficients, so no spectra are stored)."""
from __future__ import annotations

import torch

from . import api
from . import binding as B


class FOFSEFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, frame, rho, gamma, avail, blocks, specs, precision):
        rho_v = rho.detach().reshape(-1).cpu().tolist()
        gam_v = gamma.detach().reshape(-1).cpu().tolist()
        plans = [api.Plan(s.block, s.border, s.fft_size, rho_v[i], gam_v[i], s.iters,
                          getattr(s, "support", 0), precision) for i, s in enumerate(specs)]
        frame_c = frame.detach().contiguous()
        res = api.extrapolate(plans, blocks, frame_c, avail)
        ctx.save_for_backward(frame_c, avail, blocks, res.trace, res.w0)
        ctx.plans = plans
        ctx.rho_shape, ctx.gamma_shape = rho.shape, gamma.shape
        ctx.mark_non_differentiable(res.status)
        return res.blocks, res.status

    @staticmethod
    def backward(ctx, grad_blocks, _grad_status):
        frame, avail, blocks, trace, w0 = ctx.saved_tensors
        need_f, need_r, need_g = ctx.needs_input_grad[0], ctx.needs_input_grad[1], ctx.needs_input_grad[2]
        gf = torch.zeros_like(frame) if need_f else None
        grg = torch.zeros((len(ctx.plans), 2), dtype=torch.float32, device=frame.device)
        ws = api.workspace(ctx.plans, int(blocks.shape[0]), frame.device)
        B.fofse_backward([p.handle for p in ctx.plans], blocks, frame, avail, trace, w0,
                         grad_blocks.contiguous(), grad_frame=gf,
                         grad_rho_gamma=grg if (need_r or need_g) else None, workspace=ws)
        gr = grg[:, 0].reshape(ctx.rho_shape) if need_r else None
        gg = grg[:, 1].reshape(ctx.gamma_shape) if need_g else None
        return gf, gr, gg, None, None, None, None


def extrapolate(frame, avail, blocks, specs, rho, gamma, precision: str = "fp32"):
    """Differentiable batch extrapolation.

    frame: (H, W) float32 CUDA tensor (may require grad); avail: (H, W) uint8;
    blocks: (n, 3) int32 (y, x, plan index); specs: per-plan objects with
    block, border, fft_size, iters (and optional support); rho, gamma: float
    tensors with one entry per plan (may require grad).
    Returns (B_hat (n, bmax, bmax), status (n,))."""
    specs = list(specs)
    rho = torch.as_tensor(rho, dtype=torch.float32).reshape(len(specs))
    gamma = torch.as_tensor(gamma, dtype=torch.float32).reshape(len(specs))
    return FOFSEFunction.apply(frame, rho, gamma, avail, blocks, specs, precision)
