"""Helpers shared by the GPU parity tests: run the CUDA path and the FP64
oracle on the same seeded workload and compare them."""
from __future__ import annotations

import numpy as np

import oracle


def to_device(wl, device="cuda"):
    import torch
    frame = torch.from_numpy(np.ascontiguousarray(wl.frame, dtype=np.float32)).to(device)
    avail = torch.from_numpy(np.ascontiguousarray(wl.avail, dtype=np.uint8)).to(device)
    blocks = torch.from_numpy(np.ascontiguousarray(wl.blocks, dtype=np.int32)).to(device)
    return frame, avail, blocks


def run_gpu(wl, precision="fp32", out_frame=False, with_gamma=False):
    import torch
    from paper_2207_01205_gb300 import api
    plans = [api.Plan.from_spec(p, precision) for p in wl.plans]
    frame, avail, blocks = to_device(wl)
    of = frame.clone() if out_frame else None
    res = api.extrapolate(plans, blocks, frame, avail, out_frame=of, with_gamma=with_gamma)
    torch.cuda.synchronize()
    from paper_2207_01205_gb300 import binding
    binding.fofse_check()
    return res, plans


def compare(wl, res, ora, *, tol_abs=1e-3, dc_rel=1e-5):
    """Returns a dict of parity figures; paths compared per block."""
    n = wl.n_blocks
    g_blocks = res.blocks.cpu().numpy().astype(np.float64)
    g_status = res.status.cpu().numpy()
    g_path = res.path()
    g_dc = res.dc()
    same_path = np.zeros(n, dtype=bool)
    max_err = 0.0
    max_dc = 0.0
    first_div = {}
    for i in range(n):
        p = wl.plans[wl.blocks[i, 2]]
        b, it = p.block, p.iters
        if g_status[i] != ora.status[i]:
            continue
        if ora.status[i] != 0:
            same_path[i] = True
            max_err = max(max_err, float(np.abs(g_blocks[i, :b, :b]).max()))
            continue
        eq = (g_path[i, :it] == ora.path[i, :it]).all(axis=1)
        if eq.all():
            same_path[i] = True
            max_err = max(max_err, float(np.abs(g_blocks[i, :b, :b] - ora.blocks[i, :b, :b]).max()))
            scale = np.maximum(np.abs(ora.dc[i, :it]), 1e-3)
            max_dc = max(max_dc, float(np.max(np.abs(g_dc[i, :it] - ora.dc[i, :it]) / scale)))
        else:
            first_div[i] = int(np.argmin(eq))
    near_tie = {i: float(ora.gap[i, j]) for i, j in first_div.items()}
    return dict(n=n, same=int(same_path.sum()), frac=float(same_path.mean()), max_err=max_err,
                max_dc_rel=max_dc, diverged=first_div, gaps=near_tie,
                status_equal=bool(np.array_equal(g_status, ora.status)))


def psnr(blocks, truth_blocks, mask):
    b = np.clip(blocks, 0, 255)[mask]
    t = truth_blocks[mask]
    mse = np.mean((b - t) ** 2)
    return 10 * np.log10(255.0 ** 2 / mse)


def truth_blocks(wl):
    n = wl.n_blocks
    bmax = max(p.block for p in wl.plans)
    out = np.zeros((n, bmax, bmax))
    mask = np.zeros((n, bmax, bmax), dtype=bool)
    for i, (y, x, pi) in enumerate(wl.blocks):
        b = wl.plans[pi].block
        out[i, :b, :b] = wl.truth[y:y + b, x:x + b]
        mask[i, :b, :b] = True
    return out, mask
