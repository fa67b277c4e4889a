"""Parity of the CUDA adjoint (frozen selection path) with the FP64 oracle's
adjoint of the spatial recursion, through the C ABI and through autograd.

Tolerances: relative L2 error <= 1e-3 on the frame gradient; relative error
<= 1e-3 on d/drho and d/dgamma (blocks whose paths match the oracle's)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2207_01205_gb300 import api, autograd, binding, synth

from parity_util import run_gpu, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib(gpu_lib):
    return gpu_lib


def _gpu_grads(wl, res, plans, e, split=True):
    """split: with a workspace (solve kernel + sample-pass kernel); else the
    one-kernel-per-block form."""
    frame, avail, blocks = to_device(wl)
    gf = torch.zeros_like(frame)
    grg = torch.zeros((len(plans), 2), dtype=torch.float32, device="cuda")
    ge = torch.from_numpy(np.ascontiguousarray(e, dtype=np.float32)).cuda()
    ws = api.workspace(plans, len(wl.blocks), frame.device) if split else None
    binding.fofse_backward([p.handle for p in plans], blocks, frame, avail, res.trace, res.w0, ge,
                           grad_frame=gf, grad_rho_gamma=grg, workspace=ws)
    torch.cuda.synchronize()
    binding.fofse_check()
    return gf.cpu().numpy().astype(np.float64), grg.cpu().numpy().astype(np.float64)


def _rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _check(wl, e_fn, tol=1e-3, tol_rho=1e-3):
    res, plans = run_gpu(wl, "fp32")
    path = res.path()
    ora = oracle.run_batch(wl.frame, wl.avail, wl.blocks, wl.plans)
    assert np.array_equal(path, ora.path)
    e = e_fn(res.blocks.cpu().numpy().astype(np.float64))
    ogf, ogrg = oracle.batch_adjoint(wl.frame, wl.avail, wl.blocks, wl.plans, ora.path, e)
    for split in (True, False):
        gf, grg = _gpu_grads(wl, res, plans, e, split)
        assert _rel_l2(gf, ogf) <= tol, (split, _rel_l2(gf, ogf))
        assert np.all(gf[wl.avail == 0] == 0)
        for p in range(len(wl.plans)):
            assert grg[p, 0] == pytest.approx(ogrg[p, 0], rel=tol_rho), (split, grg, ogrg)
            assert grg[p, 1] == pytest.approx(ogrg[p, 1], rel=tol), (split, grg, ogrg)
    return res, plans, gf, grg, ogf, ogrg


@pytest.mark.parametrize("spec", [synth.PlanSpec(16, 16, 64, 0.8, 0.5, 60),
                                  synth.PlanSpec(8, 8, 32, 0.8, 0.5, 50),
                                  synth.PlanSpec(4, 4, 32, 0.7, 0.3, 40),
                                  synth.PlanSpec(8, 8, 32, 0.8, 0.5, 64, support=1)])
def test_adjoint_matches_oracle_small_frames(spec):
    """Overlapping supports of neighbouring blocks, blocks in the frame corners."""
    wl = synth.small_frame(21, plan=spec, n_lost=8)
    rng = np.random.default_rng(1)
    _check(wl, lambda g: rng.normal(size=g.shape))


def test_adjoint_fft128_class():
    """32x32 blocks, border 16, 128x128 FFT, 400 iterations."""
    spec = synth.PlanSpec(32, 16, 128, 0.8, 0.5, 400)
    wl = synth.small_frame(33, height=160, width=192, plan=spec, n_lost=4)
    rng = np.random.default_rng(3)
    _check(wl, lambda g: rng.normal(size=g.shape))


def test_adjoint_of_squared_error_on_1080p_workload():
    """l = sum over B of (B_hat - f_true)^2 on the 804-block 1080p workload."""
    wl = synth.frame_concealment()
    truth = np.zeros((wl.n_blocks, 16, 16))
    for i, (y, x, _) in enumerate(wl.blocks):
        truth[i] = wl.truth[y:y + 16, x:x + 16]
    _check(wl, lambda g: 2.0 * (g - truth))


def test_adjoint_against_finite_differences_of_frozen_path():
    """Central differences (step 1e-3) of the FP64 frozen-path forward in a few
    support samples; the map is linear in f, so they are exact."""
    wl = synth.small_frame(4, plan=synth.PlanSpec(8, 8, 32, 0.8, 0.5, 30), n_lost=3,
                           edge_blocks=False)
    rng = np.random.default_rng(2)
    res, plans = run_gpu(wl, "fp32")
    e = rng.normal(size=res.blocks.shape)
    gf, _ = _gpu_grads(wl, res, plans, e)
    path = res.path()
    y, x, _ = wl.blocks[0]
    p = wl.plans[0]

    def loss(frame):
        tot = 0.0
        for i, (yy, xx, _) in enumerate(wl.blocks):
            fL, aL = oracle.cut_area(frame, wl.avail, yy, xx, 8, 8)
            w = oracle.weights(8, 8, p.rho, aL)
            g, _ = oracle.replay_area(fL, w, 32, p.gamma, path[i])
            tot += float(np.sum(g[8:16, 8:16] * e[i]))
        return tot

    H, W = wl.frame.shape
    checked = 0
    for (dy, dx) in [(-1, 0), (-3, 4), (2, -2), (9, 3), (-8, -8), (16, 5), (5, 17)]:
        fy, fx = y + dy, x + dx
        if not (0 <= fy < H and 0 <= fx < W) or wl.avail[fy, fx] == 0:
            continue
        h = 1e-3
        fp = wl.frame.copy()
        fm = wl.frame.copy()
        fp[fy, fx] += h
        fm[fy, fx] -= h
        # divide by the step the float32 frame actually represents
        step = float(fp[fy, fx]) - float(fm[fy, fx])
        fd = (loss(fp) - loss(fm)) / step
        assert gf[fy, fx] == pytest.approx(fd, rel=2e-3, abs=1e-6)
        checked += 1
    assert checked >= 3


def test_autograd_function_matches_direct_call_and_is_linear_in_grad():
    wl = synth.small_frame(6, plan=synth.PlanSpec(16, 16, 64, 0.8, 0.5, 40), n_lost=5)
    frame, avail, blocks = to_device(wl)
    frame = frame.clone().requires_grad_(True)
    rho = torch.tensor([0.8], device="cuda", requires_grad=True)
    gamma = torch.tensor([0.5], device="cuda", requires_grad=True)
    out, status = autograd.extrapolate(frame, avail, blocks, wl.plans, rho, gamma)
    assert int(status.max()) == 0
    truth = torch.stack([torch.from_numpy(wl.truth[y:y + 16, x:x + 16]) for (y, x, _) in wl.blocks]).cuda()
    loss = ((out - truth) ** 2).sum()
    gf, gr, gg = torch.autograd.grad(loss, (frame, rho, gamma), retain_graph=True)
    res, plans = run_gpu(wl, "fp32")
    e = 2.0 * (res.blocks.cpu().numpy().astype(np.float64) - truth.cpu().numpy())
    dgf, dgrg = _gpu_grads(wl, res, plans, e)
    # shared-memory and global float atomics make the summation order (and so
    # the last bits) differ between two runs; d/drho is a cancelling sum
    assert _rel_l2(gf.cpu().numpy().astype(np.float64), dgf) < 1e-4
    assert float(gr) == pytest.approx(dgrg[0, 0], rel=1e-2, abs=1e-3), (float(gr), dgrg)
    assert float(gg) == pytest.approx(dgrg[0, 1], rel=1e-4), (float(gg), dgrg)
    gf2, gr2 = torch.autograd.grad((2.0 * loss), (frame, rho))
    assert _rel_l2(gf2.cpu().numpy(), 2.0 * gf.cpu().numpy()) < 1e-4
    assert float(gr2) == pytest.approx(2.0 * float(gr), rel=1e-2, abs=1e-3)
