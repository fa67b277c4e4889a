"""Degenerate supports.  Zero supports (black picture areas): the exact
residual is zero in every bin from the start, so every iteration selects the
smallest index, (0, 0), with a zero coefficient; the kernels resolve the first
such iteration exactly and write the remaining ones as such instead of running
them.  Flat supports (a constant value): the residual decays geometrically
while the bound of the FP32 working spectrum does not, until nearly every bin
is a near-tie candidate; the kernels then take the exact values of every bin
as a new R0 and restart the bound.  Paths, coefficients and blocks must equal
the oracle's, beside ordinary blocks of the same batch (DFT and DCT bases,
every precision, video volumes)."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
from paper_2207_01205_gb300 import api, synth

from parity_util import compare, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib(gpu_lib):
    return gpu_lib


SPECS = [synth.PlanSpec(16, 16, 64, 0.8, 0.5, 60), synth.PlanSpec(8, 8, 32, 0.8, 0.5, 40),
         synth.PlanSpec(32, 16, 128, 0.8, 0.5, 30)]
CASES = [(s, basis, prec) for s in SPECS for basis in (0, 1) for prec in ("fp32", "fp32_fullff", "fp64")
         if not (basis == 1 and (s.fft_size == 128 or prec == "fp64"))
         and not (prec != "fp32" and s.fft_size == 128)]


@pytest.mark.parametrize("spec,basis,precision", CASES,
                         ids=[f"T{s.fft_size}-basis{b}-{q}" for s, b, q in CASES])
def test_zero_support_blocks_match_the_oracle(spec, basis, precision):
    spec = dataclasses.replace(spec, basis=basis)
    wl = synth.small_frame(41, height=160, width=256, plan=spec, n_lost=10)
    wl.frame[:, : wl.frame.shape[1] // 2] = 0.0  # a black left half
    ora = oracle.run_batch(wl.frame, wl.avail, wl.blocks, wl.plans)
    res, _ = run_gpu(wl, precision)
    c = compare(wl, res, ora)
    assert c["status_equal"]
    assert c["same"] == c["n"], (c["diverged"], c["gaps"])
    assert c["max_err"] <= 1e-3, c
    zero = [i for i in range(wl.n_blocks) if ora.status[i] == 0 and np.all(ora.dc[i] == 0)]
    assert zero, "the batch holds a block with a zero support"
    assert len(zero) < wl.n_blocks, "and ordinary blocks"
    path, dc = res.path(), res.dc()
    for i in zero:
        assert np.all(path[i, :spec.iters] == 0) and np.all(dc[i, :spec.iters] == 0)
        assert np.all(res.blocks[i].cpu().numpy() == 0)


def test_zero_video_areas_match_the_oracle():
    spec = synth.VolumePlanSpec(8, 4, 1, 16, 4, 0.8, 0.5, 40)
    wl = synth.small_video(43, plan=spec, n_lost=6)
    wl.video[:, :, : wl.video.shape[2] // 2] = 0.0
    plan = api.VolumePlan.from_spec(wl.plan)
    res = api.extrapolate_volume(plan, torch.from_numpy(np.ascontiguousarray(wl.blocks)).cuda(),
                                 torch.from_numpy(wl.video).cuda(), torch.from_numpy(wl.avail).cuda())
    torch.cuda.synchronize()
    ora = oracle.run_batch_volume(wl.video, wl.avail, wl.blocks, wl.plan)
    np.testing.assert_array_equal(res.status.cpu().numpy(), ora.status)
    path = res.path.cpu().numpy()
    assert all(np.array_equal(path[i], ora.path[i]) for i in range(len(ora.status)))
    g = res.blocks.cpu().numpy().astype(np.float64)
    assert np.abs(g - ora.blocks).max() <= 1e-3
    coef = res.coef.cpu().numpy()
    dc = coef[..., 0] + 1j * coef[..., 1]
    assert np.abs(dc - ora.dc).max() <= 1e-6 * max(1.0, float(np.abs(ora.dc).max()))
    zero = [i for i in range(len(ora.status)) if ora.status[i] == 0 and np.all(ora.dc[i] == 0)]
    assert zero and len(zero) < len(ora.status)
    for i in zero:
        assert np.all(path[i] == 0) and np.all(dc[i] == 0)


FLAT = [(synth.PlanSpec(16, 16, 64, 0.8, 0.5, 35), 0), (synth.PlanSpec(8, 8, 32, 0.8, 0.5, 35), 0),
        (synth.PlanSpec(32, 16, 128, 0.8, 0.5, 35), 0), (synth.PlanSpec(16, 16, 64, 0.8, 0.5, 35), 1),
        (synth.PlanSpec(8, 8, 32, 0.8, 0.5, 35), 1)]


@pytest.mark.parametrize("spec,basis", FLAT, ids=[f"T{s.fft_size}-basis{b}" for s, b in FLAT])
def test_flat_support_blocks_match_the_oracle(spec, basis):
    """35 iterations at gamma 0.5 take a flat block's residual down by 2^-35,
    past the point where the bound covers every bin (about 2^-20), and stay
    well above the float-float and FP64 rounding.  A flat block on a support
    that is symmetric under transposition has bins of equal energy
    ((k1, k2) and (k2, k1) with the DCT basis): there both the oracle and the
    kernel pick by their own rounding, so a divergence is allowed only where
    the oracle's relative gap is at its rounding level (below 1e-12)."""
    spec = dataclasses.replace(spec, basis=basis)
    wl = synth.small_frame(44, height=160, width=256, plan=spec, n_lost=10)
    wl.frame[:, : wl.frame.shape[1] // 2] = 100.0  # a flat left half
    ora = oracle.run_batch(wl.frame, wl.avail, wl.blocks, wl.plans)
    res, _ = run_gpu(wl, "fp32")
    c = compare(wl, res, ora)
    assert c["status_equal"]
    assert all(g < 1e-12 for g in c["gaps"].values()), (c["diverged"], c["gaps"])
    assert c["same"] >= c["n"] - 2, (c["diverged"], c["gaps"])
    assert c["max_err"] <= 1e-3, c
    assert c["max_dc_rel"] < 1e-5, c


def test_flat_video_areas_match_the_oracle():
    spec = synth.VolumePlanSpec(8, 4, 1, 16, 4, 0.8, 0.5, 35)
    wl = synth.small_video(45, plan=spec, n_lost=6)
    wl.video[:, :, : wl.video.shape[2] // 2] = 100.0
    plan = api.VolumePlan.from_spec(wl.plan)
    res = api.extrapolate_volume(plan, torch.from_numpy(np.ascontiguousarray(wl.blocks)).cuda(),
                                 torch.from_numpy(wl.video).cuda(), torch.from_numpy(wl.avail).cuda())
    torch.cuda.synchronize()
    ora = oracle.run_batch_volume(wl.video, wl.avail, wl.blocks, wl.plan)
    np.testing.assert_array_equal(res.status.cpu().numpy(), ora.status)
    path = res.path.cpu().numpy()
    assert all(np.array_equal(path[i], ora.path[i]) for i in range(len(ora.status)))
    g = res.blocks.cpu().numpy().astype(np.float64)
    assert np.abs(g - ora.blocks).max() <= 1e-3
