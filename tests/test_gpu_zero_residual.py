"""Blocks whose support is zero (black picture areas): the exact residual is
zero in every bin from the start, so every iteration selects the smallest
index, (0, 0), with a zero coefficient.  The kernels resolve the first such
iteration exactly and write the remaining ones as such instead of running
them; paths, coefficients and blocks must equal the oracle's, beside ordinary
blocks of the same batch (DFT and DCT bases, every precision, video
volumes)."""
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
