"""The forward entry point for callers that cannot allocate device memory
(fofse_extrapolate_batch_noalloc), checked against the regular entry point.

Some callers cannot call cudaMalloc: code that runs where allocation is not
allowed, or a host framework that owns every device buffer.  The no-alloc call
takes only inputs and outputs and uses a fixed counter array inside the
library, so its results must equal those of fofse_extrapolate_batch (same
kernels), on consecutive calls too (the array keeps the previous call's
counters and must be cleared by each call).  This file is collected last."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2207_01205_gb300 import api, binding, synth

from parity_util import to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib(gpu_lib):
    return gpu_lib


def _outputs(plans, n):
    return api.alloc_outputs(plans, n, "cuda")


def test_noalloc_matches_workspace_entry_point_on_two_calls():
    spec64 = synth.PlanSpec(16, 16, 64, 0.8, 0.5, 80)
    wl = synth.small_frame(41, plan=spec64, n_lost=7, fill=np.nan)
    # add a second plan (8x8 blocks, 32x32 FFT) on free tiles of the same frame
    spec32 = synth.PlanSpec(8, 8, 32, 0.7, 0.4, 60)
    extra = [(y, x, 1) for (y, x) in [(40, 72), (72, 8), (8, 104)]
             if wl.avail[y:y + 8, x:x + 8].all()]
    for (y, x, _) in extra:
        wl.avail[y:y + 8, x:x + 8] = 0
        wl.frame[y:y + 8, x:x + 8] = np.nan
    wl.blocks = np.concatenate([wl.blocks, np.array(extra, dtype=np.int32).reshape(-1, 3)])
    wl.plans = [spec64, spec32]
    plans = [api.Plan.from_spec(p) for p in wl.plans]
    handles = [p.handle for p in plans]
    frame, avail, blocks = to_device(wl)
    n = wl.n_blocks
    ref = api.extrapolate(plans, blocks, frame, avail)
    for _ in range(2):
        ob, tr, w0, st = _outputs(plans, n)
        binding.fofse_extrapolate_batch_noalloc(handles, blocks, frame, avail, out_blocks=ob,
                                                trace=tr, w0=w0, status=st)
        torch.cuda.synchronize()
        binding.fofse_check()
        assert torch.equal(st, ref.status)
        assert torch.equal(tr, ref.trace)                       # identical selection paths
        assert float((ob - ref.blocks).abs().max()) <= 1e-3     # the tests' sample tolerance
        assert torch.allclose(w0, ref.w0, rtol=0, atol=0)


def test_noalloc_rejects_what_its_fixed_array_cannot_hold():
    lib = binding.load()
    p128 = api.Plan(32, 16, 128, 0.8, 0.5, 10)
    null = ctypes.c_void_p()
    one = (ctypes.c_void_p * 1)(p128.handle)
    assert lib.fofse_extrapolate_batch_noalloc(one, 1, null, 1, null, null, 8, 8, 8, null, null,
                                               null, null, null, null) in (binding.E_ARG,
                                                                           binding.E_UNSUPPORTED)
    frame = torch.zeros((64, 64), device="cuda")
    avail = torch.ones((64, 64), dtype=torch.uint8, device="cuda")
    blocks = torch.tensor([[16, 16, 0]], dtype=torch.int32, device="cuda")
    with pytest.raises(binding.FofseError) as ei:
        binding.fofse_extrapolate_batch_noalloc([p128.handle], blocks, frame, avail)
    assert ei.value.status == binding.E_UNSUPPORTED
    p64 = api.Plan(16, 16, 64, 0.8, 0.5, 10)
    with pytest.raises(binding.FofseError) as ei:
        binding.fofse_extrapolate_batch_noalloc([p64.handle] * 65, blocks, frame, avail)
    assert ei.value.status == binding.E_ARG
