"""The forward entry point for callers that cannot allocate device memory
(fofse_extrapolate_batch_noalloc), checked against the regular entry point.

Some callers cannot call cudaMalloc: code that runs where allocation is not
allowed, or a host framework that owns every device buffer.  The no-alloc call
takes only inputs and outputs and uses a fixed counter array inside the
library.  Without a workspace there is no scratch for the exact spectra, so
FOFSE_FP32 plans run the kernel that updates every bin in float-float, while
the regular call with a workspace runs the register-blocked kernel: for those
plans this is a comparison of two kernels that both take exact decisions
(identical selection paths, coefficients equal up to their float-float
rounding, samples within the tests' 1e-3).  DCT and FP64-validation plans run
the same kernel on both entry points, so their results are bitwise equal.
Every case runs two calls in a row (the array keeps the previous call's
counters, so each call must clear it), and one runs a larger batch right after
a smaller one.  This file is collected last."""
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


def _noalloc(handles, plans, blocks, frame, avail):
    n = int(blocks.shape[0])
    ob, tr, w0, st = _outputs(plans, n)
    binding.fofse_extrapolate_batch_noalloc(handles, blocks, frame, avail, out_blocks=ob,
                                            trace=tr, w0=w0, status=st)
    torch.cuda.synchronize()
    binding.fofse_check()
    return ob, tr, w0, st


def _two_plan_frame():
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
    return wl


def _same_paths_and_close(got, ref):
    ob, tr, w0, st = got
    assert torch.equal(st, ref.status)
    assert torch.equal(tr.view(torch.int16)[..., :2], ref.trace.view(torch.int16)[..., :2])  # paths
    dc, rdc = tr[..., 1:].view(torch.float32), ref.trace[..., 1:].view(torch.float32)
    assert float((dc - rdc).abs().max()) <= 1e-6 * max(1.0, float(rdc.abs().max()))
    assert float((ob - ref.blocks).abs().max()) <= 1e-3     # the tests' sample tolerance
    assert torch.equal(w0, ref.w0)


def test_noalloc_fp32_plans_match_the_workspace_entry_point_on_two_calls():
    wl = _two_plan_frame()
    plans = [api.Plan.from_spec(p) for p in wl.plans]
    handles = [p.handle for p in plans]
    frame, avail, blocks = to_device(wl)
    ref = api.extrapolate(plans, blocks, frame, avail)
    for _ in range(2):
        _same_paths_and_close(_noalloc(handles, plans, blocks, frame, avail), ref)


@pytest.mark.parametrize("kind", ["dct", "fp64"])
def test_noalloc_runs_dct_and_fp64_plans_bitwise_like_the_workspace_entry_point(kind):
    spec = synth.PlanSpec(8, 8, 32, 0.8, 0.5, 40, basis=1 if kind == "dct" else 0)
    wl = synth.small_frame(43, plan=spec, n_lost=6, fill=np.nan)
    prec = "fp64" if kind == "fp64" else "fp32"
    plans = [api.Plan.from_spec(p, prec) for p in wl.plans]
    handles = [p.handle for p in plans]
    frame, avail, blocks = to_device(wl)
    ref = api.extrapolate(plans, blocks, frame, avail)
    for _ in range(2):
        ob, tr, w0, st = _noalloc(handles, plans, blocks, frame, avail)
        assert torch.equal(st, ref.status)
        assert torch.equal(tr, ref.trace)
        assert torch.equal(ob, ref.blocks)
        assert torch.equal(w0, ref.w0)


def test_noalloc_larger_batch_after_a_smaller_one_reads_cleared_counters():
    wl = _two_plan_frame()
    plans = [api.Plan.from_spec(p) for p in wl.plans]
    handles = [p.handle for p in plans]
    frame, avail, blocks = to_device(wl)
    ref = api.extrapolate(plans, blocks, frame, avail)
    small = blocks[:3].contiguous()
    _noalloc(handles, plans, small, frame, avail)
    # the small call left its plans' counters at 3: the full batch must start from 0
    _same_paths_and_close(_noalloc(handles, plans, blocks, frame, avail), ref)


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
