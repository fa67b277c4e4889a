"""Whole-workload checks on the GPU: CUDA-graph capture of a mixed batch, and
the streamed prediction workload (every 8x8 block of a 1280x720 frame from its
causal L-shaped support, 32x32 FFT, 64 iterations) forward and backward."""
import numpy as np
import pytest
import torch

import oracle
from paper_2207_01205_gb300 import api, autograd, binding, synth

from parity_util import compare, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib(gpu_lib):
    return gpu_lib


def test_cuda_graph_capture_of_a_mixed_batch_replays_bitwise():
    """One captured call (work-queue reset + one persistent launch per plan)
    replayed twice gives the eager results bit for bit."""
    specs = [synth.PlanSpec(16, 16, 64, 0.8, 0.5, 60), synth.PlanSpec(8, 8, 32, 0.7, 0.4, 40)]
    wl = synth.small_frame(51, height=128, width=192, plan=specs[0], n_lost=6)
    extra = [(y, x, 1) for (y, x) in [(40, 104), (72, 152), (104, 8), (8, 120)]
             if wl.avail[y:y + 8, x:x + 8].all()]
    for (y, x, _) in extra:
        wl.avail[y:y + 8, x:x + 8] = 0
    wl.blocks = np.concatenate([wl.blocks, np.array(extra, dtype=np.int32).reshape(-1, 3)])
    wl.plans = specs
    plans = [api.Plan.from_spec(p) for p in specs]
    frame, avail, blocks = to_device(wl)
    n = wl.n_blocks
    eager = api.extrapolate(plans, blocks, frame, avail)
    ob, tr, w0, st = api.alloc_outputs(plans, n, "cuda")
    ws = api.workspace(plans, n, "cuda")
    handles = [p.handle for p in plans]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):  # warm-up outside the capture (kernel attributes, driver entry points)
        binding.fofse_extrapolate_batch(handles, blocks, frame, avail, out_blocks=ob, trace=tr, w0=w0,
                                        status=st, workspace=ws, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        binding.fofse_extrapolate_batch(handles, blocks, frame, avail, out_blocks=ob, trace=tr, w0=w0,
                                        status=st, workspace=ws,
                                        stream=torch.cuda.current_stream())
    for _ in range(2):
        ob.zero_()
        tr.zero_()
        g.replay()
        torch.cuda.synchronize()
        binding.fofse_check()
        assert torch.equal(ob, eager.blocks)
        assert torch.equal(tr, eager.trace)
        assert torch.equal(st, eager.status)


@pytest.fixture(scope="module")
def pred():
    frames, blocks, plans = synth.prediction_sequence(n_frames=2)
    return frames, blocks, plans


def test_prediction_workload_forward_parity(pred):
    """14,400 causal 8x8 blocks of one 1280x720 frame; the oracle runs all of
    them (blocks on the top row / left column have partial or no support)."""
    frames, blocks, plans = pred
    frame = frames[1]
    avail = np.ones(frame.shape, dtype=np.uint8)
    wl = synth.Workload("pred", frame, frame, avail, blocks, plans)
    ora = oracle.run_batch(frame, avail, blocks, plans)
    res, _ = _run(wl)
    c = compare(wl, res, ora)
    assert c["status_equal"]
    assert (ora.status == 1).sum() == 1          # only the top-left block has no support
    assert c["frac"] >= 0.999, c
    assert c["max_err"] <= 1e-3, c


def _run(wl):
    from parity_util import run_gpu
    return run_gpu(wl, "fp32")


def test_prediction_workload_rho_gamma_gradients(pred):
    """d(total prediction SSE)/d(rho, gamma) over two frames for parameter
    tuning, against the oracle's adjoint (paths frozen)."""
    frames, blocks, plans = pred
    spec = plans[0]
    g_rg = np.zeros(2)
    o_rg = np.zeros(2)
    for f in frames:
        avail = np.ones(f.shape, dtype=np.uint8)
        fr = torch.from_numpy(f).cuda()
        av = torch.from_numpy(avail).cuda()
        bl = torch.from_numpy(blocks).cuda()
        rho = torch.tensor([spec.rho], device="cuda", requires_grad=True)
        gamma = torch.tensor([spec.gamma], device="cuda", requires_grad=True)
        out, st = autograd.extrapolate(fr, av, bl, plans, rho, gamma)
        truth = fr.unfold(0, 8, 8).unfold(1, 8, 8).reshape(-1, 8, 8)
        loss = ((out - truth) ** 2).sum()
        gr, gg = torch.autograd.grad(loss, (rho, gamma))
        g_rg += [float(gr), float(gg)]
        ora = oracle.run_batch(f, avail, blocks, plans)
        e = 2.0 * (ora.blocks - truth.cpu().numpy().astype(np.float64))
        e[ora.status != 0] = 0.0
        _, rg = oracle.batch_adjoint(f, avail, blocks, plans, ora.path, e)
        o_rg += rg[0]
    assert g_rg[0] == pytest.approx(o_rg[0], rel=1e-3)
    assert g_rg[1] == pytest.approx(o_rg[1], rel=1e-3)


def test_autotuner_picks_a_shape_and_all_shapes_agree(tmp_path):
    """Every launch shape gives the same selection paths (and samples within
    the parity tolerance); the tuned choice is cached and reused."""
    from paper_2207_01205_gb300 import autotune
    wl = synth.small_frame(61, plan=synth.PlanSpec(16, 16, 64, 0.8, 0.5, 80), n_lost=9)
    plans = [api.Plan.from_spec(p) for p in wl.plans]
    frame, avail, blocks = to_device(wl)
    count = binding.fofse_plan_variant_count(plans[0].handle)
    assert count >= 2
    outs = []
    for v in range(count):
        binding.fofse_plan_set_variant(plans[0].handle, v)
        outs.append(api.extrapolate(plans, blocks, frame, avail))
    torch.cuda.synchronize()
    for r in outs[1:]:
        assert np.array_equal(r.path(), outs[0].path())
        assert float((r.blocks - outs[0].blocks).abs().max()) <= 1e-3
    path = str(tmp_path / "tune.json")
    first = autotune.autotune(plans, blocks, frame, avail, cache_path=path)
    assert first["cached"] == [False] and 0 <= first["choices"][0] < count
    again = autotune.autotune(plans, blocks, frame, avail, cache_path=path)
    assert again["cached"] == [True] and again["choices"] == first["choices"]
    with pytest.raises(binding.FofseError):
        binding.fofse_plan_set_variant(plans[0].handle, count)


def test_measurement_probes_run_and_report_their_work():
    """The shared-memory and FMA probe kernels used for the rooflines."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    sink = torch.empty(sms * 1024, dtype=torch.float32, device="cuda")
    b = binding.fofse_probe_smem(sms, 10, sink)
    f = binding.fofse_probe_fma(sms, 10, sink)
    torch.cuda.synchronize()
    binding.fofse_check()
    assert b == sms * 1024 * 10 * 8 * 16
    assert f == sms * 1024 * 10 * 8
    with pytest.raises(binding.FofseError):
        binding.fofse_probe_smem(0, 10, sink)
