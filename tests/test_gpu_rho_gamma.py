"""Device-side (rho, gamma) of the C ABI (d_rho_gamma): values read on the
device, weights rebuilt there, usable inside CUDA graphs and tuning loops."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2207_01205_gb300 import synth

from parity_util import compare, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib(gpu_lib):
    return gpu_lib


def _run(plans, wl, rg=None):
    import torch
    from paper_2207_01205_gb300 import api
    fr, av, bl = to_device(wl)
    res = api.extrapolate(plans, bl, fr, av, rho_gamma=rg)
    torch.cuda.synchronize()
    return res


@pytest.mark.parametrize("precision", ["fp32", "fp64", "fp32_fullff"])
def test_device_values_equal_plan_values_bitwise(precision):
    """A plan built with other values and given (rho, gamma) on the device
    computes exactly what a plan built with those values computes (the same
    kernel builds the weights in both cases)."""
    import torch
    from paper_2207_01205_gb300 import api, binding
    spec = synth.PlanSpec(16, 16, 64, 0.8, 0.5, 60)
    wl = synth.small_frame(41, plan=spec, n_lost=5)
    own = [api.Plan.from_spec(spec, precision)]
    other = [api.Plan(16, 16, 64, 0.6, 0.3, 60, 0, precision)]
    rg = torch.tensor([[spec.rho, spec.gamma]], dtype=torch.float32, device="cuda")
    a = _run(own, wl)
    b = _run(other, wl, rg)
    binding.fofse_check()
    assert torch.equal(a.blocks, b.blocks)
    assert torch.equal(a.trace, b.trace)
    assert torch.equal(a.w0, b.w0)


def test_device_values_match_the_oracle_with_those_values():
    import torch
    from paper_2207_01205_gb300 import api, binding
    specs = [synth.PlanSpec(8, 8, 32, 0.7, 0.35, 80), synth.PlanSpec(4, 4, 32, 0.9, 0.8, 40)]
    wl = synth.small_frame(43, plan=specs[0], n_lost=8)
    wl.plans = specs
    wl.blocks[::3, 2] = 1
    ora = oracle.run_batch(wl.frame, wl.avail, wl.blocks, wl.plans)
    plans = [api.Plan(8, 8, 32, 0.5, 0.5, 80), api.Plan(4, 4, 32, 0.5, 0.5, 40)]
    rg = torch.tensor([[s.rho, s.gamma] for s in specs], dtype=torch.float32, device="cuda")
    res = _run(plans, wl, rg)
    binding.fofse_check()
    c = compare(wl, res, ora)
    assert c["same"] == c["n"], c
    assert c["max_err"] <= 1e-3


def test_cuda_graph_replay_follows_the_device_values():
    """The batch call with device-side values captured once; new values
    copied into the tensor between replays give the results of direct calls
    with those values."""
    import torch
    from paper_2207_01205_gb300 import api, binding
    spec = synth.PlanSpec(8, 8, 32, 0.8, 0.5, 50)
    wl = synth.small_frame(44, plan=spec, n_lost=6)
    plans = [api.Plan.from_spec(spec)]
    fr, av, bl = to_device(wl)
    n = wl.n_blocks
    ob, tr, w0, st = api.alloc_outputs(plans, n, fr.device)
    ws = api.workspace(plans, n, fr.device)
    rg = torch.tensor([[0.8, 0.5]], dtype=torch.float32, device="cuda")
    h = [p.handle for p in plans]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        binding.fofse_extrapolate_batch(h, bl, fr, av, out_blocks=ob, trace=tr, w0=w0, status=st,
                                        workspace=ws, rho_gamma=rg, stream=s)   # warm-up
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        binding.fofse_extrapolate_batch(h, bl, fr, av, out_blocks=ob, trace=tr, w0=w0, status=st,
                                        workspace=ws, rho_gamma=rg, stream=s)
    for rho, gamma in [(0.8, 0.5), (0.65, 0.25), (0.95, 0.9)]:
        rg.copy_(torch.tensor([[rho, gamma]]))
        g.replay()
        torch.cuda.synchronize()
        ref = _run([api.Plan(8, 8, 32, rho, gamma, 50)], wl)
        assert torch.equal(ob, ref.blocks), (rho, gamma)
        assert torch.equal(tr, ref.trace), (rho, gamma)
    binding.fofse_check()


def test_out_of_range_device_values_are_reported():
    """rho = 1.5 on the device: that plan's blocks get status NONFINITE and
    zero output, fofse_check reports FOFSE_E_ARG; the next good call is clean."""
    import torch
    from paper_2207_01205_gb300 import api, binding
    spec = synth.PlanSpec(8, 8, 32, 0.8, 0.5, 20)
    wl = synth.small_frame(45, plan=spec, n_lost=4)
    plans = [api.Plan.from_spec(spec)]
    for bad in ([1.5, 0.5], [0.8, 0.0], [float("nan"), 0.5]):
        res = _run(plans, wl, torch.tensor([bad], dtype=torch.float32, device="cuda"))
        assert (res.status.cpu().numpy() == 2).all(), bad
        assert float(res.blocks.abs().max()) == 0.0
        with pytest.raises(binding.FofseError) as e:
            binding.fofse_check()
        assert e.value.status == binding.E_ARG
    res = _run(plans, wl, torch.tensor([[0.8, 0.5]], dtype=torch.float32, device="cuda"))
    binding.fofse_check()
    assert (res.status.cpu().numpy() == 0).all()


def test_backward_with_device_values_equals_plan_values():
    import torch
    from paper_2207_01205_gb300 import api, binding
    spec = synth.PlanSpec(16, 16, 64, 0.8, 0.5, 40)
    wl = synth.small_frame(46, plan=spec, n_lost=5)
    fr, av, bl = to_device(wl)
    own = [api.Plan.from_spec(spec)]
    other = [api.Plan(16, 16, 64, 0.6, 0.3, 40)]
    rg = torch.tensor([[spec.rho, spec.gamma]], dtype=torch.float32, device="cuda")
    out = []
    for plans, r in ((own, None), (other, rg)):
        res = _run(plans, wl, r)
        ws = api.workspace(plans, wl.n_blocks, fr.device)
        gf = torch.zeros_like(fr)
        grg = torch.zeros((1, 2), dtype=torch.float32, device="cuda")
        binding.fofse_backward([p.handle for p in plans], bl, fr, av, res.trace, res.w0,
                               torch.ones_like(res.blocks), grad_frame=gf, grad_rho_gamma=grg,
                               workspace=ws, rho_gamma=r)
        torch.cuda.synchronize()
        binding.fofse_check()
        out.append((gf.cpu().numpy().astype(np.float64), grg.cpu().numpy().astype(np.float64)))
    (gf1, g1), (gf2, g2) = out
    # float atomics: summation order differs between runs
    assert np.linalg.norm(gf1 - gf2) <= 1e-5 * np.linalg.norm(gf1)
    np.testing.assert_allclose(g2, g1, rtol=1e-4, atol=1e-6)


def test_device_values_need_the_workspace():
    import torch
    from paper_2207_01205_gb300 import api, binding
    spec = synth.PlanSpec(8, 8, 32, 0.8, 0.5, 20)
    wl = synth.small_frame(47, plan=spec, n_lost=3)
    plans = [api.Plan.from_spec(spec)]
    fr, av, bl = to_device(wl)
    ob = torch.empty((wl.n_blocks, 8, 8), device="cuda")
    rg = torch.tensor([[0.8, 0.5]], dtype=torch.float32, device="cuda")
    with pytest.raises(binding.FofseError) as e:
        binding.fofse_extrapolate_batch([p.handle for p in plans], bl, fr, av, out_blocks=ob,
                                        rho_gamma=rg)
    assert e.value.status == binding.E_ARG
