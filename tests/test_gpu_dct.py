"""Parity of the CUDA path with the 2-D DCT-II basis against the oracle's
(same bar as the DFT basis: identical selection paths, max |B_gpu - B_oracle|
<= 1e-3 on the 0-255 scale, PSNR within 0.01 dB)."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2207_01205_gb300 import synth

from parity_util import compare, psnr, run_gpu, to_device, truth_blocks

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib(gpu_lib):
    return gpu_lib


def _dct(wl):
    wl.plans = [dataclasses.replace(p, basis=1) for p in wl.plans]
    return wl


@pytest.mark.parametrize("spec", [synth.PlanSpec(16, 16, 64, 0.8, 0.5, 120),
                                  synth.PlanSpec(8, 8, 32, 0.8, 0.5, 100),
                                  synth.PlanSpec(4, 4, 32, 0.7, 0.3, 50),
                                  synth.PlanSpec(8, 8, 32, 0.8, 0.5, 64, support=1),
                                  synth.PlanSpec(16, 8, 32, 0.8, 0.5, 60)])
@pytest.mark.parametrize("precision", ["fp32", "fp32_fullff"])
def test_dct_small_frames_with_edge_blocks(spec, precision):
    """Corner blocks (partial support), lost neighbours, NaN-poisoned lost
    samples, the causal support, and L = T (16 + 2 x 8 = 32)."""
    wl = _dct(synth.small_frame(29, plan=spec, n_lost=7, fill=np.nan))
    ora = oracle.run_batch(wl.frame, wl.avail, wl.blocks, wl.plans)
    res, _ = run_gpu(wl, precision)
    c = compare(wl, res, ora)
    assert c["status_equal"]
    assert c["same"] == c["n"], c
    assert c["max_err"] <= 1e-3, c
    assert c["max_dc_rel"] < 1e-5, c


@pytest.mark.parametrize("spec", [synth.PlanSpec(16, 16, 64, 0.8, 0.5, 80),
                                  synth.PlanSpec(8, 8, 32, 0.8, 0.5, 150)])
def test_dct_fp32_and_float_float_loops_agree(spec):
    """Variant 0 (FP32 working spectrum, exact decisions) and variant 1 (every
    bin in float-float) select the same paths; their coefficients and blocks
    agree to float-float rounding (the exact values come from different sums)."""
    import torch
    from paper_2207_01205_gb300 import api, binding
    spec = dataclasses.replace(spec, basis=1)
    wl = synth.small_frame(30, plan=spec, n_lost=5)
    fr, av, bl = to_device(wl)
    outs = []
    for v in range(2):
        p = api.Plan.from_spec(spec)
        binding.fofse_plan_set_variant(p.handle, v)
        outs.append(api.extrapolate([p], bl, fr, av))
    torch.cuda.synchronize()
    binding.fofse_check()
    t0, t1 = (o.trace_numpy() for o in outs)
    assert np.array_equal(t0["u1"], t1["u1"]) and np.array_equal(t0["u2"], t1["u2"])
    d0, d1 = t0["re"].astype(np.float64), t1["re"].astype(np.float64)
    assert np.all(np.abs(d0 - d1) <= 1e-6 * np.maximum(np.abs(d1), 1e-3))
    assert torch.allclose(outs[0].blocks, outs[1].blocks, rtol=0, atol=1e-4)


def test_dct_full_frame_1080p():
    """The 1920x1080 concealment batch (804 blocks, 64x64 grid, 200 iterations)
    with the DCT basis."""
    wl = _dct(synth.frame_concealment())
    ora = oracle.run_batch(wl.frame, wl.avail, wl.blocks, wl.plans)
    res, _ = run_gpu(wl, "fp32")
    c = compare(wl, res, ora)
    assert c["status_equal"]
    assert c["frac"] >= 0.999, c
    assert c["max_err"] <= 1e-3, c
    tb, mask = truth_blocks(wl)
    g = res.blocks.cpu().numpy().astype(np.float64)
    assert abs(psnr(g, tb, mask) - psnr(ora.blocks, tb, mask)) <= 0.01


def test_dct_unsupported_combinations():
    import torch
    from paper_2207_01205_gb300 import api, binding
    wl = synth.small_frame(31, plan=synth.PlanSpec(8, 8, 32, 0.8, 0.5, 20), n_lost=3)
    fr, av, bl = to_device(wl)
    cases = [api.Plan(8, 8, 32, 0.8, 0.5, 20, 0, "fp64", 0, 1),
             api.Plan(8, 8, 32, 0.8, 0.5, 20, 0, "fp32", 1, 1),
             api.Plan(32, 16, 128, 0.8, 0.5, 20, 0, "fp32", 0, 1)]
    for p in cases:
        with pytest.raises(binding.FofseError) as e:
            api.extrapolate([p], bl, fr, av)
        assert e.value.status == binding.E_UNSUPPORTED
    p = api.Plan(8, 8, 32, 0.8, 0.5, 20, 0, "fp32", 0, 1)
    with pytest.raises(binding.FofseError):
        binding.fofse_plan_set_basis(p.handle, 2)
    torch.cuda.synchronize()
    binding.fofse_check()


def test_dct_long_run_and_device_values():
    """3000 iterations at fft_size 32 (the trace outgrows the setup's chunk
    region), and device-side (rho, gamma) equal to a plan built with them."""
    import torch
    from paper_2207_01205_gb300 import api, binding
    spec = synth.PlanSpec(8, 8, 32, 0.8, 0.5, 3000, 0, 0, 1)
    wl = synth.small_frame(33, plan=spec, n_lost=3)
    ora = oracle.run_batch(wl.frame, wl.avail, wl.blocks, wl.plans)
    res, _ = run_gpu(wl, "fp32")
    c = compare(wl, res, ora)
    assert c["same"] == c["n"], c
    assert c["max_err"] <= 1e-3, c
    fr, av, bl = to_device(wl)
    spec2 = dataclasses.replace(spec, iters=200)
    own = api.extrapolate([api.Plan.from_spec(spec2)], bl, fr, av)
    other = api.Plan(8, 8, 32, 0.6, 0.3, 200, 0, "fp32", 0, 1)
    rg = torch.tensor([[spec2.rho, spec2.gamma]], dtype=torch.float32, device="cuda")
    dev = api.extrapolate([other], bl, fr, av, rho_gamma=rg)
    torch.cuda.synchronize()
    binding.fofse_check()
    assert torch.equal(own.blocks, dev.blocks)
    assert torch.equal(own.trace, dev.trace)


def test_dct_shared_table_equals_the_per_call_table():
    """1080p batch: every block starts from the plan's complete-support table C
    (blocks with a complete support copy it, the others subtract their missing
    samples' part); a call with device-side (rho, gamma) builds the same table
    for its rho.  Both give the same blocks and trace bit for bit; the batch
    has complete and incomplete blocks, and matches the oracle's paths."""
    import torch
    from paper_2207_01205_gb300 import api, binding
    wl = _dct(synth.frame_concealment())
    spec = wl.plans[0]
    Ls = spec.block + 2 * spec.border
    full = 0
    for y, x, _ in wl.blocks:
        y0, x0 = y - spec.border, x - spec.border
        if y0 < 0 or x0 < 0 or y0 + Ls > wl.avail.shape[0] or x0 + Ls > wl.avail.shape[1]:
            continue
        a = wl.avail[y0:y0 + Ls, x0:x0 + Ls].astype(bool).copy()
        a[spec.border:spec.border + spec.block, spec.border:spec.border + spec.block] = True
        full += bool(a.all())
    assert full >= 100, full
    fr, av, bl = to_device(wl)
    own = api.extrapolate([api.Plan.from_spec(spec)], bl, fr, av)
    other = api.Plan(spec.block, spec.border, spec.fft_size, 0.6, 0.3, spec.iters, 0, "fp32", 0, 1)
    rg = torch.tensor([[spec.rho, spec.gamma]], dtype=torch.float32, device="cuda")
    dev = api.extrapolate([other], bl, fr, av, rho_gamma=rg)
    torch.cuda.synchronize()
    binding.fofse_check()
    assert torch.equal(own.blocks, dev.blocks)
    assert torch.equal(own.trace, dev.trace)
    assert full < wl.n_blocks


def test_dct_empty_batch_is_a_no_op():
    import torch
    from paper_2207_01205_gb300 import api, binding
    p = api.Plan(8, 8, 32, 0.8, 0.5, 20, 0, "fp32", 0, 1)
    fr = torch.zeros((64, 64), dtype=torch.float32, device="cuda")
    av = torch.ones((64, 64), dtype=torch.uint8, device="cuda")
    bl = torch.zeros((0, 3), dtype=torch.int32, device="cuda")
    binding.fofse_extrapolate_batch([p.handle], bl, fr, av)
    torch.cuda.synchronize()
    binding.fofse_check()


def _rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("spec", [synth.PlanSpec(8, 8, 32, 0.8, 0.5, 60, 0, 0, 1),
                                  synth.PlanSpec(16, 16, 64, 0.8, 0.45, 80, 0, 0, 1),
                                  synth.PlanSpec(8, 8, 32, 0.7, 0.5, 40, 1, 0, 1)])
def test_dct_backward_matches_the_oracle_adjoint(spec):
    """Frozen-path gradients of sum <e, B_hat> with the DCT basis: frame
    gradient (relative L2 1e-3; float atomics over overlapping supports),
    d/drho and d/dgamma (1e-3 relative), against the FP64 reverse-mode oracle."""
    import torch
    from paper_2207_01205_gb300 import api, binding
    wl = synth.small_frame(35, plan=spec, n_lost=6)
    ora = oracle.run_batch(wl.frame, wl.avail, wl.blocks, wl.plans)
    res, plans = run_gpu(wl, "fp32")
    assert np.array_equal(res.path(), ora.path)
    rng = np.random.default_rng(3)
    e = np.zeros(res.blocks.shape)
    b = spec.block
    e[:, :b, :b] = rng.normal(size=(wl.n_blocks, b, b))
    ogf, ogrg = oracle.batch_adjoint(wl.frame, wl.avail, wl.blocks, wl.plans, ora.path, e)
    fr, av, bl = to_device(wl)
    gf = torch.zeros_like(fr)
    grg = torch.zeros((1, 2), dtype=torch.float32, device="cuda")
    binding.fofse_backward([p.handle for p in plans], bl, fr, av, res.trace, res.w0,
                           torch.from_numpy(e.astype(np.float32)).cuda(), grad_frame=gf,
                           grad_rho_gamma=grg, workspace=api.workspace(plans, wl.n_blocks, fr.device))
    torch.cuda.synchronize()
    binding.fofse_check()
    gf = gf.cpu().numpy().astype(np.float64)
    assert _rel_l2(gf, ogf) <= 1e-3, _rel_l2(gf, ogf)
    assert np.all(gf[wl.avail == 0] == 0)
    g = grg.cpu().numpy().astype(np.float64)[0]
    assert g[0] == pytest.approx(ogrg[0, 0], rel=1e-3, abs=1e-3)
    assert g[1] == pytest.approx(ogrg[0, 1], rel=1e-3)


def test_dct_autograd_through_the_device_values():
    """autograd over a DCT-basis class: gradients equal the direct backward."""
    import torch
    from paper_2207_01205_gb300 import autograd
    spec = synth.PlanSpec(8, 8, 32, 0.8, 0.5, 40, 0, 0, 1)
    wl = synth.small_frame(36, plan=spec, n_lost=5)
    fr, av, bl = to_device(wl)
    fr = fr.clone().requires_grad_(True)
    rho = torch.tensor([0.8], device="cuda", requires_grad=True)
    gamma = torch.tensor([0.5], device="cuda", requires_grad=True)
    out, status = autograd.extrapolate(fr, av, bl, wl.plans, rho, gamma)
    assert int(status.max()) == 0
    loss = (out ** 2).sum()
    gf, gr, gg = torch.autograd.grad(loss, (fr, rho, gamma))
    ora = oracle.run_batch(wl.frame, wl.avail, wl.blocks, wl.plans)
    e = 2.0 * out.detach().cpu().numpy().astype(np.float64)
    ogf, ogrg = oracle.batch_adjoint(wl.frame, wl.avail, wl.blocks, wl.plans, ora.path, e)
    assert _rel_l2(gf.cpu().numpy().astype(np.float64), ogf) <= 1e-3
    assert float(gr) == pytest.approx(ogrg[0, 0], rel=1e-3, abs=1e-3)
    assert float(gg) == pytest.approx(ogrg[0, 1], rel=1e-3)
