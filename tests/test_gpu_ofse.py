"""Parity of the CUDA path with OFSE's compensation (Sec. 3, Eq. 10-13)
against the FP64 oracle's OFSE, through the C ABI.

Same bar as the constant compensation: identical selection paths, max
|B_gpu - B_oracle| <= 1e-3 on the 0-255 scale, PSNR within 0.01 dB; the
per-iteration compensation factors agree to 1e-4 (relative to max(|gamma|, 0.05);
on the large batch: median 1e-6, 99.9 % of them 1e-4, all 1e-2).

OFSE's iteration can be ill-conditioned: once Q[u] comes close to zero the
factors leave (0, 1) (|gamma| up to tens), and each such step amplifies the
rounding of every earlier one.  On a few blocks of a large batch the FP64
oracle's own answer then moves past the tolerance when its inputs are
perturbed at the kernel's working precision; there the answer is not
determined at that precision, and such blocks are exempt from the bar if,
and only if, the oracle itself shows that instability (checked per block)."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2207_01205_gb300 import synth

from parity_util import compare, psnr, run_gpu, truth_blocks, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib(gpu_lib):
    return gpu_lib


def _ofse(wl):
    wl.plans = [dataclasses.replace(p, compensation=1) for p in wl.plans]
    return wl


def _undetermined(wl, i, eps=2.0 ** -40, runs=3, tol=1e-4):
    """True when relative perturbations of eps (a few units of the kernel's
    float-float working precision, 2^-44 per operation) of the oracle's inputs f
    and w change the oracle's path for block i or move its B_hat by more than
    tol (a tenth of the output tolerance)."""
    p = wl.plans[wl.blocks[i, 2]]
    y, x, _ = wl.blocks[i]
    fL, aL = oracle.cut_area(wl.frame, wl.avail, y, x, p.block, p.border)
    w = oracle.weights(p.block, p.border, p.rho, aL, p.support)
    ref, _ = oracle.extrapolate_area_ofse(fL, w, p.fft_size, p.iters)
    rng = np.random.default_rng(1000 + i)
    b, br = p.block, p.border
    for _ in range(runs):
        r, _ = oracle.extrapolate_area_ofse(fL * (1 + eps * rng.standard_normal(fL.shape)),
                                            w * (1 + eps * rng.standard_normal(w.shape)),
                                            p.fft_size, p.iters)
        if not np.array_equal(r.u, ref.u):
            return True
        if np.abs(r.g[br:br + b, br:br + b] - ref.g[br:br + b, br:br + b]).max() > tol:
            return True
    return False


def _gamma_errs(wl, res, ora, same_blocks):
    """Relative errors of the factors, |gamma_gpu - gamma| / max(|gamma|, 0.05),
    over every iteration of the given blocks."""
    g = res.gamma.cpu().numpy().astype(np.float64)
    g = g[..., 0] + 1j * g[..., 1]
    errs = []
    for i in same_blocks:
        it = wl.plans[wl.blocks[i, 2]].iters
        ref = ora.ofse_gamma[i, :it]
        errs.append(np.abs(g[i, :it] - ref) / np.maximum(np.abs(ref), 0.05))
    return np.concatenate(errs) if errs else np.zeros(1)


def _gamma_err(wl, res, ora, same_blocks):
    return float(_gamma_errs(wl, res, ora, same_blocks).max())


@pytest.mark.parametrize("spec", [synth.PlanSpec(16, 16, 64, 0.8, 0.5, 120),
                                  synth.PlanSpec(8, 8, 32, 0.8, 0.5, 100),
                                  synth.PlanSpec(4, 4, 32, 0.7, 0.3, 50),
                                  synth.PlanSpec(8, 8, 32, 0.8, 0.5, 64, support=1),
                                  synth.PlanSpec(32, 16, 128, 0.8, 0.5, 150)])
def test_ofse_small_frames_with_edge_blocks(spec):
    """Tiles across the frame corners (partial support), lost neighbours and
    NaN-poisoned lost samples; every fft_size."""
    wl = _ofse(synth.small_frame(23, plan=spec, n_lost=7, fill=np.nan,
                                 height=160 if spec.fft_size == 128 else 96,
                                 width=192 if spec.fft_size == 128 else 128))
    ora = oracle.run_batch(wl.frame, wl.avail, wl.blocks, wl.plans)
    res, _ = run_gpu(wl, "fp32", with_gamma=True)
    c = compare(wl, res, ora)
    assert c["status_equal"]
    assert c["same"] == c["n"], c
    assert c["max_err"] <= 1e-3, c
    same = [i for i in range(c["n"]) if ora.status[i] == 0]
    assert _gamma_err(wl, res, ora, same) <= 1e-4


def test_ofse_full_frame_1080p_and_factor_distribution():
    """The 1920x1080 concealment workload (804 blocks, 64x64 FFT, 200
    iterations) with OFSE's compensation; the distribution of the factors
    (Fig. 2) is centred where the oracle's is, about 0.2."""
    wl = _ofse(synth.frame_concealment())
    ora = oracle.run_batch(wl.frame, wl.avail, wl.blocks, wl.plans)
    res, _ = run_gpu(wl, "fp32", with_gamma=True)
    n = wl.n_blocks
    assert np.array_equal(res.status.cpu().numpy(), ora.status)
    g = res.blocks.cpu().numpy().astype(np.float64)
    g_path = res.path()
    miss = [i for i in range(n)
            if not np.array_equal(g_path[i], ora.path[i]) or np.abs(g[i] - ora.blocks[i]).max() > 1e-3]
    unexplained = [i for i in miss if not _undetermined(wl, i)]
    print(f"OFSE 1080p: {n - len(miss)} of {n} blocks identical; {len(miss)} undetermined at the "
          f"working precision")
    assert not unexplained, unexplained
    # 14 to 19 of the 804 blocks are undetermined at the working precision
    # (each shown so on the oracle above; the count moves with the last-ulp
    # rounding of the oracle's libm on the host), but a regression in OFSE's
    # handling of small Q would add tens
    assert len(miss) <= 25, len(miss)
    keep = np.ones(n, dtype=bool)
    keep[miss] = False
    tb, mask = truth_blocks(wl)
    mask = mask & keep[:, None, None]
    assert abs(psnr(g, tb, mask) - psnr(ora.blocks, tb, mask)) <= 0.01
    same = [i for i in range(n) if keep[i] and ora.status[i] == 0]
    # gamma = W0 P[u] / Q[u] divides by a cancelling sum: on a batch this
    # large some determined blocks still pass through small |Q|, where its
    # relative error is the working precision times that cancellation.  The
    # bulk agrees to the FP32 rounding of the output, a thin tail less well.
    e = _gamma_errs(wl, res, ora, same)
    q50, q999, qmax = np.median(e), np.quantile(e, 0.999), e.max()
    print(f"OFSE 1080p: factor errors on determined blocks: median {q50:.1e}, "
          f"99.9 % {q999:.1e}, max {qmax:.1e}")
    assert q50 <= 1e-6
    assert q999 <= 1e-4
    assert qmax <= 1e-2
    gm = res.gamma.cpu().numpy()[..., 0].reshape(-1)
    assert 0.12 <= float(np.median(gm)) <= 0.28


def test_gamma_output_of_constant_compensation_plans():
    """With the constant compensation the factor of every iteration is the
    plan's gamma; entries past a block's iteration count are zero."""
    import torch
    from paper_2207_01205_gb300 import api
    specs = [synth.PlanSpec(8, 8, 32, 0.8, 0.3, 40), synth.PlanSpec(8, 8, 32, 0.8, 0.3, 25)]
    wl = synth.small_frame(4, plan=specs[0], n_lost=6)
    wl.blocks[::2, 2] = 1
    wl.plans = specs
    plans = [api.Plan.from_spec(p) for p in specs]
    fr, av, bl = to_device(wl)
    res = api.extrapolate(plans, bl, fr, av, with_gamma=True)
    torch.cuda.synchronize()
    g = res.gamma.cpu().numpy()
    for i in range(wl.n_blocks):
        it = specs[wl.blocks[i, 2]].iters
        assert np.all(g[i, :it, 0] == np.float32(0.3)) and np.all(g[i, :it, 1] == 0)
        assert np.all(g[i, it:] == 0)


def test_ofse_unsupported_combinations():
    """OFSE runs only in the FOFSE_FP32 kernel with a workspace and has no
    backward: the other combinations return FOFSE_E_UNSUPPORTED (nothing is
    launched)."""
    import torch
    from paper_2207_01205_gb300 import api, binding
    wl = _ofse(synth.small_frame(6, plan=synth.PlanSpec(8, 8, 32, 0.8, 0.5, 20), n_lost=3))
    fr, av, bl = to_device(wl)
    for prec in ("fp64", "fp32_fullff"):
        plans = [api.Plan.from_spec(p, prec) for p in wl.plans]
        with pytest.raises(binding.FofseError) as e:
            api.extrapolate(plans, bl, fr, av)
        assert e.value.status == binding.E_UNSUPPORTED
    plans = [api.Plan.from_spec(p) for p in wl.plans]
    n = wl.n_blocks
    with pytest.raises(binding.FofseError) as e:
        binding.fofse_extrapolate_batch_noalloc([p.handle for p in plans], bl, fr, av,
                                                out_blocks=torch.empty((n, 8, 8), device="cuda"))
    assert e.value.status == binding.E_UNSUPPORTED
    res = api.extrapolate(plans, bl, fr, av)
    with pytest.raises(binding.FofseError) as e:
        binding.fofse_backward([p.handle for p in plans], bl, fr, av, res.trace, res.w0,
                               torch.ones_like(res.blocks), grad_frame=torch.zeros_like(fr))
    assert e.value.status == binding.E_UNSUPPORTED
    with pytest.raises(binding.FofseError):
        binding.fofse_plan_set_compensation(plans[0].handle, 2)
    torch.cuda.synchronize()
    binding.fofse_check()
