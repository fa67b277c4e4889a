"""Parity of the error-over-iterations kernel (fofse_error_curve, the
quantity behind Fig. 4 and Fig. 5) with the oracle's curve, each built from
its own run: per block the squared error over B after every iteration count
agrees to 1e-4 relative (plus 1e-3 absolute: the model is FP32), the PSNR
curve of a batch to 0.01 dB at every iteration count."""
import numpy as np
import pytest

import oracle
from paper_2207_01205_gb300 import synth

from parity_util import to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib(gpu_lib):
    return gpu_lib


def _gpu_curve(wl):
    import torch
    from paper_2207_01205_gb300 import api, binding
    plans = [api.Plan.from_spec(p) for p in wl.plans]
    fr, av, bl = to_device(wl)
    res = api.extrapolate(plans, bl, fr, av)
    truth = torch.from_numpy(np.ascontiguousarray(wl.truth, dtype=np.float32)).cuda()
    sse = torch.empty((wl.n_blocks, max(p.iters for p in wl.plans)), dtype=torch.float32, device="cuda")
    binding.fofse_error_curve([p.handle for p in plans], bl, res.trace, truth, sse)
    torch.cuda.synchronize()
    binding.fofse_check()
    return res, sse.cpu().numpy().astype(np.float64)


def _oracle_curves(wl, ora):
    out = np.zeros((wl.n_blocks, max(p.iters for p in wl.plans)))
    for i, (y, x, pi) in enumerate(wl.blocks):
        p = wl.plans[pi]
        Ls = p.block + 2 * p.border
        tb = wl.truth[y:y + p.block, x:x + p.block].astype(np.float64)
        out[i, :p.iters] = oracle.error_curve(Ls, p.fft_size, p.block, p.border,
                                              ora.path[i, :p.iters], ora.dc[i, :p.iters], tb,
                                              basis=getattr(p, "basis", 0))
    return out


def _check(wl, res, sse, ora, ref):
    g_path = res.path()
    n_same = 0
    for i, (_, _, pi) in enumerate(wl.blocks):
        it = wl.plans[pi].iters
        assert np.all(sse[i, it:] == 0)
        if ora.status[i] != 0 or not np.array_equal(g_path[i, :it], ora.path[i, :it]):
            continue
        n_same += 1
        np.testing.assert_allclose(sse[i, :it], ref[i, :it], rtol=1e-4, atol=1e-3)
    return n_same


@pytest.mark.parametrize("specs", [[synth.PlanSpec(16, 16, 64, 0.8, 0.5, 120)],
                                   [synth.PlanSpec(8, 8, 32, 0.8, 0.3, 100), synth.PlanSpec(4, 4, 32, 0.8, 0.3, 40)],
                                   [synth.PlanSpec(32, 16, 128, 0.8, 0.5, 90)],
                                   [synth.PlanSpec(16, 16, 64, 0.8, 0.5, 80, 0, 0, 1)]])
def test_curve_small_frames(specs):
    big = specs[0].fft_size == 128
    wl = synth.small_frame(31, plan=specs[0], n_lost=7, height=160 if big else 96,
                           width=192 if big else 128)
    if len(specs) > 1:   # a second plan with fewer iterations: zero tail
        wl.plans = specs
        wl.blocks[1::2, 2] = 1
    ora = oracle.run_batch(wl.frame, wl.avail, wl.blocks, wl.plans)
    res, sse = _gpu_curve(wl)
    assert _check(wl, res, sse, ora, _oracle_curves(wl, ora)) == wl.n_blocks


def test_curve_1080p_psnr_over_iterations():
    """The 1920x1080 batch: the PSNR-over-iterations curve of all 804 blocks."""
    wl = synth.frame_concealment()
    ora = oracle.run_batch(wl.frame, wl.avail, wl.blocks, wl.plans)
    res, sse = _gpu_curve(wl)
    ref = _oracle_curves(wl, ora)
    assert _check(wl, res, sse, ora, ref) >= 0.999 * wl.n_blocks
    npx = wl.n_blocks * 16 * 16
    p_gpu = 10 * np.log10(255.0 ** 2 * npx / sse.sum(axis=0))
    p_ora = 10 * np.log10(255.0 ** 2 * npx / ref.sum(axis=0))
    assert np.max(np.abs(p_gpu - p_ora)) <= 0.01
    # the curve rises from the first iterations (the model starts at zero)
    assert p_gpu[-1] > p_gpu[0] + 10


def test_curve_argument_errors():
    import torch
    from paper_2207_01205_gb300 import api, binding
    p = api.Plan(40, 8, 64, 0.8, 0.5, 10)   # block side above 32
    bl = torch.zeros((1, 3), dtype=torch.int32, device="cuda")
    tr = torch.zeros((1, 10, 3), dtype=torch.int32, device="cuda")
    truth = torch.zeros((64, 64), dtype=torch.float32, device="cuda")
    sse = torch.zeros((1, 10), dtype=torch.float32, device="cuda")
    with pytest.raises(binding.FofseError) as e:
        binding.fofse_error_curve([p.handle], bl, tr, truth, sse)
    assert e.value.status == binding.E_UNSUPPORTED
