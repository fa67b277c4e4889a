"""The video-volume backward (fofse_volume_backward: the adjoint of the volume
recursion along the frozen selection path) against the FP64 oracle's adjoint
(oracle.adjoint_volume, pinned on CPU against differences of its replay),
composed over the batch here: each block's dl/df scattered into the video's
gradient (overlapping volumes add), dl/drho through w = rho^d summed over the
blocks, dl/dgamma summed.  The GPU works in FP32: relative L2 1e-3 on the
video gradient, 1e-3 on rho and gamma."""
import numpy as np
import pytest
import torch

import oracle
from paper_2207_01205_gb300 import api, binding, synth

pytestmark = pytest.mark.gpu


def _oracle_gradients(wl, blocks, path, grad_blocks):
    spec = wl.plan
    b, e, D = spec.block, spec.border, spec.depth
    gv = np.zeros(wl.video.shape)
    rho_bar = gamma_bar = 0.0
    dist = oracle.distance3(b, e, D)
    F, H, W = wl.video.shape
    for i, (t, y, x) in enumerate(blocks):
        fL, aL = oracle.cut_volume(wl.video, wl.avail, t, y, x, b, e, D)
        wL = oracle.weights3(b, e, D, spec.rho, aL)
        if not (wL.sum() > 0) or not np.isfinite(fL[wL != 0]).all():
            continue
        gbar = np.zeros(fL.shape)
        gbar[D, e:e + b, e:e + b] = grad_blocks[i]
        fbar, wbar, gbr = oracle.adjoint_volume(fL, wL, spec.fft_size, spec.fft_time, spec.gamma,
                                                path[i], gbar)
        gamma_bar += gbr
        rho_bar += float(np.sum(wbar * wL * dist)) / spec.rho
        Lt, Ls = fL.shape[0], fL.shape[1]
        for tau in range(Lt):
            ft = t - D + tau
            if not 0 <= ft < F:
                continue
            for m in range(Ls):
                fy = y - e + m
                if not 0 <= fy < H:
                    continue
                x0, x1 = max(0, x - e), min(W, x - e + Ls)
                gv[ft, fy, x0:x1] += fbar[tau, m, x0 - (x - e):x1 - (x - e)]
    return gv, rho_bar, gamma_bar


def _gpu_gradients(wl, blocks, precision, grad_blocks):
    plan = api.VolumePlan.from_spec(wl.plan, precision)
    bl = torch.from_numpy(np.ascontiguousarray(blocks)).cuda()
    video = torch.from_numpy(wl.video).cuda()
    avail = torch.from_numpy(wl.avail).cuda()
    res = api.extrapolate_volume(plan, bl, video, avail)
    gv, grg = api.volume_backward(plan, bl, video, avail, res,
                                  torch.from_numpy(grad_blocks.astype(np.float32)).cuda())
    torch.cuda.synchronize()
    binding.fofse_check()
    return res, gv.cpu().numpy().astype(np.float64), grg.cpu().numpy().astype(np.float64)


def _check(wl, blocks, precision, seed):
    rng = np.random.default_rng(seed)
    b = wl.plan.block
    grad_blocks = rng.normal(size=(len(blocks), b, b))
    res, gv, grg = _gpu_gradients(wl, blocks, precision, grad_blocks)
    path = res.path.cpu().numpy()
    ogv, orho, ogam = _oracle_gradients(wl, blocks, path, grad_blocks)
    rel = np.linalg.norm(gv - ogv) / max(np.linalg.norm(ogv), 1e-30)
    assert rel <= 1e-3, f"video gradient relative L2 error {rel}"
    assert abs(grg[0] - orho) <= 1e-3 * abs(orho) + 1e-6, (grg[0], orho)
    assert abs(grg[1] - ogam) <= 1e-3 * abs(ogam) + 1e-6, (grg[1], ogam)
    return rel


SPECS = [
    synth.VolumePlanSpec(8, 4, 1, 16, 4, 0.8, 0.5, 40),
    synth.VolumePlanSpec(8, 4, 0, 16, 1, 0.85, 0.4, 30),
    synth.VolumePlanSpec(16, 8, 1, 32, 4, 0.8, 0.5, 60),
    synth.VolumePlanSpec(24, 12, 1, 64, 4, 0.8, 0.5, 40),   # w of the volume inside W's free frame
    synth.VolumePlanSpec(16, 8, 3, 32, 8, 0.8, 0.5, 40),    # seven frames: w beside W
]


@pytest.mark.parametrize("spec", SPECS, ids=lambda p: f"b{p.block}e{p.border}d{p.depth}T{p.fft_size}x{p.fft_time}")
def test_small_videos_match_the_oracle_adjoint(spec):
    h, w = {16: (64, 96), 32: (96, 128), 64: (128, 192)}[spec.fft_size]
    wl = synth.small_video(11, n_frames=3, height=h, width=w, plan=spec)
    _check(wl, wl.blocks, "fp32", 5)


def test_fp64_plan_gives_the_same_gradients():
    spec = SPECS[2]
    wl = synth.small_video(13, n_frames=3, height=96, width=128, plan=spec)
    _check(wl, wl.blocks, "fp64", 7)


def test_blocks_without_support_or_with_nan_contribute_nothing():
    spec = SPECS[0]
    wl = synth.small_video(3, plan=spec)
    t, y, x = (int(v) for v in wl.blocks[wl.blocks[:, 0] == 1][0])
    _, aL = oracle.cut_volume(wl.video, wl.avail, t, y, x, spec.block, spec.border, spec.depth)
    m, n = np.argwhere(aL[0])[0]
    wl.video[t - 1, y - spec.border + m, x - spec.border + n] = np.nan
    rng = np.random.default_rng(2)
    grad_blocks = rng.normal(size=(len(wl.blocks), spec.block, spec.block))
    res, gv, grg = _gpu_gradients(wl, wl.blocks, "fp32", grad_blocks)
    assert 2 in res.status.cpu().numpy()
    gv[np.isnan(gv)] = 0.0
    ogv, orho, ogam = _oracle_gradients(wl, wl.blocks, res.path.cpu().numpy(), grad_blocks)
    assert np.isfinite(grg).all()
    np.testing.assert_allclose(gv, ogv, rtol=0, atol=1e-3 * np.abs(ogv).max())
    assert abs(grg[1] - ogam) <= 1e-3 * abs(ogam) + 1e-6


def test_1080p_video_batch_on_a_sample():
    """64 blocks of the three-frame 1080p batch (32x32x4 grid, 200 iterations)."""
    wl = synth.video_concealment()
    rng = np.random.default_rng(0)
    pick = np.sort(rng.choice(wl.n_blocks, size=64, replace=False))
    _check(wl, wl.blocks[pick], "fp32", 9)


def test_volumes_beyond_the_shared_memory_limit_are_refused():
    """The solve keeps W (128 KB at 64 x 64 x 4), the row transforms of w and
    w itself in shared memory: a 3 x 64 x 64 volume needs 275 KB."""
    spec = synth.VolumePlanSpec(32, 16, 1, 64, 4, 0.8, 0.5, 10)
    wl = synth.small_video(4, n_frames=3, height=128, width=192, n_lost=1, plan=spec)
    plan = api.VolumePlan.from_spec(spec)
    bl = torch.from_numpy(wl.blocks).cuda()
    video = torch.from_numpy(wl.video).cuda()
    avail = torch.from_numpy(wl.avail).cuda()
    res = api.extrapolate_volume(plan, bl, video, avail)
    with pytest.raises(binding.FofseError) as ei:
        api.volume_backward(plan, bl, video, avail, res, torch.zeros_like(res.blocks))
    assert ei.value.status == binding.E_UNSUPPORTED


def test_forward_and_backward_replay_in_a_cuda_graph():
    """The FP32 volume forward (queue reset + one launch) and the backward (two
    launches) captured in one CUDA graph replay the eager results bit for bit."""
    spec = SPECS[2]
    wl = synth.small_video(21, n_frames=3, height=96, width=128, plan=spec)
    plan = api.VolumePlan.from_spec(spec)
    bl = torch.from_numpy(wl.blocks).cuda()
    video = torch.from_numpy(wl.video).cuda()
    avail = torch.from_numpy(wl.avail).cuda()
    n, b, it = wl.n_blocks, spec.block, spec.iters
    ge = torch.from_numpy(np.random.default_rng(3).normal(size=(n, b, b)).astype(np.float32)).cuda()
    eager = api.extrapolate_volume(plan, bl, video, avail)
    egv, egrg = api.volume_backward(plan, bl, video, avail, eager, ge)
    out = torch.empty((n, b, b), dtype=torch.float32, device="cuda")
    path = torch.empty((n, it, 3), dtype=torch.int32, device="cuda")
    coef = torch.empty((n, it, 2), dtype=torch.float64, device="cuda")
    w0 = torch.empty((n,), dtype=torch.float64, device="cuda")
    st = torch.empty((n,), dtype=torch.int32, device="cuda")
    ws = api.volume_workspace(plan, n, "cuda")
    bws = torch.empty((binding.fofse_volume_backward_workspace_bytes(plan.handle, n),),
                      dtype=torch.uint8, device="cuda")
    gv = torch.zeros_like(video)
    grg = torch.zeros((2,), dtype=torch.float32, device="cuda")

    def step(s):
        binding.fofse_extrapolate_volume_batch(plan.handle, bl, video, avail, out_blocks=out, path=path,
                                               coef=coef, w0=w0, status=st, workspace=ws, stream=s)
        gv.zero_()
        grg.zero_()
        binding.fofse_volume_backward(plan.handle, bl, video, avail, path, coef, w0, ge, status=st,
                                      grad_video=gv, grad_rho_gamma=grg, workspace=bws, stream=s)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):  # warm-up outside the capture
        step(s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step(torch.cuda.current_stream())
    for _ in range(2):
        out.zero_()
        g.replay()
        torch.cuda.synchronize()
        binding.fofse_check()
        assert torch.equal(out, eager.blocks) and torch.equal(path, eager.path)
        assert torch.allclose(gv, egv, rtol=0, atol=1e-6 * float(egv.abs().max()))
        assert torch.allclose(grg, egrg, rtol=1e-6, atol=0)
