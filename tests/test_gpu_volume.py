"""Parity of the CUDA extrapolation over video volumes with the FP64 oracle
(the method over three-dimensional sets, Sec. 1): small videos whose volumes
reach beyond the video in space and time, every supported grid shape of both
kernels, the per-block statuses, and the 1920x1080 three-frame workload on a
sample of its blocks and on every block.  The bar is the one for the product
path: identical selection paths and |B_hat - B_oracle| <= 1e-3.  The FP64
validation kernel's coefficients agree with the oracle's to FP64 rounding; the
FP32 kernel's come from its float-float exact values (relative 1e-6, the
bar of the 2-D product kernel)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2207_01205_gb300 import api, synth

pytestmark = pytest.mark.gpu

PRECISIONS = ["fp32", "fp64"]
PLANS = [
    synth.VolumePlanSpec(8, 4, 1, 16, 4, 0.8, 0.5, 40),
    synth.VolumePlanSpec(8, 4, 2, 16, 8, 0.8, 0.5, 40),
    synth.VolumePlanSpec(4, 2, 0, 16, 1, 0.8, 0.5, 30),
    synth.VolumePlanSpec(8, 4, 0, 16, 2, 0.9, 0.7, 30),
    synth.VolumePlanSpec(16, 8, 1, 32, 4, 0.8, 0.5, 60),
    synth.VolumePlanSpec(16, 8, 0, 32, 2, 0.8, 0.5, 40),
    synth.VolumePlanSpec(12, 10, 0, 32, 1, 0.85, 0.4, 40),
]
# grids of the FP32 kernel only (T = 64, and 32 x 32 x 8): up to 16384 bins
PLANS_F32 = [
    synth.VolumePlanSpec(16, 8, 3, 32, 8, 0.8, 0.5, 60),
    synth.VolumePlanSpec(32, 16, 0, 64, 1, 0.8, 0.5, 60),
    synth.VolumePlanSpec(32, 16, 0, 64, 2, 0.8, 0.5, 60),
    synth.VolumePlanSpec(24, 12, 1, 64, 4, 0.8, 0.5, 60),
]


def _video_shape(spec):
    return {16: (64, 96), 32: (96, 128), 64: (128, 192)}[spec.fft_size]


def _run(wl, blocks=None, precision="fp32"):
    blocks = wl.blocks if blocks is None else blocks
    plan = api.VolumePlan.from_spec(wl.plan, precision)
    res = api.extrapolate_volume(plan, torch.from_numpy(np.ascontiguousarray(blocks)).cuda(),
                                 torch.from_numpy(wl.video).cuda(), torch.from_numpy(wl.avail).cuda())
    torch.cuda.synchronize()
    return res


def _compare(res, ora, min_same=0.999, precision="fp32"):
    st = res.status.cpu().numpy()
    np.testing.assert_array_equal(st, ora.status)
    path = res.path.cpu().numpy()
    same = np.array([np.array_equal(path[i], ora.path[i]) for i in range(len(st))])
    assert same.mean() >= min_same, f"identical paths {same.mean():.4f}"
    g = res.blocks.cpu().numpy().astype(np.float64)
    err = np.abs(g - ora.blocks)[same]
    assert err.max() <= 1e-3, f"max abs error {err.max()}"
    coef = res.coef.cpu().numpy()
    dc = coef[..., 0] + 1j * coef[..., 1]
    scale = max(1.0, float(np.abs(ora.dc).max()))
    if precision == "fp64":
        assert np.abs(dc[same] - ora.dc[same]).max() <= 1e-9 * scale
        np.testing.assert_allclose(res.w0.cpu().numpy(), ora.w0, rtol=1e-12, atol=0)
    else:
        assert np.abs(dc[same] - ora.dc[same]).max() <= 1e-6 * scale
        np.testing.assert_allclose(res.w0.cpu().numpy(), ora.w0, rtol=1e-9, atol=0)
    return same, err


def _spec_id(p):
    return f"b{p.block}e{p.border}d{p.depth}T{p.fft_size}x{p.fft_time}"


CASES = [(p, prec) for p in PLANS for prec in PRECISIONS] + [(p, "fp32") for p in PLANS_F32]


@pytest.mark.parametrize("spec,precision", CASES, ids=[f"{_spec_id(p)}-{q}" for p, q in CASES])
def test_small_videos_match_the_oracle(spec, precision):
    n_frames = max(3, 2 * spec.depth + 1)
    h, w = _video_shape(spec)
    wl = synth.small_video(7 + spec.fft_time, n_frames=n_frames, height=h, width=w, plan=spec)
    res = _run(wl, precision=precision)
    ora = oracle.run_batch_volume(wl.video, wl.avail, wl.blocks, wl.plan)
    same, _ = _compare(res, ora, min_same=1.0, precision=precision)
    assert same.all()


@pytest.mark.parametrize("spec", PLANS_F32, ids=_spec_id)
def test_fp64_validation_kernel_refuses_the_fp32_only_grids(spec):
    api.VolumePlan.from_spec(spec)                  # the FP32 kernel takes it
    with pytest.raises(RuntimeError):
        api.VolumePlan.from_spec(spec, "fp64")


def test_the_two_kernels_take_the_same_path():
    """FP32 product and FP64 validation kernel on the same volumes: the same
    selection path, blocks within 1e-3, coefficients within 1e-6 relative."""
    spec = PLANS[4]
    wl = synth.small_video(101, n_frames=3, height=96, width=128, n_lost=8, plan=spec)
    a, b = _run(wl, precision="fp32"), _run(wl, precision="fp64")
    np.testing.assert_array_equal(a.status.cpu().numpy(), b.status.cpu().numpy())
    np.testing.assert_array_equal(a.path.cpu().numpy(), b.path.cpu().numpy())
    assert (a.blocks - b.blocks).abs().max().item() <= 1e-3
    ca, cb = a.coef.cpu().numpy(), b.coef.cpu().numpy()
    assert np.abs(ca - cb).max() <= 1e-6 * max(1.0, np.abs(cb).max())


@pytest.mark.parametrize("precision", PRECISIONS)
def test_statuses_of_blocks_without_support_and_with_nan(precision):
    spec = PLANS[0]
    wl = synth.small_video(3, plan=spec)
    t, y, x = (int(v) for v in wl.blocks[wl.blocks[:, 0] == 1][0])
    _, aL = oracle.cut_volume(wl.video, wl.avail, t, y, x, spec.block, spec.border, spec.depth)
    m, n = np.argwhere(aL[0])[0]
    wl.video[t - 1, y - spec.border + m, x - spec.border + n] = np.nan
    avail = wl.avail.copy()
    wl.avail[:] = 0                                  # first call: nothing usable anywhere
    res0 = _run(wl, precision=precision)
    assert (res0.status.cpu().numpy() == 1).all()
    assert (res0.blocks.cpu().numpy() == 0).all() and (res0.path.cpu().numpy() == 0).all()
    wl.avail[:] = avail
    res = _run(wl, precision=precision)
    ora = oracle.run_batch_volume(wl.video, wl.avail, wl.blocks, wl.plan)
    assert 2 in ora.status
    _compare(res, ora, min_same=1.0, precision=precision)
    bad = res.status.cpu().numpy() == 2
    assert (res.blocks.cpu().numpy()[bad] == 0).all()


@pytest.mark.parametrize("precision", PRECISIONS)
def test_empty_batch_launches_nothing(precision):
    wl = synth.small_video(2, plan=PLANS[0])
    res = _run(wl, blocks=np.zeros((0, 3), np.int32), precision=precision)
    assert res.blocks.shape == (0, 8, 8)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_1080p_three_frame_workload_on_a_sample(precision):
    """The bench's workload (804 lost 16x16 blocks in the centre frame of a
    three-frame 1920x1080 pan, border 8, depth 1, 32x32x4 grid, 200
    iterations) in one launch; the oracle checks 48 blocks spread over it."""
    wl = synth.video_concealment()
    res = _run(wl, precision=precision)
    rng = np.random.default_rng(0)
    pick = np.sort(rng.choice(wl.n_blocks, size=48, replace=False))
    ora = oracle.run_batch_volume(wl.video, wl.avail, wl.blocks[pick], wl.plan)
    st = res.status.cpu().numpy()
    assert (st == 0).all()
    np.testing.assert_array_equal(st[pick], ora.status)
    path = res.path.cpu().numpy()[pick]
    same = np.array([np.array_equal(path[i], ora.path[i]) for i in range(len(pick))])
    assert same.all(), f"{(~same).sum()} of {len(pick)} sampled paths differ"
    g = res.blocks.cpu().numpy()[pick].astype(np.float64)
    assert np.abs(g - ora.blocks).max() <= 1e-3


def test_1080p_three_frame_workload_every_block():
    """The FP32 kernel on all 804 blocks of the workload against the FP64
    transform-domain form of the oracle (pinned to the spatial form on CPU)."""
    wl = synth.video_concealment()
    res = _run(wl)
    ora = oracle.run_batch_volume(wl.video, wl.avail, wl.blocks, wl.plan, transform_domain=True)
    np.testing.assert_array_equal(res.status.cpu().numpy(), ora.status)
    path = res.path.cpu().numpy()
    same = np.array([np.array_equal(path[i], ora.path[i]) for i in range(wl.n_blocks)])
    assert same.all(), f"{(~same).sum()} of {wl.n_blocks} paths differ"
    g = res.blocks.cpu().numpy().astype(np.float64)
    assert np.abs(g - ora.blocks).max() <= 1e-3


LIMIT_PLANS = [  # (plan, seed of the test video)
    (synth.VolumePlanSpec(24, 4, 1, 32, 4, 0.8, 0.5, 60), 45),   # b^2 > threads: two samples of B per thread
    (synth.VolumePlanSpec(20, 6, 0, 32, 1, 0.8, 0.5, 60), 41),   # the same with 256 threads
    (synth.VolumePlanSpec(16, 0, 3, 16, 8, 0.8, 0.5, 40), 337),  # deepest volume of its grid (7 frames), no border
    (synth.VolumePlanSpec(8, 4, 1, 16, 4, 0.8, 0.9, 500), 29),   # long run
]


LIMIT_CASES = [(p, s, q) for p, s in LIMIT_PLANS for q in PRECISIONS]


@pytest.mark.parametrize("spec,seed,precision", LIMIT_CASES,
                         ids=[f"{_spec_id(p)}I{p.iters}-{q}" for p, _, q in LIMIT_CASES])
def test_largest_blocks_deepest_volumes_and_long_runs(spec, seed, precision):
    """Seeds chosen so that no selection of the oracle is an exact tie: where
    the usable frames of a volume alias temporal frequencies (one usable
    frame, or every other frame) two bins have equal magnitude in exact
    arithmetic, and the pick between them depends on rounding (both are
    correct)."""
    n_frames = max(3, 2 * spec.depth + 1)
    h, w = _video_shape(spec)
    wl = synth.small_video(seed, n_frames=n_frames, height=h, width=w, n_lost=3, plan=spec)
    ora = oracle.run_batch_volume(wl.video, wl.avail, wl.blocks, wl.plan)
    assert ora.gap[ora.status == 0].min() > 0.0
    res = _run(wl, precision=precision)
    same, _ = _compare(res, ora, min_same=1.0, precision=precision)
    assert same.all()


@pytest.mark.parametrize("spec", [PLANS[4], PLANS[1], PLANS_F32[0], PLANS_F32[3]], ids=_spec_id)
def test_every_launch_shape_gives_the_same_result(spec):
    """The FP32 kernel's launch shapes (threads per CTA, CTAs per SM) differ
    only in how the work is spread: paths, coefficients and blocks are
    identical bit for bit."""
    from paper_2207_01205_gb300 import binding
    n_frames = max(3, 2 * spec.depth + 1)
    h, w = _video_shape(spec)
    wl = synth.small_video(31, n_frames=n_frames, height=h, width=w, plan=spec)
    plan = api.VolumePlan.from_spec(spec)
    count = binding.fofse_volume_plan_variant_count(plan.handle)
    assert count >= 2
    args = (torch.from_numpy(wl.blocks).cuda(), torch.from_numpy(wl.video).cuda(),
            torch.from_numpy(wl.avail).cuda())
    ref = None
    for v in range(count):
        binding.fofse_volume_plan_set_variant(plan.handle, v)
        res = api.extrapolate_volume(plan, *args)
        got = [t.cpu().numpy() for t in (res.path, res.coef, res.blocks, res.status)]
        if ref is None:
            ref = got
        for a, b in zip(got, ref):
            np.testing.assert_array_equal(a, b)
    with pytest.raises(RuntimeError):
        binding.fofse_volume_plan_set_variant(plan.handle, count)


def test_volume_autotuner_picks_a_shape_and_caches_it(tmp_path):
    """The volume autotuner times every launch shape on the caller's batch,
    keeps one (the default unless another is clearly faster), caches the
    choice per GPU, grid and batch size, and the plan then runs with it."""
    from paper_2207_01205_gb300 import autotune, binding
    spec = PLANS[4]
    wl = synth.small_video(17, n_frames=3, height=96, width=128, n_lost=8, plan=spec)
    plan = api.VolumePlan.from_spec(spec)
    args = (torch.from_numpy(wl.blocks).cuda(), torch.from_numpy(wl.video).cuda(),
            torch.from_numpy(wl.avail).cuda())
    ref = api.extrapolate_volume(plan, *args)
    path = str(tmp_path / "tune.json")
    first = autotune.autotune_volume(plan, *args, cache_path=path)
    count = binding.fofse_volume_plan_variant_count(plan.handle)
    assert not first["cached"] and 0 <= first["choice"] < count and len(first["timings_ms"]) == count
    again = autotune.autotune_volume(plan, *args, cache_path=path)
    assert again["cached"] and again["choice"] == first["choice"]
    res = api.extrapolate_volume(plan, *args)
    torch.cuda.synchronize()
    assert torch.equal(res.path, ref.path) and torch.equal(res.blocks, ref.blocks)
