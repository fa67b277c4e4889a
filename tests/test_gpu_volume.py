"""Parity of the CUDA extrapolation over video volumes with the FP64 oracle
(the method over three-dimensional sets, Sec. 1): small videos whose volumes
reach beyond the video in space and time, every supported grid shape with a
kernel, the per-block statuses, and the 1920x1080 three-frame workload on a
sample of its blocks.  Both sides compute in FP64, so the bar is the one for
the product path (identical selection paths, |B_hat - B_oracle| <= 1e-3) and
the coefficients agree to FP64 rounding."""
import numpy as np
import pytest
import torch

import oracle
from paper_2207_01205_gb300 import api, synth

pytestmark = pytest.mark.gpu

PLANS = [
    synth.VolumePlanSpec(8, 4, 1, 16, 4, 0.8, 0.5, 40),
    synth.VolumePlanSpec(8, 4, 2, 16, 8, 0.8, 0.5, 40),
    synth.VolumePlanSpec(4, 2, 0, 16, 1, 0.8, 0.5, 30),
    synth.VolumePlanSpec(8, 4, 0, 16, 2, 0.9, 0.7, 30),
    synth.VolumePlanSpec(16, 8, 1, 32, 4, 0.8, 0.5, 60),
    synth.VolumePlanSpec(16, 8, 0, 32, 2, 0.8, 0.5, 40),
    synth.VolumePlanSpec(12, 10, 0, 32, 1, 0.85, 0.4, 40),
]


def _run(wl, blocks=None):
    blocks = wl.blocks if blocks is None else blocks
    plan = api.VolumePlan.from_spec(wl.plan)
    res = api.extrapolate_volume(plan, torch.from_numpy(np.ascontiguousarray(blocks)).cuda(),
                                 torch.from_numpy(wl.video).cuda(), torch.from_numpy(wl.avail).cuda())
    torch.cuda.synchronize()
    return res


def _compare(res, ora, min_same=0.999):
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
    assert np.abs(dc[same] - ora.dc[same]).max() <= 1e-9 * scale
    np.testing.assert_allclose(res.w0.cpu().numpy(), ora.w0, rtol=1e-12, atol=0)
    return same, err


@pytest.mark.parametrize("spec", PLANS, ids=lambda p: f"b{p.block}e{p.border}d{p.depth}T{p.fft_size}x{p.fft_time}")
def test_small_videos_match_the_oracle(spec):
    n_frames = max(3, 2 * spec.depth + 1)
    h, w = (64, 96) if spec.fft_size == 16 else (96, 128)
    wl = synth.small_video(7 + spec.fft_time, n_frames=n_frames, height=h, width=w, plan=spec)
    res = _run(wl)
    ora = oracle.run_batch_volume(wl.video, wl.avail, wl.blocks, wl.plan)
    same, _ = _compare(res, ora, min_same=1.0)
    assert same.all()


def test_statuses_of_blocks_without_support_and_with_nan():
    spec = PLANS[0]
    wl = synth.small_video(3, plan=spec)
    t, y, x = (int(v) for v in wl.blocks[wl.blocks[:, 0] == 1][0])
    _, aL = oracle.cut_volume(wl.video, wl.avail, t, y, x, spec.block, spec.border, spec.depth)
    m, n = np.argwhere(aL[0])[0]
    wl.video[t - 1, y - spec.border + m, x - spec.border + n] = np.nan
    avail = wl.avail.copy()
    wl.avail[:] = 0                                  # first call: nothing usable anywhere
    res0 = _run(wl)
    assert (res0.status.cpu().numpy() == 1).all()
    assert (res0.blocks.cpu().numpy() == 0).all() and (res0.path.cpu().numpy() == 0).all()
    wl.avail[:] = avail
    res = _run(wl)
    ora = oracle.run_batch_volume(wl.video, wl.avail, wl.blocks, wl.plan)
    assert 2 in ora.status
    _compare(res, ora, min_same=1.0)
    bad = res.status.cpu().numpy() == 2
    assert (res.blocks.cpu().numpy()[bad] == 0).all()


def test_empty_batch_launches_nothing():
    wl = synth.small_video(2, plan=PLANS[0])
    res = _run(wl, blocks=np.zeros((0, 3), np.int32))
    assert res.blocks.shape == (0, 8, 8)


def test_1080p_three_frame_workload_on_a_sample():
    """The bench's workload (804 lost 16x16 blocks in the centre frame of a
    three-frame 1920x1080 pan, border 8, depth 1, 32x32x4 grid, 200
    iterations) in one launch; the oracle checks 48 blocks spread over it."""
    wl = synth.video_concealment()
    res = _run(wl)
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


LIMIT_PLANS = [  # (plan, seed of the test video)
    (synth.VolumePlanSpec(24, 4, 1, 32, 4, 0.8, 0.5, 60), 45),   # b^2 > threads: two samples of B per thread
    (synth.VolumePlanSpec(20, 6, 0, 32, 1, 0.8, 0.5, 60), 41),   # the same with 256 threads
    (synth.VolumePlanSpec(16, 0, 3, 16, 8, 0.8, 0.5, 40), 337),  # deepest volume of its grid (7 frames), no border
    (synth.VolumePlanSpec(8, 4, 1, 16, 4, 0.8, 0.9, 500), 29),   # long run
]


@pytest.mark.parametrize("spec,seed", LIMIT_PLANS,
                         ids=[f"b{p.block}e{p.border}d{p.depth}T{p.fft_size}x{p.fft_time}I{p.iters}"
                              for p, _ in LIMIT_PLANS])
def test_largest_blocks_deepest_volumes_and_long_runs(spec, seed):
    """Seeds chosen so that no selection of the oracle is an exact tie: where
    the usable frames of a volume alias temporal frequencies (one usable
    frame, or every other frame) two bins have equal magnitude in exact
    arithmetic, and the pick between them depends on rounding (both are
    correct)."""
    n_frames = max(3, 2 * spec.depth + 1)
    h, w = (96, 128) if spec.fft_size == 32 else (64, 96)
    wl = synth.small_video(seed, n_frames=n_frames, height=h, width=w, n_lost=3, plan=spec)
    ora = oracle.run_batch_volume(wl.video, wl.avail, wl.blocks, wl.plan)
    assert ora.gap[ora.status == 0].min() > 0.0
    res = _run(wl)
    same, _ = _compare(res, ora, min_same=1.0)
    assert same.all()
