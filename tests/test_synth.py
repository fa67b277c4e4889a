"""The seeded synthetic inputs (no method arithmetic): determinism, the loss
patterns and masks the workloads state, and the camera pan of the video
workloads."""
import numpy as np

from paper_2207_01205_gb300 import synth


def test_frame_concealment_loses_ten_percent_of_the_tiles():
    a = synth.frame_concealment()
    b = synth.frame_concealment()
    assert np.array_equal(a.frame, b.frame) and np.array_equal(a.blocks, b.blocks)
    assert a.frame.shape == (1080, 1920) and a.n_blocks == 804
    lost = np.zeros(a.avail.shape, dtype=bool)
    for (y, x, _) in a.blocks:
        assert y % 16 == 0 and x % 16 == 0
        lost[y:y + 16, x:x + 16] = True
    assert np.array_equal(a.avail == 0, lost)
    assert (a.frame[lost] == 0).all() and np.array_equal(a.frame[~lost], a.truth[~lost])
    assert a.truth.min() >= 0 and a.truth.max() <= 255 and (a.truth == np.rint(a.truth)).all()


def test_video_concealment_loses_tiles_in_every_frame():
    wl = synth.video_concealment()
    again = synth.video_concealment()
    assert np.array_equal(wl.video, again.video) and np.array_equal(wl.blocks, again.blocks)
    F, H, W = wl.video.shape
    assert (F, H, W) == (3, 1080, 1920) and wl.n_blocks == 804
    assert (wl.blocks[:, 0] == 1).all()                      # the centre frame's blocks
    tiles = (H // 16) * (W // 16)
    for t in range(F):
        lost_t = (wl.avail[t] == 0).sum() // 256
        assert lost_t == round(0.10 * tiles)                  # 10 % of every frame
    for (t, y, x) in wl.blocks:
        assert (wl.avail[t, y:y + 16, x:x + 16] == 0).all()
        assert (wl.video[t, y:y + 16, x:x + 16] == 0).all()
    ok = wl.avail == 1
    assert np.array_equal(wl.video[ok], wl.truth[ok])
    assert wl.truth.dtype == np.float32 and (wl.truth == np.rint(wl.truth)).all()


def test_moving_frames_are_a_pan_of_one_canvas():
    """Without noise, frame i + 1 is frame i shifted by a step of 0..max_step
    px per axis: the shift that makes them agree is found by search."""
    rng = np.random.Generator(np.random.PCG64(9))
    f = synth.moving_frames(rng, 4, 64, 80, max_step=2, noise_sigma=0.0, n_sines=4, n_polys=3)
    assert f.shape == (4, 64, 80) and f.dtype == np.float32
    for i in range(3):
        best = None
        for dy in range(3):
            for dx in range(3):
                a = f[i, dy:, dx:]
                b = f[i + 1, :64 - dy, :80 - dx]
                err = np.abs(a - b).max()
                best = err if best is None else min(best, err)
        assert best == 0.0


def test_small_video_covers_the_corners_of_the_first_and_last_frames():
    plan = synth.VolumePlanSpec(8, 4, 1, 16, 4, 0.8, 0.5, 40)
    wl = synth.small_video(3, n_frames=4, plan=plan)
    rows = {tuple(r) for r in wl.blocks}
    assert (0, 0, 0) in rows and (3, 64 - 8, 96 - 8) in rows
    for (t, y, x) in wl.blocks:
        assert (wl.avail[t, y:y + 8, x:x + 8] == 0).all()
    assert plan.rho == float(np.float32(0.8)) and plan.gamma == 0.5
