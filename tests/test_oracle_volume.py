"""Pins of the oracle's extrapolation over video volumes (Sec. 1: the method
carried over to three-dimensional sets).

The paper gives no formulas for volumes; the oracle's readings (a volume of
2 depth + 1 frames around the lost block's frame, Eq. 15's distance over three
coordinates, the 3-D DFT on a T x T x Tt grid, the canonical set by the
row-major index (k1 T + k2) Tt + k3) are pinned here to what fixes them:
numpy's FFT for the transform, brute force over the conjugate pairs for the
selection, integer distances (Pythagorean quadruples) for the weights, the
reduction to the (separately pinned) two-dimensional oracle at depth 0 and
Tt = 1, the symmetry under reversing time about the lost block's frame, and
one iteration on a pure temporal oscillation for the pair weight."""
import numpy as np
import pytest

import oracle
from paper_2207_01205_gb300 import synth


def _lin(k, T, Tt):
    return (k[0] * T + k[1]) * Tt + k[2]


def _neg(k, T, Tt):
    return ((-k[0]) % T, (-k[1]) % T, (-k[2]) % Tt)


@pytest.mark.parametrize("Lt,Ls,T,Tt", [(3, 5, 8, 4), (1, 6, 8, 1), (5, 4, 4, 8), (2, 3, 6, 3)])
def test_projection_is_the_3d_dft(Lt, Ls, T, Tt):
    """P[k] is numpy's forward DFT of the zero-padded volume, the volume's
    (tau, m, n) on the grid's (k3, k1, k2) axes."""
    rng = np.random.default_rng(Lt * 100 + Ls)
    rw = rng.normal(size=(Lt, Ls, Ls))
    Z = np.zeros((T, T, Tt))
    Z[:Ls, :Ls, :Lt] = np.transpose(rw, (1, 2, 0))
    ref = np.fft.fftn(Z)
    P = oracle.project3(rw, T, Tt)
    assert np.abs(P - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("T,Tt", [(4, 4), (4, 2), (6, 3), (4, 1)])
def test_selection_takes_the_canonical_member_of_each_pair(T, Tt):
    """A spectrum holding one conjugate pair (as a real volume's does): the
    pick is the member with the smaller row-major index, for every pair;
    a self-conjugate index is picked as itself."""
    for k in np.ndindex(T, T, Tt):
        mk = _neg(k, T, Tt)
        P = np.zeros((T, T, Tt), dtype=complex)
        P[k] = 1.0 + 0.5j
        P[mk] = np.conj(P[k]) if mk != k else 1.0
        u, gap = oracle.select3(P)
        want = min(k, mk, key=lambda q: _lin(q, T, Tt))
        assert u == want, (k, u, want)
        assert gap == 1.0


def test_selection_ties_go_to_the_smallest_index():
    """Two pairs of equal magnitude: the canonical member with the smallest
    row-major index wins; the relative gap is 0."""
    T, Tt = 8, 4
    rng = np.random.default_rng(5)
    for _ in range(50):
        a, b = (tuple(int(v) for v in rng.integers(0, [T, T, Tt])) for _ in range(2))
        pairs = [a, _neg(a, T, Tt), b, _neg(b, T, Tt)]
        if len({min(a, _neg(a, T, Tt)), min(b, _neg(b, T, Tt))}) < 2:
            continue
        P = np.zeros((T, T, Tt), dtype=complex)
        for q in pairs:
            P[q] = 2.0
        u, gap = oracle.select3(P)
        cands = [min(q, _neg(q, T, Tt), key=lambda r: _lin(r, T, Tt)) for q in (a, b)]
        assert u == min(cands, key=lambda r: _lin(r, T, Tt))
        assert gap == 0.0


def test_weights_at_integer_distances():
    """b = 1 puts B's centre on a sample: Pythagorean quadruples give integer
    distances, so w = rho^d exactly (frame offsets count as samples); B is
    outside A in its own frame only; unusable samples weigh 0."""
    rho, depth, border = 0.8, 6, 7
    Lt, Ls = 2 * depth + 1, 2 * border + 1
    aL = np.ones((Lt, Ls, Ls), dtype=np.uint8)
    aL[depth + 1, border + 1, border + 2] = 0
    w = oracle.weights3(1, border, depth, rho, aL)
    c = border
    cases = {  # (dtau, dm, dn) -> distance
        (2, 3, 6): 7, (-6, 2, 3): 7, (0, 3, -4): 5, (1, 0, 0): 1, (-1, 0, 0): 1,
        (2, -1, 2): 3, (-4, 4, 2): 6, (6, 0, 0): 6, (0, -7, 0): 7,
    }
    for (dt, dm, dn), d in cases.items():
        assert w[depth + dt, c + dm, c + dn] == pytest.approx(rho ** d, rel=1e-14), (dt, dm, dn)
    assert w[depth, c, c] == 0.0                       # B in its own frame
    assert w[depth + 1, c + 1, c + 2] == 0.0           # unusable sample
    # b = 3: the centre of B is the middle sample; B's position in the
    # neighbouring frames is in A, at distance 1 from the centre
    w3 = oracle.weights3(3, 2, 1, rho, np.ones((3, 7, 7), dtype=np.uint8))
    assert (w3[1, 2:5, 2:5] == 0).all()
    assert w3[0, 3, 3] == pytest.approx(rho, rel=1e-15)
    assert w3[2, 3, 3] == pytest.approx(rho, rel=1e-15)
    assert w3[0, 3, 5] == pytest.approx(rho ** np.sqrt(5.0), rel=1e-14)


def test_cut_volume_marks_samples_beyond_the_video_unusable():
    rng = np.random.default_rng(1)
    video = rng.uniform(0, 255, size=(3, 20, 24)).astype(np.float32)
    avail = np.ones(video.shape, dtype=np.uint8)
    avail[1, 5, 7] = 0
    fL, aL = oracle.cut_volume(video, avail, 0, 0, 20, 4, 4, 1)
    assert fL.shape == (3, 12, 12)
    assert not aL[0].any() and (fL[0] == 0).all()          # frame -1 does not exist
    assert not aL[1:, :4].any() and not aL[1:, :, 8:].any()  # rows < 0, columns >= 24
    assert aL[1:, 4:, :8].all()
    np.testing.assert_array_equal(fL[1:, 4:, :8], video[0:2, 0:8, 16:24])
    fL, aL = oracle.cut_volume(video, avail, 2, 4, 4, 4, 2, 1)
    assert aL[0, 2 + 1, 2 + 3] == 0 and aL[0].sum() == 8 * 8 - 1  # frame 1, sample (5, 7)
    assert not aL[2].any()                                 # frame 3 does not exist


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_depth_zero_reduces_to_the_2d_oracle(seed):
    """One frame, Tt = 1: weights, path, coefficients and model are those of
    the two-dimensional oracle."""
    wl = synth.small_frame(seed, plan=synth.PlanSpec(8, 8, 32, 0.8, 0.5, 30), n_lost=4)
    for (y, x, _) in wl.blocks:
        fL, aL = oracle.cut_area(wl.frame, wl.avail, int(y), int(x), 8, 8)
        w2 = oracle.weights(8, 8, 0.8, aL)
        w3 = oracle.weights3(8, 8, 0, 0.8, aL[None])
        np.testing.assert_array_equal(w3[0], w2)
        r2 = oracle.extrapolate_area(fL, w2, 32, 0.5, 30)
        r3 = oracle.extrapolate_volume(fL[None], w3, 32, 1, 0.5, 30)
        assert r3.status == r2.status
        np.testing.assert_array_equal(r3.u[:, :2], r2.u)
        assert (r3.u[:, 2] == 0).all()
        np.testing.assert_allclose(r3.dc, r2.dc, rtol=0, atol=1e-12 * max(1.0, np.abs(r2.dc).max()))
        np.testing.assert_allclose(r3.g[0], r2.g, rtol=0, atol=1e-10)
    # the batch drivers agree too (block lists (t, y, x) against (y, x, plan))
    vb = np.concatenate([np.zeros((wl.n_blocks, 1), np.int32), wl.blocks[:, :2]], axis=1)
    r3 = oracle.run_batch_volume(wl.frame[None], wl.avail[None], vb,
                                 synth.VolumePlanSpec(8, 8, 0, 32, 1, 0.8, 0.5, 30))
    r2 = oracle.run_batch(wl.frame, wl.avail, wl.blocks, wl.plans)
    np.testing.assert_array_equal(r3.path[:, :, :2], r2.path)
    np.testing.assert_allclose(r3.blocks, r2.blocks[:, :8, :8], rtol=0, atol=1e-10)


def test_reversing_time_leaves_the_centre_frame_unchanged():
    """Volumes symmetric in time around B's frame: reversing the frame order
    maps every pair (u1, u2, u3) to (u1, u2, -u3) with the same magnitude, so
    the model of the reversed video is the reversed model, and B_hat (in the
    centre frame) is unchanged."""
    plan = synth.VolumePlanSpec(8, 4, 2, 16, 8, 0.8, 0.5, 25)
    wl = synth.small_video(11, n_frames=5, plan=plan)
    pick = wl.blocks[wl.blocks[:, 0] == 2]
    a = oracle.run_batch_volume(wl.video, wl.avail, pick, plan)
    b = oracle.run_batch_volume(wl.video[::-1], wl.avail[::-1], pick, plan)
    assert (a.status == 0).all()
    np.testing.assert_allclose(b.blocks, a.blocks, rtol=0, atol=1e-9 * np.abs(a.blocks).max())
    T, Tt = plan.fft_size, plan.fft_time
    for pa, pb in zip(a.path.reshape(-1, 3), b.path.reshape(-1, 3)):
        mapped = (int(pa[0]), int(pa[1]), (-int(pa[2])) % Tt)
        assert tuple(int(v) for v in pb) in (mapped, _neg(mapped, T, Tt))


def test_one_iteration_on_a_temporal_oscillation():
    """f = 100 cos(pi tau / 2 + 0.3) over 4 full frames (Tt = 4, the lost
    block in frame 2 excluded): the first pick is the temporal frequency
    (0, 0, 1) of the pair {1, 3}; c = gamma P[u] / W0 with P from numpy's FFT;
    and the model is 2 Re(c phi_u), the basis function and its conjugate."""
    Ls, T, Tt, gamma = 8, 8, 4, 0.7
    tau = np.arange(3)[:, None, None]
    f = np.broadcast_to(100.0 * np.cos(np.pi * tau / 2 + 0.3), (3, Ls, Ls)).copy()
    aL = np.ones((3, Ls, Ls), dtype=np.uint8)
    w = oracle.weights3(2, 3, 1, 0.9, aL)
    r = oracle.extrapolate_volume(f, w, T, Tt, gamma, 1)
    assert tuple(r.u[0]) == (0, 0, 1)
    Z = np.zeros((T, T, Tt))
    Z[:Ls, :Ls, :3] = np.transpose(w * f, (1, 2, 0))
    c = gamma * np.fft.fftn(Z)[0, 0, 1] / w.sum()
    assert r.dc[0] == pytest.approx(c, rel=1e-12)
    model = 2.0 * np.real(c * np.exp(2j * np.pi * tau / 4))
    np.testing.assert_allclose(r.g, np.broadcast_to(model, (3, Ls, Ls)), rtol=0, atol=1e-10)


def test_self_conjugate_pick_has_a_real_coefficient_and_single_weight():
    """A volume oscillating at the temporal Nyquist frequency (u = (0, 0, 2)
    for Tt = 4, self-conjugate): the coefficient is real and the model is
    c phi_u, not doubled."""
    Ls, T, Tt, gamma = 6, 8, 4, 1.0
    tau = np.arange(3)[:, None, None]
    f = np.broadcast_to(50.0 * np.cos(np.pi * tau), (3, Ls, Ls)).copy()
    w = oracle.weights3(2, 2, 1, 0.85, np.ones((3, Ls, Ls), dtype=np.uint8))
    r = oracle.extrapolate_volume(f, w, T, Tt, gamma, 1)
    assert tuple(r.u[0]) == (0, 0, 2)
    assert r.dc[0].imag == 0.0
    Z = np.zeros((T, T, Tt))
    Z[:Ls, :Ls, :3] = np.transpose(w * f, (1, 2, 0))
    c = gamma * np.fft.fftn(Z)[0, 0, 2].real / w.sum()
    np.testing.assert_allclose(r.g, np.broadcast_to(c * np.cos(np.pi * tau), (3, Ls, Ls)),
                               rtol=0, atol=1e-10)


def test_statuses_and_temporal_support_helps():
    """No usable sample gives NO_SUPPORT and a zero block; on the camera pan
    the volume's estimate is closer to the truth than the single frame's."""
    plan = synth.VolumePlanSpec(8, 4, 1, 16, 4, 0.8, 0.5, 40)
    wl = synth.small_video(4, plan=plan)
    avail0 = np.zeros_like(wl.avail)
    r = oracle.run_batch_volume(wl.video, avail0, wl.blocks[:2], plan)
    assert (r.status == oracle.STATUS_NO_SUPPORT).all() and (r.blocks == 0).all()
    # a NaN at one usable sample of a block's volume (the neighbouring frame)
    t, y, x = (int(v) for v in wl.blocks[wl.blocks[:, 0] == 1][0])
    _, aL = oracle.cut_volume(wl.video, wl.avail, t, y, x, 8, 4, 1)
    m, n = np.argwhere(aL[0])[0]
    bad = wl.video.copy()
    bad[t - 1, y - 4 + m, x - 4 + n] = np.nan
    r = oracle.run_batch_volume(bad, wl.avail, np.array([[t, y, x]]), plan)
    assert r.status[0] == oracle.STATUS_NONFINITE
    centre = wl.blocks[wl.blocks[:, 0] == 1]
    truth = np.stack([wl.truth[t, y:y + 8, x:x + 8] for (t, y, x) in centre])
    r3 = oracle.run_batch_volume(wl.video, wl.avail, centre, plan)
    r2 = oracle.run_batch_volume(wl.video, wl.avail, centre,
                                 synth.VolumePlanSpec(8, 4, 0, 16, 1, 0.8, 0.5, 40))
    e3 = np.mean((np.clip(r3.blocks, 0, 255) - truth) ** 2)
    e2 = np.mean((np.clip(r2.blocks, 0, 255) - truth) ** 2)
    assert e3 < e2


@pytest.mark.parametrize("plan,seed", [
    (synth.VolumePlanSpec(8, 4, 1, 16, 4, 0.8, 0.5, 40), 1),
    (synth.VolumePlanSpec(8, 4, 2, 16, 8, 0.8, 0.7, 40), 2),
    (synth.VolumePlanSpec(4, 2, 0, 8, 2, 0.9, 0.5, 30), 3),
])
def test_transform_domain_form_equals_the_reprojection(plan, seed):
    """The transform-domain form (spectra transformed once, the spectrum of
    each added pair subtracted from every bin) and the spatial re-projection
    take the same path, coefficients to 1e-9 and models to 1e-9."""
    n_frames = max(3, 2 * plan.depth + 1)
    wl = synth.small_video(seed, n_frames=n_frames, plan=plan)
    a = oracle.run_batch_volume(wl.video, wl.avail, wl.blocks, plan)
    b = oracle.run_batch_volume(wl.video, wl.avail, wl.blocks, plan, transform_domain=True)
    np.testing.assert_array_equal(a.status, b.status)
    np.testing.assert_array_equal(a.path, b.path)
    np.testing.assert_allclose(b.dc, a.dc, rtol=0, atol=1e-9 * np.abs(a.dc).max())
    np.testing.assert_allclose(b.blocks, a.blocks, rtol=0, atol=1e-9 * np.abs(a.blocks).max())
