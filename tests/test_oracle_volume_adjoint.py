"""Pins of the oracle's frozen-path companions for video volumes (the method
over three-dimensional sets, Sec. 1, differentiated along a fixed selection
path as for images): the replay reproduces the forward run; the adjoint in f
equals central differences of the replay, exactly, since along a frozen path
the model is linear in f; in gamma and rho it equals Richardson-extrapolated
differences; at depth 0 with Tt = 1 it is the (separately pinned)
two-dimensional adjoint."""
import numpy as np
import pytest

import oracle
from paper_2207_01205_gb300 import synth

PLAN = synth.VolumePlanSpec(4, 2, 1, 8, 4, 0.8, 0.5, 25)


def _case(seed, plan=PLAN):
    wl = synth.small_video(seed, n_frames=3, height=24, width=32, n_lost=3, plan=plan)
    t, y, x = (int(v) for v in wl.blocks[wl.blocks[:, 0] == 1][0])
    fL, aL = oracle.cut_volume(wl.video, wl.avail, t, y, x, plan.block, plan.border, plan.depth)
    w = oracle.weights3(plan.block, plan.border, plan.depth, plan.rho, aL)
    r = oracle.extrapolate_volume(fL, w, plan.fft_size, plan.fft_time, plan.gamma, plan.iters)
    assert r.status == 0
    rng = np.random.default_rng(seed)
    gbar = np.zeros(fL.shape)
    b, e, D = plan.block, plan.border, plan.depth
    gbar[D, e:e + b, e:e + b] = rng.normal(size=(b, b))
    return fL, aL, w, r, gbar


def _loss(fL, w, gamma, path, gbar, plan=PLAN):
    st, g, _ = oracle.replay_volume(fL, w, plan.fft_size, plan.fft_time, gamma, path)
    assert st == 0
    return float(np.sum(gbar * g))


@pytest.mark.parametrize("seed", [1, 2])
def test_replay_reproduces_the_forward_run(seed):
    fL, _, w, r, _ = _case(seed)
    st, g, dc = oracle.replay_volume(fL, w, PLAN.fft_size, PLAN.fft_time, PLAN.gamma, r.u)
    assert st == 0
    np.testing.assert_allclose(dc, r.dc, rtol=0, atol=1e-12 * np.abs(r.dc).max())
    np.testing.assert_allclose(g, r.g, rtol=0, atol=1e-10)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_adjoint_in_f_is_the_exact_derivative(seed):
    fL, _, w, r, gbar = _case(seed)
    fbar, _, _ = oracle.adjoint_volume(fL, w, PLAN.fft_size, PLAN.fft_time, PLAN.gamma, r.u, gbar)
    assert (fbar[w == 0] == 0).all()
    rng = np.random.default_rng(100 + seed)
    for _ in range(3):
        d = rng.normal(size=fL.shape) * (w != 0)
        fd = (_loss(fL + d, w, PLAN.gamma, r.u, gbar) - _loss(fL - d, w, PLAN.gamma, r.u, gbar)) / 2
        assert np.sum(fbar * d) == pytest.approx(fd, rel=1e-9, abs=1e-9)
    # samples outside A do not move the model
    d = rng.normal(size=fL.shape) * (w == 0)
    assert _loss(fL + d, w, PLAN.gamma, r.u, gbar) == pytest.approx(
        _loss(fL, w, PLAN.gamma, r.u, gbar), rel=0, abs=1e-9)


def _richardson(fun, x, h):
    d = lambda hh: (fun(x + hh) - fun(x - hh)) / (2 * hh)
    return (4 * d(h / 2) - d(h)) / 3


@pytest.mark.parametrize("seed", [1, 4])
def test_adjoint_in_gamma_and_rho(seed):
    fL, aL, w, r, gbar = _case(seed)
    _, wbar, gam = oracle.adjoint_volume(fL, w, PLAN.fft_size, PLAN.fft_time, PLAN.gamma, r.u, gbar)
    num_g = _richardson(lambda g_: _loss(fL, w, g_, r.u, gbar), PLAN.gamma, 1e-3)
    assert gam == pytest.approx(num_g, rel=1e-6, abs=1e-9)
    dist = oracle.distance3(PLAN.block, PLAN.border, PLAN.depth)
    rho_bar = oracle.rho_chain(w, dist, PLAN.rho, wbar)

    def loss_rho(rho):
        return _loss(fL, oracle.weights3(PLAN.block, PLAN.border, PLAN.depth, rho, aL), PLAN.gamma,
                     r.u, gbar)
    num_r = _richardson(loss_rho, PLAN.rho, 1e-3)
    assert rho_bar == pytest.approx(num_r, rel=1e-6, abs=1e-9)


def test_depth_zero_equals_the_2d_adjoint():
    wl = synth.small_frame(4, plan=synth.PlanSpec(8, 8, 32, 0.8, 0.5, 20), n_lost=3)
    y, x, _ = wl.blocks[1]
    fL, aL = oracle.cut_area(wl.frame, wl.avail, int(y), int(x), 8, 8)
    w = oracle.weights(8, 8, 0.8, aL)
    r = oracle.extrapolate_area(fL, w, 32, 0.5, 20)
    gbar = np.zeros(fL.shape)
    gbar[8:16, 8:16] = np.random.default_rng(0).normal(size=(8, 8))
    f2, w2, g2 = oracle.adjoint_area(fL, w, 32, 0.5, r.u, gbar)
    path3 = np.concatenate([r.u, np.zeros((20, 1), np.int32)], axis=1)
    f3, w3, g3 = oracle.adjoint_volume(fL[None], w[None], 32, 1, 0.5, path3, gbar[None])
    np.testing.assert_allclose(f3[0], f2, rtol=0, atol=1e-12 * np.abs(f2).max())
    np.testing.assert_allclose(w3[0], w2, rtol=0, atol=1e-9 * np.abs(w2).max())
    assert g3 == pytest.approx(g2, rel=1e-10)
