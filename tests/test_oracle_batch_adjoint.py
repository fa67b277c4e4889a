"""Pins of the oracle's batch adjoint, the reference of every GPU gradient test.

``oracle.batch_adjoint`` composes the per-area adjoint (pinned in
test_oracle_pins.py) over a batch: the frame gradient is scattered from each
block's area L into the frame and summed where supports overlap, and the
(rho, gamma) gradients are summed per plan.  The loss is
sum_i <e_i, B_hat_i> with every selection path frozen (the frozen-path
derivative of the extrapolation of Sec. 2, Eq. 2-5, Eq. 14 with the weights of
Eq. 15).  The pins, on a small frame with two plans, overlapping supports and
an area that crosses the frame edge:
  * the batch result equals the per-block adjoints scattered and summed here;
  * the frame gradient equals central differences of the batch loss (exact up
    to rounding: along a frozen path B_hat is linear in the samples);
  * each plan's d/drho and d/dgamma equal Richardson-extrapolated central
    differences of the batch loss;
  * the result does not depend on the number of threads.
"""
import numpy as np
import pytest

import oracle
from paper_2207_01205_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore")

H, W = 40, 56
PLANS = [synth.PlanSpec(4, 4, 16, np.float32(0.8).item(), np.float32(0.45).item(), 10),
         synth.PlanSpec(8, 4, 16, np.float32(0.75).item(), np.float32(0.6).item(), 8)]
# (y, x, plan) of B's top-left corner: the first two areas overlap the third
# one, the fourth crosses the top edge of the frame, the fifth its right edge
BLOCKS = np.array([[4, 4, 0], [8, 20, 0], [12, 8, 1], [2, 36, 0], [24, 48, 1]], dtype=np.int32)


def _case(seed=11):
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:H, 0:W]
    base = 128 + 40 * np.sin(2 * np.pi * (0.07 * yy + 0.03 * xx)) + 25 * np.cos(0.31 * xx - 0.2 * yy)
    frame = np.clip(np.round(base + rng.normal(0, 6, size=(H, W))), 0, 255).astype(np.float32)
    avail = np.ones((H, W), dtype=np.uint8)
    for y, x, p in BLOCKS:
        b = PLANS[p].block
        avail[y:y + b, x:x + b] = 0
    res = oracle.run_batch(frame, avail, BLOCKS, PLANS, threads=2)
    assert np.all(res.status == oracle.STATUS_OK)
    e = np.zeros((len(BLOCKS), 8, 8))
    for i, (_, _, p) in enumerate(BLOCKS):
        b = PLANS[p].block
        e[i, :b, :b] = rng.normal(size=(b, b))
    return frame, avail, res.path, e


def _batch_loss(frame, avail, path, e, plans):
    """sum_i <e_i, B_hat_i> with every path frozen, block by block."""
    tot = 0.0
    for i, (y, x, p) in enumerate(BLOCKS):
        P = plans[p]
        b, br = P.block, P.border
        fL, aL = oracle.cut_area(frame, avail, y, x, b, br)
        w = oracle.weights(b, br, P.rho, aL)
        g, _ = oracle.replay_area(fL, w, P.fft_size, P.gamma, path[i, :P.iters])
        tot += float(np.sum(g[br:br + b, br:br + b] * e[i, :b, :b]))
    return tot


def _support_counts():
    """How many blocks' supports (w != 0) contain each frame sample."""
    frame, avail, _, _ = _case()
    cnt = np.zeros((H, W), dtype=int)
    for y, x, p in BLOCKS:
        P = PLANS[p]
        b, br = P.block, P.border
        _, aL = oracle.cut_area(frame, avail, y, x, b, br)
        w = oracle.weights(b, br, P.rho, aL)
        for m, n in np.argwhere(w != 0):
            cnt[y - br + m, x - br + n] += 1
    return cnt


def test_batch_adjoint_equals_per_block_adjoints_scattered_and_summed():
    frame, avail, path, e = _case()
    gf, grg = oracle.batch_adjoint(frame, avail, BLOCKS, PLANS, path, e, threads=3)
    ref_f = np.zeros((H, W))
    ref_rg = np.zeros((len(PLANS), 2))
    for i, (y, x, p) in enumerate(BLOCKS):
        P = PLANS[p]
        b, br = P.block, P.border
        fbar, rbar, gbar = oracle.block_gradients(frame, avail, y, x, P, path[i, :P.iters],
                                                  e[i, :b, :b])
        Ls = b + 2 * br
        for m in range(Ls):
            for n in range(Ls):
                fy, fx = y - br + m, x - br + n
                if 0 <= fy < H and 0 <= fx < W:
                    ref_f[fy, fx] += fbar[m, n]
                else:
                    assert fbar[m, n] == 0.0  # samples outside the frame are not in A
        ref_rg[p] += (rbar, gbar)
    scale = np.abs(ref_f).max()
    np.testing.assert_allclose(gf, ref_f, rtol=1e-12, atol=1e-13 * scale)
    np.testing.assert_allclose(grg, ref_rg, rtol=1e-12)
    # the case does exercise the composition: overlapping supports, several
    # blocks per plan, gradients outside every support are zero
    cnt = _support_counts()
    assert cnt.max() >= 2
    assert np.all(gf[cnt == 0] == 0.0)
    assert np.all(np.bincount(BLOCKS[:, 2]) >= 2)


def test_batch_frame_gradient_matches_central_differences():
    frame, avail, path, e = _case()
    gf, _ = oracle.batch_adjoint(frame, avail, BLOCKS, PLANS, path, e, threads=2)
    cnt = _support_counts()
    rng = np.random.default_rng(5)
    shared = [tuple(i) for i in np.argwhere(cnt >= 2)]
    single = [tuple(i) for i in np.argwhere(cnt == 1)]
    picks = [shared[j] for j in rng.choice(len(shared), min(8, len(shared)), replace=False)]
    picks += [single[j] for j in rng.choice(len(single), 6, replace=False)]
    for (yy, xx) in picks:
        h = 1.0  # integer frame: f +- 1 is exact in float32; the loss is linear in f
        fp, fm = frame.copy(), frame.copy()
        fp[yy, xx] += h
        fm[yy, xx] -= h
        fd = (_batch_loss(fp, avail, path, e, PLANS) - _batch_loss(fm, avail, path, e, PLANS)) / (2 * h)
        assert gf[yy, xx] == pytest.approx(fd, rel=1e-7, abs=1e-9), (yy, xx, cnt[yy, xx])


def _richardson(fun, x, h):
    d = lambda hh: (fun(x + hh) - fun(x - hh)) / (2 * hh)
    d1, d2, d3 = d(h), d(h / 2), d(h / 4)
    e1 = (4 * d2 - d1) / 3
    e2 = (4 * d3 - d2) / 3
    return (16 * e2 - e1) / 15


@pytest.mark.parametrize("p", [0, 1])
def test_batch_rho_gamma_gradients_match_richardson_per_plan(p):
    frame, avail, path, e = _case()
    _, grg = oracle.batch_adjoint(frame, avail, BLOCKS, PLANS, path, e, threads=2)
    import types

    def with_param(**kw):
        # plain namespaces: PlanSpec would round rho +- h to single precision,
        # which spoils the difference quotients
        plans = [types.SimpleNamespace(**vars(q)) for q in PLANS]
        for k, v in kw.items():
            setattr(plans[p], k, v)
        return plans

    fd_rho = _richardson(lambda r: _batch_loss(frame, avail, path, e, with_param(rho=r)),
                         PLANS[p].rho, 1e-3)
    fd_gam = _richardson(lambda g: _batch_loss(frame, avail, path, e, with_param(gamma=g)),
                         PLANS[p].gamma, 1e-3)
    assert grg[p, 0] == pytest.approx(fd_rho, rel=1e-6)
    assert grg[p, 1] == pytest.approx(fd_gam, rel=1e-6)


def test_batch_adjoint_is_independent_of_the_thread_count():
    frame, avail, path, e = _case()
    g1, r1 = oracle.batch_adjoint(frame, avail, BLOCKS, PLANS, path, e, threads=1)
    for t in (2, 5):
        g, r = oracle.batch_adjoint(frame, avail, BLOCKS, PLANS, path, e, threads=t)
        np.testing.assert_allclose(g, g1, rtol=1e-13, atol=1e-13 * np.abs(g1).max())
        np.testing.assert_allclose(r, r1, rtol=1e-13)
