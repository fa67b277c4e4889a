"""Pins of the oracle's FOFSE with the 2-D DCT-II basis (Sec. 2: the DCT, like
the DFT, admits the complete transform-domain formulation).

Basis phi_k[m,n] = cos(pi k1 (2m+1)/(2T)) cos(pi k2 (2n+1)/(2T)) on the T x T
grid with L at its origin; selection by the orthonormal DCT magnitude;
coefficient by Eq. 5 with the weighted norm sum w phi_u^2.  The pins use
scipy's DCT (a library routine), the orthogonal case, the product-to-sum
identities behind the transform-domain update, and an independent numpy
restatement of the transform-domain recursion."""
import numpy as np
import pytest
import scipy.fft

import oracle
from paper_2207_01205_gb300 import synth


def _cos(T, Ls, a_max=None):
    a = np.arange(a_max if a_max else T)[:, None]
    m = np.arange(Ls)[None, :]
    return np.cos(np.pi * a * (2 * m + 1) / (2 * T))


def _area(seed=3):
    wl = synth.single_block(seed=seed)
    fL, aL = oracle.cut_area(wl.frame, wl.avail, 16, 16, 16, 16)
    return fL, oracle.weights(16, 16, 0.8, aL)


def test_first_iteration_by_scipy_dct():
    """P = DCT-II of the zero-padded weighted area (scipy's unnormalised
    type-2 DCT is twice the cosine sum per axis); the pick maximises the
    orthonormal DCT's magnitude; c = gamma P[u] / sum w phi_u^2."""
    fL, w = _area()
    T, gamma = 64, 0.5
    res = oracle.extrapolate_area_dct(fL, w, T, gamma, 1)
    Z = np.zeros((T, T))
    Z[:48, :48] = w * fL
    P = scipy.fft.dctn(Z, type=2) / 4.0
    E = scipy.fft.dctn(Z, type=2, norm="ortho") ** 2
    u = np.unravel_index(np.argmax(E), E.shape)
    assert tuple(res.u[0]) == tuple(u)
    C = _cos(T, 48)
    phi = np.outer(C[u[0]], C[u[1]])
    c = gamma * P[u] / np.sum(w * phi * phi)
    assert abs(res.dc[0].real - c) <= 1e-12 * abs(c)
    assert np.max(np.abs(res.g - c * phi)) <= 1e-12 * abs(c)


@pytest.mark.parametrize("u,amp", [((3, 5), 40.0), ((0, 7), -25.0), ((0, 0), 100.0), ((15, 1), 12.0)])
def test_orthogonal_case_recovers_a_single_basis_function(u, amp):
    """w = 1 on the whole T x T grid: the DCT basis is orthogonal there, so
    f = amp phi_u is picked at once with c = gamma amp."""
    T = 16
    C = _cos(T, T)
    f = amp * np.outer(C[u[0]], C[u[1]])
    for gamma in (1.0, 0.4):
        res = oracle.extrapolate_area_dct(f, np.ones((T, T)), T, gamma, 1)
        assert tuple(res.u[0]) == u
        assert abs(res.dc[0].real - gamma * amp) <= 1e-12 * abs(amp)
        assert np.max(np.abs(res.g - gamma * f)) <= 1e-11 * abs(amp)


def test_product_to_sum_identities_of_the_update():
    """sum w phi_k phi_u = 1/4 sum over the four sign choices of
    C[|k1 +- u1|, |k2 +- u2|], C[a] = sum w cos(pi a1 (2m+1)/(2T)) cos(pi a2 (2n+1)/(2T))
    for 0 <= a < 2T - 1 (the table the transform-domain update gathers)."""
    rng = np.random.default_rng(5)
    T, Ls = 8, 6
    w = rng.uniform(0, 1, size=(Ls, Ls))
    Ce = _cos(T, Ls, 2 * T - 1)
    Ct = Ce @ w @ Ce.T
    C = _cos(T, Ls)
    for k in [(0, 0), (1, 2), (7, 7), (3, 0)]:
        for u in [(0, 0), (2, 5), (7, 1), (4, 4)]:
            direct = np.sum(w * np.outer(C[k[0]], C[k[1]]) * np.outer(C[u[0]], C[u[1]]))
            s = sum(Ct[abs(k[0] + s1 * u[0]), abs(k[1] + s2 * u[1])] for s1 in (1, -1) for s2 in (1, -1)) / 4
            assert abs(direct - s) <= 1e-12


def _spectral_dct(fL, wL, T, gamma, iters):
    """Independent transform-domain restatement: R = DCT-II of w f once, the
    table C of w once; each iteration R[k] -= c/4 sum C[|k +- u|] for the
    picked u, c = gamma R[u] / (1/4 sum C[|u +- u|])."""
    Ls = fL.shape[0]
    Ce = _cos(T, Ls, 2 * T - 1)
    C = Ce[:T]
    x = np.where(wL != 0, wL * fL, 0)
    R = C @ x @ C.T
    Ct = Ce @ wL @ Ce.T
    k = np.arange(T)
    scale = np.outer(np.where(k > 0, 2.0, 1.0), np.where(k > 0, 2.0, 1.0))
    path, cs = [], []
    for _ in range(iters):
        u1, u2 = np.unravel_index(np.argmax(R * R * scale), R.shape)
        nrm = sum(Ct[abs(u1 + s1 * u1), abs(u2 + s2 * u2)] for s1 in (1, -1) for s2 in (1, -1)) / 4
        c = gamma * R[u1, u2] / nrm
        i1p, i1m = np.abs(k + u1), np.abs(k - u1)
        i2p, i2m = np.abs(k + u2), np.abs(k - u2)
        upd = (Ct[np.ix_(i1p, i2p)] + Ct[np.ix_(i1p, i2m)] + Ct[np.ix_(i1m, i2p)] + Ct[np.ix_(i1m, i2m)]) / 4
        R = R - c * upd
        path.append((u1, u2))
        cs.append(c)
    return np.array(path), np.array(cs)


@pytest.mark.parametrize("seed", [0, 1])
def test_transform_domain_recursion_equals_spatial_reprojection(seed):
    fL, w = _area(seed + 7)
    T = 64
    res = oracle.extrapolate_area_dct(fL, w, T, 0.5, 60)
    path, cs = _spectral_dct(fL, w, T, 0.5, 60)
    assert np.array_equal(res.u, path)
    assert np.max(np.abs(res.dc.real - cs)) <= 1e-9 * np.max(np.abs(cs))


def test_batch_with_the_dct_basis_matches_single_area_calls():
    plan = synth.PlanSpec(8, 8, 32, 0.8, 0.5, 30, 0, 0, 1)
    wl = synth.small_frame(9, plan=plan, n_lost=5)
    out = oracle.run_batch(wl.frame, wl.avail, wl.blocks, [plan], with_path=True)
    for i, (y, x, _) in enumerate(wl.blocks):
        fL, aL = oracle.cut_area(wl.frame, wl.avail, y, x, 8, 8)
        w = oracle.weights(8, 8, plan.rho, aL)
        res = oracle.extrapolate_area_dct(fL, w, 32, plan.gamma, 30)
        assert out.status[i] == res.status
        assert np.array_equal(out.path[i], res.u)
        assert np.array_equal(out.blocks[i], res.g[8:16, 8:16])
        assert np.all(out.dc[i].imag == 0)


def _grad_case(seed=4, b=4, br=4, T=16, iters=12):
    rng = np.random.default_rng(seed)
    Ls = b + 2 * br
    f = rng.uniform(0, 255, size=(Ls, Ls))
    a = (rng.uniform(size=(Ls, Ls)) > 0.1).astype(np.uint8)
    rho, gamma = 0.8, 0.45
    w = oracle.weights(b, br, rho, a)
    path = oracle.extrapolate_area_dct(f, w, T, gamma, iters).u
    e = np.zeros((Ls, Ls))
    e[br:br + b, br:br + b] = rng.normal(size=(b, b))
    return f, a, w, path, e, rho, gamma, T, b, br


def test_dct_replay_reproduces_the_coefficients():
    f, a, w, path, e, rho, gamma, T, b, br = _grad_case()
    res = oracle.extrapolate_area_dct(f, w, T, gamma, len(path))
    g, dc = oracle.replay_area_dct(f, w, T, gamma, path)
    assert np.max(np.abs(dc - res.dc.real)) <= 1e-12 * np.max(np.abs(dc))
    assert np.max(np.abs(g - res.g)) <= 1e-10


def test_dct_adjoint_in_f_matches_finite_differences():
    """Along a frozen path B_hat is linear in f: central differences are exact
    up to rounding."""
    f, a, w, path, e, rho, gamma, T, b, br = _grad_case()
    fbar, wbar, gbar = oracle.adjoint_area(f, w, T, gamma, path, e, basis=1)
    rng = np.random.default_rng(1)
    for _ in range(6):
        m, n = rng.integers(0, f.shape[0], size=2)
        if w[m, n] == 0:
            continue
        h = 1e-3
        fp, fm = f.copy(), f.copy()
        fp[m, n] += h
        fm[m, n] -= h
        lp = np.sum(oracle.replay_area_dct(fp, w, T, gamma, path)[0] * e)
        lm = np.sum(oracle.replay_area_dct(fm, w, T, gamma, path)[0] * e)
        assert fbar[m, n] == pytest.approx((lp - lm) / (2 * h), rel=1e-6, abs=1e-9)


def test_dct_adjoint_in_rho_and_gamma_matches_richardson():
    f, a, w, path, e, rho, gamma, T, b, br = _grad_case()
    fbar, wbar, gbar = oracle.adjoint_area(f, w, T, gamma, path, e, basis=1)
    dist = oracle.distance(b, br)
    rbar = oracle.rho_chain(w, dist, rho, wbar)

    def loss(r, g_):
        return np.sum(oracle.replay_area_dct(f, oracle.weights(b, br, r, a), T, g_, path)[0] * e)

    def rich(fun, x, h):
        d1 = (fun(x + h) - fun(x - h)) / (2 * h)
        d2 = (fun(x + h / 2) - fun(x - h / 2)) / h
        return (4 * d2 - d1) / 3
    assert rbar == pytest.approx(rich(lambda r: loss(r, gamma), rho, 1e-4), rel=1e-6, abs=1e-8)
    assert gbar == pytest.approx(rich(lambda g_: loss(rho, g_), gamma, 1e-4), rel=1e-6, abs=1e-8)
