"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test names the passage it checks.  None of them re-types the oracle's own
formula: they use closed forms, invariants, library routines (numpy's FFT),
brute force on tiny inputs, an independent transform-domain restatement, and
finite differences.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2207_01205_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore")


def _canonical_mask(T):
    k1, k2 = np.meshgrid(np.arange(T), np.arange(T), indexing="ij")
    return (k1 * T + k2) <= (((T - k1) % T) * T + (T - k2) % T)


def _random_area(rng, Ls, b, br, lost_frac=0.0):
    f = rng.uniform(0, 255, size=(Ls, Ls))
    a = np.ones((Ls, Ls), dtype=np.uint8)
    if lost_frac:
        a[rng.uniform(size=(Ls, Ls)) < lost_frac] = 0
    return f, a


# --------------------------------------------------------------------------
# Transform operator (Eq. 8) and projection (Eq. 5)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("Ls,T", [(12, 16), (24, 32), (6, 8), (16, 16)])
def test_projection_is_numpy_fft2_of_zero_padded_area(Ls, T):
    """Eq. 8 with the 2-D DFT basis is the forward DFT of r_w embedded at the
    grid origin: a library routine (numpy.fft.fft2, axis 0 = m)."""
    rng = np.random.default_rng(Ls * 100 + T)
    rw = rng.normal(size=(Ls, Ls)) * 50
    Z = np.zeros((T, T))
    Z[:Ls, :Ls] = rw
    P = oracle.project(rw, T)
    ref = np.fft.fft2(Z)
    assert np.max(np.abs(P - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_projection_matches_bruteforce_inner_products():
    """Eq. 5 numerator: the weighted scalar product of the residual with every
    basis function, brute force O(T^4) with the conjugated basis."""
    rng = np.random.default_rng(7)
    Ls, T = 6, 8
    rw = rng.normal(size=(Ls, Ls))
    m, n = np.meshgrid(np.arange(Ls), np.arange(Ls), indexing="ij")
    ref = np.zeros((T, T), dtype=complex)
    for k1 in range(T):
        for k2 in range(T):
            phi = np.exp(2j * np.pi * (k1 * m + k2 * n) / T)
            ref[k1, k2] = np.sum(rw * np.conj(phi))
    assert np.max(np.abs(oracle.project(rw, T) - ref)) < 1e-12


def test_parseval_on_projection():
    """Parseval: sum_k |P[k]|^2 = T^2 sum r_w^2 for any weighted residual."""
    rng = np.random.default_rng(3)
    rw = rng.normal(size=(20, 20))
    P = oracle.project(rw, 32)
    assert abs(np.sum(np.abs(P) ** 2) - 32 * 32 * np.sum(rw ** 2)) < 1e-9 * np.sum(np.abs(P) ** 2)


# --------------------------------------------------------------------------
# Selection (Eq. 9) over one index per conjugate pair
# --------------------------------------------------------------------------

def test_select_returns_canonical_member_of_a_hermitian_pair():
    T = 8
    rng = np.random.default_rng(1)
    P = np.fft.fft2(rng.normal(size=(T, T)) * 0.01)
    # plant a dominant pair at (5, 6) and its mirror (3, 2); the canonical member is (3, 2)
    P[5, 6] = 100 + 30j
    P[3, 2] = 100 - 30j
    u1, u2, gap = oracle.select(P)
    assert (u1, u2) == (3, 2)
    assert 0 < gap <= 1


def test_select_exact_tie_goes_to_smallest_row_major_index():
    T = 8
    P = np.zeros((T, T), dtype=complex)
    P[2, 5] = P[6, 3] = 3 + 4j          # pair (2,5)/(6,3): canonical (2,5)
    P[1, 7] = P[7, 1] = 5j              # pair (1,7)/(7,1): canonical (1,7), same |P|
    u1, u2, gap = oracle.select(P)
    assert (u1, u2) == (1, 7)
    assert gap == 0.0


def test_select_ignores_non_canonical_duplicates():
    """A value planted only at a non-canonical index is never selected."""
    T = 8
    P = np.full((T, T), 1.0 + 0j)
    P[7, 7] = 50.0                       # mirror of (1, 1), not in H
    H = _canonical_mask(T)
    assert not H[7, 7]
    u1, u2, _ = oracle.select(P)
    assert (u1, u2) == (0, 0)


# --------------------------------------------------------------------------
# Weighting function (Eq. 4) with the isotropic model (Eq. 15)
# --------------------------------------------------------------------------

def test_weights_mask_B_and_decay_isotropically():
    b, br = 4, 5
    Ls = b + 2 * br
    a = np.ones((Ls, Ls), dtype=np.uint8)
    w = oracle.weights(b, br, 0.8, a)
    assert np.all(w[br:br + b, br:br + b] == 0)
    A = np.ones((Ls, Ls), bool)
    A[br:br + b, br:br + b] = False
    # the 8 symmetries of the square about the B centre (B is central in L)
    for t in (w.T, w[::-1], w[:, ::-1], w[::-1, ::-1]):
        assert np.allclose(t, w, rtol=0, atol=1e-15)
    # strictly decreasing along a row moving away from B
    row = w[br + 1, :br]
    assert np.all(np.diff(row) > 0)
    # rho_hat = 1 gives the plain mask
    assert np.array_equal(oracle.weights(b, br, 1.0, a), A.astype(float))
    # corner value: distance sqrt(2) * (br + (b - 1) / 2) from the centre (Eq. 15)
    assert w[0, 0] == pytest.approx(0.8 ** (math.sqrt(2) * (br + 1.5)), rel=1e-14)


def test_weights_respect_availability_and_causal_shape():
    b, br = 8, 8
    Ls = 24
    a = np.ones((Ls, Ls), dtype=np.uint8)
    w = oracle.weights(b, br, 0.8, a, support=1)
    nz = w != 0
    assert nz.sum() == 192                        # top-left, top and left 8x8 neighbours
    assert nz[:8, :16].all() and nz[8:16, :8].all()
    assert not nz[:8, 16:].any() and not nz[8:, 8:].any() and not nz[16:].any()
    a[0, 0] = 0
    assert oracle.weights(b, br, 0.8, a, support=1)[0, 0] == 0


# --------------------------------------------------------------------------
# The iteration (Eq. 1-3, 5, 9, 14)
# --------------------------------------------------------------------------

def test_first_iteration_equals_library_fft():
    """Iteration 1: P = fft2(w f) (g = 0); u = argmax over one member per
    pair; c = gamma P[u] / sum w."""
    wl = synth.single_block()
    fL, aL = oracle.cut_area(wl.frame, wl.avail, 16, 16, 16, 16)
    w = oracle.weights(16, 16, 0.8, aL)
    res = oracle.extrapolate_area(fL, w, 64, 0.5, 3)
    Z = np.zeros((64, 64))
    Z[:48, :48] = w * fL
    F = np.fft.fft2(Z)
    mag = np.where(_canonical_mask(64), np.abs(F) ** 2, -1)
    u = np.unravel_index(np.argmax(mag), mag.shape)
    assert tuple(res.u[0]) == tuple(u)
    assert abs(res.dc[0] - 0.5 * F[u] / w.sum()) < 1e-12 * abs(res.dc[0])
    assert res.w0 == pytest.approx(w.sum(), rel=1e-15)


@pytest.mark.parametrize("gamma", [0.2, 0.5, 1.0])
def test_constant_signal_closed_form(gamma):
    """f = c on A: the residual spectrum is (c - g) W, its largest entry is the
    DC one (|W[k]| < W[0] for k != 0), so g = c (1 - (1 - gamma)^nu) exactly."""
    rng = np.random.default_rng(11)
    b, br, T = 8, 8, 32
    Ls = b + 2 * br
    a = (rng.uniform(size=(Ls, Ls)) > 0.2).astype(np.uint8)
    w = oracle.weights(b, br, 0.8, a)
    c = 137.0
    for nu in (1, 3, 10):
        res = oracle.extrapolate_area(np.full((Ls, Ls), c), w, T, gamma, nu)
        assert np.all(res.u == 0)
        assert np.allclose(res.g, c * (1 - (1 - gamma) ** nu), rtol=0, atol=1e-10)


@pytest.mark.parametrize("u,coef", [((3, 5), 7.0 - 2.0j), ((0, 1), 3.0 + 4.0j), ((8, 8), -5.0),
                                    ((0, 8), 2.5)])
@pytest.mark.parametrize("gamma", [1.0, 0.3])
def test_single_basis_pair_recovered_in_orthogonal_case(u, coef, gamma):
    """With w = 1 on the whole T x T grid the basis is orthogonal (K is
    diagonal, Eq. 12) and a single pair f = 2 Re(c phi_u) (or c phi_u for a
    self-conjugate u) is picked every iteration with c_u = gamma * p_u, so
    after nu iterations g = (1 - (1 - gamma)^nu) f."""
    T = 16
    m, n = np.meshgrid(np.arange(T), np.arange(T), indexing="ij")
    phi = np.exp(2j * np.pi * (u[0] * m + u[1] * n) / T)
    selfconj = (2 * u[0]) % T == 0 and (2 * u[1]) % T == 0
    f = np.real(coef * phi) if selfconj else 2 * np.real(coef * phi)
    nu = 1 if gamma == 1.0 else 4
    res = oracle.extrapolate_area(f, np.ones((T, T)), T, gamma, nu)
    assert np.allclose(res.g, (1 - (1 - gamma) ** nu) * f, rtol=0, atol=1e-11)
    canon = u if _canonical_mask(T)[u] else ((T - u[0]) % T, (T - u[1]) % T)
    assert tuple(res.u[0]) == canon
    c0 = coef if canon == u else np.conj(coef)
    assert abs(res.dc[0] - gamma * c0) < 1e-12


def _spectral_fofse(fL, wL, T, gamma, iters):
    """Independent restatement of the transform-domain recursion (Sec. 2,
    'complete formulation in the transform domain'): R_w and W are
    transformed once; each iteration subtracts the spectrum of the added
    pair, c W[k - u] + conj(c) W[k + u]."""
    Ls = fL.shape[0]
    x = np.zeros((T, T))
    w = np.zeros((T, T))
    x[:Ls, :Ls] = np.where(wL != 0, wL * fL, 0)
    w[:Ls, :Ls] = wL
    R, W = np.fft.fft2(x), np.fft.fft2(w)
    W0 = W[0, 0].real
    H = _canonical_mask(T)
    path, dcs = [], []
    for _ in range(iters):
        mag = np.where(H, np.abs(R) ** 2, -1)
        u1, u2 = np.unravel_index(np.argmax(mag), mag.shape)
        sc = (2 * u1) % T == 0 and (2 * u2) % T == 0
        c = gamma * R[u1, u2] / W0
        if sc:
            c = c.real
        R = R - c * np.roll(W, (u1, u2), axis=(0, 1))
        if not sc:
            R = R - np.conj(c) * np.roll(W, (-u1, -u2), axis=(0, 1))
        path.append((u1, u2))
        dcs.append(c)
    return np.array(path), np.array(dcs)


@pytest.mark.parametrize("seed", [0, 1])
def test_transform_domain_recursion_equals_spatial_reprojection(seed):
    wl = synth.single_block(seed=seed + 5)
    fL, aL = oracle.cut_area(wl.frame, wl.avail, 16, 16, 16, 16)
    w = oracle.weights(16, 16, 0.8, aL)
    res = oracle.extrapolate_area(fL, w, 64, 0.5, 60)
    path, dcs = _spectral_fofse(fL, w, 64, 0.5, 60)
    assert np.array_equal(path, res.u)
    assert np.max(np.abs(dcs - res.dc)) < 1e-12 * np.max(np.abs(res.dc))


@pytest.mark.parametrize("seed", [0, 1])
def test_c_transform_domain_form_matches_numpy_restatement_and_spatial_oracle(seed):
    """The C transform-domain form (the CPU program timed beside the GPU) agrees
    with the numpy restatement above and with the spatial re-projection:
    identical paths, coefficients to 1e-12, samples to 1e-9."""
    wl = synth.single_block(seed=seed + 9)
    fL, aL = oracle.cut_area(wl.frame, wl.avail, 16, 16, 16, 16)
    w = oracle.weights(16, 16, 0.8, aL)
    sp = oracle.extrapolate_area(fL, w, 64, 0.5, 60)
    fd = oracle.extrapolate_area(fL, w, 64, 0.5, 60, transform_domain=True)
    path, dcs = _spectral_fofse(fL, w, 64, 0.5, 60)
    assert fd.status == 0 and np.array_equal(fd.u, sp.u) and np.array_equal(fd.u, path)
    scale = np.max(np.abs(sp.dc))
    assert np.max(np.abs(fd.dc - sp.dc)) < 1e-12 * scale
    assert np.max(np.abs(fd.dc - dcs)) < 1e-12 * scale
    assert np.max(np.abs(fd.g - sp.g)) < 1e-9


def test_c_transform_domain_batch_matches_oracle_batch():
    wl = synth.small_frame(17, plan=synth.PlanSpec(8, 8, 32, 0.7, 0.4, 40), n_lost=5)
    a = oracle.run_batch(wl.frame, wl.avail, wl.blocks, wl.plans, threads=2)
    b = oracle.run_batch(wl.frame, wl.avail, wl.blocks, wl.plans, threads=2, transform_domain=True)
    assert np.array_equal(a.status, b.status) and np.array_equal(a.path, b.path)
    assert np.max(np.abs(a.blocks - b.blocks)) < 1e-9


def test_cyclic_translation_of_L_inside_the_grid():
    """|DFT| is invariant under a cyclic shift, and the model update uses the
    same basis, so moving L inside the T x T grid leaves the path and the
    extrapolated samples unchanged (coefficients pick up the shift's phase)."""
    rng = np.random.default_rng(5)
    b, br, T, s = 4, 4, 32, (3, 5)
    Ls = b + 2 * br
    f, a = _random_area(rng, Ls, b, br, lost_frac=0.1)
    w = oracle.weights(b, br, 0.8, a)
    ref = oracle.extrapolate_area(f, w, T, 0.4, 25)
    big = Ls + max(s)
    f2 = np.zeros((big, big))
    w2 = np.zeros((big, big))
    f2[s[0]:s[0] + Ls, s[1]:s[1] + Ls] = f
    w2[s[0]:s[0] + Ls, s[1]:s[1] + Ls] = w
    got = oracle.extrapolate_area(f2, w2, T, 0.4, 25)
    assert np.array_equal(got.u, ref.u)
    assert np.allclose(got.g[s[0]:s[0] + Ls, s[1]:s[1] + Ls], ref.g, rtol=0, atol=1e-9)
    ph = np.exp(-2j * np.pi * (ref.u[:, 0] * s[0] + ref.u[:, 1] * s[1]) / T)
    assert np.allclose(got.dc, ref.dc * ph, rtol=0, atol=1e-10)


def test_model_is_real_and_dc_real_for_self_conjugate_picks():
    wl = synth.single_block()
    fL, aL = oracle.cut_area(wl.frame, wl.avail, 16, 16, 16, 16)
    w = oracle.weights(16, 16, 0.8, aL)
    res = oracle.extrapolate_area(fL, w, 64, 0.5, 40)
    sc = ((2 * res.u) % 64 == 0).all(axis=1)
    assert sc.any()
    assert np.all(res.dc[sc].imag == 0)
    assert np.all(np.isfinite(res.g))
    assert np.all(res.gap >= 0) and np.all(res.gap <= 1)


def test_replay_along_own_path_reproduces_coefficients():
    wl = synth.single_block()
    fL, aL = oracle.cut_area(wl.frame, wl.avail, 16, 16, 16, 16)
    w = oracle.weights(16, 16, 0.8, aL)
    res = oracle.extrapolate_area(fL, w, 64, 0.5, 30)
    g, dc = oracle.replay_area(fL, w, 64, 0.5, res.u)
    # the replay projects onto one basis function directly (not separably): equal up to rounding
    assert np.max(np.abs(g - res.g)) < 1e-10
    assert np.max(np.abs(dc - res.dc)) < 1e-12 * np.max(np.abs(res.dc))


def test_frozen_path_output_is_linear_in_f():
    rng = np.random.default_rng(9)
    b, br, T = 4, 4, 16
    Ls = 12
    f1, a = _random_area(rng, Ls, b, br)
    f2 = rng.normal(size=(Ls, Ls)) * 30
    w = oracle.weights(b, br, 0.7, a)
    path = oracle.extrapolate_area(f1, w, T, 0.5, 15).u
    g1, _ = oracle.replay_area(f1, w, T, 0.5, path)
    g2, _ = oracle.replay_area(f2, w, T, 0.5, path)
    g12, _ = oracle.replay_area(2.0 * f1 - 3.0 * f2, w, T, 0.5, path)
    assert np.allclose(g12, 2.0 * g1 - 3.0 * g2, rtol=0, atol=1e-9)


# --------------------------------------------------------------------------
# Status cases
# --------------------------------------------------------------------------

def test_no_support_and_nonfinite_status():
    b, br, T = 4, 4, 16
    Ls = 12
    f = np.full((Ls, Ls), 10.0)
    res = oracle.extrapolate_area(f, np.zeros((Ls, Ls)), T, 0.5, 5)
    assert res.status == oracle.STATUS_NO_SUPPORT and np.all(res.g == 0)
    w = oracle.weights(b, br, 0.8, np.ones((Ls, Ls), np.uint8))
    f_nan = f.copy()
    f_nan[0, 0] = np.nan
    assert oracle.extrapolate_area(f_nan, w, T, 0.5, 5).status == oracle.STATUS_NONFINITE
    # a non-finite value inside B (w = 0) is never read
    f_b = f.copy()
    f_b[5, 5] = np.inf
    res_b = oracle.extrapolate_area(f_b, w, T, 0.5, 5)
    assert res_b.status == oracle.STATUS_OK
    assert np.array_equal(res_b.g, oracle.extrapolate_area(f, w, T, 0.5, 5).g)


def test_batch_matches_single_area_calls_and_ignores_lost_content():
    wl = synth.small_frame(3, plan=synth.PlanSpec(8, 8, 32, 0.8, 0.5, 20), n_lost=5)
    res = oracle.run_batch(wl.frame, wl.avail, wl.blocks, wl.plans, threads=3)
    poisoned = wl.frame.copy()
    poisoned[wl.avail == 0] = np.nan
    res2 = oracle.run_batch(poisoned, wl.avail, wl.blocks, wl.plans, threads=2)
    assert np.array_equal(res.blocks, res2.blocks)
    for i, (y, x, _) in enumerate(wl.blocks):
        fL, aL = oracle.cut_area(wl.frame, wl.avail, y, x, 8, 8)
        P = wl.plans[0]  # rho and gamma as the plan holds them (single precision)
        w = oracle.weights(8, 8, P.rho, aL)
        one = oracle.extrapolate_area(fL, w, 32, P.gamma, 20)
        assert res.status[i] == one.status
        assert np.array_equal(res.blocks[i], one.g[8:16, 8:16])
        assert np.array_equal(res.path[i], one.u)
    # the top-left corner block still has support to its right and below
    assert res.status[0] == oracle.STATUS_OK


# --------------------------------------------------------------------------
# Frozen-path derivatives
# --------------------------------------------------------------------------

def _setup_grad_case(seed=2, b=4, br=4, T=16, iters=12, support=0):
    rng = np.random.default_rng(seed)
    Ls = b + 2 * br
    f, a = _random_area(rng, Ls, b, br, lost_frac=0.1)
    rho, gamma = 0.8, 0.45
    w = oracle.weights(b, br, rho, a, support)
    path = oracle.extrapolate_area(f, w, T, gamma, iters).u
    e = np.zeros((Ls, Ls))
    e[br:br + b, br:br + b] = rng.normal(size=(b, b))
    return f, a, w, path, e, rho, gamma, T


def _loss(f, a, rho, gamma, path, e, T, b=4, br=4, support=0):
    w = oracle.weights(b, br, rho, a, support)
    g, _ = oracle.replay_area(f, w, T, gamma, path)
    return float(np.sum(g * e))


def test_adjoint_in_f_matches_finite_differences():
    """The frozen-path output is linear in f, so a central difference is exact
    up to rounding."""
    f, a, w, path, e, rho, gamma, T = _setup_grad_case()
    fbar, wbar, _ = oracle.adjoint_area(f, w, T, gamma, path, e)
    rng = np.random.default_rng(0)
    idx = [tuple(i) for i in np.argwhere(w != 0)[rng.choice(int((w != 0).sum()), 12, replace=False)]]
    for i in idx:
        h = 1e-3
        fp, fm = f.copy(), f.copy()
        fp[i] += h
        fm[i] -= h
        fd = (_loss(fp, a, rho, gamma, path, e, T) - _loss(fm, a, rho, gamma, path, e, T)) / (2 * h)
        assert fbar[i] == pytest.approx(fd, rel=1e-7, abs=1e-9)
    assert np.all(fbar[w == 0] == 0)


def _richardson(fun, x, h):
    d = lambda hh: (fun(x + hh) - fun(x - hh)) / (2 * hh)
    d1, d2, d3 = d(h), d(h / 2), d(h / 4)
    e1 = (4 * d2 - d1) / 3
    e2 = (4 * d3 - d2) / 3
    return (16 * e2 - e1) / 15


@pytest.mark.parametrize("support", [0, 1])
def test_adjoint_and_tangent_in_rho_gamma_match_richardson(support):
    b, br, T = (4, 4, 16) if support == 0 else (8, 8, 32)
    f, a, w, path, e, rho, gamma, T = _setup_grad_case(seed=4, b=b, br=br, T=T, support=support)
    fbar, wbar, gbar = oracle.adjoint_area(f, w, T, gamma, path, e)
    dist = oracle.distance(b, br)
    rbar = oracle.rho_chain(w, dist, rho, wbar)
    fd_rho = _richardson(lambda r: _loss(f, a, r, gamma, path, e, T, b, br, support), rho, 1e-3)
    fd_gam = _richardson(lambda g: _loss(f, a, rho, g, path, e, T, b, br, support), gamma, 1e-3)
    assert rbar == pytest.approx(fd_rho, rel=1e-6)
    assert gbar == pytest.approx(fd_gam, rel=1e-6)
    # forward-mode tangents as a third opinion
    wdot = np.where(w != 0, dist * rho ** (dist - 1), 0.0)
    g_rho = oracle.tangent_area(f, w, wdot, T, gamma, 0.0, path)
    g_gam = oracle.tangent_area(f, w, np.zeros_like(w), T, gamma, 1.0, path)
    assert np.sum(g_rho * e) == pytest.approx(rbar, rel=1e-10)
    assert np.sum(g_gam * e) == pytest.approx(gbar, rel=1e-10)
