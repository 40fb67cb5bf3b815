"""Pins of the FP64 oracle against what the paper and mathematics fix (no GPU).

Each test compares the oracle with something other than its own code: a closed form, a library
routine that the method reduces to in a special case, the dense normal equations of Eq. 7, or an
invariant the paper states.  A plausible slip (a dropped term, a wrong sign or index, a
transposed operand, sigma^2 for 2 sigma^2, a missing wrap) fails at least one of them.
"""
import math

import numpy as np
import pytest
import scipy.ndimage as ndi

import oracle


def _rng(seed):
    return np.random.default_rng(seed)


# ------------------------------------------------------------------------------------------
# Gradients (Section II-B: forward differences D_x, D_y; periodic reading)
# ------------------------------------------------------------------------------------------
def test_gradients_of_a_ramp_closed_form():
    H, W, a, b = 5, 7, 0.3, -1.1
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    f = a * xx + b * yy
    gx, gy = oracle.gradients(f)
    want_gx = np.full((H, W), a)
    want_gx[:, W - 1] = -a * (W - 1)          # wrap from x = W-1 back to x = 0
    want_gy = np.full((H, W), b)
    want_gy[H - 1, :] = -b * (H - 1)
    np.testing.assert_allclose(gx, want_gx, atol=1e-14)
    np.testing.assert_allclose(gy, want_gy, atol=1e-14)


# ------------------------------------------------------------------------------------------
# Bilateral filter (Section II-A, Eq. 1)
# ------------------------------------------------------------------------------------------
def test_blf_radius_zero_is_identity():
    g = _rng(0).normal(size=(6, 9))
    np.testing.assert_array_equal(oracle.blf(g, 0, 2.0, 0.1), g)


def test_blf_constant_field_is_invariant():
    g = np.full((7, 5), -0.37)
    v = oracle.blf(g, 2, 1.5, 0.05)
    np.testing.assert_allclose(v, g, rtol=0, atol=1e-15)


def _spike_closed_form(H, W, r, ss, sr, a, py, px):
    """BLF of a field that is `a` at (py, px) and 0 elsewhere, written out by hand.

    For s != p: Z_s = sum_o G(o) - G(p-s)(1 - R), v_s = a G(p-s) R / Z_s;
    for s == p: Z_p = 1 + R sum_{o != 0} G(o), v_p = a / Z_p,
    with G(o) = exp(-|o|^2 / (2 ss^2)), R = exp(-a^2 / (2 sr^2)) and p-s the wrapped offset
    when it lies in the window (otherwise v_s = 0)."""
    offs = [(dy, dx) for dy in range(-r, r + 1) for dx in range(-r, r + 1)]
    G = {o: math.exp(-(o[0] ** 2 + o[1] ** 2) / (2 * ss * ss)) for o in offs}
    sumG = sum(G.values())
    R = math.exp(-a * a / (2 * sr * sr))
    v = np.zeros((H, W))
    for y in range(H):
        for x in range(W):
            if (y, x) == (py, px):
                v[y, x] = a / (1.0 + R * (sumG - 1.0))
                continue
            hits = [o for o in offs if ((y + o[0]) % H, (x + o[1]) % W) == (py, px)]
            if not hits:
                continue
            assert len(hits) == 1
            gp = G[hits[0]]
            v[y, x] = a * gp * R / (sumG - gp * (1.0 - R))
    return v


@pytest.mark.parametrize("H,W,r,ss,sr,a,p", [
    (3, 3, 1, 0.9, 0.3, 0.8, (1, 1)),      # the window covers the whole 3x3 torus
    (5, 7, 2, 1.3, 0.4, 0.7, (2, 3)),
    (5, 7, 2, 1.3, 0.4, -0.5, (0, 6)),     # spike at a corner: every tap wraps
    (9, 6, 1, 2.0, 0.25, 1.0, (8, 0)),
])
def test_blf_spike_closed_form(H, W, r, ss, sr, a, p):
    g = np.zeros((H, W))
    g[p] = a
    want = _spike_closed_form(H, W, r, ss, sr, a, *p)
    np.testing.assert_allclose(oracle.blf(g, r, ss, sr), want, rtol=0, atol=1e-15)


@pytest.mark.parametrize("H,W,r,ss", [(16, 11, 3, 1.7), (9, 23, 4, 2.5), (12, 12, 1, 0.6)])
def test_blf_infinite_range_sigma_is_periodic_gaussian_correlation(H, W, r, ss):
    """sigma_r = inf removes the range kernel: Eq. 1 becomes correlation with the normalised,
    truncated spatial Gaussian -- scipy.ndimage.correlate with wrap-around boundaries."""
    g = _rng(1).normal(size=(H, W))
    d = np.arange(-r, r + 1, dtype=np.float64)
    K = np.exp(-(d[:, None] ** 2 + d[None, :] ** 2) / (2 * ss * ss))
    K /= K.sum()
    want = ndi.correlate(g, K, mode="wrap")
    np.testing.assert_allclose(oracle.blf(g, r, ss, math.inf), want, rtol=0, atol=1e-13)
    # a huge but finite sigma_r gives the same result up to exp(-d^2/2e12) - 1
    np.testing.assert_allclose(oracle.blf(g, r, ss, 1e6), want, rtol=0, atol=1e-10)


def test_blf_both_sigmas_infinite_is_box_mean():
    g = _rng(2).normal(size=(10, 13))
    want = ndi.uniform_filter(g, size=5, mode="wrap")
    np.testing.assert_allclose(oracle.blf(g, 2, math.inf, math.inf), want, atol=1e-13)


def test_blf_two_level_field_keeps_its_edge():
    """A jump of 1 with sigma_r = 0.05: taps across the edge weigh exp(-200), so both sides stay
    at their own level; without a range kernel the edge would blur by O(1)."""
    H, W = 8, 16
    g = np.zeros((H, W))
    g[:, W // 2:] = 1.0
    v = oracle.blf(g, 3, 2.0, 0.05)
    assert np.max(np.abs(v - g)) < 1e-80
    v_blur = oracle.blf(g, 3, 2.0, math.inf)
    assert np.max(np.abs(v_blur - g)) > 0.1


def test_blf_at_samples_the_full_field():
    g = _rng(3).normal(size=(17, 29))
    full = oracle.blf(g, 3, 1.5, 0.3)
    ys = np.array([0, 5, 16, 16, 3])
    xs = np.array([0, 28, 0, 28, 14])
    np.testing.assert_array_equal(oracle.blf_at(g, 3, 1.5, 0.3, ys, xs), full[ys, xs])


# ------------------------------------------------------------------------------------------
# Solve of Eq. 8 (and its special cases)
# ------------------------------------------------------------------------------------------
def _diff_matrices(H, W):
    """Dense periodic forward-difference matrices on the row-major pixel vector
    (Section II-B: (D_x f)[y,x] = f[y,x+1] - f[y,x], (D_y f)[y,x] = f[y+1,x] - f[y,x])."""
    n = H * W
    Dx = np.zeros((n, n))
    Dy = np.zeros((n, n))
    for y in range(H):
        for x in range(W):
            p = y * W + x
            Dx[p, y * W + (x + 1) % W] += 1.0
            Dx[p, p] -= 1.0
            Dy[p, ((y + 1) % H) * W + x] += 1.0
            Dy[p, p] -= 1.0
    return Dx, Dy


@pytest.mark.parametrize("H,W", [(8, 8), (8, 5), (7, 8), (1, 6), (5, 1)])
@pytest.mark.parametrize("lam", [0.1, 20.0, 1024.0])
def test_P6_fft_solve_matches_dense_normal_equations(H, W, lam):
    """Eq. 7 is strictly convex; its stationarity condition is
    (I + lam (Dx^T Dx + Dy^T Dy)) u = f + lam (Dx^T v_x + Dy^T v_y)  (Eq. 4 with W = I).
    Solved densely by LAPACK, it must agree with the Fourier solve of Eq. 8."""
    rng = _rng(int(lam * 10) + H * 31 + W)
    f = rng.uniform(size=(H, W))
    vx = rng.normal(scale=0.3, size=(H, W))
    vy = rng.normal(scale=0.3, size=(H, W))
    Dx, Dy = _diff_matrices(H, W)
    A = np.eye(H * W) + lam * (Dx.T @ Dx + Dy.T @ Dy)
    rhs = f.ravel() + lam * (Dx.T @ vx.ravel() + Dy.T @ vy.ravel())
    u_dense = np.linalg.solve(A, rhs).reshape(H, W)
    u = oracle.solve_eq8(f, vx, vy, lam)
    np.testing.assert_allclose(u, u_dense, rtol=0, atol=1e-12 * (1.0 + lam))


def test_P1_lambda_zero_returns_input():
    f = _rng(5).uniform(size=(3, 12, 10))
    u = oracle.blfls(f, 0.0, 2.0, 0.1, 2)
    np.testing.assert_allclose(u, f, rtol=0, atol=1e-14)


def test_P2_identity_filter_returns_input():
    """v = g (the filter replaced by the identity) makes Eq. 8's numerator the denominator times
    F(f), so u = f; radius 0 is the same case reached through the filter."""
    f = _rng(6).uniform(size=(11, 14))
    gx, gy = oracle.gradients(f)
    np.testing.assert_allclose(oracle.solve_eq8(f, gx, gy, 50.0), f, atol=1e-13)
    np.testing.assert_allclose(oracle.blfls(f, 50.0, 3.0, 0.1, 0), f, atol=1e-13)


def test_P3_constant_image_is_invariant():
    f = np.full((2, 9, 13), 0.625)
    np.testing.assert_allclose(oracle.blfls(f, 30.0, 2.0, 0.08, 3), f, atol=1e-14)


def test_P4_mean_is_preserved():
    f = _rng(7).uniform(size=(16, 20))
    u = oracle.blfls(f, 30.0, 2.5, 0.1, 3)
    assert abs(u.sum() - f.sum()) < 1e-11


@pytest.mark.parametrize("H,W,r,ss,lam", [(48, 64, 3, 1.5, 20.0), (64, 48, 5, 3.0, 1024.0)])
def test_P5_infinite_range_sigma_closed_form(H, W, r, ss, lam):
    """sigma_r = inf: BLF(D f) = K * (D f) = D (K * f) on the torus, so
    u = F^-1[F f (1 + lam K^ sum|F d|^2) / (1 + lam sum|F d|^2)],  |F d_x|^2 = 4 sin^2(pi kx/W)."""
    f = _rng(8).uniform(size=(H, W))
    d = np.arange(-r, r + 1)
    K = np.exp(-(d[:, None] ** 2 + d[None, :] ** 2) / (2.0 * ss * ss))
    K /= K.sum()
    kimg = np.zeros((H, W))
    for i, dy in enumerate(d):
        for j, dx in enumerate(d):
            kimg[dy % H, dx % W] += K[i, j]
    Khat = np.fft.fft2(kimg).real
    sx = 4.0 * np.sin(np.pi * np.arange(W) / W) ** 2
    sy = 4.0 * np.sin(np.pi * np.arange(H) / H) ** 2
    L = sy[:, None] + sx[None, :]
    want = np.fft.ifft2(np.fft.fft2(f) * (1.0 + lam * Khat * L) / (1.0 + lam * L)).real
    np.testing.assert_allclose(oracle.blfls(f, lam, ss, math.inf, r), want, atol=1e-12)
    np.testing.assert_allclose(oracle.blfls(f, lam, ss, 1e6, r), want, atol=1e-9)


def test_P7_lambda_monotonicity():
    """Section III-C / Fig. 5: as lam grows, |grad u - v|^2 does not increase and |u - f|^2
    does not decrease (the path of a quadratic penalty)."""
    rng = _rng(9)
    f = rng.uniform(size=(24, 20))
    # guidance = gradients of another image plus a little noise, so large lam can track it
    vx, vy = oracle.gradients(rng.uniform(size=f.shape))
    vx = vx + rng.normal(scale=0.01, size=f.shape)
    vy = vy + rng.normal(scale=0.01, size=f.shape)
    eg, ed = [], []
    for lam in [1.0, 4.0, 32.0, 256.0, 1024.0]:
        u = oracle.solve_eq8(f, vx, vy, lam)
        ux, uy = oracle.gradients(u)
        eg.append(np.sum((ux - vx) ** 2 + (uy - vy) ** 2))
        ed.append(np.sum((u - f) ** 2))
    assert all(b <= a * (1 + 1e-12) for a, b in zip(eg, eg[1:]))
    assert all(b >= a * (1 - 1e-12) for a, b in zip(ed, ed[1:]))
    assert eg[-1] < 0.5 * eg[0]


@pytest.mark.parametrize("lam", [1.0, 20.0, 50.0, 1024.0])
def test_P10_guidance_error_gain_bound(lam):
    """Per frequency the map dv -> du has gain lam sqrt(a) / (1 + lam a) <= sqrt(lam)/2, so
    |du|_2 <= sqrt(lam)/2 |(dv_x, dv_y)|_2 (Parseval)."""
    rng = _rng(10)
    f = rng.uniform(size=(32, 40))
    vx = rng.normal(size=f.shape)
    vy = rng.normal(size=f.shape)
    dvx = rng.normal(scale=1e-3, size=f.shape)
    dvy = rng.normal(scale=1e-3, size=f.shape)
    du = oracle.solve_eq8(f, vx + dvx, vy + dvy, lam) - oracle.solve_eq8(f, vx, vy, lam)
    bound = math.sqrt(lam) / 2 * math.sqrt(np.sum(dvx ** 2) + np.sum(dvy ** 2))
    assert math.sqrt(np.sum(du ** 2)) <= bound * (1 + 1e-9)


def test_blf_ls_reduces_to_ls_when_guidance_is_zero():
    """v = 0 turns Eq. 8 into the plain LS solve of Eq. 6: u = F^-1[F f / (1 + lam sum|Fd|^2)]."""
    H, W, lam = 12, 18, 7.0
    f = _rng(11).uniform(size=(H, W))
    sx = 4.0 * np.sin(np.pi * np.arange(W) / W) ** 2
    sy = 4.0 * np.sin(np.pi * np.arange(H) / H) ** 2
    want = np.fft.ifft2(np.fft.fft2(f) / (1.0 + lam * (sy[:, None] + sx[None, :]))).real
    z = np.zeros_like(f)
    np.testing.assert_allclose(oracle.solve_eq8(f, z, z, lam), want, atol=1e-14)


def test_iterations_compose_and_channels_are_independent():
    f = _rng(12).uniform(size=(2, 10, 12))
    one = oracle.blfls(f, 10.0, 1.5, 0.1, 2, iters=1)
    two = oracle.blfls(f, 10.0, 1.5, 0.1, 2, iters=2)
    np.testing.assert_array_equal(two, oracle.blfls(one, 10.0, 1.5, 0.1, 2, iters=1))
    np.testing.assert_array_equal(one[1], oracle.blfls(f[1], 10.0, 1.5, 0.1, 2))
    np.testing.assert_array_equal(oracle.blfls(f, 10.0, 1.5, 0.1, 2, iters=0), f)


def test_residual_form_matches_eq8():
    """u = f + (I + lam L)^-1 lam (D_x^T e_x + D_y^T e_y) with e = v - g is Eq. 8 rewritten by
    linearity (D f = g); checked here on the oracle's own residuals with the dense operator."""
    H, W, lam = 8, 6, 25.0
    f = _rng(13).uniform(size=(H, W))
    ex, ey = oracle.blf_residuals(f, 2, 1.2, 0.15)
    Dx, Dy = _diff_matrices(H, W)
    A = np.eye(H * W) + lam * (Dx.T @ Dx + Dy.T @ Dy)
    du = np.linalg.solve(A, lam * (Dx.T @ ex[0].ravel() + Dy.T @ ey[0].ravel()))
    want = f + du.reshape(H, W)
    np.testing.assert_allclose(oracle.blfls(f, lam, 1.2, 0.15, 2), want, atol=1e-12)


def test_normalised_gradients_are_the_filter_with_the_range_scaled():
    """Section IV normalises the gradients to [0, 1]: normalising a field of range R around
    Eq. 1 and restoring it equals Eq. 1 on the raw field with sigma_r R (the weights sum to 1 and
    the range kernel sees only differences), per field and channel."""
    f = np.random.default_rng(21).uniform(size=(2, 20, 24))
    got = oracle.blfls(f, 20.0, 3.0, 0.1, 4, normalize_grad=True)
    for c in range(2):
        gx, gy = oracle.gradients(f[c])
        rx, ry = gx.max() - gx.min(), gy.max() - gy.min()
        want = oracle.solve_eq8(f[c], oracle.blf(gx, 4, 3.0, 0.1 * rx), oracle.blf(gy, 4, 3.0, 0.1 * ry),
                                20.0)
        np.testing.assert_allclose(got[c], want, rtol=0, atol=1e-12)


def test_normalised_gradients_make_the_smoother_scale_invariant():
    """With normalised gradients the result scales with the image (u(a f) = a u(f)); without
    them it does not (sigma_r is absolute)."""
    f = np.random.default_rng(22).uniform(size=(18, 22))
    u1 = oracle.blfls(f, 30.0, 3.0, 0.1, 3, iters=2, normalize_grad=True)
    u2 = oracle.blfls(3.7 * f, 30.0, 3.0, 0.1, 3, iters=2, normalize_grad=True)
    np.testing.assert_allclose(u2, 3.7 * u1, rtol=0, atol=1e-12)
    v1 = oracle.blfls(f, 30.0, 3.0, 0.1, 3)
    v2 = oracle.blfls(3.7 * f, 30.0, 3.0, 0.1, 3)
    assert np.max(np.abs(v2 - 3.7 * v1)) > 1e-3


def test_normalised_constant_field_is_left_alone():
    """A field of zero range (here the x-gradient of an image constant along x) is returned
    unchanged, so its residual is zero."""
    f = np.tile(np.random.default_rng(23).uniform(size=(16, 1)), (1, 12))
    gx, _ = oracle.gradients(f)
    assert np.all(gx == 0.0)
    np.testing.assert_array_equal(oracle.blf_field(gx, 3, 2.0, 0.1, normalize=True), gx)
