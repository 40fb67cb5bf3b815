"""Pins of the FP64 oracle of the LS model (Section II-B, Eqs. 5-6) and of the base/detail
applications (Section IV) against closed forms and dense linear algebra (no GPU)."""
import math

import numpy as np
import pytest

import oracle


def _rng(seed):
    return np.random.default_rng(seed)


def _laplacian(H, W):
    """Dense L = Dx^T Dx + Dy^T Dy for the periodic forward differences (Section II-B)."""
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
    return Dx, Dy, Dx.T @ Dx + Dy.T @ Dy


@pytest.mark.parametrize("H,W", [(8, 8), (8, 5), (7, 8), (1, 6), (5, 1)])
@pytest.mark.parametrize("lam", [0.1, 20.0, 1024.0])
def test_ls_matches_dense_normal_equations(H, W, lam):
    """Eq. 5's stationarity condition is (I + lam L) u = f; solved densely it must equal Eq. 6."""
    f = _rng(H * 13 + W + int(lam)).uniform(size=(H, W))
    _, _, L = _laplacian(H, W)
    want = np.linalg.solve(np.eye(H * W) + lam * L, f.ravel()).reshape(H, W)
    np.testing.assert_allclose(oracle.ls(f, lam), want, rtol=0, atol=1e-12 * (1 + lam))


@pytest.mark.parametrize("k,l", [(1, 0), (0, 2), (3, 5), (7, 1)])
def test_ls_fourier_mode_is_scaled_by_the_eq6_denominator(k, l):
    """A single real Fourier mode is an eigenvector of L with eigenvalue
    4 sin^2(pi k / W) + 4 sin^2(pi l / H), so Eq. 6 only scales it."""
    H, W, lam = 16, 24, 3.5
    y, x = np.mgrid[0:H, 0:W]
    f = np.cos(2 * math.pi * (k * x / W + l * y / H) + 0.3)
    gain = 1.0 / (1.0 + lam * (4 * math.sin(math.pi * k / W) ** 2 + 4 * math.sin(math.pi * l / H) ** 2))
    np.testing.assert_allclose(oracle.ls(f, lam), gain * f, rtol=0, atol=1e-13)


def test_ls_special_cases_and_gradient_energy():
    f = _rng(3).uniform(size=(2, 12, 10))
    np.testing.assert_allclose(oracle.ls(f, 0.0), f, rtol=0, atol=1e-14)          # lam = 0
    c = np.full((9, 7), 0.4)
    np.testing.assert_allclose(oracle.ls(c, 50.0), c, rtol=0, atol=1e-14)         # constant
    u = oracle.ls(f, 6.0)
    np.testing.assert_allclose(u.sum(axis=(1, 2)), f.sum(axis=(1, 2)), rtol=1e-13)  # mean
    # the LS model penalises every gradient: the smoothed image's gradient energy is smaller
    for ch in range(2):
        gx, gy = oracle.gradients(f[ch])
        ux, uy = oracle.gradients(u[ch])
        assert np.sum(ux ** 2 + uy ** 2) < np.sum(gx ** 2 + gy ** 2)
    np.testing.assert_array_equal(oracle.ls(f, 6.0, iters=2), oracle.ls(u, 6.0))


def test_detail_enhance_special_cases():
    f = _rng(4).uniform(size=(2, 14, 12))
    np.testing.assert_allclose(oracle.detail_enhance(f, 20.0, 2.0, 0.1, 3, 1, 0.0), f,
                               rtol=0, atol=0)                                      # m = 0
    np.testing.assert_allclose(oracle.detail_enhance(f, 0.0, 2.0, 0.1, 3, 1, 2.5), f,
                               rtol=0, atol=1e-14)                                  # lam = 0: u = f
    np.testing.assert_allclose(oracle.detail_enhance(f, 20.0, 2.0, 0.1, 0, 1, 2.5), f,
                               rtol=0, atol=1e-13)                                  # r = 0: BLF = id
    u = oracle.blfls(f, 20.0, 2.0, 0.1, 3)
    np.testing.assert_allclose(oracle.detail_enhance(f, 20.0, 2.0, 0.1, 3, 1, 1.5),
                               f + 1.5 * (f - u), rtol=0, atol=1e-15)


def test_log_tone_closed_forms():
    f = _rng(5).uniform(0.05, 1.0, size=(1, 12, 14))
    # c = 1: exp(b + l - b) = f
    np.testing.assert_allclose(oracle.log_tone(f, 20.0, 2.0, 0.1, 3, 1, 1.0), f, rtol=1e-13)
    # r = 0 (BLF identity) or lam = 0: b = l, so out = exp(c l) = f^c
    for kw in (dict(lam=20.0, radius=0), dict(lam=0.0, radius=3)):
        out = oracle.log_tone(f, kw["lam"], 2.0, 0.1, kw["radius"], 1, 0.4)
        np.testing.assert_allclose(out, f ** 0.4, rtol=1e-12)
    # constant image a: out = a^c; values below the floor are clamped to it
    a = np.full((1, 6, 8), 0.25)
    np.testing.assert_allclose(oracle.log_tone(a, 30.0, 2.0, 0.1, 2, 1, 0.5), np.sqrt(a), rtol=1e-13)
    z = np.zeros((1, 6, 8))
    np.testing.assert_allclose(oracle.log_tone(z, 30.0, 2.0, 0.1, 2, 1, 0.5, floor=1e-4),
                               np.full_like(z, 1e-2), rtol=1e-12)
