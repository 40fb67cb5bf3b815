"""Pins of the FP64 oracle of joint (guided) BLF-LS, the periodic Gaussian and rolling guidance
(Section III-D) against independent code, library routines and closed forms (no GPU)."""
import math

import numpy as np
import pytest
import scipy.ndimage as ndi

import oracle


def _rng(seed):
    return np.random.default_rng(seed)


@pytest.mark.parametrize("H,W,r,ss,sr", [(9, 11, 2, 1.5, 0.2), (16, 7, 3, 2.0, 0.05), (6, 6, 2, 3.0, 1.0)])
def test_joint_filter_guided_by_its_own_field_is_the_plain_filter(H, W, r, ss, sr):
    """h = g: the joint filter is Eq. 1 itself; compared with the independent C brute force."""
    g = _rng(H * W).normal(scale=0.3, size=(H, W))
    np.testing.assert_allclose(oracle.blf_joint(g, g, r, ss, sr), oracle.blf(g, r, ss, sr),
                               rtol=0, atol=1e-14)


def test_joint_filter_with_a_constant_guide_is_the_spatial_gaussian():
    """Constant guidance: every range weight is 1, leaving the normalised truncated periodic
    Gaussian -- scipy's correlate with mode='wrap'."""
    H, W, r, ss = 12, 10, 3, 1.7
    g = _rng(2).normal(size=(H, W))
    y, x = np.mgrid[-r:r + 1, -r:r + 1]
    k = np.exp(-(x * x + y * y) / (2 * ss * ss))
    want = ndi.correlate(g, k / k.sum(), mode="wrap")
    np.testing.assert_allclose(oracle.blf_joint(g, np.full((H, W), 0.3), r, ss, 0.1), want,
                               rtol=0, atol=1e-13)


def test_joint_filter_two_level_guide_separates_the_regions():
    """A guide with a jump much larger than sigma_r cuts the window: each pixel averages only the
    input values on its own side (hand-checkable case: constant input per side)."""
    H, W = 8, 12
    h = np.zeros((H, W))
    h[:, 6:] = 10.0
    g = np.where(h > 0, 2.0, -1.0) + 0.0
    v = oracle.blf_joint(g, h, 2, 1.5, 0.05)
    # the guide jumps at columns 0|11 (wrap) and 5|6; no window straddles both sides' values
    np.testing.assert_allclose(v, g, rtol=0, atol=1e-12)
    # the plain filter of the same input (guided by itself) does the same; a guide that is
    # constant mixes the sides at the jump
    assert np.max(np.abs(oracle.blf_joint(g, np.zeros_like(h), 2, 1.5, 0.05) - g)) > 0.1


def test_joint_blfls_with_itself_as_guide_is_blfls_and_constant_guide_is_closed_form():
    f = _rng(3).uniform(size=(2, 12, 14))
    np.testing.assert_allclose(oracle.blfls_joint(f, f, 20.0, 2.0, 0.1, 3),
                               oracle.blfls(f, 20.0, 2.0, 0.1, 3), rtol=0, atol=1e-13)
    # constant guide: v = K * g with the spatial Gaussian K, so u = F^-1[F f (1 + lam K^ L^)/(1 + lam L^)]
    H, W, r, ss, lam = 12, 14, 3, 2.0, 20.0
    y, x = np.mgrid[-r:r + 1, -r:r + 1]
    k = np.exp(-(x * x + y * y) / (2 * ss * ss))
    k /= k.sum()
    kern = np.zeros((H, W))
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            kern[dy % H, dx % W] += k[dy + r, dx + r]
    Kh = np.fft.fft2(kern).real          # symmetric kernel: real spectrum
    L = (4 * np.sin(np.pi * np.arange(H) / H) ** 2)[:, None] + (4 * np.sin(np.pi * np.arange(W) / W) ** 2)[None, :]
    want = np.fft.ifft2(np.fft.fft2(f[0]) * (1 + lam * Kh * L) / (1 + lam * L)).real
    got = oracle.blfls_joint(f[0], np.full((H, W), 0.5), lam, ss, 0.1, r)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)
    # a single-channel guide is shared by every channel
    np.testing.assert_allclose(oracle.blfls_joint(f, f[:1], 20.0, 2.0, 0.1, 3)[0],
                               oracle.blfls_joint(f[0], f[0], 20.0, 2.0, 0.1, 3), atol=1e-15)


@pytest.mark.parametrize("sigma", [0.5, 1.3, 4.0])
def test_gaussian_is_scipy_wrap_correlation(sigma):
    a = _rng(4).uniform(size=(2, 17, 23))
    w = oracle.gaussian_weights(sigma)
    assert w.size == 2 * math.ceil(3 * sigma) + 1 and abs(w.sum() - 1) < 1e-15
    want = np.stack([ndi.correlate1d(ndi.correlate1d(a[c], w, axis=1, mode="wrap"), w, axis=0,
                                     mode="wrap") for c in range(2)])
    np.testing.assert_allclose(oracle.gaussian(a, sigma), want, rtol=0, atol=1e-14)
    np.testing.assert_allclose(oracle.gaussian(np.full((5, 6), 0.7), sigma), 0.7, atol=1e-15)
    np.testing.assert_allclose(oracle.gaussian(a, sigma).sum(axis=(1, 2)), a.sum(axis=(1, 2)),
                               rtol=1e-13)


def test_rolling_guidance_passes_compose():
    f = _rng(5).uniform(size=(1, 14, 12))
    args = (20.0, 2.0, 0.1, 3)
    g0 = oracle.gaussian(f, 1.0)
    one = oracle.blfls_joint(f, g0, *args)
    np.testing.assert_array_equal(oracle.blfls_rolling(f, *args, 1, 1.0), one)
    two = oracle.blfls_joint(f, one, *args)
    np.testing.assert_array_equal(oracle.blfls_rolling(f, *args, 2, 1.0), two)
    np.testing.assert_array_equal(oracle.blfls_rolling(f, *args, 0, 1.0), f)
    # a rolling pass keeps the input as its data term: lam = 0 returns f whatever the guidance
    np.testing.assert_allclose(oracle.blfls_rolling(f, 0.0, 2.0, 0.1, 3, 3, 1.0), f, atol=1e-14)
