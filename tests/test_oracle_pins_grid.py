"""Pins of the FP64 oracle of the bilateral-grid BLF (the fast approximation the paper uses,
Section III-A / IV) and of BLF-LS on it, against closed forms, scipy and the brute-force
filter (no GPU)."""
import math

import numpy as np
import pytest
import scipy.ndimage as ndi

import oracle


def _rng(seed):
    return np.random.default_rng(seed)


def test_grid_shape():
    # floor((W-1)/s)+1 cells of data plus 2 pads on each side, per axis
    assert oracle.grid_shape(10, 21, -0.5, 0.5, 5.0, 0.25) == (4 + 1 + 4, 1 + 1 + 4, 4 + 1 + 4)


def test_grid_constant_field_is_exact():
    g = np.full((17, 23), 0.37)
    np.testing.assert_allclose(oracle.blf_grid(g, 3.0, 0.1), g, rtol=0, atol=1e-15)


def test_grid_unit_spatial_step_single_range_bin_is_normalised_convolution():
    """s_s = 1 puts every pixel in its own cell and slices at cell centres; with sigma_r huge
    every value sits in one range bin, so the grid filter is the zero-padded normalised
    convolution with the outer product of (e^-1/2, 1, e^-1/2)."""
    g = _rng(1).normal(size=(9, 13))
    k1 = np.array([math.exp(-0.5), 1.0, math.exp(-0.5)])
    k = np.outer(k1, k1)
    want = ndi.correlate(g, k, mode="constant") / ndi.correlate(np.ones_like(g), k, mode="constant")
    np.testing.assert_allclose(oracle.blf_grid(g, 1.0, 1e6), want, rtol=0, atol=1e-13)


def test_grid_is_affine_equivariant():
    """(a g + b) with sigma_r scaled by a lands in the same cells: the output is a v + b.  The
    values are dyadic and a is a power of two, so every cell coordinate is the same exact value
    (some exactly on a rounding boundary, decided alike)."""
    g = _rng(2).integers(-16, 17, size=(20, 24)) / 64.0
    v = oracle.blf_grid(g, 2.0, 0.125)
    np.testing.assert_allclose(oracle.blf_grid(2.0 * g + 0.25, 2.0, 0.25), 2.0 * v + 0.25,
                               rtol=0, atol=1e-12)


def test_grid_keeps_a_jump_far_above_sigma_r():
    """Values more than two range cells apart never mix (the range blur reaches one cell and the
    slice interpolates between neighbouring cells only)."""
    g = np.zeros((16, 20))
    g[:, 10:] = 1.0
    np.testing.assert_allclose(oracle.blf_grid(g, 2.0, 0.05), g, rtol=0, atol=1e-15)


def test_grid_approximates_the_brute_force_filter_in_the_interior():
    """On a smooth field the grid output is closer to the brute-force filter (radius 2 sigma_s)
    than the filter's own effect is large."""
    y, x = np.mgrid[0:64, 0:80]
    g = 0.3 * np.sin(2 * np.pi * x / 80 * 3) * np.cos(2 * np.pi * y / 64 * 2)
    g = g + 0.02 * _rng(3).normal(size=g.shape)
    for ss, sr in ((3.0, 0.2), (4.0, 0.05)):
        v = oracle.blf_grid(g, ss, sr)
        b = oracle.blf(g, int(2 * ss), ss, sr)
        m = slice(8, -8)
        err = np.sqrt(np.mean((v - b)[m, m] ** 2))
        effect = np.sqrt(np.mean((b - g)[m, m] ** 2))
        assert err < 0.5 * effect


def test_grid_blfls_special_cases():
    f = _rng(4).uniform(size=(2, 18, 22))
    np.testing.assert_allclose(oracle.blfls_grid(f, 0.0, 2.0, 0.1), f, rtol=0, atol=1e-14)
    c = np.full((12, 14), 0.6)
    np.testing.assert_allclose(oracle.blfls_grid(c, 30.0, 2.0, 0.1), c, rtol=0, atol=1e-13)
    u = oracle.blfls_grid(f, 20.0, 2.0, 0.1)
    np.testing.assert_allclose(u.sum(axis=(1, 2)), f.sum(axis=(1, 2)), rtol=1e-12)
    np.testing.assert_array_equal(oracle.blfls_grid(f, 20.0, 2.0, 0.1, iters=2),
                                  oracle.blfls_grid(u, 20.0, 2.0, 0.1))


def test_a_flipped_cell_is_the_decision_just_across_the_boundary():
    """A pixel whose range coordinate t is exactly an integer goes to cell t (floor(t + 1/2) of
    the exact value); moving it to the other candidate cell equals lowering its value by a
    hair, which puts t just below the boundary (the value itself changes by 1e-12)."""
    g = _rng(5).integers(0, 32, size=(12, 14)) / 32.0
    g[0, 0] = 0.0                      # min g = 0, so t = 4 g + 1/2: an integer where 32 g = 2 mod 4
    sr = 0.125
    t, lo = oracle.grid_z_coords(g, sr)
    assert lo == 0.0
    p = tuple(np.argwhere(np.abs(t - np.rint(t)) == 0)[0])   # a pixel exactly on a boundary
    flip = np.zeros_like(g, dtype=bool)
    flip[p] = True
    got = oracle.blf_grid(g, 2.0, sr, flip)
    h = g.copy()
    h[p] -= 1e-12
    want = oracle.blf_grid(h, 2.0, sr)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-10)
    assert np.max(np.abs(got - oracle.blf_grid(g, 2.0, sr))) > 1e-4
