"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, element by element.

Tolerance for the FP32 path: max-abs 1e-4 on images in [0, 1] (the accuracy target of the
FP32 form).  Sizes span several 32x32 bilateral tiles with ragged edges, odd and prime
dimensions (the prime ones run the Bluestein FFT), and the 4K RGB workload in full.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1812_07122_gb300 import blfls, synth

from gpu_util import blf_residual, maxabs, smooth, solve_residual

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-4


@pytest.fixture(scope="module")
def h():
    import __graft_entry__
    __graft_entry__.build()
    handle = blfls.blfls_create(0)
    yield handle
    blfls.blfls_destroy(handle)


def _img(H, W, C=1, seed=0):
    return synth.sinusoid_disc_image(H, W, C, n_disc=max(3, H * W // 2000), noise=0.03, seed=seed)


# ------------------------------------------------------------------------------------------
# Step 1: bilateral residuals e = BLF(g) - g
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("H,W,C,r,ss,sr", [
    (64, 48, 1, 3, 1.5, 0.1),
    (37, 53, 2, 5, 3.0, 0.1),       # ragged tiles, two channels
    (100, 70, 1, 10, 5.0, 0.08),
    (33, 33, 1, 16, 8.0, 0.05),     # 2r+1 = H: the window wraps onto the whole column
    (80, 120, 1, 20, 10.0, 0.1),    # runtime-radius tiled kernel
    (130, 120, 1, 50, 25.0, 0.2),   # global-memory kernel
    (45, 61, 1, 4, 2.0, math.inf),  # no range kernel
    (45, 61, 1, 4, math.inf, 0.1),  # no spatial kernel
    (20, 9, 1, 0, 1.0, 0.1),        # radius 0: residual is exactly zero
    (7, 300, 3, 2, 1.0, 0.3),
])
def test_blf_residual_matches_oracle(h, H, W, C, r, ss, sr):
    f = _img(H, W, C, seed=H * 7 + W)
    ex, ey = blf_residual(h, f, ss, sr, r)
    wx, wy = oracle.blf_residuals(f, r, ss, sr)
    err = max(maxabs(ex, wx), maxabs(ey, wy))
    assert err <= TOL_FP32, err
    if r == 0:
        assert not np.any(ex) and not np.any(ey)


# ------------------------------------------------------------------------------------------
# Step 2: Fourier solve given residuals (oracle residuals in, so the solve is tested alone)
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("H,W", [(256, 256), (30, 50), (97, 61), (1, 64), (64, 1), (3, 5),
                                 (2160, 3840), (1536, 2048), (211, 4096), (4093, 17),
                                 (1080, 1920), (1080, 3840), (3840, 2160)])
@pytest.mark.parametrize("lam", [0.0, 20.0, 1024.0])
def test_solve_residual_matches_eq8(h, H, W, lam):
    rng = np.random.default_rng(H + 3 * W)
    f = rng.uniform(size=(H, W)).astype(np.float32)
    ex = rng.normal(scale=0.05, size=(H, W)).astype(np.float32)
    ey = rng.normal(scale=0.05, size=(H, W)).astype(np.float32)
    got = solve_residual(h, f, ex, ey, lam)[0]
    gx, gy = oracle.gradients(f)
    want = oracle.solve_eq8(f, gx + ex.astype(np.float64), gy + ey.astype(np.float64), lam)
    err = maxabs(got, want)
    assert err <= TOL_FP32, err
    if lam == 0.0:
        assert np.array_equal(got, f)


@pytest.mark.parametrize("H,W", [(211, 128), (1523, 96), (97, 300), (11, 40), (13, 2), (37, 1),
                                 (8191, 3)])
@pytest.mark.parametrize("lam", [0.5, 1.0e4, 2.0e4])
def test_solve_recursion_columns_match_eq8(h, H, W, lam):
    """Column lengths without a mixed-radix plan: up to lambda = 1e4 the column transform, divide
    and inverse are the cyclic recursion they equal (its rounding grows like sqrt(lambda), largest
    at 1e4), above it Bluestein transforms; both match Eq. 8, with more than one 32-column block
    and a ragged last block (W = 300: 151 columns), a single segment (11, 13, 37 rows), one or two
    columns, and 256 segments (8191 rows, a prime)."""
    rng = np.random.default_rng(H + 7 * W)
    f = rng.uniform(size=(H, W)).astype(np.float32)
    ex = rng.normal(scale=0.05, size=(H, W)).astype(np.float32)
    ey = rng.normal(scale=0.05, size=(H, W)).astype(np.float32)
    got = solve_residual(h, f, ex, ey, lam)[0]
    gx, gy = oracle.gradients(f)
    want = oracle.solve_eq8(f, gx + ex.astype(np.float64), gy + ey.astype(np.float64), lam)
    err = maxabs(got, want)
    assert err <= TOL_FP32, err


@pytest.mark.parametrize("H,W,log2_len", [(2160, 96, 12), (1080, 70, 11), (8, 3840, 3),
                                          (9, 1920, 4)])
def test_solve_compile_time_plans_every_column_block(tmp_path, H, W, log2_len):
    """The lengths with compile-time plans (columns of 2160 and 1080, rows of 3840 and 1920),
    with every column block the column driver can take (chosen through a tune table; 16 columns
    of 2160 points exceed the shared-memory budget and run as 13) and with the column driver's
    own choice (an empty table): each matches Eq. 8, and all blocks give the same bits (a
    column's arithmetic does not depend on how columns are grouped)."""
    import json
    rng = np.random.default_rng(H * 7 + W)
    f = rng.uniform(size=(H, W)).astype(np.float32)
    ex = rng.normal(scale=0.05, size=(H, W)).astype(np.float32)
    ey = rng.normal(scale=0.05, size=(H, W)).astype(np.float32)
    gx, gy = oracle.gradients(f)
    want = oracle.solve_eq8(f, gx + ex.astype(np.float64), gy + ey.astype(np.float64), 30.0)
    outs = []
    for cb in (1, 2, 4, 7, 8, 13, 16, None):
        path = tmp_path / f"tune_{cb}.json"
        blocks = [] if cb is None else [{"log2_len": log2_len, "col_block": cb}]
        path.write_text(json.dumps({"blfls_tune_table": 1, "k1_tile_h": [],
                                    "k3_col_block": blocks}))
        h2 = blfls.blfls_create(0, tune_table_path=str(path))
        try:
            outs.append(solve_residual(h2, f, ex, ey, 30.0)[0])
        finally:
            blfls.blfls_destroy(h2)
        assert maxabs(outs[-1], want) <= TOL_FP32, (cb, maxabs(outs[-1], want))
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])


# ------------------------------------------------------------------------------------------
# The whole smoother
# ------------------------------------------------------------------------------------------
def test_small_grey_rectangles_workload(h):
    """256x256 grey rectangles + noise, r = 5, sigma_s = 3, sigma_r = 0.1, lam = 20, 1 pass."""
    f = synth.image_256_rectangles()
    got = smooth(h, f, 20.0, 3.0, 0.1, 5, 1)
    want = oracle.blfls(f, 20.0, 3.0, 0.1, 5, 1)
    err = maxabs(got, want)
    assert err <= TOL_FP32, err


@pytest.mark.parametrize("H,W,C,lam,ss,sr,r,iters", [
    (96, 128, 3, 30.0, 5.0, 0.08, 10, 3),
    (61, 97, 1, 50.0, 2.0, 0.05, 3, 1),     # prime sizes: Bluestein in both directions
    (120, 90, 2, 1024.0, 4.0, 0.12, 8, 2),  # the paper's default lambda
    (64, 64, 1, 0.0, 3.0, 0.1, 5, 1),        # lam = 0 returns f exactly
    (50, 70, 1, 20.0, 3.0, math.inf, 5, 1),  # no range kernel
    (40, 33, 4, 10.0, 1.0, 0.2, 1, 2),
    (11, 13, 1, 5.0, 1.0, 0.1, 5, 1),        # 2r+1 = H
])
def test_smooth_matches_oracle(h, H, W, C, lam, ss, sr, r, iters):
    f = _img(H, W, C, seed=C * 1000 + H)
    got = smooth(h, f, lam, ss, sr, r, iters)
    want = oracle.blfls(f, lam, ss, sr, r, iters)
    err = maxabs(got, want)
    assert err <= TOL_FP32, err
    if lam == 0.0:
        assert np.array_equal(got, f)


@pytest.mark.parametrize("H,W", [(8192, 5), (5, 8192)])
def test_maximum_dimension_lines(h, H, W):
    """BLFLS_MAX_DIM along each axis (the plain FFT drivers take over where the staged buffers
    no longer fit)."""
    f = _img(H, W, 1, seed=H + W)
    got = smooth(h, f, 20.0, 1.5, 0.1, 2, 1)
    want = oracle.blfls(f, 20.0, 1.5, 0.1, 2, 1)
    assert maxabs(got, want) <= TOL_FP32


def test_maximum_dimension_square(h):
    """8192 x 8192 (BLFLS_MAX_DIM on both axes), radius 2, one pass: every pixel against the
    oracle (about half a minute of FP64 work on the host cores)."""
    f = np.random.default_rng(5).uniform(size=(1, 8192, 8192)).astype(np.float32)
    got = smooth(h, f, 30.0, 1.5, 0.1, 2, 1)
    want = oracle.blfls(f, 30.0, 1.5, 0.1, 2, 1)
    err = maxabs(got, want)
    print(f"8192x8192 r=2: max-abs {err:.3e}")
    assert err <= TOL_FP32, err


def test_constant_image_and_radius_zero(h):
    f = np.full((1, 40, 56), 0.3125, dtype=np.float32)
    assert maxabs(smooth(h, f, 30.0, 3.0, 0.1, 5), f) <= 1e-6
    g = _img(40, 56, 1, seed=5)
    assert maxabs(smooth(h, g, 30.0, 3.0, 0.1, 0), g) <= 1e-6


def test_in_place_equals_out_of_place(h):
    f = _img(70, 90, 3, seed=9)
    a = smooth(h, f, 25.0, 2.5, 0.1, 5, 2)
    b = smooth(h, f, 25.0, 2.5, 0.1, 5, 2, inplace=True)
    assert np.array_equal(a, b)


def test_iters_zero_copies(h):
    f = _img(20, 30, 2, seed=2)
    assert np.array_equal(smooth(h, f, 25.0, 2.5, 0.1, 3, 0), f)


def test_host_entry_point_equals_device_entry_point(h):
    import torch
    f = _img(64, 80, 3, seed=4)
    dev = smooth(h, f, 30.0, 3.0, 0.1, 5, 2)
    src = torch.from_numpy(f).pin_memory()
    dst = torch.empty_like(src).pin_memory()
    blfls.blfls_smooth_host(h, src, dst, 64, 80, 3, 30.0, 3.0, 0.1, 5, 2)
    assert np.array_equal(dst.numpy(), dev)


def test_host_entry_point_in_place_pageable_and_zero_iters(h):
    """The host entry point overlaps per-channel copies with compute on its own copy stream;
    in-place buffers, pageable memory and iters = 0 must give the device entry point's result."""
    import torch
    f = _img(48, 72, 3, seed=6)
    dev = smooth(h, f, 30.0, 3.0, 0.1, 4, 2)
    buf = torch.from_numpy(f.copy()).pin_memory()
    blfls.blfls_smooth_host(h, buf, buf, 48, 72, 3, 30.0, 3.0, 0.1, 4, 2)
    assert np.array_equal(buf.numpy(), dev)
    src = torch.from_numpy(f.copy())
    dst = torch.zeros_like(src)
    blfls.blfls_smooth_host(h, src, dst, 48, 72, 3, 30.0, 3.0, 0.1, 4, 2)
    assert np.array_equal(dst.numpy(), dev)
    dst.zero_()
    blfls.blfls_smooth_host(h, src, dst, 48, 72, 3, 30.0, 3.0, 0.1, 4, 0)
    assert np.array_equal(dst.numpy(), f)


def test_mean_is_preserved_on_gpu(h):
    f = _img(128, 96, 1, seed=3)
    u = smooth(h, f, 30.0, 3.0, 0.1, 5, 1)
    assert abs(float(u.astype(np.float64).mean()) - float(f.astype(np.float64).mean())) < 1e-6


@pytest.mark.parametrize("bad", [
    dict(radius=40),            # 2r+1 > min(H, W)
    dict(sigma_s=0.0),
    dict(sigma_r=-1.0),
    dict(lam=float("nan")),
    dict(lam=-1.0),
    dict(iters=-1),
    dict(C=5),
    dict(prec=7),
])
def test_invalid_arguments_are_rejected(h, bad):
    import torch
    args = dict(H=64, W=64, C=1, lam=10.0, sigma_s=2.0, sigma_r=0.1, radius=3, iters=1, prec=0)
    args.update(bad)
    x = torch.zeros(4, 64, 64, device="cuda")
    with pytest.raises(blfls.BlflsError) as ei:
        blfls.blfls_smooth(h, x, x, args["H"], args["W"], args["C"], args["lam"],
                           args["sigma_s"], args["sigma_r"], args["radius"], args["iters"],
                           args["prec"])
    assert ei.value.code == blfls.BLFLS_EINVAL


def test_memory_budget_is_enforced():
    import torch
    h2 = blfls.blfls_create(0, mem_budget_bytes=1 << 20)
    try:
        x = torch.zeros(1, 512, 512, device="cuda")
        with pytest.raises(blfls.BlflsError) as ei:
            blfls.blfls_smooth(h2, x, x, 512, 512, 1, 10.0, 2.0, 0.1, 3, 1)
        assert ei.value.code == blfls.BLFLS_ENOMEM
    finally:
        blfls.blfls_destroy(h2)


TOL_HALF = 2e-3    # accuracy target of the FP16/BF16-weight forms (images in [0, 1])


@pytest.mark.parametrize("prec", [blfls.BLFLS_FP16W, blfls.BLFLS_BF16W])
@pytest.mark.parametrize("H,W,C,lam,ss,sr,r,iters", [
    (96, 128, 3, 30.0, 5.0, 0.08, 10, 1),
    (61, 97, 1, 50.0, 2.0, 0.05, 3, 2),
    (256, 256, 1, 20.0, 3.0, 0.1, 5, 1),
    (70, 66, 2, 1024.0, 8.0, 0.12, 16, 1),
    (50, 70, 1, 20.0, 3.0, math.inf, 5, 1),
])
def test_precision_forms_match_oracle(h, prec, H, W, C, lam, ss, sr, r, iters):
    f = _img(H, W, C, seed=C * 77 + W)
    got = smooth(h, f, lam, ss, sr, r, iters, prec=prec)
    want = oracle.blfls(f, lam, ss, sr, r, iters)
    err = maxabs(got, want)
    assert err <= TOL_HALF, err


@pytest.mark.parametrize("prec", [blfls.BLFLS_FP16W, blfls.BLFLS_BF16W])
def test_precision_forms_on_sharp_rectangles(h, prec):
    """The 256x256 grey rectangles workload: gradients up to ~1 against sigma_r = 0.1 are the
    hardest case for a half-precision exponent."""
    f = synth.image_256_rectangles()
    got = smooth(h, f, 20.0, 3.0, 0.1, 5, 1, prec=prec)
    want = oracle.blfls(f, 20.0, 3.0, 0.1, 5, 1)
    err = maxabs(got, want)
    print(f"256x256 rectangles prec={prec}: max-abs {err:.3e}")
    assert err <= TOL_HALF, err


def test_precision_forms_reject_large_radius(h):
    import torch
    x = torch.zeros(1, 64, 64, device="cuda")
    with pytest.raises(blfls.BlflsError) as ei:
        blfls.blfls_smooth(h, x, x, 64, 64, 1, 10.0, 9.0, 0.1, 20, 1, blfls.BLFLS_FP16W)
    assert ei.value.code == blfls.BLFLS_EINVAL


def test_4k_rgb_three_iterations_full_image(h):
    """3840x2160 RGB, r = 10, sigma_s = 5, sigma_r = 0.08, lam = 30, 3 passes: every pixel of the
    benchmark workload against the oracle (about a minute of FP64 work on the host cores), for
    the FP32 path (1e-4) and the FP16/BF16-weight forms (2e-3); per-channel errors printed."""
    f = synth.image_4k_rgb()
    want = oracle.blfls(f, 30.0, 5.0, 0.08, 10, 3)
    for prec, tol, name in [(blfls.BLFLS_FP32, TOL_FP32, "fp32"),
                            (blfls.BLFLS_FP16W, TOL_HALF, "fp16w"),
                            (blfls.BLFLS_BF16W, TOL_HALF, "bf16w")]:
        got = smooth(h, f, 30.0, 5.0, 0.08, 10, 3, prec=prec).astype(np.float64)
        per_c = [(float(np.max(np.abs(got[c] - want[c]))),
                  float(np.sqrt(np.mean((got[c] - want[c]) ** 2)))) for c in range(3)]
        print(f"4K RGB x3 {name}: " + "; ".join(f"c{c} max-abs {m:.3e} rms {q:.3e}"
                                                for c, (m, q) in enumerate(per_c)))
        err = max(m for m, _ in per_c)
        assert err <= tol, (name, err)
