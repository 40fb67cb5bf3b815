"""GPU parity of joint (guided) BLF-LS, the periodic Gaussian and rolling guidance
(Section III-D) against the FP64 oracle, through the C ABI.

Tolerances as for the plain smoother: FP32 max-abs 1e-4, FP16W/BF16W 2e-3 (images in [0, 1]);
the Gaussian (a normalised average) within 1e-6.  A guidance image equal to the input makes the
joint kernels compute exactly the plain kernels' arithmetic, so those results must be equal bit
for bit."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1812_07122_gb300 import blfls, synth

from gpu_util import DEV, maxabs, smooth, stream, to_dev

pytestmark = pytest.mark.gpu

TOL = {blfls.BLFLS_FP32: 1e-4, blfls.BLFLS_FP16W: 2e-3, blfls.BLFLS_BF16W: 2e-3}


@pytest.fixture(scope="module")
def h():
    import __graft_entry__
    __graft_entry__.build()
    handle = blfls.blfls_create(0)
    yield handle
    blfls.blfls_destroy(handle)


def _img(H, W, C=1, seed=0):
    return synth.sinusoid_disc_image(H, W, C, n_disc=max(3, H * W // 2000), noise=0.03, seed=seed)


def _guided(h, f, g, lam, ss, sr, r, iters=1, prec=blfls.BLFLS_FP32, inplace=False):
    C, H, W = f.shape
    x, gd = to_dev(f), to_dev(g)
    out = x if inplace else torch.empty_like(x)
    blfls.blfls_smooth_guided(h, x, gd, out, H, W, C, g.shape[0], lam, ss, sr, r, iters, prec,
                              stream())
    torch.cuda.synchronize(DEV)
    return out.cpu().numpy()


def _rolling(h, f, lam, ss, sr, r, iters, sg, prec=blfls.BLFLS_FP32):
    C, H, W = f.shape
    x = to_dev(f)
    out = torch.empty_like(x)
    blfls.blfls_smooth_rolling(h, x, out, H, W, C, lam, ss, sr, r, iters, sg, prec, stream())
    torch.cuda.synchronize(DEV)
    return out.cpu().numpy()


@pytest.mark.parametrize("prec", [blfls.BLFLS_FP32, blfls.BLFLS_FP16W, blfls.BLFLS_BF16W])
@pytest.mark.parametrize("H,W,C,r", [(64, 80, 1, 5), (45, 61, 3, 10), (33, 33, 1, 16)])
def test_guided_by_itself_equals_plain_bit_for_bit(h, prec, H, W, C, r):
    """One pass (a later joint pass keeps the first guidance, a plain pass does not).  FP32 and
    BF16W: bit for bit.  FP16W: the joint and plain kernels are compiled separately, and how a
    subnormal FP16 weight is rounded is the compiler's choice per kernel, so they may differ
    by an output ulp or so (as the batched and single FP16W drivers do); bound 1e-6, far below
    the FP16W tolerance of 2e-3."""
    f = _img(H, W, C, seed=H + W)
    want = smooth(h, f, 20.0, r / 2, 0.1, r, 1, prec)
    got = _guided(h, f, f, 20.0, r / 2, 0.1, r, 1, prec)
    if prec == blfls.BLFLS_FP16W:
        assert maxabs(got, want) <= 1e-6
    else:
        np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("prec", [blfls.BLFLS_FP32, blfls.BLFLS_FP16W, blfls.BLFLS_BF16W])
@pytest.mark.parametrize("H,W,C,Cg,r,ss,sr,lam,iters", [
    (64, 80, 1, 1, 5, 3.0, 0.1, 20.0, 1),
    (57, 70, 3, 3, 8, 4.0, 0.08, 30.0, 2),     # ragged tiles, a guide per channel
    (48, 64, 3, 1, 3, 1.5, 0.2, 1024.0, 1),    # one guide shared by three channels
    (40, 40, 1, 1, 16, 8.0, 0.05, 20.0, 1),
])
def test_guided_matches_oracle(h, prec, H, W, C, Cg, r, ss, sr, lam, iters):
    f = _img(H, W, C, seed=3 * H + W)
    g = _img(H, W, Cg, seed=H * W + 7)          # an unrelated guidance image
    got = _guided(h, f, g, lam, ss, sr, r, iters, prec)
    want = oracle.blfls_joint(f, g, lam, ss, sr, r, iters)
    assert maxabs(got, want) <= TOL[prec]


@pytest.mark.parametrize("r", [20, 50])
def test_guided_large_radius_per_pixel_kernel(h, r):
    H, W = 110, 120
    f = _img(H, W, 1, seed=r)
    g = _img(H, W, 1, seed=r + 1)
    got = _guided(h, f, g, 30.0, r / 2, 0.1, r)
    assert maxabs(got, oracle.blfls_joint(f, g, 30.0, r / 2, 0.1, r)) <= 1e-4


def test_guided_constant_guide_and_in_place(h):
    f = _img(50, 66, 2, seed=9)
    c = np.full((1, 50, 66), 0.3, np.float32)
    got = _guided(h, f, c, 20.0, 2.0, 0.1, 4)
    # constant guidance = no range kernel: the plain smoother with sigma_r = inf
    assert maxabs(got, smooth(h, f, 20.0, 2.0, math.inf, 4)) <= 1e-5
    np.testing.assert_array_equal(_guided(h, f, c, 20.0, 2.0, 0.1, 4, inplace=True), got)


@pytest.mark.parametrize("H,W,C,sigma", [(64, 80, 1, 1.0), (37, 53, 3, 2.5), (20, 16, 1, 6.0)])
def test_gaussian_matches_oracle(h, H, W, C, sigma):
    f = _img(H, W, C, seed=5)
    x = to_dev(f)
    out = torch.empty_like(x)
    blfls.blfls_gaussian(h, x, out, H, W, C, sigma, stream())
    torch.cuda.synchronize(DEV)
    assert maxabs(out.cpu().numpy(), oracle.gaussian(f, sigma)) <= 1e-6


@pytest.mark.parametrize("prec", [blfls.BLFLS_FP32, blfls.BLFLS_FP16W])
@pytest.mark.parametrize("iters", [1, 3])
def test_rolling_matches_oracle(h, prec, iters):
    f = _img(72, 90, 3, seed=iters)
    got = _rolling(h, f, 20.0, 3.0, 0.05, 6, iters, 1.0, prec)
    want = oracle.blfls_rolling(f, 20.0, 3.0, 0.05, 6, iters, 1.0)
    assert maxabs(got, want) <= TOL[prec]


def test_guided_and_rolling_reject_invalid_arguments(h):
    f = to_dev(_img(32, 32, 2, seed=1))
    g1 = to_dev(_img(32, 32, 1, seed=2))
    out = torch.empty_like(f)
    bad_calls = [
        lambda: blfls.blfls_smooth_guided(h, f, None, out, 32, 32, 2, 1, 20.0, 2.0, 0.1, 3),
        lambda: blfls.blfls_smooth_guided(h, f, g1, out, 32, 32, 2, 3, 20.0, 2.0, 0.1, 3),
        lambda: blfls.blfls_smooth_guided(h, f, out, out, 32, 32, 2, 2, 20.0, 2.0, 0.1, 3),
        lambda: blfls.blfls_smooth_guided(h, f, g1, out, 32, 32, 2, 1, 20.0, 2.0, 0.1, 20, 1, 1),
        lambda: blfls.blfls_smooth_rolling(h, f, f, 32, 32, 2, 20.0, 2.0, 0.1, 3, 2, 1.0),
        lambda: blfls.blfls_smooth_rolling(h, f, out, 32, 32, 2, 20.0, 2.0, 0.1, 3, 2, 0.0),
        lambda: blfls.blfls_gaussian(h, f, out, 32, 32, 2, 40.0),
        lambda: blfls.blfls_gaussian(h, f, out, 32, 32, 2, float("nan")),
    ]
    for call in bad_calls:
        with pytest.raises(blfls.BlflsError) as ei:
            call()
        assert ei.value.code == blfls.BLFLS_EINVAL
