"""GPU parity of NC-LS (the domain-transform normalised convolution in place of the BLF,
Section III-D) against the FP64 oracle, through the C ABI.

Which samples enter each box is decided in FP32 on both sides with the same operations
(a floating-point decision); the averages are FP32 on the GPU and FP64 in the oracle, so the FP32
bound of 1e-4 (images in [0, 1]) applies."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1812_07122_gb300 import blfls, synth

from gpu_util import DEV, maxabs, stream, to_dev

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def h():
    import __graft_entry__
    __graft_entry__.build()
    handle = blfls.blfls_create(0)
    yield handle
    blfls.blfls_destroy(handle)


def _img(H, W, C=1, seed=0):
    return synth.sinusoid_disc_image(H, W, C, n_disc=max(3, H * W // 2000), noise=0.03, seed=seed)


def _nc(h, f, lam, ss, sr, iters=1, nc_iters=3, inplace=False):
    C, H, W = f.shape
    x = to_dev(f)
    out = x if inplace else torch.empty_like(x)
    blfls.blfls_smooth_nc(h, x, out, H, W, C, lam, ss, sr, iters, nc_iters, stream())
    torch.cuda.synchronize(DEV)
    return out.cpu().numpy()


@pytest.mark.parametrize("H,W,C,lam,ss,sr,iters,nit", [
    (64, 80, 1, 20.0, 3.0, 0.1, 1, 3),
    (57, 71, 3, 30.0, 5.0, 0.05, 2, 3),     # ragged sizes, three channels, two passes
    (100, 37, 1, 1024.0, 12.0, 0.05, 1, 3), # radius above a third of the width (wrapping boxes)
    (33, 45, 1, 20.0, 4.0, math.inf, 1, 2), # plain box iterations
    (211, 64, 1, 20.0, 2.0, 0.2, 1, 1),     # prime height (Bluestein solve), one iteration
    (72, 96, 2, 30.0, 8.0, 0.1, 1, 3),      # box radii 12, 6, 3
    (24, 7, 1, 20.0, 8.0, 0.1, 1, 3),       # radii above the width: boxes wrap several periods
    (9, 130, 1, 20.0, 45.0, 0.5, 1, 2),     # radii 69 (sliding-window passes) and 34 (tiles)
])
def test_ncls_matches_oracle(h, H, W, C, lam, ss, sr, iters, nit):
    f = _img(H, W, C, seed=7 * H + W)
    got = _nc(h, f, lam, ss, sr, iters, nit)
    want = oracle.ncls(f, lam, ss, sr, iters, nit)
    assert maxabs(got, want) <= TOL


def test_ncls_4k_channel(h):
    f = synth.image_4k_rgb()[:1]
    assert maxabs(_nc(h, f, 30.0, 5.0, 0.08), oracle.ncls(f, 30.0, 5.0, 0.08)) <= TOL


def test_ncls_in_place_zero_iters_constant(h):
    f = _img(40, 48, 2, seed=2)
    a = _nc(h, f, 20.0, 3.0, 0.1, 2)
    np.testing.assert_array_equal(_nc(h, f, 20.0, 3.0, 0.1, 2, inplace=True), a)
    np.testing.assert_array_equal(_nc(h, f, 20.0, 3.0, 0.1, 0), f)
    c = np.full((1, 24, 30), 0.4, np.float32)
    assert maxabs(_nc(h, c, 20.0, 3.0, 0.1), c) <= 1e-6


def test_ncls_rejects_invalid_arguments(h):
    f = to_dev(_img(32, 32, 1))
    out = torch.empty_like(f)
    for ss, sr, nit in ((0.0, 0.1, 3), (300.0, 0.1, 3), (3.0, 0.0, 3), (3.0, 0.1, 0), (3.0, 0.1, 9)):
        with pytest.raises(blfls.BlflsError) as ei:
            blfls.blfls_smooth_nc(h, f, out, 32, 32, 1, 20.0, ss, sr, 1, nit, stream())
        assert ei.value.code == blfls.BLFLS_EINVAL
