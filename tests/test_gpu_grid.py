"""GPU parity of BLF-LS with the bilateral-grid filter (the fast approximation of Eq. 1 that the
paper uses) against the FP64 grid oracle, through the C ABI.

Both sides decide every pixel's grid cell in FP32 (a quantisation decided by floating point);
sums, blur and slicing are FP32 on the GPU and FP64 in the oracle, so the FP32 bound of 1e-4
(images in [0, 1]) applies."""
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


def _grid(h, f, lam, ss, sr, iters=1, inplace=False):
    C, H, W = f.shape
    x = to_dev(f)
    out = x if inplace else torch.empty_like(x)
    blfls.blfls_smooth_grid(h, x, out, H, W, C, lam, ss, sr, iters, stream())
    torch.cuda.synchronize(DEV)
    return out.cpu().numpy()


@pytest.mark.parametrize("H,W,C,lam,ss,sr,iters", [
    (64, 80, 1, 20.0, 2.0, 0.05, 1),
    (57, 71, 3, 30.0, 3.0, 0.08, 2),      # ragged sizes, three channels, two passes
    (128, 96, 1, 1024.0, 4.0, 0.1, 1),
    (7, 300, 2, 20.0, 5.0, 0.2, 1),       # a grid one data cell high
    (211, 128, 1, 20.0, 1.0, 0.05, 1),    # unit spatial step, prime height (Bluestein solve)
    (40, 40, 1, 20.0, 6.0, math.inf, 1),  # one range cell
])
def test_grid_blfls_matches_oracle(h, H, W, C, lam, ss, sr, iters):
    f = _img(H, W, C, seed=H + 5 * W)
    got = _grid(h, f, lam, ss, sr, iters)
    want = oracle.blfls_grid(f, lam, ss, sr, iters)
    assert maxabs(got, want) <= TOL


def test_grid_4k_channel(h):
    f = synth.image_4k_rgb()[:1]
    got = _grid(h, f, 30.0, 5.0, 0.08)
    assert maxabs(got, oracle.blfls_grid(f, 30.0, 5.0, 0.08)) <= TOL


def test_grid_in_place_zero_iters_and_constant(h):
    f = _img(48, 64, 2, seed=3)
    a = _grid(h, f, 20.0, 3.0, 0.1, 2)
    np.testing.assert_array_equal(_grid(h, f, 20.0, 3.0, 0.1, 2, inplace=True), a)
    np.testing.assert_array_equal(_grid(h, f, 20.0, 3.0, 0.1, 0), f)
    c = np.full((1, 30, 40), 0.25, np.float32)
    assert maxabs(_grid(h, c, 20.0, 3.0, 0.1), c) <= 1e-6


def test_grid_rejects_invalid_arguments(h):
    f = to_dev(_img(32, 32, 1))
    out = torch.empty_like(f)
    for ss, sr, lam in ((0.25, 0.1, 20.0), (math.inf, 0.1, 20.0), (2.0, 0.0, 20.0),
                        (2.0, 0.1, -1.0), (2.0, 1e-9, 20.0)):
        with pytest.raises(blfls.BlflsError) as ei:
            blfls.blfls_smooth_grid(h, f, out, 32, 32, 1, lam, ss, sr, 1, stream())
        assert ei.value.code == blfls.BLFLS_EINVAL
