"""GPU parity of BLF-LS on normalised gradients (every gradient field mapped to [0, 1] around the
bilateral filter, per channel and pass: the setting of Section IV) against the FP64 oracle, which
normalises, filters and restores each field literally; the GPU filters the raw field with
sigma_r scaled by the field's range.  Tolerances as for the plain smoother: FP32 max-abs 1e-4,
FP16W/BF16W 2e-3 (images in [0, 1])."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1812_07122_gb300 import blfls, synth

from gpu_util import DEV, maxabs, stream, to_dev

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


def _norm(h, f, lam, ss, sr, r, iters=1, prec=blfls.BLFLS_FP32, inplace=False):
    C, H, W = f.shape
    x = to_dev(f)
    out = x if inplace else torch.empty_like(x)
    blfls.blfls_smooth_normalized(h, x, out, H, W, C, lam, ss, sr, r, iters, prec, stream())
    torch.cuda.synchronize(DEV)
    return out.cpu().numpy()


@pytest.mark.parametrize("H,W,C,lam,ss,sr,r,iters,prec", [
    (64, 80, 1, 20.0, 3.0, 0.1, 5, 1, blfls.BLFLS_FP32),
    (57, 71, 3, 30.0, 4.0, 0.2, 8, 2, blfls.BLFLS_FP32),     # ragged tiles, two passes
    (96, 128, 2, 30.0, 5.0, 0.1, 10, 1, blfls.BLFLS_FP32),
    (48, 50, 1, 20.0, 6.0, 0.15, 20, 1, blfls.BLFLS_FP32),   # runtime-radius tiled kernel
    (61, 67, 1, 20.0, 3.0, math.inf, 4, 1, blfls.BLFLS_FP32),
    (64, 80, 2, 20.0, 3.0, 0.1, 5, 1, blfls.BLFLS_FP16W),
    (64, 80, 2, 20.0, 3.0, 0.1, 5, 1, blfls.BLFLS_BF16W),
])
def test_normalized_matches_oracle(h, H, W, C, lam, ss, sr, r, iters, prec):
    f = _img(H, W, C, seed=H + 5 * W)
    got = _norm(h, f, lam, ss, sr, r, iters, prec)
    want = oracle.blfls(f, lam, ss, sr, r, iters, normalize_grad=True)
    err = maxabs(got, want)
    assert err <= TOL[prec], err


def test_normalized_is_scale_invariant(h):
    """u(a f) = a u(f) with normalised gradients (FP32 rounding only)."""
    f = _img(72, 90, 2, seed=9)
    u1 = _norm(h, f, 30.0, 4.0, 0.1, 6, 2)
    u2 = _norm(h, (3.0 * f).astype(np.float32), 30.0, 4.0, 0.1, 6, 2)
    assert maxabs(u2, 3.0 * u1.astype(np.float64)) <= 3e-5


def test_normalized_in_place_zero_iters_and_rejects_bad_arguments(h):
    f = _img(40, 48, 2, seed=3)
    a = _norm(h, f, 20.0, 3.0, 0.1, 5, 2)
    np.testing.assert_array_equal(_norm(h, f, 20.0, 3.0, 0.1, 5, 2, inplace=True), a)
    np.testing.assert_array_equal(_norm(h, f, 20.0, 3.0, 0.1, 5, 0), f)
    x = to_dev(f)
    out = torch.empty_like(x)
    for args in ((20.0, 3.0, 0.1, -1, 1, 0), (20.0, 3.0, 0.0, 5, 1, 0), (-1.0, 3.0, 0.1, 5, 1, 0),
                 (20.0, 3.0, 0.1, 5, 1, 7), (20.0, 3.0, 0.1, 20, 1, blfls.BLFLS_FP16W)):
        lam, ss, sr, r, iters, prec = args
        with pytest.raises(blfls.BlflsError) as ei:
            blfls.blfls_smooth_normalized(h, x, out, 40, 48, 2, lam, ss, sr, r, iters, prec,
                                          stream())
        assert ei.value.code == blfls.BLFLS_EINVAL


def test_normalized_call_does_not_wait_for_the_gpu(h):
    """The fields' ranges and range constants are computed on the device: with the stream held
    busy by a bounded spin, the call returns while the stream is still busy, and its result is
    the same as the same call made on an idle stream."""
    f = _img(96, 128, 3, seed=21)
    want = _norm(h, f, 20.0, 3.0, 0.1, 4, iters=2)       # also builds plans and scratch
    x = to_dev(f)
    out = torch.empty_like(x)
    torch.cuda.synchronize(DEV)
    s = stream()
    torch.cuda._sleep(200_000_000)                        # ~0.1 s of spinning on the stream
    blfls.blfls_smooth_normalized(h, x, out, 96, 128, 3, 20.0, 3.0, 0.1, 4, 2,
                                  blfls.BLFLS_FP32, s)
    done = torch.cuda.Event()
    done.record(s)
    assert not done.query(), "the call waited for the stream"
    torch.cuda.synchronize(DEV)
    np.testing.assert_array_equal(out.cpu().numpy(), want)
