"""GPU parity of the LS model (Section II-B, Eqs. 5-6) and of the base/detail applications of
Section IV (detail enhancement, log-domain tone mapping) against the FP64 oracle.

Tolerances: the LS model and detail enhancement are linear in the image, so the FP32 bound of
1e-4 (images in [0, 1]) applies, scaled by 1 + m for the enhancement (out = f + m (f - u)).  The
tone map smooths the logarithmic image l, whose range D is several units: the smoother's error
scales with D, and out = exp(c b + l - b) carries (1 - c) times the error of b, so the bound is
1e-4 D (1 - c) plus a rounding allowance for logf/expf."""
import numpy as np
import pytest
import torch

import oracle
from paper_1812_07122_gb300 import blfls, synth

from gpu_util import DEV, maxabs, stream, to_dev

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-4


@pytest.fixture(scope="module")
def h():
    import __graft_entry__
    __graft_entry__.build()
    handle = blfls.blfls_create(0)
    yield handle
    blfls.blfls_destroy(handle)


def _img(H, W, C=1, seed=0, lo=0.0):
    f = synth.sinusoid_disc_image(H, W, C, n_disc=max(3, H * W // 2000), noise=0.03, seed=seed)
    return (lo + (1.0 - lo) * f).astype(np.float32)


def _ls(h, f, lam, iters=1, inplace=False):
    C, H, W = f.shape
    x = to_dev(f)
    out = x if inplace else torch.empty_like(x)
    blfls.blfls_smooth_ls(h, x, out, H, W, C, lam, iters, stream())
    torch.cuda.synchronize(DEV)
    return out.cpu().numpy()


def _layers(h, f, mode, strength, lam, ss, sr, r, iters=1, prec=blfls.BLFLS_FP32, inplace=False):
    C, H, W = f.shape
    x = to_dev(f)
    out = x if inplace else torch.empty_like(x)
    blfls.blfls_layers(h, x, out, H, W, C, mode, strength, lam, ss, sr, r, iters, prec, stream())
    torch.cuda.synchronize(DEV)
    return out.cpu().numpy()


@pytest.mark.parametrize("H,W,C,lam,iters", [
    (64, 80, 1, 20.0, 1),
    (211, 256, 3, 30.0, 2),     # prime height: Bluestein column transform
    (37, 53, 2, 1024.0, 1),     # the paper's default lambda
    (2160, 3840, 1, 30.0, 1),   # 4K plane
    (1, 64, 1, 5.0, 1),         # one row: the y difference wraps onto itself
    (48, 1, 1, 5.0, 1),         # one column
])
def test_ls_matches_oracle(h, H, W, C, lam, iters):
    f = _img(H, W, C, seed=H + 3 * W)
    got = _ls(h, f, lam, iters)
    want = oracle.ls(f, lam, iters)
    assert maxabs(got, want) <= TOL_FP32


def test_ls_in_place_zero_iters_and_lambda_zero(h):
    f = _img(40, 56, 2, seed=8)
    a = _ls(h, f, 12.0, 2)
    np.testing.assert_array_equal(_ls(h, f, 12.0, 2, inplace=True), a)
    np.testing.assert_array_equal(_ls(h, f, 12.0, 0), f)
    assert maxabs(_ls(h, f, 0.0, 1), f) <= 1e-6


@pytest.mark.parametrize("H,W,C,m,lam,ss,sr,r,iters", [
    (64, 80, 1, 2.0, 20.0, 3.0, 0.1, 5, 1),
    (96, 130, 3, 4.0, 30.0, 5.0, 0.08, 10, 2),
    (45, 61, 1, 0.0, 20.0, 2.0, 0.1, 3, 1),
])
def test_detail_enhance_matches_oracle(h, H, W, C, m, lam, ss, sr, r, iters):
    f = _img(H, W, C, seed=W)
    got = _layers(h, f, blfls.BLFLS_DETAIL_ENHANCE, m, lam, ss, sr, r, iters)
    want = oracle.detail_enhance(f, lam, ss, sr, r, iters, m)
    assert maxabs(got, want) <= TOL_FP32 * (1.0 + m)
    if m == 0.0:
        np.testing.assert_array_equal(got, f)


@pytest.mark.parametrize("H,W,C,c,lam,ss,sr,r", [
    (64, 80, 1, 0.5, 20.0, 3.0, 0.1, 5),
    (90, 128, 3, 0.3, 30.0, 5.0, 0.2, 8),
    (50, 50, 1, 1.0, 20.0, 2.0, 0.1, 3),
])
def test_log_tone_matches_oracle(h, H, W, C, c, lam, ss, sr, r):
    f = _img(H, W, C, seed=H * W, lo=0.02)
    got = _layers(h, f, blfls.BLFLS_LOG_TONE, c, lam, ss, sr, r)
    want = oracle.log_tone(f, lam, ss, sr, r, 1, c)
    lg = np.log(np.maximum(f.astype(np.float64), 1e-6))
    D = float(lg.max() - lg.min())
    assert maxabs(got, want) <= TOL_FP32 * D * (1.0 - c) + 1e-5 * float(np.max(want))


def test_layers_in_place_equals_out_of_place(h):
    f = _img(48, 64, 3, seed=11, lo=0.05)
    for mode, s in ((blfls.BLFLS_DETAIL_ENHANCE, 1.5), (blfls.BLFLS_LOG_TONE, 0.4)):
        a = _layers(h, f, mode, s, 20.0, 3.0, 0.1, 4)
        b = _layers(h, f, mode, s, 20.0, 3.0, 0.1, 4, inplace=True)
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("bad", [
    dict(mode=7), dict(strength=float("nan")), dict(strength=-1.0),
    dict(mode=blfls.BLFLS_LOG_TONE, strength=1.5), dict(iters=0), dict(radius=40),
])
def test_layers_rejects_invalid_arguments(h, bad):
    f = _img(32, 32, 1, seed=1)
    args = dict(mode=blfls.BLFLS_DETAIL_ENHANCE, strength=1.0, iters=1, radius=3)
    args.update(bad)
    with pytest.raises(blfls.BlflsError) as ei:
        _layers(h, f, args["mode"], args["strength"], 20.0, 2.0, 0.1, args["radius"], args["iters"])
    assert ei.value.code == blfls.BLFLS_EINVAL


def test_ls_rejects_invalid_arguments(h):
    f = _img(16, 16, 1)
    for lam, iters in ((float("nan"), 1), (-1.0, 1), (5.0, -1), (5.0, 65)):
        with pytest.raises(blfls.BlflsError) as ei:
            _ls(h, f, lam, iters)
        assert ei.value.code == blfls.BLFLS_EINVAL
