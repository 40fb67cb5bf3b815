"""GPU parity of NC-LS (the domain-transform normalised convolution in place of the BLF,
Section III-D) against the FP64 oracle, through the C ABI.

The oracle decides box membership on the FP64 transform distance; the GPU sums transform steps
held in units of 2^-q (rounded down; q as the C interface states), so a member whose FP64
distance lies within (number of steps) x 2^-q of the radius is ambiguous: both decisions are
correct.  Those decisions are listed from the oracle's values, must be rare, and are handled as
described in ``ambiguity`` (element-wise comparison at the FP32 bound of 1e-4 everywhere else,
either decision inside their reach).  Multi-pass calls are checked pass by pass (each pass from
the GPU's previous output) and against the single passes bit for bit."""
import math

import numpy as np
import pytest
import torch

import ambiguity
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


def unit_exponent(sigma_s, nit):
    """q of the C interface: the largest integer <= 30 with floor(r_1 2^q) + 1 < 2^32."""
    r1 = oracle.nc_schedule(float(np.float32(sigma_s)), nit)[0]
    q = 30
    while q > 0 and math.floor(math.ldexp(r1, q)) + 1 >= 2 ** 32:
        q -= 1
    return q


def nc_ambiguous(f, ss, sr, nit):
    """(c, y, x, key) of every box decision within the GPU's step rounding of the radius; one key
    per pair of samples (the decision seen from both ends), key = (c, field, k, axis, y, x, d)
    for the pair (i, i + d), d > 0."""
    unit = 2.0 ** -unit_exponent(ss, nit)
    out = []
    for c in range(f.shape[0]):
        for fi, g in enumerate(oracle.gradients(np.asarray(f[c], np.float64))):
            for k, axis, d, m in oracle.nc_margins(g, ss, sr, nit):
                if d < 0:
                    continue
                for y, x in np.argwhere(np.abs(m) <= d * unit * 1.001 + 1e-9):
                    out.append((c, int(y), int(x), (c, fi, k, axis, int(y), int(x), d)))
    return out


def check_nc_pass(h, f, lam, ss, sr, nit):
    """One pass of the GPU against the FP64 oracle (see the module notes); returns the GPU's
    output."""
    f = np.asarray(f, np.float32)
    C, H, W = f.shape
    got = _nc(h, f, lam, ss, sr, 1, nit)
    base = oracle.ncls(f, lam, ss, sr, 1, nit)
    amb = nc_ambiguous(f, ss, sr, nit)

    def evaluate(keys):
        flips = [[{}, {}] for _ in range(C)]
        for (c, fi, k, axis, y, x, d) in keys:
            per = flips[c][fi].setdefault((k, axis), {})
            up = per.setdefault(d, np.zeros((H, W), dtype=bool))
            dn = per.setdefault(-d, np.zeros((H, W), dtype=bool))
            up[y, x] = True
            if axis == 1:
                dn[y, (x + d) % W] = True
            else:
                dn[(y + d) % H, x] = True
        return oracle.ncls(f, lam, ss, sr, 1, nit, flips)

    radii = oracle.nc_schedule(float(np.float32(ss)), nit)
    rho = 2 * sum(int(math.ceil(r)) for r in radii) + 2 + ambiguity.solve_reach(lam, TOL)
    n_dec = C * 2 * H * W * sum(2 * int(math.floor(r)) for r in radii)
    summary = ambiguity.check(got, base, amb, evaluate, rho, TOL, n_decisions=n_dec)
    print("nc", (H, W, C, lam, ss, sr, nit), summary)
    return got


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
    u = f
    for _ in range(iters):
        u = check_nc_pass(h, u, lam, ss, sr, nit)
    if iters > 1:
        np.testing.assert_array_equal(_nc(h, f, lam, ss, sr, iters, nit), u)


def test_ncls_4k_channel(h):
    f = synth.image_4k_rgb()[:1]
    check_nc_pass(h, f, 30.0, 5.0, 0.08, 3)


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
