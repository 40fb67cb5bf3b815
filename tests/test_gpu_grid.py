"""GPU parity of BLF-LS with the bilateral-grid filter (the fast approximation of Eq. 1 that the
paper uses) against the FP64 grid oracle, through the C ABI.

The oracle decides every pixel's range cell from the FP64 gradient; the GPU holds the gradient in
FP32 (and takes the decision in FP64 near a rounding boundary), so a pixel whose FP64 coordinate
lies closer to a boundary than the FP32 representation of its gradient and of the field's minimum
can move is ambiguous: both cells are correct.  Those pixels are listed from the oracle's values,
must be rare, and are handled as described in ``ambiguity`` (element-wise comparison at the FP32
bound of 1e-4 everywhere else, either decision inside their reach).  Multi-pass calls are checked
pass by pass (each pass from the GPU's previous output) and against the single passes bit for
bit."""
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


def _grid(h, f, lam, ss, sr, iters=1, inplace=False):
    C, H, W = f.shape
    x = to_dev(f)
    out = x if inplace else torch.empty_like(x)
    blfls.blfls_smooth_grid(h, x, out, H, W, C, lam, ss, sr, iters, stream())
    torch.cuda.synchronize(DEV)
    return out.cpu().numpy()


def grid_ambiguous(f, sigma_r):
    """(c, y, x, key) of every range-cell decision an FP32 gradient can place on either side of a
    rounding boundary (key = (c, field, y, x))."""
    sr = float(np.float32(sigma_r))
    out = []
    for c in range(f.shape[0]):
        for fi, g in enumerate(oracle.gradients(np.asarray(f[c], np.float64))):
            t, lo = oracle.grid_z_coords(g, sr)
            # how far the FP32 representation of the gradient and of the minimum can move t
            dg = np.abs(g - g.astype(np.float32)) + abs(lo - float(np.float32(lo)))
            delta = dg / sr + np.where(dg > 0, 8 * 2.0 ** -52 * np.abs(t), 0.0)
            for y, x in np.argwhere(np.abs(t - np.rint(t)) < delta):
                out.append((c, int(y), int(x), (c, fi, int(y), int(x))))
    return out


def check_grid_pass(h, f, lam, ss, sr):
    """One pass of the GPU against the FP64 oracle (see the module notes); returns the GPU's
    output."""
    f = np.asarray(f, np.float32)
    C, H, W = f.shape
    got = _grid(h, f, lam, ss, sr, 1)
    base = oracle.blfls_grid(f, lam, ss, sr, 1)
    amb = grid_ambiguous(f, sr)

    def evaluate(keys):
        flips = np.zeros((C, 2, H, W), dtype=bool)
        for (c, fi, y, x) in keys:
            flips[c, fi, y, x] = True
        return oracle.blfls_grid(f, lam, ss, sr, 1, flips)

    rho = int(math.ceil(3 * ss)) + 3 + ambiguity.solve_reach(lam, TOL)
    summary = ambiguity.check(got, base, amb, evaluate, rho, TOL, n_decisions=2 * C * H * W)
    print("grid", (H, W, C, lam, ss, sr), summary)
    return got


@pytest.mark.parametrize("H,W,C,lam,ss,sr,iters", [
    (64, 80, 1, 20.0, 2.0, 0.05, 1),
    (57, 71, 3, 30.0, 3.0, 0.08, 2),      # ragged sizes, three channels, two passes
    (128, 96, 1, 1024.0, 4.0, 0.1, 1),
    (7, 300, 2, 20.0, 5.0, 0.2, 1),       # a grid one data cell high
    (211, 128, 1, 20.0, 1.0, 0.05, 1),    # unit spatial step, prime height (Bluestein solve)
    (40, 40, 1, 20.0, 6.0, math.inf, 1),  # one range cell
    (96, 128, 2, 30.0, 2.5, 0.03, 1),     # many range cells, a non-integer spatial step
])
def test_grid_blfls_matches_oracle(h, H, W, C, lam, ss, sr, iters):
    f = _img(H, W, C, seed=H + 5 * W)
    u = f
    for _ in range(iters):
        u = check_grid_pass(h, u, lam, ss, sr)
    if iters > 1:
        np.testing.assert_array_equal(_grid(h, f, lam, ss, sr, iters), u)


def test_grid_dyadic_values_on_rounding_boundaries(h):
    """Values on a 1/64 lattice with sigma_r = 1/8: exact in FP32, so the gradients and the cell
    coordinates are exact and many lie exactly on a rounding boundary; the GPU must decide all
    of them as the FP64 definition does (no ambiguity is allowed: the representation is exact)."""
    rng = np.random.default_rng(9)
    f = (rng.integers(0, 65, size=(1, 48, 64)) / 64.0).astype(np.float32)
    assert not grid_ambiguous(f, 0.125)
    check_grid_pass(h, f, 20.0, 3.0, 0.125)


def test_grid_4k_channel(h):
    f = synth.image_4k_rgb()[:1]
    check_grid_pass(h, f, 30.0, 5.0, 0.08)


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
                        (2.0, 0.1, -1.0)):
        with pytest.raises(blfls.BlflsError) as ei:
            blfls.blfls_smooth_grid(h, f, out, 32, 32, 1, lam, ss, sr, 1, stream())
        assert ei.value.code == blfls.BLFLS_EINVAL


def test_grid_wide_range_in_many_chunks(h):
    """A field far wider than the range the grid buffers are sized for (an image in [0, 40],
    sigma_r = 0.5: about 160 range cells in chunks of 9 levels) is filtered chunk by chunk on the
    device and still matches the FP64 oracle."""
    f = (40.0 * _img(48, 64, 1, seed=11)).astype(np.float32)
    check_grid_pass(h, f, 20.0, 3.0, 0.5)


def test_grid_range_beyond_the_cell_cap_gives_nan(h):
    """A range of more than BLFLS_GRID_MAX_RANGE_CELLS cells of sigma_r cannot be gridded: the
    call (which never reads the range back) succeeds and the channel's output is NaN; a channel
    within the cap beside it is unaffected."""
    f = _img(32, 32, 2, seed=4)
    f[1] *= 1e-6                                    # channel 1: range about 2e-6 -> 2 cells
    got = _grid(h, f, 20.0, 2.0, 1e-9)
    assert np.isnan(got[0]).all()
    np.testing.assert_array_equal(got[1], _grid(h, f[1:], 20.0, 2.0, 1e-9)[0])
    assert np.isfinite(got[1]).all()


def test_grid_does_not_wait_for_the_stream(h):
    """The ranges stay on the device: the call returns while the stream is still busy, and the
    result is the same as a call on an idle stream."""
    f = _img(96, 128, 3, seed=6)
    want = _grid(h, f, 20.0, 3.0, 0.1, 2)
    x = to_dev(f)
    out = torch.empty_like(x)
    torch.cuda.synchronize(DEV)
    s = stream()
    torch.cuda._sleep(200_000_000)                        # ~0.1 s of spinning on the stream
    blfls.blfls_smooth_grid(h, x, out, 96, 128, 3, 20.0, 3.0, 0.1, 2, s)
    done = torch.cuda.Event()
    done.record(s)
    assert not done.query(), "the call waited for the stream"
    torch.cuda.synchronize(DEV)
    np.testing.assert_array_equal(out.cpu().numpy(), want)
