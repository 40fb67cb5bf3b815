"""TEST INFRASTRUCTURE ONLY -- FP64 oracle of the bilateral-grid approximation of the BLF and of
BLF-LS built on it.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this module.  It shares no code with the CUDA path and never calls it.

The paper computes the BLF of Eq. 1 with the fast approximation of Paris and Durand
(Section III-A and IV): the signal is lifted into a coarse 3-D grid (two spatial axes and the
range axis), blurred there with a small Gaussian, and read back by interpolation.  The paper
gives no further detail, so this oracle fixes the steps (listed as readings in the design
notes), for one field g of size H x W with spatial and range parameters sigma_s, sigma_r:

1. sampling steps s_s = sigma_s (space) and s_r = sigma_r (range); padding P = 2 cells;
   grid sizes Gx = floor((W - 1) / s_s) + 1 + 2P, Gy likewise with H,
   Gz = floor((max g - min g) / s_r) + 1 + 2P;
2. splat: pixel (x, y) adds (g, 1) to the cell (round(z), round(y / s_s) + P,
   round(x / s_s) + P) with z = (g - min g) / s_r + P, round(t) = floor(t + 1/2);
3. blur both grids with the 3-tap kernel (exp(-1/2), 1, exp(-1/2)) (a Gaussian of one cell)
   along x, then y, then z, zero outside the grid;
4. slice: trilinear interpolation of both grids at (z, y / s_s + P, x / s_s + P);
   v = (interpolated sum of g) / (interpolated count).

Image borders are open (the grid is not periodic), as in the grid method itself.

Everything is FP64 on the values as given: the gradients are the exact FP64 differences of the
input, min g their exact minimum, and the cell of a pixel is floor(t + 1/2) of the FP64 value of
t.  sigma_s and sigma_r enter as the FP32 values the C interface receives.

A cell is an integer decided by a real number, so an implementation that holds the gradients in
a narrower type can land on the other side of a rounding boundary when t is within that type's
rounding of it.  ``grid_z_coords`` exposes the FP64 range coordinate t of every pixel (so a test
can find those pixels) and ``blf_grid`` / ``blfls_grid`` accept ``flip`` masks that put the
marked pixels in the other candidate cell (the neighbour across the nearest boundary), so a test
can evaluate the definition with either decision.
"""
from __future__ import annotations

import math

import numpy as np

from .blfls_ref import gradients, solve_eq8

PAD = 2
_EDGE = math.exp(-0.5)


def _params(sigma_s: float, sigma_r: float) -> tuple[float, float]:
    """sigma_s, sigma_r as the FP32 values the C interface receives, widened to FP64."""
    return float(np.float32(sigma_s)), float(np.float32(sigma_r))


def grid_shape(H: int, W: int, lo: float, hi: float, sigma_s: float, sigma_r: float):
    gx = int(math.floor((W - 1) / sigma_s)) + 1 + 2 * PAD
    gy = int(math.floor((H - 1) / sigma_s)) + 1 + 2 * PAD
    gz = int(math.floor((hi - lo) / sigma_r)) + 1 + 2 * PAD
    return gz, gy, gx


def grid_z_coords(g: np.ndarray, sigma_r: float) -> tuple[np.ndarray, float]:
    """The FP64 range coordinate t = (g - min g) / s_r + 1/2 whose floor is a pixel's range cell
    (before the padding), and min g."""
    g = np.asarray(g, dtype=np.float64)
    _, sr = _params(1.0, sigma_r)
    lo = float(g.min())
    return (g - lo) / sr + 0.5, lo


def _flipped_cell(t: np.ndarray) -> np.ndarray:
    """The other candidate cell of a coordinate near a rounding boundary: the neighbour of
    floor(t) across the nearest integer."""
    n = np.floor(t)
    near = np.rint(t)
    return np.where(n == near, n - 1.0, n + 1.0)


def _blur_axis(a: np.ndarray, axis: int) -> np.ndarray:
    out = a.copy()
    n = a.shape[axis]
    lo = [slice(None)] * a.ndim
    hi = [slice(None)] * a.ndim
    # out[i] += e * a[i-1] + e * a[i+1], zero outside
    lo[axis] = slice(1, n)
    hi[axis] = slice(0, n - 1)
    out[tuple(lo)] += _EDGE * a[tuple(hi)]
    out[tuple(hi)] += _EDGE * a[tuple(lo)]
    return out


def _trilinear(grid: np.ndarray, z: np.ndarray, y: np.ndarray, x: np.ndarray) -> np.ndarray:
    z0, y0, x0 = np.floor(z).astype(int), np.floor(y).astype(int), np.floor(x).astype(int)
    fz, fy, fx = z - z0, y - y0, x - x0
    out = np.zeros_like(z)
    for dz in (0, 1):
        wz = fz if dz else 1.0 - fz
        for dy in (0, 1):
            wy = fy if dy else 1.0 - fy
            for dx in (0, 1):
                wx = fx if dx else 1.0 - fx
                out += wz * wy * wx * grid[z0 + dz, y0 + dy, x0 + dx]
    return out


def blf_grid(g: np.ndarray, sigma_s: float, sigma_r: float,
             flip: np.ndarray | None = None) -> np.ndarray:
    """The bilateral-grid approximation of Eq. 1 on one field (FP64).  `flip` (bool, H x W)
    puts the marked pixels in their other candidate range cell (see the module notes)."""
    g = np.asarray(g, dtype=np.float64)
    H, W = g.shape
    ss, sr = _params(sigma_s, sigma_r)
    t, lo = grid_z_coords(g, sr)
    hi = float(g.max())
    gz, gy, gx = grid_shape(H, W, lo, hi, ss, sr)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    zc = np.floor(t)
    if flip is not None:
        zc = np.where(flip, _flipped_cell(t), zc)
        gz = max(gz, int(zc.max()) + 1 + 2 * PAD)   # a flip upwards may need one more cell
    cz = zc.astype(int) + PAD
    cy = np.floor(yy / ss + 0.5).astype(int) + PAD
    cx = np.floor(xx / ss + 0.5).astype(int) + PAD
    zf = t - 0.5 + PAD
    yf = yy / ss + PAD
    xf = xx / ss + PAD
    wi = np.zeros((gz, gy, gx))
    w = np.zeros((gz, gy, gx))
    np.add.at(wi, (cz, cy, cx), g)
    np.add.at(w, (cz, cy, cx), 1.0)
    for axis in (2, 1, 0):
        wi = _blur_axis(wi, axis)
        w = _blur_axis(w, axis)
    return _trilinear(wi, zf, yf, xf) / _trilinear(w, zf, yf, xf)


def blfls_grid(img: np.ndarray, lam: float, sigma_s: float, sigma_r: float,
               iters: int = 1, flips: np.ndarray | None = None) -> np.ndarray:
    """BLF-LS with the grid BLF on each gradient field, then Eq. 8 (periodic solve).
    `flips` (bool [C][2][H][W], one pass only) marks, per channel and field (x, y), the pixels
    whose range cell takes the other candidate."""
    a = np.asarray(img, dtype=np.float64)
    squeeze = a.ndim == 2
    if squeeze:
        a = a[None]
    if flips is not None and int(iters) != 1:
        raise ValueError("flips apply to one pass")
    u = a.copy()
    for _ in range(int(iters)):
        chans = []
        for c in range(u.shape[0]):
            gx, gy = gradients(u[c])
            fx = None if flips is None else flips[c][0]
            fy = None if flips is None else flips[c][1]
            chans.append(solve_eq8(u[c], blf_grid(gx, sigma_s, sigma_r, fx),
                                   blf_grid(gy, sigma_s, sigma_r, fy), lam))
        u = np.stack(chans)
    return u[0] if squeeze else u
