"""TEST INFRASTRUCTURE ONLY -- FP64 oracle of joint (guided) BLF-LS and rolling guidance.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this module.  It shares no code with the CUDA path and never calls it.

Section III-D (model extensions):
* joint filtering, as the joint bilateral filter does: the range weights of the bilateral filter
  come from the gradients of another (guidance) image, while the values averaged are still the
  input's gradients.  Per field: v[s] = sum_t w_st g[t] / sum_t w_st with
  w_st = G_ss(|s - t|) G_sr(h[s] - h[t]), g = D f (input), h = D guide (same field);
* rolling guidance: the input is smoothed jointly again and again, each pass guided by the
  previous pass's output; the first guidance is the input smoothed by a Gaussian of standard
  deviation sigma.

Readings (listed in the design notes): G_sigma(x) = exp(-x^2 / (2 sigma^2)), square periodic
window of radius r as in the plain smoother; the initial Gaussian is periodic, truncated at
radius ceil(3 sigma) and normalised to sum 1, applied along rows then columns; a rolling pass
takes its data term and averaged gradients from the input f, and only the guidance from the
previous output; a joint (non-rolling) pass k > 1 smooths u_(k-1) with the fixed guidance.
"""
from __future__ import annotations

import math

import numpy as np

from .blfls_ref import gradients, solve_eq8


def blf_joint(g: np.ndarray, h: np.ndarray, radius: int, sigma_s: float,
              sigma_r: float) -> np.ndarray:
    """Joint bilateral filter of the field g with range weights from the field h (FP64)."""
    g = np.asarray(g, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    acc = np.zeros_like(g)
    z = np.zeros_like(g)
    for dy in range(-radius, radius + 1):
        for dx in range(-radius, radius + 1):
            # t = s + (dy, dx): rolling by (-dy, -dx) brings t's value to s
            gt = np.roll(g, (-dy, -dx), axis=(0, 1))
            ht = np.roll(h, (-dy, -dx), axis=(0, 1))
            ws = math.exp(-(dx * dx + dy * dy) / (2.0 * sigma_s * sigma_s)) if math.isfinite(sigma_s) else 1.0
            wr = np.exp(-(h - ht) ** 2 / (2.0 * sigma_r * sigma_r)) if math.isfinite(sigma_r) else 1.0
            w = ws * wr
            acc += w * gt
            z += w
    return acc / z


def blfls_joint_channel(f: np.ndarray, guide: np.ndarray, lam: float, sigma_s: float,
                        sigma_r: float, radius: int) -> np.ndarray:
    gx, gy = gradients(f)
    hx, hy = gradients(guide)
    vx = blf_joint(gx, hx, radius, sigma_s, sigma_r)
    vy = blf_joint(gy, hy, radius, sigma_s, sigma_r)
    return solve_eq8(f, vx, vy, lam)


def _chw(a):
    a = np.asarray(a, dtype=np.float64)
    return (a[None], True) if a.ndim == 2 else (a, False)


def blfls_joint(img: np.ndarray, guide: np.ndarray, lam: float, sigma_s: float, sigma_r: float,
                radius: int, iters: int = 1) -> np.ndarray:
    """Joint BLF-LS with a fixed guidance image ([C,H,W] or [1,H,W] shared by every channel);
    pass k smooths u_(k-1)."""
    u, squeeze = _chw(img)
    gd, _ = _chw(guide)
    u = u.copy()
    for _ in range(int(iters)):
        u = np.stack([blfls_joint_channel(u[c], gd[c if gd.shape[0] > 1 else 0], lam, sigma_s,
                                          sigma_r, radius) for c in range(u.shape[0])])
    return u[0] if squeeze else u


def gaussian_weights(sigma: float) -> np.ndarray:
    """Normalised taps exp(-x^2 / (2 sigma^2)), |x| <= ceil(3 sigma)."""
    R = int(math.ceil(3.0 * sigma))
    x = np.arange(-R, R + 1, dtype=np.float64)
    w = np.exp(-x * x / (2.0 * sigma * sigma))
    return w / w.sum()


def gaussian(img: np.ndarray, sigma: float) -> np.ndarray:
    """Periodic separable Gaussian blur, rows then columns (FP64)."""
    a, squeeze = _chw(img)
    w = gaussian_weights(sigma)
    R = (w.size - 1) // 2
    rows = np.zeros_like(a)
    for k in range(-R, R + 1):
        rows += w[k + R] * np.roll(a, -k, axis=2)
    out = np.zeros_like(a)
    for k in range(-R, R + 1):
        out += w[k + R] * np.roll(rows, -k, axis=1)
    return out[0] if squeeze else out


def blfls_rolling(img: np.ndarray, lam: float, sigma_s: float, sigma_r: float, radius: int,
                  iters: int, sigma_g: float) -> np.ndarray:
    """Rolling guidance: guide_1 = gaussian(f, sigma_g); u_k = joint BLF-LS(f; guide_k);
    guide_(k+1) = u_k.  Returns u_iters (f for iters = 0)."""
    f, squeeze = _chw(img)
    guide = gaussian(f, sigma_g)
    u = f.copy()
    for _ in range(int(iters)):
        u = blfls_joint(f, guide, lam, sigma_s, sigma_r, radius, 1)
        guide = u
    return u[0] if squeeze else u
