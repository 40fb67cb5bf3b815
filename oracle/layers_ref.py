"""TEST INFRASTRUCTURE ONLY -- FP64 oracle of the LS model and of the base/detail applications.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this module.  It shares no code with the CUDA path and never calls it.

* ``ls``: the un-weighted least-squares smoother of Section II-B, Eq. 5, solved in the Fourier
  domain as Eq. 6: u = F^-1[ F(f) / (F(1) + lam (conj F(d_x) F(d_x) + conj F(d_y) F(d_y))) ],
  with the same periodic forward differences and DFT conventions as the BLF-LS oracle.
* ``detail_enhance``: Section IV, image detail enhancement: the detail layer f - u (input minus
  its smoothed version) is magnified and added back to the input.  Reading: out = f + m (f - u)
  with the magnification m >= 0 given by the caller (m = 0 returns f).
* ``log_tone``: Section IV, HDR tone mapping in the layer framework the paper adopts
  (decomposition of the logarithmic image into a smoothed base and a detail layer, the base
  compressed, the layers recombined).  Reading: l = ln(max(f, floor)), b = BLFLS(l),
  out = exp(c b + (l - b)) with the base compression factor c in (0, 1] given by the caller;
  no further normalisation (the caller rescales the result for display).
"""
from __future__ import annotations

import numpy as np

from .blfls_ref import blfls, difference_otfs


def ls_channel(f: np.ndarray, lam: float) -> np.ndarray:
    """One pass of Eq. 6 on one channel (FP64)."""
    f = np.asarray(f, dtype=np.float64)
    H, W = f.shape
    fdx, fdy = difference_otfs(H, W)
    den = 1.0 + lam * (np.conj(fdx) * fdx + np.conj(fdy) * fdy)   # F(1) = 1
    u = np.fft.ifft2(np.fft.fft2(f) / den)
    scale = max(1.0, float(np.max(np.abs(u.real))) if u.size else 1.0)
    if u.size and float(np.max(np.abs(u.imag))) > 1e-10 * scale:
        raise AssertionError("Eq. 6 solve left an imaginary residual above FP64 rounding")
    return u.real


def ls(img: np.ndarray, lam: float, iters: int = 1) -> np.ndarray:
    """The LS model (Eqs. 5-6) on a [C, H, W] (or [H, W]) image, applied ``iters`` times."""
    a = np.asarray(img, dtype=np.float64)
    squeeze = a.ndim == 2
    if squeeze:
        a = a[None]
    u = a.copy()
    for _ in range(int(iters)):
        u = np.stack([ls_channel(u[c], lam) for c in range(u.shape[0])])
    return u[0] if squeeze else u


def detail_enhance(img: np.ndarray, lam: float, sigma_s: float, sigma_r: float, radius: int,
                   iters: int, strength: float, threads: int | None = None) -> np.ndarray:
    """out = f + m (f - u), u = BLF-LS^iters(f)."""
    f = np.asarray(img, dtype=np.float64)
    u = blfls(f, lam, sigma_s, sigma_r, radius, iters, threads)
    return f + float(strength) * (f - u)


def log_tone(img: np.ndarray, lam: float, sigma_s: float, sigma_r: float, radius: int,
             iters: int, compression: float, floor: float = 1e-6,
             threads: int | None = None) -> np.ndarray:
    """l = ln(max(f, floor)); b = BLF-LS^iters(l); out = exp(c b + (l - b))."""
    f = np.asarray(img, dtype=np.float64)
    lg = np.log(np.maximum(f, floor))
    b = blfls(lg, lam, sigma_s, sigma_r, radius, iters, threads)
    return np.exp(float(compression) * b + (lg - b))


__all__ = ["ls_channel", "ls", "detail_enhance", "log_tone"]
