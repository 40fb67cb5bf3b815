"""TEST INFRASTRUCTURE ONLY -- the plain, slow FP64 oracle of the BLF-LS smoother.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this module.  It shares no code with the CUDA path and never calls it.

What it computes, step by step in the paper's order (Section III-A, "two steps"):

1. gradients ``g_x = D_x f``, ``g_y = D_y f`` with the periodic forward differences of
   Section II-B (Eq. 4: D_x, D_y forward; their transposes backward differences);
2. ``v_* = f_BLF(g_*)``: the brute-force bilateral filter of Eq. 1 on each gradient field
   (C, ``blf_ref.c``);
3. the closed-form minimiser of Eq. 7 given by Eq. 8:
       u = F^-1[ (F(f) + lam * sum_* conj(F(d_*)) F(v_*)) / (F(1) + lam * sum_* conj(F(d_*)) F(d_*)) ]
   with three forward 2-D DFTs and one inverse (NumPy's FFT serves as the DFT; F(1) = 1 is the
   transform of the unit impulse, Eq. 6).

Readings of points the paper leaves open (each also listed in the design notes):
* F(d_x)(k) = exp(2 pi i k_x / W) - 1, the transfer function of the same forward difference
  used in step 1 under NumPy's sign convention F(k) = sum_n x_n exp(-2 pi i k n / N);
* unnormalised forward DFT, 1/(HW) on the inverse;
* ``iters`` applies the whole smoother repeatedly, u_k = BLFLS(u_{k-1}) (the paper defines one
  pass; iteration appears only in its rolling-guidance extension, Section III-D);
* channels are smoothed independently; no clamping of the output.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.oracle_blf_f64.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_int]
        lib.oracle_blf_f64.restype = ctypes.c_int
        lib.oracle_blf_at_f64.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_double, ctypes.c_double, ip, ip,
                                          ctypes.c_int, dp, ctypes.c_int]
        lib.oracle_blf_at_f64.restype = ctypes.c_int
        _LIB = lib
    return _LIB


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


# --------------------------------------------------------------------------------------------
# Step 1: periodic forward differences (Section II-B, Eq. 4 operators; used in Eq. 7)
# --------------------------------------------------------------------------------------------
def gradients(f: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """g_x[y,x] = f[y, x+1 mod W] - f[y,x];  g_y[y,x] = f[y+1 mod H, x] - f[y,x]."""
    f = np.asarray(f, dtype=np.float64)
    gx = np.roll(f, -1, axis=1) - f
    gy = np.roll(f, -1, axis=0) - f
    return gx, gy


# --------------------------------------------------------------------------------------------
# Step 2: brute-force bilateral filter (Section II-A, Eq. 1)
# --------------------------------------------------------------------------------------------
def blf(g: np.ndarray, radius: int, sigma_s: float, sigma_r: float,
        threads: int | None = None) -> np.ndarray:
    """v = f_BLF(g) over the square periodic window of the given radius (FP64)."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    H, W = g.shape
    v = np.empty_like(g)
    rc = _lib().oracle_blf_f64(_dptr(g), _dptr(v), H, W, int(radius), float(sigma_s),
                               float(sigma_r), int(threads or default_threads()))
    if rc != 0:
        raise ValueError("oracle_blf_f64 rejected its arguments")
    return v


def blf_at(g: np.ndarray, radius: int, sigma_s: float, sigma_r: float, ys, xs,
           threads: int | None = None) -> np.ndarray:
    """f_BLF(g) evaluated only at the pixels (ys[i], xs[i])."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    H, W = g.shape
    ys = np.ascontiguousarray(ys, dtype=np.int32)
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    out = np.empty(ys.shape[0], dtype=np.float64)
    rc = _lib().oracle_blf_at_f64(_dptr(g), H, W, int(radius), float(sigma_s),
                                  float(sigma_r), _iptr(ys), _iptr(xs), int(ys.shape[0]),
                                  _dptr(out), int(threads or default_threads()))
    if rc != 0:
        raise ValueError("oracle_blf_at_f64 rejected its arguments")
    return out


# --------------------------------------------------------------------------------------------
# Step 3: Fourier-domain least-squares solve (Eq. 8; Eq. 6 when v = 0)
# --------------------------------------------------------------------------------------------
def difference_otfs(H: int, W: int) -> tuple[np.ndarray, np.ndarray]:
    """Transfer functions of the periodic forward differences: F(d_x) of shape (1, W) and
    F(d_y) of shape (H, 1), so that F(D_x f) = F(d_x) * F(f)."""
    kx = np.arange(W, dtype=np.float64)
    ky = np.arange(H, dtype=np.float64)
    fdx = np.exp(2j * math.pi * kx / W) - 1.0
    fdy = np.exp(2j * math.pi * ky / H) - 1.0
    return fdx[None, :], fdy[:, None]


def solve_eq8(f: np.ndarray, vx: np.ndarray, vy: np.ndarray, lam: float) -> np.ndarray:
    """u = F^-1[(F f + lam (conj(F d_x) F v_x + conj(F d_y) F v_y)) /
                (1 + lam (|F d_x|^2 + |F d_y|^2))]   (Eq. 8, literal: three forward DFTs)."""
    f = np.asarray(f, dtype=np.float64)
    H, W = f.shape
    fdx, fdy = difference_otfs(H, W)
    Ff = np.fft.fft2(f)
    Fvx = np.fft.fft2(np.asarray(vx, dtype=np.float64))
    Fvy = np.fft.fft2(np.asarray(vy, dtype=np.float64))
    num = Ff + lam * (np.conj(fdx) * Fvx + np.conj(fdy) * Fvy)
    den = 1.0 + lam * (np.conj(fdx) * fdx + np.conj(fdy) * fdy)
    u = np.fft.ifft2(num / den)
    scale = max(1.0, float(np.max(np.abs(u.real))) if u.size else 1.0)
    if u.size and float(np.max(np.abs(u.imag))) > 1e-10 * scale:
        raise AssertionError("Eq. 8 solve left an imaginary residual above FP64 rounding")
    return u.real


def blf_field(g: np.ndarray, radius: int, sigma_s: float, sigma_r: float,
              threads: int | None = None, normalize: bool = False) -> np.ndarray:
    """Eq. 1 on one gradient field.  With `normalize` (Section IV normalises images and gradients
    to [0, 1]) the field is mapped to [0, 1] by (g - min) / (max - min), filtered, and mapped
    back; a constant field is returned unchanged."""
    if not normalize:
        return blf(g, radius, sigma_s, sigma_r, threads)
    lo, hi = float(np.min(g)), float(np.max(g))
    if hi == lo:
        return np.array(g, dtype=np.float64)
    return blf((g - lo) / (hi - lo), radius, sigma_s, sigma_r, threads) * (hi - lo) + lo


def blfls_channel(f: np.ndarray, lam: float, sigma_s: float, sigma_r: float, radius: int,
                  threads: int | None = None, normalize_grad: bool = False) -> np.ndarray:
    """One BLF-LS pass on one channel: gradients -> BLF on each -> Eq. 8 (with
    `normalize_grad`, each field normalised to [0, 1] around its filter)."""
    gx, gy = gradients(f)
    vx = blf_field(gx, radius, sigma_s, sigma_r, threads, normalize_grad)
    vy = blf_field(gy, radius, sigma_s, sigma_r, threads, normalize_grad)
    return solve_eq8(f, vx, vy, lam)


def blfls(img: np.ndarray, lam: float, sigma_s: float, sigma_r: float, radius: int,
          iters: int = 1, threads: int | None = None, normalize_grad: bool = False) -> np.ndarray:
    """BLF-LS on a [C, H, W] (or [H, W]) image; returns FP64 of the same shape.

    ``iters`` repeats the whole smoother, u_k = BLFLS(u_{k-1}); iters = 0 returns the input.
    ``normalize_grad`` normalises every gradient field of every pass to [0, 1] around its filter
    (the setting of Section IV)."""
    a = np.asarray(img, dtype=np.float64)
    squeeze = a.ndim == 2
    if squeeze:
        a = a[None]
    u = a.copy()
    for _ in range(int(iters)):
        u = np.stack([blfls_channel(u[c], lam, sigma_s, sigma_r, radius, threads, normalize_grad)
                      for c in range(u.shape[0])])
    return u[0] if squeeze else u


def blf_residuals(img: np.ndarray, radius: int, sigma_s: float, sigma_r: float,
                  threads: int | None = None) -> tuple[np.ndarray, np.ndarray]:
    """Per channel: e_* = f_BLF(g_*) - g_*, the amount the bilateral filter moves each
    gradient field.  Shapes [C, H, W]."""
    a = np.asarray(img, dtype=np.float64)
    if a.ndim == 2:
        a = a[None]
    ex = np.empty_like(a)
    ey = np.empty_like(a)
    for c in range(a.shape[0]):
        gx, gy = gradients(a[c])
        ex[c] = blf(gx, radius, sigma_s, sigma_r, threads) - gx
        ey[c] = blf(gy, radius, sigma_s, sigma_r, threads) - gy
    return ex, ey
