"""TEST INFRASTRUCTURE ONLY -- FP64 oracle of NC-LS: BLF-LS with the bilateral filter replaced by
the normalised-convolution filter of the domain transform (Section III-D).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this module.  It shares no code with the CUDA path and never calls it.

The paper names the filter (the normalised convolution of Gastal and Oliveira's domain
transform) and embeds it in place of the BLF; its steps, restated here:

* the domain transform of a 1-D signal s is the running sum
  ct[i] = sum_{j = 1..i} (1 + (sigma_s / sigma_r) |s[j] - s[j-1]|), ct[0] = 0;
* one normalised-convolution pass with radius r averages, for every sample i, the samples j with
  |ct[i] - ct[j]| <= r (a box of radius r in the transformed domain);
* N iterations; iteration k (1-based) uses sigma_k = sigma_s sqrt(3) 2^(N-k) / sqrt(4^N - 1) and
  r_k = sigma_k sqrt(3), first along every row, then along every column.

Readings (listed in the design notes): each gradient field is filtered with its own domain
transform (rows: the transform of each row of that field; columns: of each column), computed
once from the unfiltered field and used in every iteration; rows and columns are periodic -- the
copy of a row one period to the right sits at ct + T, T = ct[W-1] + 1 + a |s[0] - s[W-1]|; N = 3
by default.

Which samples enter a box must not depend on rounding order, so the transform is kept exact:
FP32 gradients; each increment 1 + a |ds| with a = sigma_s / sigma_r (FP32 division) is one FP32
multiply then one add (no fused multiply-add), capped at 2^20 (an increment beyond every box
radius separates the samples either way, so no decision changes); an FP32 value >= 1 is a
multiple of 2^-23, so ct and T are held exactly as integers in units of 2^-23 and summed in any
order; r_k is computed in FP64 and rounded to FP32; the test |(ct[j] + k T) - ct[i]| <= r_k is
then an exact comparison.  The averaged values are FP64.
"""
from __future__ import annotations

import math

import numpy as np

from .blfls_ref import gradients, solve_eq8

UNIT = 2 ** 23           # the transform is held in integer units of 2^-23
INC_CAP = 2.0 ** 20      # increments are capped here (beyond every box radius)


def nc_schedule(sigma_s: float, n_iter: int) -> list[float]:
    """Box radii r_k = sigma_k sqrt(3) of the N iterations (FP64)."""
    N = int(n_iter)
    return [sigma_s * math.sqrt(3.0) * 2.0 ** (N - k) / math.sqrt(4.0 ** N - 1.0) * math.sqrt(3.0)
            for k in range(1, N + 1)]


def _increments(s_hi: np.ndarray, s_lo: np.ndarray, a32: np.float32) -> np.ndarray:
    """FP32 increments 1 + a |s_hi - s_lo| (multiply, then add), capped, as exact int64 units."""
    d = np.float32(1.0) + a32 * np.abs(s_hi - s_lo)
    d = np.minimum(d, np.float32(INC_CAP))
    return (d.astype(np.float64) * UNIT).astype(np.int64)


def domain_transform(s: np.ndarray, a, axis: int) -> tuple[np.ndarray, np.ndarray]:
    """Periodic domain transform along `axis` (see the module notes): ct (same shape) and the
    period T (one per line), both int64 in units of 2^-23."""
    s32 = np.moveaxis(np.asarray(s, dtype=np.float32), axis, -1)
    a32 = np.float32(a)
    D = _increments(s32[..., 1:], s32[..., :-1], a32)
    ct = np.zeros(s32.shape, dtype=np.int64)
    ct[..., 1:] = np.cumsum(D, axis=-1)
    T = ct[..., -1] + _increments(s32[..., 0], s32[..., -1], a32)
    return np.moveaxis(ct, -1, axis), T


def nc_pass(v: np.ndarray, ct: np.ndarray, T: np.ndarray, r: float, axis: int) -> np.ndarray:
    """One normalised-convolution pass of radius r along `axis` with periodic lines; the
    inclusion test exact on the integer transform."""
    v = np.moveaxis(np.asarray(v, dtype=np.float64), axis, -1)
    c = np.moveaxis(np.asarray(ct, dtype=np.int64), axis, -1)
    T = np.asarray(T, dtype=np.int64)
    r32 = np.float32(r)
    r_units = int(math.floor(float(r32) * UNIT))   # |L| <= r  <=>  |L| <= floor(r 2^23) for integer L
    n = v.shape[-1]
    R = int(math.floor(r32))        # ct grows by >= 1 per sample, so |i - j| <= r
    acc = np.zeros_like(v)
    cnt = np.zeros_like(v)
    idx = np.arange(n)
    for d in range(-R, R + 1):
        j = idx + d
        wraps = np.floor_divide(j, n)              # which period the neighbour sits in
        jm = j - wraps * n
        cj = c[..., jm] + wraps * T[..., None]
        inside = np.abs(cj - c) <= r_units
        acc += np.where(inside, v[..., jm], 0.0)
        cnt += inside
    return np.moveaxis(acc / cnt, -1, axis)


def nc_filter(g: np.ndarray, sigma_s: float, sigma_r: float, n_iter: int = 3) -> np.ndarray:
    """The domain-transform normalised convolution of one field, guided by itself."""
    g = np.asarray(g, dtype=np.float64)
    ss32, sr32 = np.float32(sigma_s), np.float32(sigma_r)
    a = ss32 / sr32 if math.isfinite(sr32) else np.float32(0.0)
    ct_h, T_h = domain_transform(g, a, axis=1)
    ct_v, T_v = domain_transform(g, a, axis=0)
    v = g.copy()
    for r in nc_schedule(float(ss32), n_iter):
        v = nc_pass(v, ct_h, T_h, r, axis=1)
        v = nc_pass(v, ct_v, T_v, r, axis=0)
    return v


def ncls(img: np.ndarray, lam: float, sigma_s: float, sigma_r: float, iters: int = 1,
         n_iter: int = 3) -> np.ndarray:
    """NC-LS: gradients -> NC filter on each field -> Eq. 8, per channel, `iters` times."""
    a = np.asarray(img, dtype=np.float64)
    squeeze = a.ndim == 2
    if squeeze:
        a = a[None]
    u = a.copy()
    for _ in range(int(iters)):
        chans = []
        for c in range(u.shape[0]):
            gx, gy = gradients(u[c])
            chans.append(solve_eq8(u[c], nc_filter(gx, sigma_s, sigma_r, n_iter),
                                   nc_filter(gy, sigma_s, sigma_r, n_iter), lam))
        u = np.stack(chans)
    return u[0] if squeeze else u
