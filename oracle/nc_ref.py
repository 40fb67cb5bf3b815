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
line continues into its next period, whose first step is 1 + a |s[0] - s[W-1]|; N = 3 by
default.

Everything is FP64: the gradients are the exact FP64 differences of the input, a = sigma_s /
sigma_r is the FP64 quotient of the FP32 parameters the C interface receives, every increment is
1 + a |s[j] - s[j-1]| in FP64, and the transform distance between i and j is the sum of the
increments between them (ct[j] - ct[i] written out, so it carries the rounding of a few terms,
not of a whole line's running sum).

Box membership is a decision taken on a real number: an implementation that rounds the
increments can land on the other side of |ct[j] - ct[i]| = r when the distance is within that
rounding of r.  ``nc_margins`` exposes, for every iteration, axis, sample and offset, the FP64
value of |ct[j] - ct[i]| - r (so a test can find those decisions), and ``nc_filter`` / ``ncls``
accept ``flips`` that reverse the marked decisions, so a test can evaluate the definition with
either one.
"""
from __future__ import annotations

import math

import numpy as np

from .blfls_ref import gradients, solve_eq8


def nc_schedule(sigma_s: float, n_iter: int) -> list[float]:
    """Box radii r_k = sigma_k sqrt(3) of the N iterations (FP64)."""
    N = int(n_iter)
    return [sigma_s * math.sqrt(3.0) * 2.0 ** (N - k) / math.sqrt(4.0 ** N - 1.0) * math.sqrt(3.0)
            for k in range(1, N + 1)]


def _params(sigma_s: float, sigma_r: float) -> tuple[float, float]:
    """sigma_s and a = sigma_s / sigma_r from the FP32 values the C interface receives."""
    ss, sr = float(np.float32(sigma_s)), float(np.float32(sigma_r))
    return ss, (ss / sr if math.isfinite(sr) else 0.0)


def increments(s: np.ndarray, a: float, axis: int) -> np.ndarray:
    """inc[p] = 1 + a |s[p] - s[p-1]| along `axis` (periodic: inc[0] joins the previous period's
    last sample to sample 0), FP64."""
    s = np.asarray(s, dtype=np.float64)
    return 1.0 + a * np.abs(s - np.roll(s, 1, axis=axis))


def domain_transform(s: np.ndarray, a: float, axis: int) -> tuple[np.ndarray, np.ndarray]:
    """Running sum ct (ct = 0 at the first sample) and period T of each line along `axis`
    (FP64)."""
    inc = np.moveaxis(increments(s, a, axis), axis, -1)
    ct = np.zeros_like(inc)
    ct[..., 1:] = np.cumsum(inc[..., 1:], axis=-1)
    T = ct[..., -1] + inc[..., 0]
    return np.moveaxis(ct, -1, axis), T


def _distances(inc: np.ndarray, R: int):
    """Yields (d, dist) and (-d, dist') for d = 1..R: dist[..., i] = |ct(i + d) - ct(i)|, the sum
    of the d increments into samples i+1 .. i+d along the last axis (periodic), and
    dist'[..., i] = |ct(i - d) - ct(i)|, the same sum for the pair (i - d, i), so both ends of a
    pair see the same number."""
    acc = np.zeros_like(inc)
    for d in range(1, R + 1):
        acc = acc + np.roll(inc, -d, axis=-1)       # + inc[i + d]
        yield d, acc
        yield -d, np.roll(acc, d, axis=-1)          # the pair (i - d, i)


def nc_pass(v: np.ndarray, inc: np.ndarray, r: float, axis: int,
            flip: dict | None = None) -> np.ndarray:
    """One normalised-convolution pass of radius r along `axis` with periodic lines, given the
    line's increments `inc` (see ``increments``).  `flip` maps an offset d to a bool array (the
    shape of v) of decisions to reverse."""
    v = np.moveaxis(np.asarray(v, dtype=np.float64), axis, -1)
    inc = np.moveaxis(np.asarray(inc, dtype=np.float64), axis, -1)
    R = int(math.floor(r))          # every increment is >= 1, so only |d| <= r can be inside
    acc = v.copy()
    cnt = np.ones_like(v)
    for d, dist in _distances(inc, R):
        inside = dist <= r
        if flip is not None and d in flip:
            inside = inside ^ np.moveaxis(flip[d], axis, -1)
        vj = np.roll(v, -d, axis=-1)                 # v[i + d], periodic
        acc += np.where(inside, vj, 0.0)
        cnt += inside
    return np.moveaxis(acc / cnt, -1, axis)


def nc_margins(g: np.ndarray, sigma_s: float, sigma_r: float, n_iter: int = 3):
    """For iteration k (1-based), axis (1 rows, 0 columns) and offset d: the FP64 margin
    |ct(i + d) - ct(i)| - r_k of every sample i (the shape of g).  Yields (k, axis, d, margin)."""
    g = np.asarray(g, dtype=np.float64)
    ss, a = _params(sigma_s, sigma_r)
    incs = {1: increments(g, a, 1), 0: increments(g, a, 0)}
    for k, r in enumerate(nc_schedule(ss, n_iter), start=1):
        for axis in (1, 0):
            inc = np.moveaxis(incs[axis], axis, -1)
            for d, dist in _distances(inc, int(math.floor(r))):
                yield k, axis, d, np.moveaxis(dist - r, -1, axis)


def nc_filter(g: np.ndarray, sigma_s: float, sigma_r: float, n_iter: int = 3,
              flips: dict | None = None) -> np.ndarray:
    """The domain-transform normalised convolution of one field, guided by itself.  `flips` maps
    (k, axis) to the `flip` argument of ``nc_pass`` for that iteration and axis."""
    g = np.asarray(g, dtype=np.float64)
    ss, a = _params(sigma_s, sigma_r)
    inc_h = increments(g, a, 1)
    inc_v = increments(g, a, 0)
    v = g.copy()
    for k, r in enumerate(nc_schedule(ss, n_iter), start=1):
        f_h = None if flips is None else flips.get((k, 1))
        f_v = None if flips is None else flips.get((k, 0))
        v = nc_pass(v, inc_h, r, axis=1, flip=f_h)
        v = nc_pass(v, inc_v, r, axis=0, flip=f_v)
    return v


def ncls(img: np.ndarray, lam: float, sigma_s: float, sigma_r: float, iters: int = 1,
         n_iter: int = 3, flips: list | None = None) -> np.ndarray:
    """NC-LS: gradients -> NC filter on each field -> Eq. 8, per channel, `iters` times.
    `flips` (one pass only): flips[c][field] is the `flips` argument of ``nc_filter`` for that
    channel and field (x = 0, y = 1), or None."""
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
            chans.append(solve_eq8(u[c], nc_filter(gx, sigma_s, sigma_r, n_iter, fx),
                                   nc_filter(gy, sigma_s, sigma_r, n_iter, fy), lam))
        u = np.stack(chans)
    return u[0] if squeeze else u
