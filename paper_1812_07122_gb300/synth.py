"""Seeded synthetic inputs shaped like the paper's smoothing workloads.

The paper evaluates on natural photographs, HDR images, flash/no-flash pairs and clip-art
(Section IV); none of them ship with it, so these generators stand in for them.  Every image is
built in FP64 from ``numpy.random.default_rng(seed)`` (PCG64), clipped to [0, 1] and cast to
FP32, so the FP64 oracle and the CUDA path read identical bits.

This module holds none of the smoothing method's arithmetic (no gradients, no bilateral
weights, no Fourier solve).  It is the one module shared by the oracle's tests and the CUDA
path's tests and benchmark.

Recipes
-------
* ``rectangles_image``: a background level U[0,1] and ``n_rect`` axis-aligned rectangles painted
  in order (later ones overwrite), corners drawn as integers in [0, W] x [0, H], levels U[0,1];
  additive N(0, noise^2); clip.  Piecewise-constant content with sharp edges (the clip-art and
  cartoon inputs of Section IV).
* ``sinusoid_disc_image``: per channel a sum of 8 periodic sinusoids with integer frequencies
  (kx, ky) in [-4, 4]^2 minus the origin, phases U[0, 2pi), amplitudes U[0,1], min-max rescaled to
  [0.2, 0.8]; then ``n_disc`` discs (centre uniform, radius log-uniform in [8, 200] px, one colour
  U[0,1]^C per disc); additive N(0, noise^2); clip.  Smooth shading plus strong edges plus
  texture-like noise (the detail-enhancement and tone-mapping inputs of Section IV).
* ``batch_jobs`` / ``serving_requests``: job lists with log-uniform sizes, mixed channel counts
  and per-job smoothing parameters, for the batched and served forms.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "rectangles_image",
    "sinusoid_disc_image",
    "image_256_rectangles",
    "image_4k_rgb",
    "Job",
    "batch_jobs",
    "serving_requests",
    "job_image",
]


def rectangles_image(H: int = 256, W: int = 256, n_rect: int = 12, noise: float = 0.05,
                     seed: int = 1) -> np.ndarray:
    """Grey piecewise-constant rectangles plus Gaussian noise; returns float32 [1, H, W]."""
    rng = np.random.default_rng(seed)
    img = np.full((H, W), rng.uniform(0.0, 1.0), dtype=np.float64)
    for _ in range(n_rect):
        while True:
            x0, x1 = np.sort(rng.integers(0, W + 1, size=2))
            y0, y1 = np.sort(rng.integers(0, H + 1, size=2))
            if x1 > x0 and y1 > y0:
                break
        img[y0:y1, x0:x1] = rng.uniform(0.0, 1.0)
    img += rng.normal(0.0, noise, size=(H, W))
    return np.clip(img, 0.0, 1.0).astype(np.float32)[None]


def _sinusoid_background(rng: np.random.Generator, H: int, W: int) -> np.ndarray:
    yy = np.arange(H, dtype=np.float64)[:, None] / H
    xx = np.arange(W, dtype=np.float64)[None, :] / W
    bg = np.zeros((H, W), dtype=np.float64)
    for _ in range(8):
        while True:
            kx, ky = rng.integers(-4, 5, size=2)
            if kx != 0 or ky != 0:
                break
        phase = rng.uniform(0.0, 2.0 * math.pi)
        amp = rng.uniform(0.0, 1.0)
        bg += amp * np.cos(2.0 * math.pi * (kx * xx + ky * yy) + phase)
    lo, hi = bg.min(), bg.max()
    if hi - lo < 1e-12:
        return np.full((H, W), 0.5)
    return 0.2 + 0.6 * (bg - lo) / (hi - lo)


def sinusoid_disc_image(H: int, W: int, C: int = 3, n_disc: int = 200, noise: float = 0.03,
                        seed: int = 2) -> np.ndarray:
    """Smooth periodic background + constant-colour discs + noise; float32 [C, H, W]."""
    rng = np.random.default_rng(seed)
    img = np.stack([_sinusoid_background(rng, H, W) for _ in range(C)])
    lo_r, hi_r = math.log(8.0), math.log(200.0)
    for _ in range(n_disc):
        cy, cx = rng.uniform(0, H), rng.uniform(0, W)
        rad = math.exp(rng.uniform(lo_r, hi_r))
        colour = rng.uniform(0.0, 1.0, size=C)
        y0, y1 = max(0, int(cy - rad)), min(H, int(cy + rad) + 1)
        x0, x1 = max(0, int(cx - rad)), min(W, int(cx + rad) + 1)
        if y1 <= y0 or x1 <= x0:
            continue
        yy = np.arange(y0, y1)[:, None] + 0.5 - cy
        xx = np.arange(x0, x1)[None, :] + 0.5 - cx
        mask = yy * yy + xx * xx <= rad * rad
        for c in range(C):
            img[c, y0:y1, x0:x1][mask] = colour[c]
    img += rng.normal(0.0, noise, size=img.shape)
    return np.clip(img, 0.0, 1.0).astype(np.float32)


def image_256_rectangles() -> np.ndarray:
    """The small grey workload: 256x256, 12 rectangles, noise 0.05, seed 1."""
    return rectangles_image(256, 256, 12, 0.05, seed=1)


def image_4k_rgb() -> np.ndarray:
    """The 4K workload: 3840x2160 RGB, sinusoids + 200 discs + noise 0.03, seed 2."""
    return sinusoid_disc_image(2160, 3840, 3, 200, 0.03, seed=2)


@dataclass
class Job:
    """One smoothing job: image shape, parameters and the seed of its image."""
    H: int
    W: int
    C: int
    lam: float
    sigma_s: float
    sigma_r: float
    radius: int
    iters: int = 1
    seed: int = 0
    arrival_s: float = 0.0
    meta: dict = field(default_factory=dict)

    @property
    def pixels(self) -> int:
        return self.H * self.W


def _log_uniform_int(rng: np.random.Generator, lo: int, hi: int) -> int:
    return int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))


def _draw_params(rng: np.random.Generator):
    lam = float(rng.uniform(5.0, 50.0))
    sigma_r = float(rng.uniform(0.05, 0.2))
    radius = int(rng.choice([3, 5, 8, 10]))
    return lam, radius / 2.0, sigma_r, radius


def batch_jobs(n: int = 64, seed: int = 4, h_range=(256, 1536), w_range=(256, 2048)) -> list[Job]:
    """Uneven batch: H, W log-uniform integers, C in {1, 3}, lambda~U[5,50],
    sigma_r~U[0.05,0.2], radius in {3,5,8,10}, sigma_s = radius/2, one iteration."""
    rng = np.random.default_rng(seed)
    jobs = []
    for i in range(n):
        H = _log_uniform_int(rng, *h_range)
        W = _log_uniform_int(rng, *w_range)
        C = 1 if rng.uniform() < 0.5 else 3
        lam, ss, sr, r = _draw_params(rng)
        r = min(r, (min(H, W) - 1) // 2)
        jobs.append(Job(H, W, C, lam, ss, sr, r, 1, seed=seed * 100003 + i))
    return jobs


def serving_requests(n: int = 10000, seed: int = 5, rate_hz: float = 200.0,
                     size_range=(128, 4096)) -> list[Job]:
    """Poisson arrivals (exponential gaps, mean 1/rate) of jobs with H, W log-uniform in
    ``size_range``, C in {1, 3}, parameters as in ``batch_jobs``."""
    rng = np.random.default_rng(seed)
    t = 0.0
    jobs = []
    for i in range(n):
        t += float(rng.exponential(1.0 / rate_hz))
        H = _log_uniform_int(rng, *size_range)
        W = _log_uniform_int(rng, *size_range)
        C = 1 if rng.uniform() < 0.5 else 3
        lam, ss, sr, r = _draw_params(rng)
        r = min(r, (min(H, W) - 1) // 2)
        jobs.append(Job(H, W, C, lam, ss, sr, r, 1, seed=seed * 100003 + i, arrival_s=t))
    return jobs


def job_image(job: Job) -> np.ndarray:
    """The image of a batched or served job: the sinusoid + disc recipe with the disc count
    scaled by area relative to 3840x2160 (at least 1)."""
    n_disc = max(1, int(round(200 * job.H * job.W / (3840 * 2160))))
    return sinusoid_disc_image(job.H, job.W, job.C, n_disc, 0.03, seed=job.seed)
