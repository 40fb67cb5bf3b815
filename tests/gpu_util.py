"""Helpers for the GPU tests: run the C ABI on numpy inputs and return numpy outputs."""
import numpy as np
import torch

from paper_1812_07122_gb300 import blfls

DEV = torch.device("cuda:0")


def to_dev(a) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV)


def stream():
    return torch.cuda.current_stream(DEV)


def smooth(h, f, lam, ss, sr, r, iters=1, prec=blfls.BLFLS_FP32, inplace=False):
    f = np.asarray(f, dtype=np.float32)
    if f.ndim == 2:
        f = f[None]
    C, H, W = f.shape
    x = to_dev(f)
    out = x if inplace else torch.empty_like(x)
    blfls.blfls_smooth(h, x, out, H, W, C, lam, ss, sr, r, iters, prec, stream())
    torch.cuda.synchronize(DEV)
    return out.cpu().numpy()


def blf_residual(h, f, ss, sr, r, prec=blfls.BLFLS_FP32):
    f = np.asarray(f, dtype=np.float32)
    if f.ndim == 2:
        f = f[None]
    C, H, W = f.shape
    x = to_dev(f)
    ex = torch.empty_like(x)
    ey = torch.empty_like(x)
    blfls.blfls_blf_residual(h, x, ex, ey, H, W, C, ss, sr, r, prec, stream())
    torch.cuda.synchronize(DEV)
    return ex.cpu().numpy(), ey.cpu().numpy()


def solve_residual(h, f, ex, ey, lam):
    f = np.asarray(f, dtype=np.float32)
    if f.ndim == 2:
        f, ex, ey = f[None], ex[None], ey[None]
    C, H, W = f.shape
    x, dex, dey = to_dev(f), to_dev(ex), to_dev(ey)
    out = torch.empty_like(x)
    blfls.blfls_solve_residual(h, x, dex, dey, out, H, W, C, lam, stream())
    torch.cuda.synchronize(DEV)
    return out.cpu().numpy()


def maxabs(a, b) -> float:
    return float(np.max(np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64))))
