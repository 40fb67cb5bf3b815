"""The allocation-free solve entry point (GPU).

blfls_solve_residual_noalloc serves callers that cannot call cudaMalloc -- for instance a plug-in
whose host application owns all device memory, or a real-time path that cannot risk an
allocation stalling the device.  Its scratch is a static device array inside the library, so
this test calls it twice in a row with different sizes (the second call finds the first call's
leftovers in that array) and checks each result against the handle-based blfls_solve_residual,
within the FP32 tolerance used by the other parity tests.  The file name makes pytest collect it
last.
"""
import numpy as np
import pytest

from paper_1812_07122_gb300 import blfls

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-4


def _inputs(H, W, C, seed):
    rng = np.random.default_rng(seed)
    f = rng.uniform(size=(C, H, W)).astype(np.float32)
    ex = rng.normal(scale=0.05, size=(C, H, W)).astype(np.float32)
    ey = rng.normal(scale=0.05, size=(C, H, W)).astype(np.float32)
    return f, ex, ey


def test_noalloc_solve_matches_handle_solve_on_consecutive_calls():
    import torch

    import __graft_entry__
    __graft_entry__.build()
    lib = blfls.load()
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    h = blfls.blfls_create(0)
    try:
        # two calls in a row with different sizes and parameters, then the first size again
        cases = [(256, 320, 3, 30.0, 1), (97, 61, 1, 1024.0, 2), (256, 320, 3, 30.0, 3)]
        for H, W, C, lam, seed in cases:
            f, ex, ey = (torch.from_numpy(a).to(dev) for a in _inputs(H, W, C, seed))
            want = torch.empty_like(f)
            blfls.blfls_solve_residual(h, f, ex, ey, want, H, W, C, lam, stream)
            got = torch.full_like(f, float("nan"))
            rc = lib.blfls_solve_residual_noalloc(f.data_ptr(), ex.data_ptr(), ey.data_ptr(),
                                                  got.data_ptr(), H, W, C, lam,
                                                  stream.cuda_stream)
            assert rc == blfls.BLFLS_OK, blfls.blfls_last_error()
            torch.cuda.synchronize(dev)
            err = float((got.double() - want.double()).abs().max())
            assert err <= TOL_FP32, (H, W, err)
    finally:
        blfls.blfls_destroy(h)


def test_noalloc_solve_rejects_sizes_beyond_its_static_scratch():
    import torch
    lib = blfls.load()
    x = torch.zeros(1, 8, 8, device="cuda")
    p = x.data_ptr()
    rc = lib.blfls_solve_residual_noalloc(p, p, p, p, 2048, 2048, 1, 10.0, None)
    assert rc == blfls.BLFLS_EINVAL
    assert "exceed" in blfls.blfls_last_error()
    rc = lib.blfls_solve_residual_noalloc(p, p, p, p, 8192, 8, 1, 10.0, None)
    assert rc == blfls.BLFLS_EINVAL
