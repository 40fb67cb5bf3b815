"""The allocation-free solve entry point (GPU).

blfls_solve_residual_noalloc serves callers that cannot call cudaMalloc -- for instance a plug-in
whose host application owns all device memory, or a real-time path that cannot risk an
allocation stalling the device.  Its scratch is a static device array inside the library, so
this test calls it several times in a row with different sizes (each call finds the previous
call's leftovers in that array) and checks each result against the handle-based
blfls_solve_residual and against the FP64 oracle's Eq. 8 with v = D f + e, within the FP32
tolerance used by the other parity tests.  The sizes include rows of 1920 and columns of 540 and
1080, which run the compile-time FFT plans on the tables bound inside the static array.  The file
name makes pytest collect it last.
"""
import numpy as np
import pytest

import oracle
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
        # calls in a row with different sizes and parameters, then the first size again
        cases = [(256, 320, 3, 30.0, 1), (97, 61, 1, 1024.0, 2), (540, 1920, 1, 30.0, 4),
                 (1080, 512, 2, 20.0, 5), (256, 320, 3, 30.0, 3)]
        for H, W, C, lam, seed in cases:
            fn, exn, eyn = _inputs(H, W, C, seed)
            f, ex, ey = (torch.from_numpy(a).to(dev) for a in (fn, exn, eyn))
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
            g = got.cpu().numpy()
            for c in range(C):
                gx, gy = oracle.gradients(fn[c].astype(np.float64))
                ref = oracle.solve_eq8(fn[c], gx + exn[c], gy + eyn[c], lam)
                e = float(np.max(np.abs(g[c] - ref)))
                assert e <= TOL_FP32, (H, W, c, e)
    finally:
        blfls.blfls_destroy(h)


def test_noalloc_solve_rejects_sizes_beyond_its_static_scratch():
    import torch

    import __graft_entry__
    __graft_entry__.build()
    lib = blfls.load()
    x = torch.zeros(1, 8, 8, device="cuda")
    p = x.data_ptr()
    rc = lib.blfls_solve_residual_noalloc(p, p, p, p, 2048, 2048, 1, 10.0, None)
    assert rc == blfls.BLFLS_EINVAL
    assert "exceed" in blfls.blfls_last_error()
    rc = lib.blfls_solve_residual_noalloc(p, p, p, p, 8192, 8, 1, 10.0, None)
    assert rc == blfls.BLFLS_EINVAL
