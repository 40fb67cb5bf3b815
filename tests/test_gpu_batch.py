"""Batched form (blfls_smooth_batch): uneven jobs in persistent launches under a CUDA graph.

Each job's result must equal blfls_smooth on that job alone -- bit for bit, since both run the
same device functions -- including when the batch's launch sequence is captured into a graph
and replayed on new data, and for the 64-job uneven workload.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1812_07122_gb300 import blfls, synth

from gpu_util import DEV, maxabs, smooth, stream

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    import __graft_entry__
    __graft_entry__.build()
    handle = blfls.blfls_create(0)
    yield handle
    blfls.blfls_destroy(handle)


def _run_batch(h, specs, seed=0, inplace=False):
    """specs: list of (H, W, C, lam, ss, sr, r, iters, prec).  Returns (inputs, outputs)."""
    import torch
    ins, outs, jobs, keep = [], [], [], []
    for k, (H, W, C, lam, ss, sr, r, iters, prec) in enumerate(specs):
        f = synth.sinusoid_disc_image(H, W, C, n_disc=max(2, H * W // 3000), seed=seed * 1000 + k)
        x = torch.from_numpy(f).to(DEV)
        keep.append(x)      # the jobs hold raw pointers: keep every input alive until the end
        y = x if inplace else torch.empty_like(x)
        ins.append(f)
        outs.append(y)
        jobs.append(blfls.make_job(x, y, H, W, C, lam, ss, sr, r, iters, prec))
        if inplace:
            outs[-1] = x
    blfls.blfls_smooth_batch(h, jobs, stream())
    torch.cuda.synchronize(DEV)
    return ins, [o.cpu().numpy() for o in outs]


MIXED = [
    (96, 128, 3, 30.0, 5.0, 0.08, 10, 1, 0),
    (61, 97, 1, 50.0, 2.0, 0.05, 3, 1, 0),     # prime sizes (Bluestein)
    (256, 256, 1, 20.0, 3.0, 0.1, 5, 2, 0),
    (40, 33, 2, 10.0, 1.0, 0.2, 1, 1, 0),
    (70, 66, 2, 1024.0, 8.0, 0.12, 16, 1, 0),
    (50, 70, 1, 20.0, 3.0, math.inf, 5, 1, 0),
    (33, 200, 3, 30.0, 4.0, 0.08, 8, 3, 1),    # FP16 weights in the same batch
    (45, 45, 1, 25.0, 2.5, 0.1, 5, 1, 2),      # BF16 weights
    (11, 13, 1, 5.0, 1.0, 0.1, 5, 1, 0),       # 2r+1 = H
    (64, 64, 1, 0.0, 3.0, 0.1, 5, 1, 0),       # lam = 0
    (30, 30, 1, 10.0, 2.0, 0.1, 0, 1, 0),      # radius 0
    (120, 90, 2, 30.0, 10.0, 0.1, 20, 1, 0),   # radius above the batched kernels: single path
    (20, 24, 1, 30.0, 2.0, 0.1, 3, 0, 0),      # iters = 0: copy
]


def test_batch_equals_single_job_runs(h):
    """FP32 and BF16-weight jobs are bit-identical to their single runs.  FP16-weight jobs agree
    to 1e-5: the half-precision K1 arithmetic compiled into the batched driver may round a
    subnormal half weight differently from the single-image driver (far below FP16's own
    rounding unit of 4.9e-4)."""
    ins, outs = _run_batch(h, MIXED, seed=1)
    for (H, W, C, lam, ss, sr, r, iters, prec), f, got in zip(MIXED, ins, outs):
        want = smooth(h, f, lam, ss, sr, r, iters, prec=prec)
        if prec == blfls.BLFLS_FP16W:
            assert maxabs(got, want) <= 1e-5, (H, W, C, r, prec, maxabs(got, want))
        else:
            assert np.array_equal(got, want), (H, W, C, r, prec, maxabs(got, want))


def test_batch_against_oracle(h):
    specs = MIXED[:3]
    ins, outs = _run_batch(h, specs, seed=2)
    for (H, W, C, lam, ss, sr, r, iters, prec), f, got in zip(specs, ins, outs):
        want = oracle.blfls(f, lam, ss, sr, r, iters)
        assert maxabs(got, want) <= 1e-4


def test_batch_graph_replay_on_new_data(h):
    """Same shapes three times: the second call captures a graph, the third replays it; each
    call brings new image data and must still match the single-job path."""
    specs = MIXED[:6]
    for rep in range(3):
        ins, outs = _run_batch(h, specs, seed=10 + rep)
        for (H, W, C, lam, ss, sr, r, iters, prec), f, got in zip(specs, ins, outs):
            want = smooth(h, f, lam, ss, sr, r, iters, prec=prec)
            assert np.array_equal(got, want), (rep, H, W)


def test_batch_in_place(h):
    specs = MIXED[:4]
    ins, outs = _run_batch(h, specs, seed=3, inplace=True)
    for (H, W, C, lam, ss, sr, r, iters, prec), f, got in zip(specs, ins, outs):
        assert np.array_equal(got, smooth(h, f, lam, ss, sr, r, iters, prec=prec))


def test_batch_rejects_a_bad_job_before_enqueueing(h):
    import torch
    x = torch.zeros(1, 32, 32, device=DEV)
    good = blfls.make_job(x, x, 32, 32, 1, 10.0, 2.0, 0.1, 3)
    bad = blfls.make_job(x, x, 32, 32, 1, 10.0, 2.0, 0.1, 40)   # 2r+1 > 32
    with pytest.raises(blfls.BlflsError) as ei:
        blfls.blfls_smooth_batch(h, [good, bad], stream())
    assert ei.value.code == blfls.BLFLS_EINVAL
    blfls.blfls_smooth_batch(h, [], stream())                  # empty batch is fine


def test_uneven_64_job_workload_equals_single_runs(h):
    """64 jobs: H log-uniform 256..1536, W 256..2048, C in {1,3}, lam~U[5,50],
    sigma_r~U[0.05,0.2], r in {3,5,8,10}, sigma_s = r/2, one pass."""
    import torch
    jobs = synth.batch_jobs(64, seed=4)
    xs, ys, cj = [], [], []
    for j in jobs:
        x = torch.from_numpy(synth.job_image(j)).to(DEV)
        y = torch.empty_like(x)
        xs.append(x)
        ys.append(y)
        cj.append(blfls.make_job(x, y, j.H, j.W, j.C, j.lam, j.sigma_s, j.sigma_r, j.radius,
                                 j.iters))
    for _ in range(3):    # direct, captured, replayed
        blfls.blfls_smooth_batch(h, cj, stream())
    torch.cuda.synchronize(DEV)
    for j, x, y in zip(jobs, xs, ys):
        alone = torch.empty_like(x)
        blfls.blfls_smooth(h, x, alone, j.H, j.W, j.C, j.lam, j.sigma_s, j.sigma_r, j.radius,
                           j.iters, 0, stream())
        torch.cuda.synchronize(DEV)
        assert torch.equal(alone, y), (j.H, j.W, j.C, j.radius)
