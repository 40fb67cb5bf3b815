"""Served form: continuous batching under a device-memory budget (GPU).

Each request's result must be the same whether it ran alone or was batched with others, the
server must stay within its budget while admitting work as memory frees up, and bad or
oversized requests are refused at submit time.
"""
import numpy as np
import pytest

from paper_1812_07122_gb300 import blfls, synth

from gpu_util import smooth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    import __graft_entry__
    __graft_entry__.build()
    handle = blfls.blfls_create(0)
    yield handle
    blfls.blfls_destroy(handle)


def _make(n, seed, lo=16, hi=384):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        H, W = int(rng.integers(lo, hi)), int(rng.integers(lo, hi))
        C = int(rng.choice([1, 3]))
        r = min(int(rng.choice([3, 5, 8, 10])), (min(H, W) - 1) // 2)
        p = dict(H=H, W=W, C=C, lam=float(rng.uniform(5, 50)), ss=max(r / 2, 0.5),
                 sr=float(rng.uniform(0.05, 0.2)), r=r)
        f = synth.sinusoid_disc_image(H, W, C, n_disc=3, seed=seed * 1000 + i)
        out.append((f, p))
    return out


def _submit(srv, f, p, out):
    req = blfls.make_request(f, out, p["H"], p["W"], p["C"], p["lam"], p["ss"], p["sr"], p["r"])
    return blfls.blfls_server_submit(srv, req)


def test_results_are_the_same_alone_and_in_the_mix(h):
    reqs = _make(40, seed=1)
    outs = [np.full_like(f, np.nan) for f, _ in reqs]
    srv = blfls.blfls_server_create(0, 512 << 20, slots=3, max_batch=8)
    try:
        tickets = [_submit(srv, f, p, o) for (f, p), o in zip(reqs, outs)]
        for t in tickets:
            blfls.blfls_server_wait(srv, t, 60000)
        stats = blfls.blfls_server_get_stats(srv)
    finally:
        blfls.blfls_server_destroy(srv)
    for (f, p), got in zip(reqs, outs):
        alone = smooth(h, f, p["lam"], p["ss"], p["sr"], p["r"], 1)
        assert np.array_equal(got, alone), p
    assert stats["completed"] == 40 and stats["failed"] == 0
    assert stats["max_batch_seen"] > 1          # requests really were batched together
    assert 0 < stats["p50_ms"] <= stats["p99_ms"] <= stats["max_ms"]
    assert stats["device_bytes_peak"] <= stats["device_bytes_budget"]


def test_admission_stays_within_a_small_budget(h):
    """256 MiB: the I/O arena holds about 19 requests of 1024x1024 in + out; 30 are queued at
    once, so later ones are admitted only as earlier ones release their buffers."""
    rng = np.random.default_rng(7)
    f = rng.uniform(size=(1, 1024, 1024)).astype(np.float32)
    outs = [np.empty_like(f) for _ in range(30)]
    srv = blfls.blfls_server_create(0, 256 << 20, slots=2, max_batch=4)
    try:
        p = dict(H=1024, W=1024, C=1, lam=20.0, ss=2.5, sr=0.1, r=5)
        tickets = [_submit(srv, f, p, o) for o in outs]
        for t in tickets:
            blfls.blfls_server_wait(srv, t, 120000)
        stats = blfls.blfls_server_get_stats(srv)
    finally:
        blfls.blfls_server_destroy(srv)
    assert stats["completed"] == 30
    assert stats["device_bytes_peak"] <= stats["device_bytes_budget"]
    alone = smooth(h, f, 20.0, 2.5, 0.1, 5, 1)
    for o in outs:
        assert np.array_equal(o, alone)


def test_oversized_and_malformed_requests_are_refused():
    srv = blfls.blfls_server_create(0, 256 << 20, slots=1, max_batch=2)
    try:
        big = np.zeros((3, 4096, 4096), dtype=np.float32)
        with pytest.raises(blfls.BlflsError) as ei:
            _submit(srv, big, dict(H=4096, W=4096, C=3, lam=10.0, ss=2.0, sr=0.1, r=3), big)
        assert ei.value.code == blfls.BLFLS_ENOMEM
        small = np.zeros((1, 32, 32), dtype=np.float32)
        with pytest.raises(blfls.BlflsError) as ei:
            _submit(srv, small, dict(H=32, W=32, C=1, lam=10.0, ss=2.0, sr=0.1, r=40), small)
        assert ei.value.code == blfls.BLFLS_EINVAL
        stats = blfls.blfls_server_get_stats(srv)
        assert stats["rejected"] == 1 and stats["submitted"] == 0
    finally:
        blfls.blfls_server_destroy(srv)


def test_cancel_a_queued_request():
    rng = np.random.default_rng(3)
    f = rng.uniform(size=(3, 1024, 1024)).astype(np.float32)
    outs = [np.empty_like(f) for _ in range(12)]
    srv = blfls.blfls_server_create(0, 1 << 30, slots=1, max_batch=1)
    try:
        p = dict(H=1024, W=1024, C=3, lam=20.0, ss=5.0, sr=0.1, r=10)
        tickets = [_submit(srv, f, p, o) for o in outs]
        last = tickets[-1]
        try:
            blfls.blfls_server_cancel(srv, last)
            cancelled = True
        except blfls.BlflsError as e:           # it was already admitted: also valid
            assert e.code == blfls.BLFLS_EBUSY
            cancelled = False
        for t in tickets[:-1]:
            blfls.blfls_server_wait(srv, t, 120000)
        state = blfls.blfls_server_poll(srv, last)
        if cancelled:
            assert state == 2
            with pytest.raises(blfls.BlflsError):
                blfls.blfls_server_wait(srv, last, 10)
        blfls.blfls_server_release(srv, tickets[0])
        with pytest.raises(blfls.BlflsError):
            blfls.blfls_server_poll(srv, tickets[0])      # released: unknown ticket
    finally:
        blfls.blfls_server_destroy(srv)


def test_handle_submit_poll_equals_smooth_bit_for_bit(h):
    """blfls_submit / blfls_poll on the handle (device-pointer jobs, continuous batching on the
    handle's own queue): every result equals blfls_smooth on the job alone, bit for bit, the
    ticket is forgotten once reported done, and invalid jobs are refused at submit."""
    import time

    import torch

    from gpu_util import DEV, to_dev

    reqs = _make(24, seed=3)
    q = blfls.blfls_create(0)
    try:
        ins = [to_dev(f) for f, _ in reqs]
        outs = [torch.full_like(x, float("nan")) for x in ins]
        torch.cuda.synchronize(DEV)       # the inputs hold their data before the jobs are queued
        tickets = []
        for (f, p), x, o in zip(reqs, ins, outs):
            job = blfls.make_job(x, o, p["H"], p["W"], p["C"], p["lam"], p["ss"], p["sr"], p["r"])
            tickets.append(blfls.blfls_submit(q, job))
        pending = set(tickets)
        deadline = time.monotonic() + 120
        while pending and time.monotonic() < deadline:
            pending = {t for t in pending if not blfls.blfls_poll(q, t)}
            time.sleep(0.001)
        assert not pending, f"{len(pending)} jobs unfinished"
        with pytest.raises(blfls.BlflsError) as ei:
            blfls.blfls_poll(q, tickets[0])           # reported done once: forgotten
        assert ei.value.code == blfls.BLFLS_EINVAL
        bad = blfls.make_job(ins[0], outs[0], 8, 8, 1, -1.0, 1.0, 0.1, 1)
        with pytest.raises(blfls.BlflsError) as ei:
            blfls.blfls_submit(q, bad)
        assert ei.value.code == blfls.BLFLS_EINVAL
        got = [o.cpu().numpy() for o in outs]
    finally:
        blfls.blfls_destroy(q)
    for (f, p), g in zip(reqs, got):
        alone = smooth(h, f, p["lam"], p["ss"], p["sr"], p["r"], 1)
        assert np.array_equal(g, alone), p
