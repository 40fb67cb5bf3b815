#!/usr/bin/env python
"""Benchmark of the GB300 BLF-LS smoother: megapixels/s on the 3840x2160 RGB workload.

One step = one ``blfls_smooth`` call on a 3840x2160x3 FP32 image (radius 10, sigma_s 5,
sigma_r 0.08, lambda 30, 3 passes): per pass and channel the bilateral kernel (K1) and the three
FFT-solve kernels (K2-K4).  MP/s counts H*W per completed call (channels and passes included).

Timing: W untimed warm-up steps; then K steps, each bracketed by CUDA events on the launching
stream, with a 512 MB device write (L2 flush) before every step outside the events; barrier +
synchronize on both sides of the timed loop; max over ranks.  Under torchrun each rank smooths
its own copy of the image (independent replicas, weak scaling).

Also reported: ``roofline`` for K1 (ALU-bound on the MUFU ex2 pipe; live per-launch timing from
events the library records around each launch, in a second timed loop where a profiled call runs
the channels in order so that no other kernel overlaps a K1 launch), ``e2e`` (host buffers through
``blfls_smooth_host``, copies included), ``clocks`` sampled by nvidia-smi during the timed loop,
``cpu_baseline`` (the FP64 oracle on the host cores, bounded sample, rank 0 at N=1 only) and
``forms`` (the FP16/BF16-weight precision forms on the same workload), ``modes`` (the LS model of
Eq. 6, the detail-enhancement / log-tone applications of Section IV, joint and rolling-guidance
smoothing of Section III-D, BLF-LS on the bilateral-grid filter, and NC-LS, on the same image),
``step_ms`` (median / p99 of the timed steps), ``small`` (the 256x256 grey workload, one pass),
the batched and served forms, and, in ``cpu_baseline``, the oracle on one core and on the small
workload.

``--impl reference`` times the FP64 oracle instead (the comparison arm; no GPU work).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "BLF-LS megapixels/s at 4K RGB, batched/FP16 vs plain FP32; p99 latency"
H, W, C = 2160, 3840, 3
PARAMS = dict(lam=30.0, sigma_s=5.0, sigma_r=0.08, radius=10, iters=3)
WORKLOAD = "3840x2160 RGB FP32, radius 10, sigma_s 5, sigma_r 0.08, lambda 30, 3 passes"
L2_FLUSH_BYTES = 512 << 20


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--no-modes", action="store_true",
                    help="skip the LS-model and base/detail lines")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-small", action="store_true",
                    help="skip the 256x256 workload line")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=10000)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--tune-table", default=None,
                    help="launch-shape table: loaded if the file exists (no autotuning), else "
                         "written by the autotuner (so a profiled run can take the shapes of a "
                         "plain one)")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x: float, device=None) -> float:
    """The maximum of x over all ranks of the default process group (x itself when there is
    none); the tensor lives on `device` (a CUDA device under NCCL, the CPU under gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank: float, max_seconds: float, world: int) -> float:
    """Whole-job throughput of `world` independent replicas: all units over the slowest rank."""
    return world * units_per_rank / max_seconds


# ------------------------------------------------------------------------------------------
# nvidia-smi clock sampling during the timed region
# ------------------------------------------------------------------------------------------
_FIELDS = ("pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, bus_id: str | None):
        self.bus_id = (bus_id or "").lower()
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={_FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) != 9:
                continue
            rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        mine = [r for r in rows if self.bus_id and r[0].lower() == self.bus_id]
        if not mine:
            vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
            ids = sorted({r[0] for r in rows})
            pick = ids[int(vis)] if vis.isdigit() and int(vis) < len(ids) else rows[0][0]
            mine = [r for r in rows if r[0] == pick]
        sm = [float(r[1]) for r in mine if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in mine if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in mine:
            for name, val in zip(names, r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(mine)}


# ------------------------------------------------------------------------------------------
def cpu_oracle_sample(f, rows: int | None, threads: int, keep: list | None = None):
    """Time the FP64 oracle on channel 0, one pass, rows [0, rows) (all rows if None).
    Returns (seconds, fraction of the whole workload's work that the sample covers); the
    result is appended to `keep` when given."""
    import oracle
    f0 = f[0] if rows is None else f[0, :rows]
    t0 = time.perf_counter()
    u = oracle.blfls_channel(f0, PARAMS["lam"], PARAMS["sigma_s"], PARAMS["sigma_r"],
                             PARAMS["radius"], threads)
    dt = time.perf_counter() - t0
    if keep is not None:
        keep.append(u)
    frac = (f0.shape[0] * f0.shape[1]) / (H * W) / C / PARAMS["iters"]
    return dt, frac


def channel_errors(a, b) -> dict:
    """Per-channel max-abs and RMS of a - b (arrays [C][H][W]), in FP64."""
    import numpy as np
    d = np.asarray(a, np.float64) - np.asarray(b, np.float64)
    return {"max_abs": [float(f"{v:.3e}") for v in np.abs(d).max(axis=(1, 2))],
            "rms": [float(f"{v:.3e}") for v in np.sqrt((d * d).mean(axis=(1, 2)))]}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_1812_07122_gb300 import synth
    f = synth.image_4k_rgb()
    threads = oracle.default_threads()
    rows = 540
    for _ in range(args.warmup):
        cpu_oracle_sample(f, rows, threads)
    times = []
    frac = None
    for _ in range(args.steps):
        dt, frac = cpu_oracle_sample(f, rows, threads)
        times.append(dt / frac)                      # seconds for the whole workload
    mean_s = sum(times) / len(times)
    value = H * W / 1e6 / mean_s
    sample = (f"channel 0, one pass, rows 0-{rows - 1} (full width) of the 3840x2160 image; "
              f"{frac:.4f} of the workload per step, scaled to the whole workload")
    line = {"metric": METRIC, "value": round(value, 4), "unit": "MP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(mean_s * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": round(value, 4), "unit": "MP/s", "cores": threads,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 4), "unit": "MP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def bench_batched(h, dev, stream, flush, steps, table=None, tuned=False):
    """64 uneven jobs (sizes log-uniform, C in {1,3}, per-job lambda, sigma_r, radius): one
    blfls_smooth_batch call (graph-replayed) vs. a loop of blfls_smooth calls, both timed with
    events after an L2 flush."""
    import torch
    from paper_1812_07122_gb300 import blfls, synth
    jobs = synth.batch_jobs(64, seed=4)
    if not tuned:   # shapes for the batch's radii (a loaded table already holds them)
        for r in sorted({j.radius for j in jobs}):
            for prec in (0, 1):
                blfls.blfls_autotune(h, 768, 1024, 1, r, prec, table)
    xs, ys, cj, cj16 = [], [], [], []
    for j in jobs:
        x = torch.from_numpy(synth.job_image(j)).to(dev)
        y = torch.empty_like(x)
        xs.append(x)
        ys.append(y)
        cj.append(blfls.make_job(x, y, j.H, j.W, j.C, j.lam, j.sigma_s, j.sigma_r, j.radius,
                                 j.iters))
        cj16.append(blfls.make_job(x, y, j.H, j.W, j.C, j.lam, j.sigma_s, j.sigma_r, j.radius,
                                   j.iters, blfls.BLFLS_FP16W))
    mp = sum(j.H * j.W for j in jobs) / 1e6

    def loop():
        for j, x, y in zip(jobs, xs, ys):
            blfls.blfls_smooth(h, x, y, j.H, j.W, j.C, j.lam, j.sigma_s, j.sigma_r, j.radius,
                               j.iters, 0, stream)

    def batch():
        blfls.blfls_smooth_batch(h, cj, stream)

    def batch16():
        blfls.blfls_smooth_batch(h, cj16, stream)

    def timed(fn, n):
        for _ in range(3):
            fn()
        torch.cuda.synchronize(dev)
        tot = 0.0
        for i in range(n):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            tot += a.elapsed_time(b)
        return tot / n

    n = max(3, steps // 6)
    t_batch = timed(batch, n)
    t_loop = timed(loop, n)
    t_batch16 = timed(batch16, n)
    return {"workload": "64 jobs, H log-uniform 256-1536, W 256-2048, C in {1,3}, lambda~U[5,50], "
                        "sigma_r~U[0.05,0.2], radius in {3,5,8,10}, sigma_s=r/2, 1 pass, FP32",
            "megapixels_per_call": round(mp, 2), "ms_batched": round(t_batch, 3),
            "ms_single_loop": round(t_loop, 3), "batched_mp_per_s": round(mp / t_batch * 1e3, 1),
            "single_loop_mp_per_s": round(mp / t_loop * 1e3, 1),
            "speedup": round(t_loop / t_batch, 3),
            "batched_fp16w_mp_per_s": round(mp / t_batch16 * 1e3, 1),
            "batched_fp16w_speedup_vs_fp32_loop": round(t_loop / t_batch16, 3),
            "launch": "graph replay of one persistent launch per phase (K1 per radius group, "
                      "K2, K3, K4)"}


def bench_serving(dev, n_req, rate):
    """Poisson arrivals of jobs with H, W log-uniform 128-4096, C in {1,3}, parameters as in
    the batched workload, served with an 80 GB budget from pinned host buffers; then the same
    server saturated (all requests queued at once) for its capacity."""
    import torch
    from paper_1812_07122_gb300 import blfls, synth
    reqs = synth.serving_requests(n_req, seed=5, rate_hz=rate)
    pool_img = synth.sinusoid_disc_image(4096, 4096, 3, 400, 0.03, seed=55)
    src = torch.from_numpy(pool_img.reshape(-1)).pin_memory()
    dst = torch.empty_like(src).pin_memory()
    n_pool = src.numel()
    rng = __import__("numpy").random.default_rng(6)
    base_in, base_out = src.data_ptr(), dst.data_ptr()

    def request(j):
        need = j.C * j.H * j.W
        off = int(rng.integers(0, (n_pool - need) // 64 + 1)) * 64
        return blfls.make_request(base_in + 4 * off, base_out + 4 * off, j.H, j.W, j.C, j.lam,
                                  j.sigma_s, j.sigma_r, j.radius, j.iters)

    def run(jobs, paced):
        srv = blfls.blfls_server_create(dev.index or 0, 80 << 30, slots=4, max_batch=16)
        try:
            tickets = []
            t0 = time.perf_counter()
            for j in jobs:
                if paced:
                    delay = j.arrival_s - (time.perf_counter() - t0)
                    if delay > 0:
                        time.sleep(delay)
                tickets.append(blfls.blfls_server_submit(srv, request(j)))
            for t in tickets:
                blfls.blfls_server_wait(srv, t, 600000)
            return blfls.blfls_server_get_stats(srv)
        finally:
            blfls.blfls_server_destroy(srv)

    warm = run(reqs[:64], paced=False)          # plans and graphs for common shapes
    st = run(reqs, paced=True)
    sat = run(reqs[: min(len(reqs), 2000)], paced=False)
    keep = ["completed", "failed", "p50_ms", "p99_ms", "mean_ms", "max_ms", "megapixels",
            "busy_s", "mp_per_s", "max_batch_seen", "device_bytes_peak"]
    return {"workload": f"{n_req} requests, Poisson {rate:g} req/s, H,W log-uniform 128-4096, "
                        "C in {1,3}, lambda~U[5,50], sigma_r~U[0.05,0.2], radius in {3,5,8,10}, "
                        "pinned host buffers, budget 80 GB, 4 slots, batches <= 16",
            "poisson": {k: (round(v, 3) if isinstance(v, float) else v) for k, v in st.items()
                        if k in keep},
            "saturated_2000": {k: (round(v, 3) if isinstance(v, float) else v)
                               for k, v in sat.items() if k in keep},
            "warmup_requests": warm["completed"]}


def hbm_peak_gbs():
    """(peak GB/s, basis): the measured HBM copy bandwidth recorded in MEASURED_PEAKS.json when
    that file is present, else the fallback figure."""
    try:
        rec = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(rec["hbm_gbs"]), "of measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, ValueError, KeyError, TypeError):
        return 6800.0, "of fallback (6.8 TB/s)"


def solve_rooflines(prof_ms, prof_n, H, W):
    """K2-K4 against the HBM roofline: algorithmic bytes per launch (one channel) over the
    average launch time of the profiled loop.  K2 reads e_x, e_y and writes the half spectrum;
    K3 reads and writes the half spectrum; K4 reads it and f and writes u."""
    try:
        spec = H * (W // 2 + 1) * 8
        plane = H * W * 4
        algo = {"K2": 2 * plane + spec, "K3": 2 * spec, "K4": spec + 2 * plane}
        peak, basis = hbm_peak_gbs()
        out = {"unit": "GB/s", "peak": peak, "peak_basis": basis}
        for i, k in ((1, "K2"), (2, "K3"), (3, "K4")):
            if prof_n[i] <= 0:
                continue
            ms = prof_ms[i] / prof_n[i]
            gbs = algo[k] / (ms / 1e3) / 1e9
            out[k] = {"ms_per_launch": round(ms, 4), "algorithmic_bytes": algo[k],
                      "achieved": round(gbs, 1), "frac": round(gbs / peak, 4)}
        return out
    except (TypeError, ValueError, IndexError, ZeroDivisionError):
        return None


def k1_traffic_per_launch():
    """DRAM bytes per K1 launch from the committed ncu summary, if it was taken on the current
    kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "k1_blf_4k_traffic.json")
    src = os.path.join(ROOT, "paper_1812_07122_gb300", "csrc", "blf_tile.cuh")
    try:
        rec = json.load(open(path))
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
        if rec.get("kernel_src_sha256") == sha:
            return rec.get("dram_bytes_per_launch")
    except (OSError, ValueError):
        pass
    return None


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    import __graft_entry__
    __graft_entry__.build()
    from paper_1812_07122_gb300 import blfls, synth

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group(backend="nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count
    bus_id = None
    try:
        bus_id = f"{props.pci_domain_id:08x}:{props.pci_bus_id:02x}:{props.pci_device_id:02x}.0"
    except AttributeError:
        pass

    f = synth.image_4k_rgb()
    x = torch.from_numpy(f).to(dev)
    out = torch.empty_like(x)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    tuned_from_file = bool(args.tune_table) and os.path.exists(args.tune_table)
    h = blfls.blfls_create(local, 0, args.tune_table if tuned_from_file else None)
    stream = torch.cuda.current_stream(dev)
    p = PARAMS

    def step(prec=blfls.BLFLS_FP32):
        blfls.blfls_smooth(h, x, out, H, W, C, p["lam"], p["sigma_s"], p["sigma_r"], p["radius"],
                           p["iters"], prec, stream)

    # launch shapes for this workload from the project autotuner (K1 tile height per precision,
    # K3 column block), untimed; they change speed only, never results
    table = args.tune_table or os.path.join(tempfile.mkdtemp(), "tune.json")
    if not tuned_from_file:
        for prec in (0, 1, 2):
            blfls.blfls_autotune(h, H, W, 1, p["radius"], prec, table)
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize(dev)
    rates = blfls.blfls_pipe_rates(local)                # results / clk / SM, measured here
    ex2_per_clk = rates["ex2_f32"]
    ex2_units = float(2 ** round(math.log2(ex2_per_clk))) if ex2_per_clk > 0 else 32.0

    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(K)]
    launches_per_step = C * p["iters"] * 4
    sampler = ClockSampler(bus_id)
    sampler.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    for i in range(K):
        flush.fill_(float(i))                        # L2 flush, outside the timed events
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    step_times = sorted(a.elapsed_time(b) for a, b in ev)
    total_ms = max_over_ranks(sum(step_times), dev)
    ms_per_step = total_ms / K
    step_ms = {"median": round(statistics.median(step_times), 3),
               "p99": round(step_times[min(K - 1, int(math.ceil(0.99 * K)) - 1)], 3),
               "min": round(step_times[0], 3), "max": round(step_times[-1], 3)}
    mp = H * W / 1e6
    value = replica_throughput(mp, ms_per_step / 1e3, world)

    # Per-kernel times: a second timed loop with the library's profiling on.  A profiled call
    # runs the channels in order on the caller's stream (the timed loop above runs them on
    # concurrent streams, where one channel's solve overlaps another's bilateral kernel), so
    # every launch's events enclose that kernel alone.
    blfls.blfls_profile_begin(h, K * C * p["iters"] * 8 + 16)
    prof_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(K)]
    for i in range(K):
        flush.fill_(float(i))
        prof_ev[i][0].record(stream)
        step()
        prof_ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    prof_ms, prof_n = blfls.blfls_profile_end(h)
    clocks = sampler.stop()
    ms_per_step_in_order = sum(a.elapsed_time(b) for a, b in prof_ev) / K

    # roofline of the dominant kernel (K1): taps per launch / average launch time
    taps_per_launch = H * W * 2 * (2 * p["radius"] + 1) ** 2          # one channel per launch
    k1_ms = prof_ms[0] / max(prof_n[0], 1)
    achieved = taps_per_launch / (k1_ms / 1e3) / 1e9                    # Gtap/s
    sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    peak = ex2_units * n_sm * sm_mhz * 1e6 / 1e9
    total_prof = sum(prof_ms)
    roofline = {"bound": "alu", "kernel": "k1_blf<10,range,fp32> (bilateral residuals)",
                "achieved": round(achieved, 1), "peak": round(peak, 1), "unit": "Gtap/s",
                "frac": round(achieved / peak, 4), "traffic": k1_traffic_per_launch(),
                "peak_basis": f"MUFU ex2.f32: {ex2_units:.0f}/clk/SM (probe measured "
                              f"{ex2_per_clk:.2f}) x {n_sm} SMs x {sm_mhz:.0f} MHz (median SM "
                              f"clock sampled in the timed loop); one ex2 per tap",
                "pipe_rates_per_clk_per_sm": {k: round(v, 2) for k, v in rates.items()},
                "k1_ms_per_launch": round(k1_ms, 4),
                "timing": "per-launch events in a second timed loop of the same workload with "
                          "the channels in order (ms per step there: "
                          f"{ms_per_step_in_order:.3f}); `value` comes from the loop with "
                          "concurrent channel streams",
                "stage_share": {k: round(v / total_prof, 4) for k, v in
                                zip(["K1", "K2", "K3", "K4"], prof_ms)} if total_prof else None,
                "solve_kernels": solve_rooflines(prof_ms, prof_n, H, W)}

    # end to end through host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        hx = torch.from_numpy(f).pin_memory()
        hy = torch.empty_like(hx).pin_memory()
        for _ in range(2):
            blfls.blfls_smooth_host(h, hx, hy, H, W, C, p["lam"], p["sigma_s"], p["sigma_r"],
                                    p["radius"], p["iters"], 0, stream)
        n_e2e = max(3, min(K, 20))
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            blfls.blfls_smooth_host(h, hx, hy, H, W, C, p["lam"], p["sigma_s"], p["sigma_r"],
                                    p["radius"], p["iters"], 0, stream)
        e2e_s = max_over_ranks((time.perf_counter() - t0) / n_e2e, dev)
        nbytes = C * H * W * 4
        e2e = {"value": round(replica_throughput(mp, e2e_s, world), 2), "unit": "MP/s",
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
               "api": "blfls_smooth_host (pinned host buffers)"}

    def timed_mp(fn, n):
        """MP/s of fn() on the 4K workload: CUDA events around each call, L2 flushed between."""
        fn()
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tot = 0.0
        for i in range(n):
            flush.fill_(float(i))
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            tot += a.elapsed_time(b)
        return round(mp / (tot / n / 1e3), 2)

    # precision forms on the same workload
    forms = None
    one_pass = {}      # precision -> this workload's image after ONE pass (for the oracle errors)
    if not args.no_forms:
        forms = {}
        full = {}
        for name, prec in [("fp32", 0), ("fp16w", 1), ("bf16w", 2)]:
            try:
                forms[name] = timed_mp(lambda: step(prec), max(3, K // 4))
                full[name] = out.cpu().numpy()
                blfls.blfls_smooth(h, x, out, H, W, C, p["lam"], p["sigma_s"], p["sigma_r"],
                                   p["radius"], 1, prec, stream)
                one_pass[name] = out.cpu().numpy()
            except blfls.BlflsError as e:
                forms[name] = f"unavailable: {e}"
        # per-channel error of the reduced-precision forms against the plain FP32 path on the
        # whole workload (3 passes, every pixel); against the FP64 oracle below (one pass)
        forms["errors_vs_fp32_path"] = {k: channel_errors(full[k], full["fp32"])
                                        for k in ("fp16w", "bf16w") if k in full and "fp32" in full}

    # the LS model (Eq. 6) and the base/detail applications on the same image and parameters
    modes = None
    if not args.no_modes:
        n = max(3, K // 4)
        ls = lambda: blfls.blfls_smooth_ls(h, x, out, H, W, C, p["lam"], p["iters"], stream)
        enh = lambda: blfls.blfls_layers(h, x, out, H, W, C, blfls.BLFLS_DETAIL_ENHANCE, 2.0,
                                         p["lam"], p["sigma_s"], p["sigma_r"], p["radius"],
                                         p["iters"], 0, stream)
        tone = lambda: blfls.blfls_layers(h, x, out, H, W, C, blfls.BLFLS_LOG_TONE, 0.5,
                                          p["lam"], p["sigma_s"], p["sigma_r"], p["radius"],
                                          p["iters"], 0, stream)
        guide = torch.empty_like(x)
        blfls.blfls_gaussian(h, x, guide, H, W, C, 2.0, stream)   # a smooth guidance image
        out2 = torch.empty_like(x)
        joint = lambda: blfls.blfls_smooth_guided(h, x, guide, out, H, W, C, C, p["lam"],
                                                  p["sigma_s"], p["sigma_r"], p["radius"],
                                                  p["iters"], 0, stream)
        rolling = lambda: blfls.blfls_smooth_rolling(h, x, out2, H, W, C, p["lam"], p["sigma_s"],
                                                     p["sigma_r"], p["radius"], p["iters"], 1.0,
                                                     0, stream)
        modes = {"workload": "the same 4K RGB image and parameters, FP32",
                 "ls_model": timed_mp(ls, n),
                 "detail_enhance_m2": timed_mp(enh, n),
                 "log_tone_c0.5": timed_mp(tone, n),
                 "joint_guided_by_gaussian2": timed_mp(joint, n),
                 "rolling_guidance_sigma1": timed_mp(rolling, n)}
        grid = lambda: blfls.blfls_smooth_grid(h, x, out, H, W, C, p["lam"], p["sigma_s"],
                                               p["sigma_r"], p["iters"], stream)
        try:
            modes["bilateral_grid_blf"] = timed_mp(grid, n)
        except blfls.BlflsError as e:
            modes["bilateral_grid_blf"] = f"unavailable: {e}"
        nc = lambda: blfls.blfls_smooth_nc(h, x, out, H, W, C, p["lam"], p["sigma_s"],
                                           p["sigma_r"], p["iters"], 3, stream)
        modes["nc_ls_3_box_iterations"] = timed_mp(nc, n)

    batched = None
    if not args.no_batch:
        batched = bench_batched(h, dev, stream, flush, K, table, tuned_from_file)
    serving = None
    if not args.no_serve and rank == 0:
        serving = bench_serving(dev, args.serve_requests, args.serve_rate)

    # the small grey workload (256x256, r 5, sigma_s 3, sigma_r 0.1, lambda 20, one pass) on the GPU
    small = None
    if not args.no_small and rank == 0:
        fs = synth.image_256_rectangles()                # [1, 256, 256]
        xs = torch.from_numpy(fs).to(dev)
        ys = torch.empty_like(xs)
        run_small = lambda: blfls.blfls_smooth(h, xs, ys, 256, 256, 1, 20.0, 3.0, 0.1, 5, 1, 0,
                                               stream)
        for _ in range(max(3, args.warmup)):
            run_small()
        torch.cuda.synchronize(dev)
        n_small = max(50, K)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(n_small):
            run_small()
        b.record(stream)
        b.synchronize()
        small_ms = a.elapsed_time(b) / n_small
        small = {"workload": "256x256 grey rectangles, radius 5, sigma_s 3, sigma_r 0.1, "
                             "lambda 20, one pass, FP32 (back-to-back calls, inputs in L2)",
                 "ms_per_call": round(small_ms, 4), "mp_per_s": round(0.065536 / small_ms * 1e3, 2)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        threads = oracle.default_threads()
        kept = []
        dt, frac = cpu_oracle_sample(f, None, threads, kept)
        cpu = {"value": round(mp / (dt / frac), 4), "unit": "MP/s", "cores": threads,
               "kind": "oracle",
               "sample": f"channel 0, one pass, whole 3840x2160 plane ({dt:.1f} s; "
                         f"{frac:.4f} of the workload), scaled to the whole workload"}
        # one core, and the small grey workload on all cores and on one
        dt1, frac1 = cpu_oracle_sample(f, 135, 1)
        fs0 = synth.image_256_rectangles()[0]
        t0 = time.perf_counter()
        oracle.blfls_channel(fs0, 20.0, 3.0, 0.1, 5, threads)
        c1_all = time.perf_counter() - t0
        t0 = time.perf_counter()
        oracle.blfls_channel(fs0, 20.0, 3.0, 0.1, 5, 1)
        c1_one = time.perf_counter() - t0
        cpu["one_core"] = {"value": round(mp / (dt1 / frac1), 5), "unit": "MP/s", "cores": 1,
                           "sample": f"channel 0, one pass, rows 0-134 ({dt1:.1f} s; "
                                     f"{frac1:.5f} of the workload), scaled"}
        if forms is not None and one_pass:
            # precision report against the FP64 oracle: one pass of every channel of the 4K
            # image (channel 0 from the timed sample above; the others untimed)
            ref = [kept[0]] + [oracle.blfls_channel(f[c], p["lam"], p["sigma_s"], p["sigma_r"],
                                                    p["radius"], threads) for c in range(1, C)]
            ref = np.stack(ref)
            forms["errors_vs_fp64_oracle_one_pass"] = {k: channel_errors(v, ref)
                                                       for k, v in one_pass.items()}
        cpu["small_workload"] = {"workload": "256x256 grey rectangles, radius 5, one pass",
                                 "all_cores_s": round(c1_all, 3), "one_core_s": round(c1_one, 3),
                                 "all_cores_mp_per_s": round(0.065536 / c1_all, 4),
                                 "one_core_mp_per_s": round(0.065536 / c1_one, 4)}

    blfls.blfls_destroy(h)
    try:
        tuned = json.load(open(table))
    except (OSError, ValueError):
        tuned = None
    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 2), "unit": "MP/s", "n_gpus": world,
                "steps": K, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "H": H, "W": W, "C": C, **PARAMS,
                           "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                           "l2": f"flushed before every step ({L2_FLUSH_BYTES >> 20} MB write)"},
                "step_ms": step_ms, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches_per_step * K, "clocks": clocks,
                "launch_shapes": {"source": "file" if tuned_from_file else "autotuner",
                                  "table": tuned},
                "forms": forms,
                "modes": modes, "small": small, "batched": batched, "serving": serving}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
