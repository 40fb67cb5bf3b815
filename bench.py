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
events the library records around each launch), ``e2e`` (host buffers through
``blfls_smooth_host``, copies included), ``clocks`` sampled by nvidia-smi during the timed loop,
``cpu_baseline`` (the FP64 oracle on the host cores, bounded sample, rank 0 at N=1 only) and
``forms`` (the FP16/BF16-weight precision forms on the same workload).

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
MUFU_EX2_PER_CLK_PER_SM = 16    # FP32 ex2 results per clock per SM (sm_100-class SFU)
L2_FLUSH_BYTES = 512 << 20


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


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
def cpu_oracle_sample(f, rows: int | None, threads: int):
    """Time the FP64 oracle on channel 0, one pass, rows [0, rows) (all rows if None).
    Returns (seconds, fraction of the whole workload's work that the sample covers)."""
    import oracle
    f0 = f[0] if rows is None else f[0, :rows]
    t0 = time.perf_counter()
    oracle.blfls_channel(f0, PARAMS["lam"], PARAMS["sigma_s"], PARAMS["sigma_r"],
                         PARAMS["radius"], threads)
    dt = time.perf_counter() - t0
    frac = (f0.shape[0] * f0.shape[1]) / (H * W) / C / PARAMS["iters"]
    return dt, frac


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


def k1_traffic_per_launch():
    """DRAM bytes per K1 launch from the committed ncu summary, if it was taken on the current
    kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "k1_blf_4k_traffic.json")
    src = os.path.join(ROOT, "paper_1812_07122_gb300", "csrc", "blf_kernels.cu")
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
    h = blfls.blfls_create(local)
    stream = torch.cuda.current_stream(dev)
    p = PARAMS

    def step(prec=blfls.BLFLS_FP32):
        blfls.blfls_smooth(h, x, out, H, W, C, p["lam"], p["sigma_s"], p["sigma_r"], p["radius"],
                           p["iters"], prec, stream)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize(dev)

    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(K)]
    launches_per_step = C * p["iters"] * 4
    sampler = ClockSampler(bus_id)
    sampler.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    blfls.blfls_profile_begin(h, K * C * p["iters"] * 8 + 16)
    for i in range(K):
        flush.fill_(float(i))                        # L2 flush, outside the timed events
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    prof_ms, prof_n = blfls.blfls_profile_end(h)
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    total_ms = sum(a.elapsed_time(b) for a, b in ev)
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / K
    mp = H * W / 1e6
    value = world * mp / (ms_per_step / 1e3)

    # roofline of the dominant kernel (K1): taps per launch / average launch time
    taps_per_launch = H * W * 2 * (2 * p["radius"] + 1) ** 2          # one channel per launch
    k1_ms = prof_ms[0] / max(prof_n[0], 1)
    achieved = taps_per_launch / (k1_ms / 1e3) / 1e9                    # Gtap/s
    sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    peak = MUFU_EX2_PER_CLK_PER_SM * n_sm * sm_mhz * 1e6 / 1e9
    total_prof = sum(prof_ms)
    roofline = {"bound": "alu", "kernel": "k1_blf_tiled<10,range> (bilateral residuals)",
                "achieved": round(achieved, 1), "peak": round(peak, 1), "unit": "Gtap/s",
                "frac": round(achieved / peak, 4), "traffic": k1_traffic_per_launch(),
                "peak_basis": f"MUFU ex2: {MUFU_EX2_PER_CLK_PER_SM}/clk/SM x {n_sm} SMs x "
                              f"{sm_mhz:.0f} MHz (median SM clock sampled in the timed loop)",
                "k1_ms_per_launch": round(k1_ms, 4),
                "stage_share": {k: round(v / total_prof, 4) for k, v in
                                zip(["K1", "K2", "K3", "K4"], prof_ms)} if total_prof else None}

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
        e2e_s = (time.perf_counter() - t0) / n_e2e
        if world > 1:
            t = torch.tensor([e2e_s], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        nbytes = C * H * W * 4
        e2e = {"value": round(world * mp / e2e_s, 2), "unit": "MP/s",
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
               "api": "blfls_smooth_host (pinned host buffers)"}

    # precision forms on the same workload
    forms = None
    if not args.no_forms:
        forms = {}
        for name, prec in [("fp32", 0), ("fp16w", 1), ("bf16w", 2)]:
            try:
                step(prec)
                torch.cuda.synchronize(dev)
                n = max(3, K // 4)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                tot = 0.0
                for i in range(n):
                    flush.fill_(float(i))
                    a.record(stream)
                    step(prec)
                    b.record(stream)
                    b.synchronize()
                    tot += a.elapsed_time(b)
                forms[name] = round(mp / (tot / n / 1e3), 2)
            except blfls.BlflsError as e:
                forms[name] = f"unavailable: {e}"

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        threads = oracle.default_threads()
        dt, frac = cpu_oracle_sample(f, None, threads)
        cpu = {"value": round(mp / (dt / frac), 4), "unit": "MP/s", "cores": threads,
               "kind": "oracle",
               "sample": f"channel 0, one pass, whole 3840x2160 plane ({dt:.1f} s; "
                         f"{frac:.4f} of the workload), scaled to the whole workload"}

    blfls.blfls_destroy(h)
    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 2), "unit": "MP/s", "n_gpus": world,
                "steps": K, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "H": H, "W": W, "C": C, **PARAMS,
                           "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                           "l2": f"flushed before every step ({L2_FLUSH_BYTES >> 20} MB write)"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches_per_step * K, "clocks": clocks, "forms": forms}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
