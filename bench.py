#!/usr/bin/env python3
"""Benchmark of the FFA periodogram on one series per GPU.

Workload (default): 2^23 samples at 64 us (the paper's benchmark series shape, Sec. 5.8),
N(0,1) noise plus three Gaussian pulse trains, periods 0.2-20 s, 240-260 bins, 11 boxcar
widths; synthetic data from a fixed seed.  One step = one whole periodogram (prefix sums,
downsampling of all 55 pseudo-octaves, 1155 FFA transforms, boxcar S/N of 662,440 trials).

metric: time-series samples searched per second = N / (device time of one step), summed
over GPUs.  Each GPU runs its own replica (series are independent; no collective is in
the data path).  Between timed steps the L2 is flushed by writing a 256 MB buffer.

--impl reference times the CPU oracle instead (a bounded sample of the same workload per
step, extrapolated to the whole periodogram); it is the slow reference program, not a
target.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "time-series samples searched/s (FFA periodogram)"
UNIT = "samples/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ffa", "reference"], default="ffa")
    ap.add_argument("--workload", choices=["survey", "plain_small"], default="survey")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-sample-stride", type=int, default=8)
    return ap.parse_args()


def workload(name):
    return synth.survey() if name == "survey" else synth.plain_small()


def recorded_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu record, or None if the
    kernel source changed since it was taken."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "roofline_traffic.json")))
        src = open(os.path.join(ROOT, "paper_2004_03701_gb300", "csrc", "ffa_kernels.cu"), "rb").read()
        if hashlib.sha256(src).hexdigest()[:16] != rec["kernel_source_sha256_prefix"]:
            return None
        return rec["dram_bytes_per_launch"] if rec["kernel"] == kernel else None
    except Exception:
        return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------ distributed
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ------------------------------------------------------------------------- CPU oracle
def oracle_sample_time(w, stride, offset=0):
    """Times the CPU oracle on a bounded sample of the workload: all downsampling, plus
    the FFA and S/N of every `stride`-th transform; extrapolates the FFA + S/N time by
    the folded-sample ratio.  Returns (seconds per whole periodogram, description)."""
    import oracle
    oracle.build()
    args = (w.tsamp, w.pmin, w.pmax, w.bmin, w.bmax)
    pl = oracle.plan(w.n, *args)
    t0 = time.perf_counter()
    for f in pl.oct_factor:
        oracle.downsample(w.x, float(f))
    t_ds = time.perf_counter() - t0
    sel = np.zeros(pl.n_transforms, bool)
    sel[offset % stride::stride] = True
    t0 = time.perf_counter()
    oracle.periodogram(w.x, *args, w.widths, select=sel)
    t_sel = time.perf_counter() - t0
    folded = (pl.tr_m * pl.tr_p).astype(np.float64)
    ratio = folded.sum() / folded[sel].sum()
    # the selected run downsampled every octave it touched again; remove that once
    touched = np.unique(pl.tr_octave[sel])
    t_ds_sel = t_ds * len(touched) / pl.n_octaves
    est = t_ds + max(t_sel - t_ds_sel, 0.0) * ratio
    desc = ("oracle (1 thread, C, FP64): downsampling of all %d octaves timed in full, FFA + "
            "direct boxcar S/N of every %d-th of %d transforms (%.1f%% of folded samples) "
            "extrapolated by folded samples; %.1f s measured" %
            (pl.n_octaves, stride, pl.n_transforms, 100.0 / ratio, t_ds + t_sel))
    return est, desc


def run_reference(a):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    w = workload(a.workload)
    stride = 64
    times = []
    for i in range(a.warmup + a.steps):
        est, desc = oracle_sample_time(w, stride, offset=i)
        if i >= a.warmup:
            times.append(est)
    t = statistics.mean(times)
    value = w.n / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "n": w.n, "tsamp": w.tsamp, "pmin": w.pmin,
                   "pmax": w.pmax, "bins": [w.bmin, w.bmax], "widths": list(w.widths)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": desc.replace("every 64-th", "every 64-th (rotating)")},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------- GPU
def run_ffa(a):
    import torch

    import paper_2004_03701_gb300 as ffa

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    ffa.build()
    ffa.library()

    w = workload(a.workload)
    x = torch.from_numpy(w.x).to(dev)
    s = ffa.Searcher(w.n, w.tsamp, w.pmin, w.pmax, w.bmin, w.bmax, w.widths, device=dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(max(3, a.warmup)):
        s(x)
    s.check()
    barrier()

    # ---- timed region (no profiling events): headline device time per step
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = ffa.launch_count()
    times = []
    for _ in range(a.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s(x)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    launches = ffa.launch_count() - launches0
    barrier()
    clk = clocks.stop()
    t_step = sum(times) / len(times)
    if world > 1:
        tt = torch.tensor([t_step], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        t_step = float(tt.item())
    value = world * w.n / (t_step * 1e-3)

    # ---- same steps with per-kernel CUDA events on the launching stream
    ffa.profile_reset()
    ffa.profile_enable(True)
    for _ in range(a.steps):
        flush.zero_()
        s(x)
    torch.cuda.synchronize()
    ffa.profile_enable(False)
    kern = {}
    for name in ffa.kernel_names():
        q = ffa.profile_query(name)
        if q["launches"]:
            kern[name] = q
    ffa.profile_reset()
    tot_ms = sum(k["ms"] for k in kern.values())
    top = max(kern, key=lambda k: kern[k]["ms"])
    kq = kern[top]
    avg_s = kq["ms"] / kq["launches"] * 1e-3
    bytes_per_launch = kq["alg_bytes"] / kq["launches"]
    peak, peak_kind = measured_peaks()
    achieved = bytes_per_launch / avg_s / 1e9
    roofline = {"bound": "hbm", "kernel": top, "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "traffic": recorded_traffic(top),
                "peak_source": peak_kind,
                "share_of_step": kq["ms"] / tot_ms if tot_ms else None,
                "launches_per_step": kq["launches"] / a.steps}

    # ---- end to end through the host-buffer C-ABI call (copies inside the timed call)
    e2e = None
    if not a.no_e2e:
        T, nw = s.info.ntrials, len(w.widths)
        xh = torch.from_numpy(w.x).pin_memory()
        per_h = torch.empty(T, dtype=torch.float64).pin_memory()
        fb_h = torch.empty(T, dtype=torch.int32).pin_memory()
        snr_h = torch.empty((T, nw), dtype=torch.float32).pin_memory()
        xs, ps, fs, ss = xh.numpy(), per_h.numpy(), fb_h.numpy(), snr_h.numpy()
        for _ in range(2):
            s.run_host(xs, ps, fs, ss)
        barrier()
        et = []
        for _ in range(a.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.run_host(xs, ps, fs, ss)
            et.append(time.perf_counter() - t0)
        te = sum(et) / len(et)
        if world > 1:
            tt = torch.tensor([te], device=dev, dtype=torch.float64)
            torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
            te = float(tt.item())
        e2e = {"value": world * w.n / te, "unit": UNIT, "h2d_bytes_per_step": 4 * w.n,
               "d2h_bytes_per_step": T * (8 + 4 + 4 * nw)}

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        est, desc = oracle_sample_time(w, a.cpu_sample_stride)
        cpu = {"value": w.n / est, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": t_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "n": w.n, "tsamp": w.tsamp, "pmin": w.pmin,
                       "pmax": w.pmax, "bins": [w.bmin, w.bmax], "widths": list(w.widths),
                       "ntrials": s.info.ntrials, "transforms": s.info.ntransforms,
                       "octaves": s.info.noctaves, "l2": "flushed (256 MB write) between steps",
                       "parallelism": "replicas" if world > 1 else "single"},
            "roofline": roofline,
            "kernels_ms_per_step": {k: v["ms"] / a.steps for k, v in kern.items()},
            "e2e": e2e,
            "cpu_baseline": cpu,
            "clocks": clk,
            "gpu_launches": launches,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ffa(a)


if __name__ == "__main__":
    main()
