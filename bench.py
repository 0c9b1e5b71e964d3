#!/usr/bin/env python3
"""Benchmark of the GB300 X-stage: complex multiply-accumulates per second.

One step is one pass of the whole X-stage over one integration of the
512-input workload: unpack the 4+4-bit samples, cross-multiply and integrate
on the tensor cores, and dump the packed int32 triangle (Sec. 2.1 / Sec. 2.4
of the paper: the GPU integrates K spectra and hands the matrix back).

Workload: 256 stations x 2 polarisations (512 inputs), 512 channels, K = 2048
samples, 4+4-bit complex Gaussian noise (sigma 2.5 levels) plus a common
plane-wave source, synthetic and seeded.  Work per step: C * K * N_i (N_i+1)/2
complex MACs.  The input (537 MB) and the output (538 MB) are both larger than
the 129 MB L2, so every step streams them from HBM.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank correlates its own band of 512 channels (the paper's
frequency parallelism, no data exchange) and rank 0 prints one JSON line.
"""

from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("X-stage complex MACs/s and % of GB300 int8 tensor peak vs CUDA-core kernel, "
          "bit-exact")
WORKLOADS = {
    # the headline: 512 inputs, 4+4-bit Gaussian + plane wave
    "ci4_512in": dict(name="512 inputs (256 stations x 2 pols), 512 channels, K=2048, 4+4-bit",
                      n_sta=256, n_chan=512, n_time=2048, seed=14018288 + 2, fmt="ci4",
                      gen="planewave", dtype="e4m3"),
    # the small field-system-sized case: 64 inputs
    "ci4_64in": dict(name="64 inputs (32 stations x 2 pols), 64 channels, K=1024, 4+4-bit",
                     n_sta=32, n_chan=64, n_time=1024, seed=14018288 + 1, fmt="ci4",
                     gen="uniform", dtype="e4m3"),
    # the precision ladder at 512 inputs: int8 and float spectra
    "ci8_512in": dict(name="512 inputs, 256 channels, K=4096, 8-bit complex (sigma 20)",
                      n_sta=256, n_chan=256, n_time=4096, seed=14018288 + 3, fmt="ci8",
                      gen="gauss8", dtype="bf16"),
    "cf32_512in": dict(name="512 inputs, 256 channels, K=4096, float32 complex (sigma 1)",
                       n_sta=256, n_chan=256, n_time=4096, seed=14018288 + 4, fmt="cf32",
                       gen="gauss32", dtype="bf16x3"),
    # 24 independent subarrays of uneven size in one launch (see batch_arm)
    "batch24": dict(name="24 subarrays, inputs 16..704, channels 64..1024, K 512..8192, 4+4-bit",
                    seed=14018288 + 4, fmt="ci4", dtype="e4m3"),
    # many small subarrays, where per-instance launches leave most SMs idle
    "batch_small": dict(name="64 subarrays, inputs 16..128, channels 16..256, K 512..4096, 4+4-bit",
                        seed=14018288 + 7, fmt="ci4", dtype="e4m3",
                        mix=dict(count=64, inputs=(16, 128), channels=(16, 256), samples=(512, 4096))),
    # the streaming server: F-engine packets -> device ring -> X-stage -> dumps (see stream_arm)
    # the engine choice for small problems: both engines over a grid of small sizes (see sweep_arm)
    "engine_sweep": dict(name="4-bit, inputs 2..256, channels 16..256, K 256..2048: tensor (a plan's first "
                              "shape and the small-problem shape) vs CUDA-core; 8-bit, inputs 2..256, channels "
                              "16..64, K 256..1024: tensor vs CUDA-core", seed=14018288 + 6, fmt="ci4", dtype="e4m3"),
    "stream1024": dict(name="1024 inputs (512 stations x 2 pols), 1024 channels, K=8192 per dump, "
                            "4+4-bit Gaussian in 8 KB packets (4 samples x 128 channels x 16 "
                            "inputs) + 16 B header, ring of 4 blocks of 2048 samples",
                       n_sta=512, n_chan=1024, block=2048, blocks_per_dump=4, nt=4, nch=128, na=16,
                       seed=14018288 + 5, fmt="ci4", dtype="e4m3"),
}
WORKLOAD = WORKLOADS["ci4_512in"]
# ncu DRAM traffic of the headline kernel per launch, stored beside the source hash it was taken on
KERNEL_SOURCES = {
    "xcorr_tc_fused_pair_kernel": ("xcorr_tc_fused_pair.cu", "fused_common.cuh", "sm103_ptx.cuh", "xcorr_internal.h"),
    "xcorr_tc_fused_ta_kernel": ("xcorr_tc_fused_ta.cu", "fused_common.cuh", "sm103_ptx.cuh", "xcorr_internal.h"),
    "xcorr_tc_fused_kernel": ("xcorr_tc_fused.cu", "fused_common.cuh", "sm103_ptx.cuh", "xcorr_internal.h"),
    "xcorr_tc_kernel": ("xcorr_tc.cu", "sm103_ptx.cuh", "xcorr_internal.h"),
}
FUSED_TA_VARIANTS = (4, 5, 6, 10)  # tuning stage_variants served by the tensor-memory-A fused kernel
FUSED_PAIR_VARIANTS = (7, 8, 9)  # ... and by the CTA-pair kernel


def profile_summary_path(kernel: str) -> str:
    return os.path.join(ROOT, "profiles", f"{kernel}_512in_512ch_2048t.json")


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the oracle timing on the host cores")
    ap.add_argument("--channels", type=int, default=0,
                    help="channels per GPU (a smaller case of the same kernels, for profiler "
                         "captures); 0 = the workload's own")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="ci4_512in",
                    help="the default is the headline 512-input 4-bit workload")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the library's default launch shape")
    ap.add_argument("--tuning", default="",
                    help="fix the launch shape instead of autotuning: variant,groups,x_streams")
    ap.add_argument("--tuning-cache", default="",
                    help="JSON-lines tuning cache to load before and save after (batch workloads)")
    ap.add_argument("--sustained-s", type=float, default=2.5,
                    help="seconds of back-to-back steps for the sustained record (0 = skip)")
    ap.add_argument("--graph", type=int, default=0, metavar="STEPS",
                    help="capture STEPS steps in one CUDA graph and time its replays (no host call per "
                         "step: for small workloads whose kernels are shorter than the host's calls); "
                         "--steps must be a multiple of STEPS")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    """Reads SM clock, power and clock-event reasons through NVML (read-only)
    every few milliseconds while the timed region runs."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown", 0x1: "gpu_idle",
               0x2: "applications_clocks_setting"}

    def __init__(self, local_rank: int):
        self.samples = []
        self.max_mhz = None
        self.ok = False
        self._stop = threading.Event()
        try:
            nv = ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                return
            count = ctypes.c_uint()
            nv.nvmlDeviceGetCount_v2(ctypes.byref(count))
            index = 0
            vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
            first = vis.split(",")[local_rank] if vis and len(vis.split(",")) > local_rank else ""
            if count.value > 1:
                index = int(first) if first.isdigit() else local_rank
            self.dev = ctypes.c_void_p()
            if nv.nvmlDeviceGetHandleByIndex_v2(index, ctypes.byref(self.dev)) != 0:
                return
            mx = ctypes.c_uint()
            nv.nvmlDeviceGetMaxClockInfo(self.dev, 1, ctypes.byref(mx))  # 1 = SM clock
            self.max_mhz = mx.value
            self.nv = nv
            self.ok = True
        except OSError:
            pass

    def _sample(self):
        clk, mw, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        self.nv.nvmlDeviceGetClockInfo(self.dev, 1, ctypes.byref(clk))
        self.nv.nvmlDeviceGetPowerUsage(self.dev, ctypes.byref(mw))
        fn = getattr(self.nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.nv.nvmlDeviceGetCurrentClocksThrottleReasons
        fn(self.dev, ctypes.byref(rs))
        self.samples.append((clk.value, mw.value / 1000.0, rs.value))

    def _run(self):
        while not self._stop.is_set():
            self._sample()
            time.sleep(0.005)

    def __enter__(self):
        if self.ok:
            self._thread = threading.Thread(target=self._run, daemon=True)
            self._thread.start()
        return self

    def __exit__(self, *exc):
        if self.ok:
            self._stop.set()
            self._thread.join()
            self._sample()

    def summary(self) -> dict:
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": [],
                    "note": "NVML unavailable"}
        reasons = 0
        for _, _, r in self.samples:
            reasons |= r
        names = [n for bit, n in self.REASONS.items() if reasons & bit and n != "gpu_idle"]
        return {"sm_mhz": statistics.median(s[0] for s in self.samples),
                "sm_max_mhz": self.max_mhz, "reasons": names,
                "power_w_max": max(s[1] for s in self.samples), "samples": len(self.samples)}


# --------------------------------------------------------------- helpers --
def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def kernel_source_hash(kernel: str) -> str:
    """Hash of a kernel's sources: a stored ncu traffic figure is only
    reported while the kernel it was taken on is unchanged."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1401_8288_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def stored_traffic(kernel: str) -> float | None:
    path = profile_summary_path(kernel)
    if not os.path.exists(path):
        return None
    with open(path) as f:
        s = json.load(f)
    if s.get("source_hash") != kernel_source_hash(kernel):
        return None
    return s.get("dram_bytes_per_launch")


def emit(obj: dict) -> None:
    print(json.dumps(obj), flush=True)


def cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sample(x, fmt: str, budget_s: float, n_pairs: int) -> dict:
    """Time the oracle, as it stands, on a bounded sample of the workload: whole
    channels, one per host core per round, until about budget_s of CPU time."""
    import oracle
    ofmt = {"ci4": oracle.FMT_CI4, "ci8": oracle.FMT_CI8, "cf32": oracle.FMT_CF32}[fmt]
    cores = cpu_cores()
    n_time, n_chan = x.shape[0], x.shape[1]
    t0 = time.perf_counter()
    done = 0
    while done < n_chan:
        c1 = min(n_chan, done + cores)
        oracle.correlate(ofmt, x, c0=done, c1=c1, threads=cores)
        done = c1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": done * n_time * n_pairs / dt / 1e12, "unit": "TCMAC/s", "cores": cores,
            "kind": "oracle", "seconds": round(dt, 3),
            "sample": f"{done} of {n_chan} channels, all {n_pairs} pairs, K={n_time}",
            "build": "gcc " + " ".join(oracle.BUILD_FLAGS) + " (portable: no -march=native)"}


def oracle_check(got, x, fmt: str, channels, n_pairs_sample: int, seed: int) -> dict:
    """The step's output against the oracle, after the timed region: whole
    triangles of a few channels, then single pairs drawn across all channels
    (each computed on its own by the oracle).  Integer formats must match bit
    for bit; float output must lie within 1e-6 of sqrt(V_ii V_jj) per entry."""
    import numpy as np

    import oracle
    ofmt = {"ci4": oracle.FMT_CI4, "ci8": oracle.FMT_CI8, "cf32": oracle.FMT_CF32}[fmt]
    n_chan, n_pairs = got.shape[0], got.shape[1]
    ni = int((np.sqrt(8 * n_pairs + 1) - 1) / 2)
    rng = np.random.default_rng(seed)
    i = rng.integers(0, ni, size=n_pairs_sample)
    j = (rng.random(n_pairs_sample) * (i + 1)).astype(np.int64)
    c = rng.integers(0, n_chan, size=n_pairs_sample)
    want_pairs = oracle.correlate_pairs(ofmt, x, np.stack([c, i, j], axis=1))
    got_pairs = got[c, i * (i + 1) // 2 + j].astype(np.float64 if fmt == "cf32" else np.int64)
    what = f"channels {list(channels)} whole + {n_pairs_sample} sampled pairs"
    if fmt != "cf32":
        ok = all(np.array_equal(got[ch].astype(np.int64),
                                oracle.correlate(ofmt, x, c0=ch, c1=ch + 1, threads=len(channels))[0])
                 for ch in channels)
        ok = ok and bool(np.array_equal(got_pairs, want_pairs))
        return {"exact": bool(ok), "checked": what}
    worst = 0.0
    idx = np.arange(ni)
    autos_idx = idx * (idx + 1) // 2 + idx
    ii, jj = np.tril_indices(ni)
    order = np.argsort(ii * (ii + 1) // 2 + jj)
    for ch in channels:
        want = oracle.correlate(ofmt, x, c0=ch, c1=ch + 1, threads=len(channels))[0]
        autos = want[autos_idx, 0]
        scale = np.sqrt(autos[ii[order]] * autos[jj[order]])
        err = np.abs((got[ch, :, 0] - want[:, 0]) + 1j * (got[ch, :, 1] - want[:, 1]))
        worst = max(worst, float(np.max(err / scale)))
    auto_i = oracle.correlate_pairs(ofmt, x, np.stack([c, i, i], axis=1))[:, 0]
    auto_j = oracle.correlate_pairs(ofmt, x, np.stack([c, j, j], axis=1))[:, 0]
    err = np.abs((got_pairs[:, 0] - want_pairs[:, 0]) + 1j * (got_pairs[:, 1] - want_pairs[:, 1]))
    worst = max(worst, float(np.max(err / np.sqrt(auto_i * auto_j))))
    return {"exact": bool(worst <= 1e-6), "max_normalised_error": worst, "tolerance": 1e-6,
            "checked": what}


def make_input(w: dict, seed: int):
    from paper_1401_8288_gb300 import synth
    args = (w["n_time"], w["n_chan"], w["n_sta"])
    if w["gen"] == "planewave":
        return synth.gaussian_planewave_ci4(*args, seed=seed)
    if w["gen"] == "uniform":
        return synth.uniform_ci4(*args, seed=seed)
    if w["gen"] == "gauss8":
        return synth.gaussian_ci8(*args, seed=seed)
    return synth.gaussian_cf32(*args, seed=seed)


# ------------------------------------------------------------ reference --
def reference_arm(args) -> int:
    from paper_1401_8288_gb300 import dist
    info = dist.rank_info()
    if info.rank != 0:
        return 0  # the oracle arm runs on rank 0 alone
    import oracle
    from paper_1401_8288_gb300 import costmodel
    oracle.build()
    if args.workload in ("batch24", "batch_small"):
        emit({"impl": "reference", "unavailable": "the oracle arm times single workloads; "
              "run it per subarray size"})
        return 0
    if args.workload == "stream1024":
        emit({"impl": "reference", "unavailable": "the oracle has no packet path; its correlation "
              "rate is the reference line of the default workload"})
        return 0
    if args.workload == "engine_sweep":
        emit({"impl": "reference", "unavailable": "the sweep compares the library's own engines"})
        return 0
    w = WORKLOADS[args.workload]
    x = make_input(w, w["seed"])
    ofmt = {"ci4": oracle.FMT_CI4, "ci8": oracle.FMT_CI8, "cf32": oracle.FMT_CF32}[w["fmt"]]
    n_pairs = costmodel.n_pairs(2 * w["n_sta"])
    cores = cpu_cores()
    per_step = max(1, cores)  # channels per step: one per host core
    times = []
    for k in range(args.warmup + args.steps):
        c0 = (k * per_step) % w["n_chan"]
        c1 = min(w["n_chan"], c0 + per_step)
        t0 = time.perf_counter()
        oracle.correlate(ofmt, x, c0=c0, c1=c1, threads=cores)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append((c1 - c0, dt))
    total_cmacs = sum(n for n, _ in times) * w["n_time"] * n_pairs
    total_s = sum(t for _, t in times)
    value = total_cmacs / total_s / 1e12
    sample = f"{per_step} channels per step (one per core), all {n_pairs} pairs, K={w['n_time']}"
    emit({"impl": "reference", "metric": METRIC, "value": value, "unit": "TCMAC/s",
          "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
          "ms_per_step": 1e3 * total_s / max(1, len(times)), "higher_is_better": True,
          "scaling": "weak", "vs_baseline": None,
          "dtype": "f64" if w["fmt"] == "cf32" else "int64", "data": "synthetic",
          "config": {"workload": w["name"], "sample": sample},
          "cpu_baseline": {"value": value, "unit": "TCMAC/s", "cores": cores, "kind": "oracle",
                           "sample": sample},
          "e2e": {"value": value, "unit": "TCMAC/s", "h2d_bytes_per_step": 0,
                  "d2h_bytes_per_step": 0}})
    return 0


# ----------------------------------------------------------------- batch --
def batch_arm(args) -> int:
    """Many uneven subarrays: one execute of a batch per step (a fused launch per
    shape class, the classes side by side), replayed as a CUDA graph, against
    the same subarrays run as separate plans (per-instance launches), eagerly
    and from one graph.  Every subarray and plan is autotuned through the
    tuning cache (--tuning-cache)."""
    import torch

    from paper_1401_8288_gb300 import dist
    info = dist.init("nccl")
    torch.cuda.set_device(info.local_rank)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1401_8288_gb300 import costmodel, synth, xcorr

    w = WORKLOADS[args.workload]
    if args.tuning_cache and os.path.exists(args.tuning_cache):
        xcorr.xcorr_tuning_cache_load(args.tuning_cache)
    subs = synth.subarray_batch(w["seed"], **w.get("mix", {}))
    sizes = [(s["n_sta"], s["n_chan"], s["n_time"]) for s in subs]
    xs = [synth.uniform_ci4_torch(nt, nc, ns, seed=s["seed"] + info.rank) for (ns, nc, nt), s in zip(sizes, subs)]
    cmacs = sum(costmodel.cmacs(nc, nt, 2 * ns) for ns, nc, nt in sizes)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, steps):
        for _ in range(max(args.warmup, 3)):
            fn()
        torch.cuda.synchronize()
        dist.barrier()
        ev0.record()
        for _ in range(steps):
            fn()
        ev1.record()
        torch.cuda.synchronize()
        return dist.max_over_ranks(ev0.elapsed_time(ev1), torch.device("cuda", info.local_rank)) / steps

    batch = xcorr.Batch(sizes)
    # batch-wide shapes (0-2 planes path, 3-5 fused kernel), by replay time
    wide = {}
    for v in range(6):
        try:
            batch.set_variant(v)
        except xcorr.XcorrError:  # a fused shape for subarrays the fused kernel does not take
            continue
        batch.capture(xs)
        wide[v] = timed(batch.replay, 3)
    # a shape per subarray (its size class), timed alone or taken from the tuning cache
    per_sub = batch.autotune(xs)
    batch.capture(xs)
    ms_classes = timed(batch.replay, 3)
    best_wide = min(wide, key=wide.get)
    if wide[best_wide] < ms_classes:
        batch.set_variant(best_wide)
        chosen = {"kind": "one shape for the batch", "stage_variant": best_wide}
    else:
        chosen = {"kind": "a shape per subarray (size class): tensor-memory-A shapes 4-6 share one launch "
                          "per shape, other shapes run their subarray alone, all side by side",
                  "subarrays_per_shape": {str(v): per_sub.count(v) for v in sorted(set(per_sub))}}
    batch.capture(xs)
    with ClockSampler(info.local_rank) as clocks:
        ms_graph = timed(batch.replay, args.steps)
    batch.sync()
    outs = batch.outputs
    # the same subarrays as separate plans (each autotuned), one after another
    plans = [xcorr.Plan(ns, nc, nt) for ns, nc, nt in sizes]
    for p, x in zip(plans, xs):
        p.autotune(x, cached=True)
    per_out = [torch.empty_like(o) for o in outs]

    def each():
        for p, x, o in zip(plans, xs, per_out):
            p.execute_dump(x, o)

    ms_each = timed(each, max(2, args.steps // 4))
    same = all(torch.equal(a, b) for a, b in zip(outs, per_out))
    each()
    torch.cuda.synchronize()
    g_each = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g_each):
        each()
    ms_each_graph = timed(g_each.replay, max(2, args.steps // 4))
    same = same and all(torch.equal(a, b) for a, b in zip(outs, per_out))
    # one subarray of each size against the oracle (whole first channel + sampled pairs)
    check = []
    for k in sorted({0, len(sizes) // 2, len(sizes) - 1}):
        check.append(oracle_check(outs[k].cpu().numpy(), xs[k].cpu().numpy(), "ci4", [0], 100,
                                  seed=w["seed"] + k))
    del g_each
    for p in plans:
        p.close()
    batch.close()
    if args.tuning_cache:
        xcorr.xcorr_tuning_cache_save(args.tuning_cache)
    value = info.world * cmacs / (ms_graph * 1e-3) / 1e12
    exact = all(c["exact"] for c in check) and same
    if info.rank == 0:
        emit({"metric": METRIC, "value": value, "unit": "TCMAC/s", "n_gpus": info.world,
              "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_graph,
              "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "e4m3",
              "data": "synthetic",
              "config": {"workload": w["name"], "subarrays": sizes, "shape": chosen,
                         "per_subarray_shapes": per_sub,
                         "batch_wide_ms": {str(v): ms for v, ms in wide.items()}, "per_class_ms": ms_classes,
                         "engine": ("fused 4-bit kernels on the raw input, launched side by side"
                                    if best_wide >= 3 or wide[best_wide] >= ms_classes
                                    else "unpack per subarray + one planes X launch"),
                         "graph": True, "cmacs_per_step_per_gpu": cmacs,
                         "l2": "inputs larger than L2" if cmacs > 1e11 else "working set partly in L2"},
              "per_instance": {"value": info.world * cmacs / (ms_each * 1e-3) / 1e12,
                               "unit": "TCMAC/s", "ms_per_step": ms_each,
                               "batch_speedup": ms_each / ms_graph, "outputs_identical": same},
              "per_instance_graph": {"value": info.world * cmacs / (ms_each_graph * 1e-3) / 1e12,
                                     "unit": "TCMAC/s", "ms_per_step": ms_each_graph,
                                     "batch_speedup": ms_each_graph / ms_graph},
              "exact": exact, "parity": check,
              "gpu_launches": (len({v for v in per_sub if 4 <= v <= 6}) + sum(1 for v in per_sub if not 4 <= v <= 6))
                              * args.steps if "subarrays_per_shape" in chosen else
                              (1 if best_wide >= 3 else len(sizes) + 1) * args.steps,
              "clocks": clocks.summary()})
    dist.barrier()
    return 0 if exact else 1


# ---------------------------------------------------------- engine sweep --
def sweep_arm(args) -> int:
    """Per-call device time of one execute_dump (inputs in HBM) for the tensor
    engine at its default shape (4) and its small-problem shape (10), and for
    the CUDA-core engine, over small problem sizes: the evidence behind
    XCORR_ENGINE_AUTO and the default shape of a plan.  Achieved HBM GB/s =
    (input + output bytes) / time."""
    import torch

    from paper_1401_8288_gb300 import dist
    info = dist.init("nccl")
    torch.cuda.set_device(info.local_rank)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1401_8288_gb300 import costmodel, synth, xcorr

    rows = []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(args.steps, 20)
    grid = [("ci4", n_in, n_chan, n_time) for n_in in (2, 8, 16, 32, 64, 128, 256) for n_chan in (16, 64, 256)
            for n_time in (256, 1024, 2048)]
    grid += [("ci8", n_in, n_chan, n_time) for n_in in (2, 8, 16, 64, 256) for n_chan in (16, 64)
             for n_time in (256, 1024)]
    for fmt, n_in, n_chan, n_time in grid:
        seed = n_in * 7 + n_chan + n_time
        if fmt == "ci4":
            xd = synth.uniform_ci4_torch(n_time, n_chan, n_in // 2, seed=seed)
        else:
            xd = torch.from_numpy(synth.uniform_ci8(n_time, n_chan, n_in // 2, seed=seed)).cuda()
        n_pairs = costmodel.n_pairs(n_in)
        out = torch.empty((n_chan, n_pairs, 2), dtype=torch.int32, device="cuda")
        row = {"fmt": fmt, "n_inputs": n_in, "n_channels": n_chan, "n_time": n_time}
        shapes = (("tensor_default", "tensor", None), ("tensor_small", "tensor", 10),
                  ("cuda_core", "cuda_core", None)) if fmt == "ci4" else \
                 (("tensor_default", "tensor", None), ("cuda_core", "cuda_core", None))
        for label, engine, tuning in shapes:
            with xcorr.Plan(n_in // 2, n_chan, n_time, fmt=fmt, engine=engine) as plan:
                if tuning is not None:
                    plan.set_tuning(tuning, 0, 2, 0)
                for _ in range(max(args.warmup, 3)):
                    plan.execute_dump(xd, out)
                torch.cuda.synchronize()
                ev0.record()
                for _ in range(reps):
                    plan.execute_dump(xd, out)
                ev1.record()
                torch.cuda.synchronize()
                row[label + "_eager_us"] = round(1e3 * ev0.elapsed_time(ev1) / reps, 2)
                # the same call, 20 times in one CUDA graph: the device's own time per call
                graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(graph):
                    for _ in range(20):
                        plan.execute_dump(xd, out)
                for _ in range(2):
                    graph.replay()
                torch.cuda.synchronize()
                n_rep = max(1, reps // 20)
                ev0.record()
                for _ in range(n_rep):
                    graph.replay()
                ev1.record()
                torch.cuda.synchronize()
                row[label + "_us"] = round(1e3 * ev0.elapsed_time(ev1) / (20 * n_rep), 2)
                plan.sync()
                del graph
        nbytes = xd.numel() * xd.element_size() + out.numel() * 4
        best = min((lab for lab, _, _ in shapes), key=lambda k: row[k + "_us"])
        row["best"] = best
        row["best_hbm_gbs"] = round(nbytes / (row[best + "_us"] * 1e-6) / 1e9, 1)
        row["tcmacs_best"] = round(costmodel.cmacs(n_chan, n_time, n_in) / (row[best + "_us"] * 1e-6) / 1e12, 4)
        rows.append(row)
    if info.rank == 0:
        emit({"metric": "per-call time of one execute_dump by engine over small sizes", "unit": "us",
              "n_gpus": info.world, "steps": reps, "warmup": args.warmup, "higher_is_better": False,
              "data": "synthetic", "config": {"workload": WORKLOADS["engine_sweep"]["name"],
                                              "timing": "CUDA events around back-to-back replays of a graph of "
                                                        "20 calls (<engine>_us, per call) and around eager "
                                                        "calls (<engine>_eager_us); inputs in HBM"},
              "rows": rows})
    dist.barrier()
    return 0


# ------------------------------------------------------------------ ours --
def our_arm(args) -> int:
    import torch

    from paper_1401_8288_gb300 import dist
    info = dist.init("nccl")
    torch.cuda.set_device(info.local_rank)
    dev = torch.device("cuda", info.local_rank)

    import __graft_entry__
    __graft_entry__.build()
    from paper_1401_8288_gb300 import costmodel, xcorr

    w = dict(WORKLOADS[args.workload])
    if args.channels and args.channels != w["n_chan"]:
        w["name"] = w["name"].replace(f"{w['n_chan']} channels", f"{args.channels} channels")
        w["n_chan"] = args.channels
    n_sta, n_chan, n_time, fmt = w["n_sta"], w["n_chan"], w["n_time"], w["fmt"]
    n_in = 2 * n_sta
    n_pairs = costmodel.n_pairs(n_in)
    cmacs_per_step = costmodel.cmacs(n_chan, n_time, n_in)
    # rank r correlates channel band r of a world * n_chan-channel observation
    x = make_input(w, w["seed"] + info.rank)
    x_pin = torch.from_numpy(x).pin_memory()
    xd = x_pin.to(dev)
    in_bytes, out_bytes = x.nbytes, n_chan * n_pairs * 8

    plan = xcorr.Plan(n_sta, n_chan, n_time, fmt=fmt, engine="tensor")
    if args.tuning:
        plan.set_tuning(*[int(v) for v in args.tuning.split(",")])
        tuning = plan.query()["tuning"]
    else:
        tuning, _ = (plan.query()["tuning"], None) if args.no_autotune else plan.autotune(xd)
    launches_per_step = plan.query()["kernels_per_execute"]  # all launches of one execute
    fused = fmt == "ci4" and tuning["unfused"] == 0
    fused_ta = fused and tuning["stage_variant"] in FUSED_TA_VARIANTS
    fused_pair = fused and tuning["stage_variant"] in FUSED_PAIR_VARIANTS
    x_kernel = (("xcorr_tc_fused_pair_kernel" if fused_pair else "xcorr_tc_fused_ta_kernel" if fused_ta
                 else "xcorr_tc_fused_kernel") if fused else "xcorr_tc_kernel")
    x_launches = launches_per_step if fused else launches_per_step // 2  # else unpack + X per channel group
    out_dtype = torch.float32 if fmt == "cf32" else torch.int32
    out = torch.empty((n_chan, n_pairs, 2), dtype=out_dtype, device=dev)

    def eager_step():
        plan.execute_dump(xd, out, reset=True)

    for _ in range(max(args.warmup, 3)):
        eager_step()
    torch.cuda.synchronize()
    if args.graph:  # args.graph steps recorded once; the timed loop replays the graph
        if args.steps % args.graph:
            raise SystemExit("--steps must be a multiple of --graph")
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            for _ in range(args.graph):
                eager_step()
        replays = args.steps // args.graph
        for _ in range(max(args.warmup, 3)):
            graph.replay()
        torch.cuda.synchronize()
    else:
        replays = args.steps
        step = eager_step

    if not args.graph:
        xcorr.xcorr_profile_enable(plan.handle, args.steps)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(info.local_rank) as clocks:
        dist.barrier()
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(replays):
            graph.replay() if args.graph else step()
        ev1.record()
        torch.cuda.synchronize()
        dist.barrier()
    ms_total = ev0.elapsed_time(ev1)
    if args.graph:  # no per-launch events inside a graph: the replay time bounds the kernels' time
        kernel_ms = [(0.0, ms_total / args.steps)] * args.steps
    else:
        kernel_ms = xcorr.xcorr_profile_read(plan.handle, args.steps)
        xcorr.xcorr_profile_enable(plan.handle, 0)
    ms_total = dist.max_over_ranks(ms_total, dev)
    value = info.world * cmacs_per_step * args.steps / (ms_total * 1e-3) / 1e12
    # the last timed step's output against the oracle (outside the timed region)
    check_channels = sorted({0, n_chan // 2 + 9, n_chan - 1})
    parity = oracle_check(out.cpu().numpy(), x, fmt, check_channels, 400, seed=w["seed"] + 7)

    # sustained: the same step back to back for a few seconds, with its own clock record
    sustained = None
    if args.sustained_s > 0 and not args.graph:
        n_sus = max(100, int(args.sustained_s / (ms_total / args.steps * 1e-3)))
        xcorr.xcorr_profile_enable(plan.handle, 512)  # kernel times of the last 512 steps
        with ClockSampler(info.local_rank) as sus_clocks:
            dist.barrier()
            torch.cuda.synchronize()
            ev0.record()
            for _ in range(n_sus):
                step()
            ev1.record()
            torch.cuda.synchronize()
            dist.barrier()
        sus_ms = dist.max_over_ranks(ev0.elapsed_time(ev1), dev)
        sus_kernel = xcorr.xcorr_profile_read(plan.handle, 512)
        xcorr.xcorr_profile_enable(plan.handle, 0)
        sustained = {"seconds": sus_ms * 1e-3, "steps": n_sus,
                     "value": info.world * cmacs_per_step * n_sus / (sus_ms * 1e-3) / 1e12,
                     "unit": "TCMAC/s", "ms_per_step": sus_ms / n_sus,
                     "kernel_ms_per_step": statistics.mean(k for _, k in sus_kernel),
                     "clocks": sus_clocks.summary()}

    # end to end through the public API: pinned host input -> device -> X-stage -> host result
    host_out = torch.empty((n_chan, n_pairs, 2), dtype=out_dtype).pin_memory()

    def e2e_step():
        # xcorr_execute_dump_host: channel groups copied up, correlated and copied
        # down in a pipeline (one piece for paths the fused kernel does not take)
        plan.execute_dump_host(x_pin, host_out)

    for _ in range(max(args.warmup, 3)):
        e2e_step()
    torch.cuda.synchronize()
    dist.barrier()
    ev0.record()
    for _ in range(args.steps):
        e2e_step()
    ev1.record()
    torch.cuda.synchronize()
    e2e_ms = dist.max_over_ranks(ev0.elapsed_time(ev1), dev)
    e2e_value = info.world * cmacs_per_step * args.steps / (e2e_ms * 1e-3) / 1e12
    e2e_parity = oracle_check(host_out.numpy(), x, fmt, check_channels[:1], 200, seed=w["seed"] + 8)

    # the plain CUDA-core kernel on the same workload (integer formats)
    cc_value = cc_ms = None
    if fmt != "cf32":
        cc_steps = max(2, min(args.steps, 5))
        with xcorr.Plan(n_sta, n_chan, n_time, fmt=fmt, engine="cuda_core") as cc:
            cc.execute_dump(xd, out)
            torch.cuda.synchronize()
            ev0.record()
            for _ in range(cc_steps):
                cc.execute_dump(xd, out)
            ev1.record()
            torch.cuda.synchronize()
            cc_ms = ev0.elapsed_time(ev1) / cc_steps
        cc_value = cmacs_per_step / (cc_ms * 1e-3) / 1e12
    plan.close()

    # measured arithmetic peaks of this device
    peak_e4m3 = xcorr.xcorr_measure_peak("tc_e4m3")
    peak_s8 = xcorr.xcorr_measure_peak("mma_sync_s8")
    peak_dp4a = xcorr.xcorr_measure_peak("dp4a")

    x_ms = statistics.mean(k for _, k in kernel_ms)
    unpack_ms = statistics.mean(u for u, _ in kernel_ms)
    # algorithmic work of one step: 8 operations per complex MAC, six times
    # that for the float path (its algorithm is six BF16 piece products)
    split = 6 if fmt == "cf32" else 1
    ops_per_step = split * costmodel.int8_ops(n_chan, n_time, n_in)
    achieved = ops_per_step / (x_ms * 1e-3) / 1e12
    peaks = measured_peaks()
    ratio = 2.0 if fmt == "ci4" else 1.0  # E4M3 runs at twice the BF16 rate
    if "bf16_tflops" in peaks:
        peak = ratio * peaks["bf16_tflops"]
        peak_note = (("E4M3 dense = 2 x " if ratio == 2 else "BF16 dense = ")
                     + "measured bf16 burst (MEASURED_PEAKS.json); of measured")
    else:
        peak = ratio * 1900.0
        peak_note = "bf16 1.9 PFLOP/s x fp8:bf16 ratio; of fallback"

    if sustained is not None:
        sus_peak = ratio * peaks.get("bf16_tflops_sustained", 1700.0)
        sus_achieved = ops_per_step / (sustained["kernel_ms_per_step"] * 1e-3) / 1e12
        sustained["roofline"] = {"achieved": sus_achieved, "peak": sus_peak, "unit": "TFLOP/s",
                                 "frac": sus_achieved / sus_peak,
                                 "peak_source": ("2 x " if ratio == 2 else "") + "measured bf16 sustained "
                                                "(MEASURED_PEAKS.json); of measured"
                                                if "bf16_tflops_sustained" in peaks else "of fallback"}

    hbm = {"bytes_per_step": in_bytes + out_bytes,
           "achieved_gbs": (in_bytes + out_bytes) / (x_ms * 1e-3) / 1e9,
           "peak_gbs": peaks.get("hbm_gbs", 6800.0),
           "peak_source": "MEASURED_PEAKS.json hbm_gbs; of measured" if "hbm_gbs" in peaks else "of fallback"}
    hbm["frac"] = hbm["achieved_gbs"] / hbm["peak_gbs"]

    result = {
        "metric": METRIC,
        "value": value,
        "unit": "TCMAC/s",
        "n_gpus": info.world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_total / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": w["dtype"],
        "data": "synthetic",
        "config": {"workload": w["name"],
                   "input": {"planewave": "4+4-bit complex, Gaussian sigma 2.5 levels + common "
                                          "plane wave 0.3 sigma",
                             "uniform": "4+4-bit complex, uniform integers in [-7, 7]",
                             "gauss8": "int8 complex, Gaussian sigma 20 clipped to +-127",
                             "gauss32": "float32 complex, Gaussian sigma 1"}[w["gen"]],
                   "engine": {"ci4": ("tcgen05 kind::f8f6f4 cta_group::2 on SM pairs (cluster of 2) "
                                      "sharing a column tile, M = 256: each SM decodes its row tile "
                                      "into tensor memory (ldmatrix.trans + tcgen05.st) and half of "
                                      "the column tile into shared memory (offset-binary E4M3 codes "
                                      "u = t + 8, exact FP32 TMEM sums, per-input sum correction, "
                                      "int32 out)") if fused_pair else
                                     ("tcgen05 kind::f8f6f4, unpack fused on chip, A operand decoded "
                                      "into tensor memory (ldmatrix.trans + tcgen05.st), B in shared "
                                      "memory (offset-binary E4M3 codes u = t + 8, exact FP32 TMEM "
                                      "sums, per-input sum correction, int32 out)") if fused_ta else
                                     ("tcgen05 kind::f8f6f4, unpack fused on chip (offset-binary "
                                      "E4M3 codes u = t + 8, exact FP32 TMEM sums, per-input sum "
                                      "correction, int32 out)") if fused else
                                     ("tcgen05 kind::f8f6f4 (E4M3 codes of 4-bit integers, exact "
                                      "FP32 TMEM sums drained to int32)"),
                              "ci8": "tcgen05 kind::f16 (BF16 copies of int8 values, exact FP32 "
                                     "sums drained to int32 every 384 samples)",
                              "cf32": "tcgen05 kind::f16 (three BF16 pieces per value, six piece "
                                      "products, FP32 sums drained every 384 samples)"}[fmt],
                   "tuning": tuning,
                   "l2": f"inputs larger than L2 ({in_bytes / 1e6:.0f} MB in, "
                         f"{out_bytes / 1e6:.0f} MB out per step)",
                   "parallelism": f"frequency bands x{info.world}",
                   "cmacs_per_step_per_gpu": cmacs_per_step},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak,
                     "traffic": stored_traffic(x_kernel) if args.workload == "ci4_512in" else None,
                     "kernel": x_kernel, "ops_per_step": ops_per_step,
                     "launches_per_step": x_launches, "kernel_ms_per_step": x_ms,
                     "peak_source": peak_note,
                     "frac_of_probe_peak": achieved / (peak_e4m3 if fmt == "ci4" else peak_e4m3 / 2)},
        "exact": parity["exact"] and e2e_parity["exact"],
        "hbm_view": hbm,
        "parity": {"timed_output": parity, "e2e_output": e2e_parity},
        "e2e": {"value": e2e_value, "unit": "TCMAC/s", "h2d_bytes_per_step": in_bytes,
                "d2h_bytes_per_step": out_bytes, "ms_per_step": e2e_ms / args.steps},
        "gpu_launches": launches_per_step * args.steps,
        "timing": (f"CUDA graphs of {args.graph} steps replayed (kernel_ms_per_step is the replay time per "
                   "step)" if args.graph else "eager calls; kernel times from events recorded around each launch"),
        "clocks": clocks.summary(),
        "sustained": sustained,
        # GB300 keeps no tcgen05 int8 kind; its int8 tensor path is warp-level mma.sync s8,
        # measured at the rate below.  The X-stage's useful integer operations per second are
        # this many times that rate.
        "x_ops_over_mma_sync_s8_rate": 8 * value * 1e12 / info.world / (peak_s8 * 1e12),
        "peaks_measured_tops": {"tcgen05_e4m3": peak_e4m3, "mma_sync_s8": peak_s8,
                                "dp4a": peak_dp4a},
        "cuda_core": {"value": cc_value, "unit": "TCMAC/s", "ms_per_step": cc_ms,
                      "speedup_tensor_vs_cuda_core": (value / info.world / cc_value)
                      if cc_value else None},
        "kernels_ms": {"unpack_span": unpack_ms, "x_tensor_sum": x_ms,
                       "note": ("per step: the fused kernel has no separate unpack (span ~0); "
                                "x_tensor_sum is its duration") if fused else
                               ("per step: start to end of the last unpack, and the summed "
                                "durations of the X launches (channel groups overlap the "
                                "unpack of the next group with the X kernel of this one)")},
    }
    if info.rank == 0 and info.world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = oracle_sample(x, fmt, budget_s=12.0, n_pairs=n_pairs)
    if info.rank == 0:
        emit(result)
    dist.barrier()
    return 0 if result["exact"] else 1


def h2d_ceiling(torch, nbytes: int, reps: int = 6) -> dict:
    """Pinned host -> device copy rate of chunk-sized copies, on one stream and
    on two streams at once (the link ceiling for the stream's input)."""
    hp = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    dps = [torch.empty(nbytes, dtype=torch.uint8, device="cuda") for _ in range(2)]
    streams = [torch.cuda.Stream() for _ in range(2)]
    out = {}
    for n_str in (1, 2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for r in range(reps):
            for q in range(n_str):
                with torch.cuda.stream(streams[q]):
                    dps[q].copy_(hp, non_blocking=True)
        torch.cuda.synchronize()
        out[f"{n_str}_stream" + ("s" if n_str > 1 else "")] = n_str * reps * nbytes / (time.perf_counter() - t0) / 1e9
    return out


def stream_arm(args) -> int:
    """The streaming server of the paper's Fig. 4 on one GPU: an F-engine
    emulator fills the stream's pinned landing chunks with packets, the stream
    places them on the device, correlates each 2048-sample block and copies
    every 8192-sample dump to host memory.  The emulator writes each chunk's
    payloads once (one block of Gaussian samples) and then only advances the
    headers' sequence numbers, the way a NIC would deliver packets by DMA
    without the CPU touching the payload; so every block carries the same
    samples and a dump must equal 4 x the block's correlation."""
    import numpy as np
    import torch

    from paper_1401_8288_gb300 import dist
    info = dist.init("nccl")
    torch.cuda.set_device(info.local_rank)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1401_8288_gb300 import costmodel, synth, xcorr

    w = WORKLOADS["stream1024"]
    n_sta, n_chan, block, bpd = w["n_sta"], w["n_chan"], w["block"], w["blocks_per_dump"]
    n_in = 2 * n_sta
    n_groups, n_feng = n_chan // w["nch"], n_in // w["na"]
    per_block = (block // w["nt"]) * n_groups * n_feng
    chunks_per_block = 8
    # two blocks of landing chunks: a chunk whose scatter waits behind a long X
    # launch does not hold up the next copies
    cfg = xcorr.stream_config(w["nt"], w["nch"], w["na"], block, n_blocks=4, blocks_per_dump=bpd,
                              stack_threshold=per_block // 4, chunk_packets=per_block // chunks_per_block,
                              n_chunks=2 * chunks_per_block, n_host_dumps=2)
    xd = synth.gaussian_ci4_torch(block, n_chan, n_sta, seed=w["seed"] + info.rank)
    x = xd.cpu().numpy().reshape(block, n_chan, n_in)
    plan = xcorr.Plan(n_sta, n_chan, block)
    tuning = plan.query()["tuning"] if args.no_autotune else plan.autotune(xd)[0]
    del xd
    packets = xcorr.xcorr_packetize(x, cfg)
    pb = xcorr.packet_bytes(cfg)
    seq_per_block = (block // w["nt"]) * n_groups

    stream = xcorr.Stream(plan, cfg)
    views = {}
    host_s = {"acquire": 0.0, "emulator": 0.0, "commit": 0.0}

    def push_block(b):
        # chunk buffer q always carries the (q mod 8)-th eighth of a block: written
        # whole once, then only moved ahead in time by whole blocks per reuse
        for k in range(chunks_per_block):
            t0 = time.perf_counter()
            ptr, cap = stream.acquire()
            t1 = time.perf_counter()
            if ptr not in views:
                views[ptr] = b
                dst = np.ctypeslib.as_array((ctypes.c_uint8 * (cap * pb)).from_address(ptr)).reshape(cap, pb)
                dst[:] = packets[k * cap:(k + 1) * cap]
                xcorr.xcorr_packets_advance(ptr, pb, cap, b * seq_per_block)
            else:
                xcorr.xcorr_packets_advance(ptr, pb, cap, (b - views[ptr]) * seq_per_block)
                views[ptr] = b
            t2 = time.perf_counter()
            stream.commit(cap)
            t3 = time.perf_counter()
            host_s["acquire"] += t1 - t0
            host_s["emulator"] += t2 - t1
            host_s["commit"] += t3 - t2

    warm_dumps = max(1, args.warmup // 4)
    n_dumps = max(2, args.steps)
    for b in range(warm_dumps * bpd):
        push_block(b)
    stream.wait_dump(warm_dumps - 1, timeout_ms=120000, copy=False)
    torch.cuda.synchronize()
    for key in host_s:
        host_s[key] = 0.0
    with ClockSampler(info.local_rank) as clocks:
        t0 = time.perf_counter()
        for b in range(warm_dumps * bpd, (warm_dumps + n_dumps) * bpd):
            push_block(b)
        recs = [stream.wait_dump(k, timeout_ms=120000, copy=False) for k in range(warm_dumps, warm_dumps + n_dumps)]
        wall = time.perf_counter() - t0
    last = stream.wait_dump(warm_dumps + n_dumps - 1, copy=True)
    counters, _ = stream.counters()
    stream.close()
    plan.close()
    h2d = h2d_ceiling(torch, cfg.chunk_packets * pb)
    # a sampled channel of the last dump against the oracle: 4 identical blocks
    import oracle
    c = 5
    want = 4 * oracle.correlate(oracle.FMT_CI4, x[:, c:c + 1].reshape(block, 1, n_sta, 2))
    exact = bool(np.array_equal(last["data"][c:c + 1].astype(np.int64), want))
    payload_bytes = n_dumps * bpd * per_block * (pb - xcorr.XCORR_PACKET_HEADER_BYTES)
    cmacs = n_dumps * bpd * costmodel.cmacs(n_chan, block, n_in)
    lat = sorted(r["latency_ms"] for r in recs)
    result = {
        "metric": "streaming X-stage sustained input rate and dump latency",
        "value": payload_bytes * 8 / wall / 1e9,
        "unit": "Gbit/s",
        "n_gpus": info.world,
        "steps": n_dumps,
        "warmup": warm_dumps,
        "ms_per_step": 1e3 * wall / n_dumps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "e4m3",
        "data": "synthetic",
        "config": {"workload": w["name"], "tuning": tuning, "step": "one dump (4 blocks)",
                   "stack_threshold": cfg.stack_threshold, "chunk_packets": cfg.chunk_packets,
                   "n_chunks": cfg.n_chunks},
        "tcmacs": cmacs / wall / 1e12,
        "dump_latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                            "max": lat[-1]},
        "packets": counters,
        "h2d_ceiling_gbs": h2d,
        "host_ms_per_dump": {k: 1e3 * v / n_dumps for k, v in host_s.items()},
        "sampled_channel_exact": exact,
        "clocks": clocks.summary(),
    }
    if info.rank == 0:
        emit(result)
    dist.barrier()
    return 0 if exact else 1


def main() -> int:
    args = parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    if args.workload in ("batch24", "batch_small"):
        return batch_arm(args)
    if args.workload == "stream1024":
        return stream_arm(args)
    if args.workload == "engine_sweep":
        return sweep_arm(args)
    return our_arm(args)


if __name__ == "__main__":
    sys.exit(main())
