#!/usr/bin/env python
"""Throughput benchmark of the n-th order DMAS + CF beamformer.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME]

A step is one frame through the whole path (signed roots, gather + power sums
+ Newton-Girard + CF, envelope) with the frame already resident in HBM.  L2 is
flushed (a 256 MB write) before every timed step, outside the step's CUDA
events.  The default workload is the 3-D hemisphere scene at 5th order: 32
microphones, 2048 directions, 16384 samples, linear (fractional) delays.

Prints ONE JSON line (rank 0).  Under torchrun each rank beamforms its own
frames on its own GPU with no data exchange (weak scaling); the step time is
the maximum over ranks.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (the reference implementation of the paper's
method is not available as code).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from workloads import scenes  # noqa: E402

METRIC = "direction·samples/s for 5th-order DMAS+CF at N=32 mics; p50/p99 frame latency"
UNIT = "direction·samples/s"

# MEASURED_PEAKS.json carries the HBM and tensor peaks; the FP32 ALU peak of
# this path is derived from the unit counts: the device's SM count x 128 FP32
# lanes x the maximum SM clock (2032 MHz on B300).
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2032.0


def measured_peaks() -> dict:
    """MEASURED_PEAKS.json next to this file (copy bandwidth and bf16 GEMM rate
    measured on this machine type), else the stated fallback figures."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "source": "measured (MEASURED_PEAKS.json)"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "source": "fallback"}

WORKLOADS = {
    "hemi_3d_n5": dict(
        scene=lambda: scenes.hemi_3d(seed=2), order=5, mode="linear",
        text="3-D hemisphere: 32 mics in a 12 cm disc, 2048 Fibonacci directions, "
             "16384 samples at 450 kHz, 8 reflectors, 10 dB SNR, n=5, linear delays, "
             "CF, 181-tap envelope"),
    "hemi_3d_n5_round": dict(
        scene=lambda: scenes.hemi_3d(seed=2), order=5, mode="round",
        text="3-D hemisphere as hemi_3d_n5 with nearest-sample delays"),
    "small_2d_n5": dict(
        scene=lambda: scenes.small_2d(seed=1), order=5, mode="round",
        text="2-D fan: 32 mics in a 12 cm disc, 91 azimuths, 4096 samples at 450 kHz, "
             "3 reflectors, 20 dB SNR, n=5, nearest-sample delays, CF, 181-tap envelope"),
    "passive64_n5": dict(
        scene=lambda: scenes.passive(seed=4, n_mics=64), order=5, mode="round",
        text="passive: 64 mics in a 0.4 m square, 8192 az/el directions, 32768 samples "
             "at 400 kHz, 4 broadband sources, 0 dB SNR, n=5, nearest-sample delays, "
             "CF, 161-tap envelope"),
    # the paper's timing workload (Table II): N = 32, 1000 directions, 163840
    # samples (the reading in which the stated sample count is processed),
    # DMAS5 without CF; delay mode unstated (nearest sample here), envelope
    # included here.  The paper's fastest GPU, an RTX 3090, took 40 ms.
    "paper_2d_1000_n5": dict(
        scene=lambda: scenes.small_2d(seed=1, n_samples=163840, n_dirs=1000), order=5,
        mode="round", cf=False, paper_rate=1000 * 163840 / 40e-3,
        text="the paper's timing configuration: 32 mics in a 12 cm disc, 1000 azimuths "
             "over -90..90 deg, 163840 samples at 450 kHz, n=5 without CF, "
             "nearest-sample delays, 181-tap envelope; vs_baseline against the paper's "
             "RTX 3090 (40 ms per frame, Table II)"),
    # the paper's full pipeline: chirp echoes, the eRTIS call (2.5 ms, 25 to
    # 50 kHz, 1125 taps) as the matched filter before the roots
    "hemi_3d_n5_mf": dict(
        scene=lambda: scenes.hemi_3d(seed=2, pulse="chirp"), order=5, mode="linear",
        mf=True,
        text="3-D hemisphere as hemi_3d_n5 with chirp echoes and the matched filter "
             "(the emitted 2.5 ms 25-50 kHz chirp, 1125 taps) before the roots"),
    "passive64_n3": dict(
        scene=lambda: scenes.passive(seed=4, n_mics=64), order=3, mode="round",
        text="passive as passive64_n5 at n=3"),
    "passive64_n5_linear": dict(
        scene=lambda: scenes.passive(seed=4, n_mics=64), order=5, mode="linear",
        text="passive as passive64_n5 with linear (fractional) delays"),
    "passive256_n3": dict(
        scene=lambda: scenes.passive(seed=4, n_mics=256), order=3, mode="round",
        text="passive as passive256_n5 at n=3"),
    "passive256_n5": dict(
        scene=lambda: scenes.passive(seed=4, n_mics=256), order=5, mode="round",
        text="passive: 256 mics in a 0.4 m square, 8192 az/el directions, 32768 samples "
             "at 400 kHz, 4 broadband sources, 0 dB SNR, n=5, nearest-sample delays, "
             "CF, 161-tap envelope"),
}


# DRAM bytes (read + write) of one beamform launch on the default workload,
# from one ncu capture of that kernel (the profile summary of the
# interpolated-delay pair kernel on the hemisphere frame), valid only while
# the kernel source is the one that was measured; otherwise the line's
# "traffic" is null and "traffic_note" says why.
TRAFFIC_RECORD = {"workload": "hemi_3d_n5", "ng": "cf32", "kernel_src_sha256_16": "9eaadf1d3864f53f",
                  # ncu dram__bytes_read.sum + dram__bytes_write.sum (bytes)
                  "bytes": 5_145_600 + 76_103_680}


def beam_traffic(workload: str, ng: str = "cf32"):
    import hashlib
    src = os.path.join(ROOT, "paper_2511_09165_b300", "csrc", "dmas_kernels.cuh")
    with open(src, "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()[:16]
    if (workload == TRAFFIC_RECORD["workload"] and ng == TRAFFIC_RECORD.get("ng", "cf32")
            and sha == TRAFFIC_RECORD["kernel_src_sha256_16"]):
        return TRAFFIC_RECORD["bytes"], "one ncu capture of this kernel on this workload"
    if workload != TRAFFIC_RECORD["workload"] or ng != TRAFFIC_RECORD.get("ng", "cf32"):
        return None, ("no DRAM capture recorded for this workload and Newton-Girard form; "
                      f"the recorded one is {TRAFFIC_RECORD['workload']} with "
                      f"{TRAFFIC_RECORD.get('ng', 'cf32')}")
    return None, "the kernel source changed since its DRAM traffic was captured"


NG_PREC = {"cf32": lambda dm: dm.NG_CF32, "f64": lambda dm: dm.NG_F64,
           "f32": lambda dm: dm.NG_F32}
NG_TEXT = {"cf32": "compensated FP32 (compensated Horner over Eqs. dmas2_impl..dmas5_impl)",
           "f64": "FP64", "f32": "plain FP32 (variant)"}


def algorithmic_ops_per_pixel(N: int, n: int, linear: bool) -> dict:
    """FP32 operations one output pixel needs (FADD, FMUL and FFMA each count 1):
    N(n+2) channel accumulations (twice with interpolation), ~n(n+1)/2 + n
    Newton-Girard mult-adds, 6 for CF and weighting; the envelope adds L."""
    main = N * (n + 2) * (2 if linear else 1)
    ng = n * (n + 1) // 2 + n
    return {"main": main, "newton_girard": ng, "cf": 6, "beam_total": main + ng + 6}


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ["clocks.sm", "clocks.max.sm", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self, t0: float, t1: float) -> dict:
        rows = []
        for ts, line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) != len(self.FIELDS):
                continue
            rows.append((ts, parts))
        inside = [r for r in rows if t0 <= r[0] <= t1] or rows
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(p[0]) for _, p in inside if p[0].replace(".", "").isdigit()]
        mx = [float(p[1]) for _, p in inside if p[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, p in inside for k in range(4)
                          if p[3 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(inside)}


# ---------------------------------------------------------------------------
# distributed plumbing (torchrun): barrier and max over ranks only
# ---------------------------------------------------------------------------
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(world: int, backend: str):
    if world <= 1:
        return None
    import torch.distributed as td
    if not td.is_initialized():
        td.init_process_group(backend=backend)
    return td


def dist_max(td, value: float, device) -> float:
    if td is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.item())


def dist_barrier(td):
    if td is not None:
        td.barrier()


# ---------------------------------------------------------------------------
# CPU oracle timing
# ---------------------------------------------------------------------------
def oracle_sample(scene, order, linear, n_dirs, cf=True, mf=False):
    import oracle
    u = scene.dir_unit if scene.dir_unit is not None else oracle.unit_vectors(scene.dir_azel)
    tau = oracle.geometric_delays(scene.mic_xyz, u, scene.c)
    taps = oracle.fir_taps(scene.fs, 5000.0)
    frame = scene.frame.astype(np.float64)
    D = min(n_dirs, scene.n_dirs)
    t0 = time.perf_counter()
    if mf:
        frame = oracle.matched_filter(frame, scenes.lfm_chirp(scene.fs).astype(np.float32))
    oracle.dmas(frame, tau, scene.fs, order, oracle.LINEAR if linear else oracle.ROUND,
                use_cf=cf, taps=taps, dir_range=(0, D))
    dt = time.perf_counter() - t0
    return D * scene.n_samples, dt


def cpu_baseline(scene, order, linear, cf=True, mf=False, min_s=10.0) -> dict:
    """The oracle as it stands, on all host cores: whole frames of the workload
    (or a direction subset if a frame takes longer than min_s), repeated until
    at least min_s seconds of CPU work."""
    import oracle
    cores = oracle.set_threads(os.cpu_count() or 1)
    px, dt = oracle_sample(scene, order, linear, 64, cf, mf)
    D = int(max(64, min(scene.n_dirs, min_s * px / dt / scene.n_samples)))
    total_px, total_s, reps = 0, 0.0, 0
    while total_s < min_s:
        px, dt = oracle_sample(scene, order, linear, D, cf, mf)
        total_px += px
        total_s += dt
        reps += 1
    what = "all" if D == scene.n_dirs else f"directions 0..{D - 1} of"
    # one core, on a smaller direction subset (about min_s / 4 seconds)
    oracle.set_threads(1)
    px1, dt1 = oracle_sample(scene, order, linear, 8, cf, mf)
    D1 = int(max(8, min(scene.n_dirs, 0.25 * min_s * px1 / dt1 / scene.n_samples)))
    px1, dt1 = oracle_sample(scene, order, linear, D1, cf, mf)
    oracle.set_threads(cores)
    return {"value": total_px / total_s, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{reps} x ({what} {scene.n_dirs} directions x {scene.n_samples} "
                      f"samples), {total_s:.1f} s, FP64",
            "single_core": {"value": px1 / dt1, "sample": f"directions 0..{D1 - 1}, "
                                                          f"{dt1:.1f} s"},
            "cpu_model": cpu_model()}


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def run_reference(args, wl, scene) -> None:
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    linear = wl["mode"] == "linear"
    cf, mf = wl.get("cf", True), bool(wl.get("mf"))
    cores = oracle.set_threads(os.cpu_count() or 1)
    px, dt = oracle_sample(scene, wl["order"], linear, 16, cf, mf)
    rate = px / dt
    D = int(max(8, min(scene.n_dirs, 0.4 * rate / scene.n_samples)))  # ~0.4 s a step
    for _ in range(args.warmup):
        oracle_sample(scene, wl["order"], linear, D, cf, mf)
    times = []
    for _ in range(args.steps):
        px, dt = oracle_sample(scene, wl["order"], linear, D, cf, mf)
        times.append(dt)
    value = px * len(times) / sum(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "description": wl["text"],
                   "step": f"oracle on directions 0..{D - 1} x {scene.n_samples} samples"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{D} directions x {scene.n_samples} samples per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our path
# ---------------------------------------------------------------------------
def run_ours(args, wl, scene) -> None:
    import torch
    import paper_2511_09165_b300 as dm

    world, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    td = dist_init(world, "nccl")
    linear = wl["mode"] == "linear"
    order = wl["order"]
    cf = wl.get("cf", True)
    mf = scenes.lfm_chirp(scene.fs).astype(np.float32) if wl.get("mf") else None
    plan_kw = dict(mic_xyz=scene.mic_xyz, dir_azel=scene.dir_azel, dir_unit=scene.dir_unit,
                   n_samples=scene.n_samples, fs=scene.fs, c=scene.c, order=order,
                   delay_mode=dm.LINEAR if linear else dm.ROUND, cf=cf, mf_signal=mf)
    plan = dm.Plan(ng_prec=NG_PREC[args.ng](dm), **plan_kw)
    info = plan.info()
    N, M, T = scene.n_mics, scene.n_dirs, scene.n_samples
    px = M * T
    stream = torch.cuda.current_stream(dev)
    frame = torch.from_numpy(scene.frame).to(dev)
    image = torch.empty((M, T), device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, device=dev)

    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        plan(frame, out=image, stream=stream)
    torch.cuda.synchronize(dev)
    plan.check()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stage = []
    dist_barrier(td)
    torch.cuda.synchronize(dev)
    wall0 = time.time()
    for k in range(args.steps):
        flush.zero_()
        ev0[k].record(stream)
        plan(frame, out=image, stream=stream)
        ev1[k].record(stream)
    torch.cuda.synchronize(dev)
    dist_barrier(td)
    wall1 = time.time()
    plan.check()
    step_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    total_ms = dist_max(td, sum(step_ms), dev)
    ms_per_step = total_ms / args.steps
    value = px * world * args.steps / (total_ms * 1e-3)

    # per-stage times, from a separate run with the plan's stage events (reading
    # them synchronises after every step, which the timed steps above avoid)
    plan.set_profiling(True)
    for _ in range(min(args.steps, 50)):
        flush.zero_()
        plan(frame, out=image, stream=stream)
        stage.append(plan.stage_ms())
    plan.set_profiling(False)
    stage = np.array(stage)

    # the other Newton-Girard arithmetics on the same frame: beamform stage
    # only (named variants, never the line's value)
    ng_variants = {}
    for name in NG_PREC:
        if name == args.ng:
            continue
        vp = dm.Plan(ng_prec=NG_PREC[name](dm), **plan_kw)
        vp.set_profiling(True)
        vt = []
        for _ in range(min(args.steps, 20)):
            flush.zero_()
            vp(frame, out=image, stream=stream)
            vt.append(vp.stage_ms()[1])
        vp.check()
        vp.close()
        ng_variants[name] = float(np.mean(vt[1:] if len(vt) > 1 else vt))

    # small frames: the same step replayed from a CUDA graph (the path only
    # enqueues kernels, so it captures), which removes the host launch gaps
    graph_ms = None
    if px <= (1 << 23):
        gs = torch.cuda.Stream(dev)
        with torch.cuda.stream(gs):
            plan.set_profiling(False)
            plan(frame, out=image, stream=gs)
            gs.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=gs):
                plan(frame, out=image, stream=gs)
            for _ in range(10):
                g.replay()
            ga, gb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            n_rep = 200
            ga.record(gs)
            for _ in range(n_rep):
                g.replay()
            gb.record(gs)
            gs.synchronize()
            graph_ms = ga.elapsed_time(gb) / n_rep
            del g
        plan.check()

    # end to end through the host-buffer entry point (pinned host memory)
    h_frame = torch.from_numpy(scene.frame).pin_memory()
    h_image = torch.empty((M, T), dtype=torch.float32).pin_memory()
    for _ in range(3):
        plan.beamform_host_ptr(h_frame.data_ptr(), h_image.data_ptr(), stream=stream)
    e2e_steps = max(3, min(args.steps, 50))
    e2e_t = []
    dist_barrier(td)
    for _ in range(e2e_steps):
        t0 = time.perf_counter()
        plan.beamform_host_ptr(h_frame.data_ptr(), h_image.data_ptr(), stream=stream)
        e2e_t.append(time.perf_counter() - t0)
    e2e_total = dist_max(td, sum(e2e_t), dev)
    clocks.stop()
    plan.close()

    # serving: a short leg of Poisson arrivals from the 16-sensor mix (the
    # metric's latency half), through the continuous-batching server and the
    # one-frame-per-launch baseline, latency to the device-resident image and
    # to the image copied to host memory
    serve = None
    if args.serve_leg_seconds > 0 and args.workload == "hemi_3d_n5":
        serve, _ = serving_measure([200.0], args.serve_leg_seconds, rank,
                                   to_host_rates=[100.0])

    if rank != 0:
        return
    ops = algorithmic_ops_per_pixel(N, order, linear)
    beam_ms = float(np.mean(stage[:, 1]))
    env_ms = float(np.mean(stage[:, 2]))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sms * FP32_LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e12   # T op/s
    achieved = ops["beam_total"] * px / (beam_ms * 1e-3) / 1e12
    # the whole per-pixel path (beamform + envelope, L taps), as one roofline
    path_ops = ops["beam_total"] + info.env_taps
    peaks = measured_peaks()
    traffic = beam_traffic(args.workload, args.ng)
    roots_ms = float(np.mean(stage[:, 0]))
    roots_bytes = N * T * 4 + N * info.row * 4 * (2 if linear else 1)
    roots_gbs = roots_bytes / (roots_ms * 1e-3) / 1e9
    path_achieved = path_ops * px / ((beam_ms + env_ms) * 1e-3) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": (value / wl["paper_rate"]) if "paper_rate" in wl else None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "description": wl["text"],
                   "n_mics": N, "n_dirs": M, "n_samples": T, "order": order,
                   "delays": wl["mode"], "cf": cf, "ng": args.ng,
                   "newton_girard": NG_TEXT[args.ng],
                   "l2": "flushed (256 MB write) before every step",
                   "parallelism": f"replicas x{world}"},
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                       "p99": float(np.percentile(step_ms, 99))},
        "stage_ms": {("matched filter + roots" if mf is not None else "roots"):
                     float(np.mean(stage[:, 0])), "beamform": beam_ms,
                     "envelope": float(np.mean(stage[:, 2]))},
        "roofline": {"bound": "alu", "kernel": "beamform_x2_kernel", "achieved": achieved,
                     "peak": peak, "unit": "Top/s", "frac": achieved / peak,
                     "ops_per_pixel": ops, "pixels_per_launch": px,
                     "peak_source": f"{sms} SMs (device properties) x 128 FP32 lanes x "
                                    f"{SM_MAX_MHZ:.0f} MHz (max SM clock)",
                     "traffic": traffic[0], "traffic_note": traffic[1],
                     "algorithmic_bytes": px * 4 + N * T * 4 * (2 if linear else 1),
                     "path": {"stages": "beamform + envelope", "ops_per_pixel": path_ops,
                              "achieved": path_achieved, "frac": path_achieved / peak},
                     # K1 alone: the roots kernel reads the frame and writes the root
                     # rows (twice with interpolation): an HBM-bound pass
                     "roots": None if mf is not None else {
                         "bound": "hbm", "unit": "GB/s", "bytes": roots_bytes,
                         "achieved": roots_gbs, "peak": peaks["hbm_gbs"],
                         "frac": roots_gbs / peaks["hbm_gbs"], "peak_source": peaks["source"]}},
        "e2e": {"value": px * world * e2e_steps / e2e_total, "unit": UNIT,
                "h2d_bytes_per_step": N * T * 4, "d2h_bytes_per_step": M * T * 4},
        "gpu_launches": (4 if mf is not None else 3) * args.steps,
        "graph_replay_ms_per_step": graph_ms,
        "clocks": clocks.summary(wall0, wall1),
        "plan": {"window": info.window, "mic_chunk": info.mic_chunk,
                 "groups": info.n_groups},
    }
    line["ng_variants_beamform_ms"] = {
        name: {"beamform_ms": ms, "frac": ops["beam_total"] * px / (ms * 1e-3) / 1e12 / peak}
        for name, ms in ng_variants.items()}
    if serve is not None:
        at = serve["200_fps"]["server"]
        line["serving_200fps"] = {
            "p50_ms": at.get("p50_ms"), "p99_ms": at.get("p99_ms"),
            "baseline_p50_ms": serve["200_fps"]["one_frame_per_launch"].get("p50_ms"),
            "baseline_p99_ms": serve["200_fps"]["one_frame_per_launch"].get("p99_ms"),
            "to_host_100fps_p50_ms": serve["100_fps_to_host"]["server"].get("p50_ms"),
            "to_host_100fps_p99_ms": serve["100_fps_to_host"]["server"].get("p99_ms"),
            "to_host_100fps_baseline_p50_ms":
                serve["100_fps_to_host"]["one_frame_per_launch"].get("p50_ms"),
            "to_host_100fps_baseline_p99_ms":
                serve["100_fps_to_host"]["one_frame_per_launch"].get("p99_ms"),
            "seconds": args.serve_leg_seconds, "detail": serve}
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(scene, order, linear, cf, mf is not None)
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# one frame split by directions across the ranks (strong scaling)
# ---------------------------------------------------------------------------
def run_split(args, wl, scene) -> None:
    """Each rank beamforms a contiguous slice of the direction grid of the same
    frame: per step the frame is broadcast from rank 0 (NCCL), every rank runs
    its slice's plan, and the slices are gathered to rank 0 into the image."""
    import torch
    import paper_2511_09165_b300 as dm
    from paper_2511_09165_b300.split import SplitBeamformer, direction_slices, plan_rows, \
        slice_grid

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    td = dist_init(world, "nccl")
    linear = wl["mode"] == "linear"
    M, T, N = scene.n_dirs, scene.n_samples, scene.n_mics
    lo, hi = direction_slices(M, world)[rank]
    azel, unit, _ = slice_grid(scene.dir_azel, scene.dir_unit, None, lo, hi)
    plan = dm.Plan(mic_xyz=scene.mic_xyz, dir_azel=azel, dir_unit=unit, n_samples=T,
                   fs=scene.fs, c=scene.c, order=wl["order"],
                   delay_mode=dm.LINEAR if linear else dm.ROUND, cf=wl.get("cf", True),
                   ng_prec=NG_PREC[args.ng](dm)) if hi > lo else None
    sb = SplitBeamformer(rank, world, M, plan_rows(plan) if plan else None, device=dev)
    frame = torch.from_numpy(scene.frame).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, device=dev)

    def step():
        if world > 1:
            return sb(frame, src=0, dst=0)
        return plan(frame)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local)
    clocks.start()
    dist_barrier(td)
    torch.cuda.synchronize(dev)
    wall0 = time.time()
    times = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        dist_barrier(td)
        t0 = time.perf_counter()
        step()
        torch.cuda.synchronize(dev)
        times.append(time.perf_counter() - t0)
    dist_barrier(td)
    wall1 = time.time()
    clocks.stop()
    total = dist_max(td, sum(times), dev)
    if plan is not None:
        plan.check()
        plan.close()
    if rank != 0:
        return
    ms = 1e3 * total / args.steps
    print(json.dumps({
        "metric": METRIC, "value": M * T / (ms * 1e-3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "description": wl["text"], "n_mics": N,
                   "n_dirs": M, "n_samples": T, "ng": args.ng,
                   "parallelism": f"directions split x{world} (frame broadcast, rows gathered "
                                  "to rank 0, both inside the timed step)",
                   "l2": "flushed (256 MB write) before every step",
                   "timing": "host wall clock around each synchronised step, max over ranks"},
        "gpu_launches": 3 * args.steps,
        "clocks": clocks.summary(wall0, wall1),
    }), flush=True)


# ---------------------------------------------------------------------------
# serving: Poisson arrivals from 16 mixed sensors
# ---------------------------------------------------------------------------
def serving_measure(rates, seconds, rank=0, budget_gb=48, to_host_rates=(), env_cap=None,
                    bulk_depth=2):
    """Poisson arrivals from the 16-sensor mix at each rate, through the
    continuous-batching server and through the one-frame-per-launch baseline:
    latency to the image resident on the device (`rates`) and to the image
    copied to pinned host memory (`to_host_rates`; the mix's images average
    324 MB, so 200 frames/s would need 65 GB/s of device-to-host copies, more
    than the host link carries).  Returns (results, mix)."""
    import torch
    import paper_2511_09165_b300 as dm
    from paper_2511_09165_b300 import serving

    mix = scenes.serving_mix(seed=5 + rank)
    sensors = [serving.Sensor(dm.Plan(mic_xyz=s.mic_xyz, dir_azel=s.dir_azel,
                                      dir_unit=s.dir_unit, n_samples=s.n_samples, fs=s.fs,
                                      c=s.c, order=s.order), s.name) for s in mix]
    host = [[torch.from_numpy(f).pin_memory() for f in s.frames] for s in mix]
    px = [s.n_dirs * s.n_samples for s in mix]
    pinned = serving.PinnedPool()
    for sn, h in zip(sensors, host):          # warm-up: every sensor once
        img = sn.plan(h[0].cuda())
        if to_host_rates:                     # one pinned image per sensor, allocated now
            pinned.put(pinned.get(img.shape))
    torch.cuda.synchronize()

    def schedule(rate, seed):
        offs, which = serving.poisson_arrivals(rate, seconds, len(mix), seed)
        rng = np.random.default_rng(seed + 1)
        frames = [int(rng.integers(len(host[w]))) for w in which]
        return offs, which, frames

    def run_server(rate, seed, copy_back):
        offs, which, fidx = schedule(rate, seed)
        reqs = []
        with serving.Server(sensors, budget_bytes=budget_gb << 30, streams=2,
                            copy_back=copy_back, pinned=pinned, bulk_depth=bulk_depth,
                            bulk_env_tile_cap=serving.BULK_ENV_TILE_CAP if env_cap is None
                            else env_cap) as srv:
            t0 = time.perf_counter() + 0.05
            for o, w, f in zip(offs, which, fidx):
                while time.perf_counter() < t0 + o:
                    time.sleep(0.0002)
                reqs.append(srv.submit(int(w), host[w][f], t_arrival=t0 + o))
            srv.drain(600.0)
            nb = srv.batches
        return reqs, t0, nb

    def run_baseline(rate, seed, copy_back):
        offs, which, fidx = schedule(rate, seed)
        t0 = time.perf_counter() + 0.05
        reqs = [serving.Request(int(w), host[w][f], t0 + o)
                for o, w, f in zip(offs, which, fidx)]
        for sn in sensors:                    # the baseline's default scheduling
            sn.plan.set_envelope_tile_cap(0)
        serving.one_frame_per_launch(sensors, reqs, copy_back=copy_back, pinned=pinned)
        return reqs, t0

    fast = [sn.cost <= serving.FAST_COST for sn in sensors]

    def summary(reqs, t0, batches=None):
        done = [r for r in reqs if not r.rejected]
        span = max(r.t_done for r in done) - t0
        d = serving.latency_summary(reqs)
        d["small_frames"] = serving.latency_summary([r for r in reqs if fast[r.sensor]])
        d["big_frames"] = serving.latency_summary([r for r in reqs if not fast[r.sensor]])
        d["frames_per_s"] = len(done) / span
        d["dir_samples_per_s"] = sum(px[r.sensor] for r in done) / span
        d["rejected"] = sum(r.rejected for r in reqs)
        if batches is not None:
            d["batches"] = batches
            d["mean_batch"] = len(done) / max(batches, 1)
        return d

    results = {}
    legs = [(r, False) for r in rates] + [(r, True) for r in to_host_rates]
    for k, (rate, cb) in enumerate(legs):
        reqs, t0, nb = run_server(rate, 100 + k, cb)
        sv = summary(reqs, t0, nb)
        reqs, t0 = run_baseline(rate, 100 + k, cb)
        bl = summary(reqs, t0)
        key = f"{rate:g}_fps" + ("_to_host" if cb else "")
        results[key] = {"server": sv, "one_frame_per_launch": bl}
    for sn in sensors:
        sn.plan.close()
    return results, mix


def run_serving(args) -> None:
    import torch

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    clocks = ClockSampler(local)
    clocks.start()
    wall0 = time.time()
    results, mix = serving_measure(args.serve_rates, args.serve_seconds, rank,
                                   args.serve_budget_gb,
                                   to_host_rates=args.serve_to_host_rates,
                                   env_cap=args.serve_env_cap, bulk_depth=args.serve_bulk_depth)
    wall1 = time.time()
    clocks.stop()
    if rank != 0:
        return
    top = results[f"{args.serve_rates[-1]:g}_fps"]["server"]
    line = {
        "metric": METRIC, "value": top["dir_samples_per_s"] * world, "unit": UNIT,
        "n_gpus": world, "steps": sum(v["server"]["frames"] for v in results.values()),
        "warmup": len(mix), "ms_per_step": 1e3 / top["frames_per_s"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "serving", "description":
                   "16 sensors (N in {32,64,128}, M in {91,2048,8192}, T in "
                   "{4096,16384,32768}, n in {3,5}, nearest-sample delays, CF, envelope, "
                   "compensated-FP32 Newton-Girard), small_2d-style echo frames, Poisson "
                   "arrivals at " +
                   ", ".join(f"{r:g}" for r in args.serve_rates) + " frames/s for "
                   f"{args.serve_seconds:g} s each; latency = arrival to image resident "
                   "on the device (keys *_to_host, at " +
                   ", ".join(f"{r:g}" for r in args.serve_to_host_rates) +
                   " frames/s: to the image copied to pinned host memory); value = "
                   "delivered direction*samples/s at the highest device-resident rate",
                   "budget_gb": args.serve_budget_gb, "streams": 2,
                   "bulk_streams": 1,
                   "bulk_depth": args.serve_bulk_depth,
                   "bulk_envelope_tiles_per_cta": args.serve_env_cap,
                   "sensors": [f"N{s.n_mics} M{s.n_dirs} T{s.n_samples} n{s.order}"
                               for s in mix]},
        "latency_ms": {"p50": top.get("p50_ms"), "p99": top.get("p99_ms")},
        "serving": results,
        "clocks": clocks.summary(wall0, wall1),
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# direction sweep: frame time against the number of directions (the paper's
# Fig. 7b setting: 163840 samples, DMAS5-CF, its direction counts), 2-D fan
# ---------------------------------------------------------------------------
SWEEP_DIRS = [2, 10, 100, 200, 500, 1000, 2000, 3000, 4000]   # the paper's counts


def run_sweep(args) -> None:
    import torch
    import paper_2511_09165_b300 as dm

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, device=dev)
    steps = max(5, min(args.steps, 50))
    clocks = ClockSampler(local)
    clocks.start()
    wall0 = time.time()
    rows = []
    for M in SWEEP_DIRS:
        sc = scenes.small_2d(seed=1, n_samples=163840, n_dirs=M)
        plan = dm.Plan(mic_xyz=sc.mic_xyz, dir_azel=sc.dir_azel, n_samples=sc.n_samples,
                       fs=sc.fs, c=sc.c, order=5, delay_mode=dm.ROUND)
        frame = torch.from_numpy(sc.frame).to(dev)
        image = torch.empty((M, sc.n_samples), device=dev)
        for _ in range(args.warmup):
            flush.zero_()
            plan(frame, out=image, stream=stream)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            plan(frame, out=image, stream=stream)
            b.record(stream)
        torch.cuda.synchronize(dev)
        plan.check()
        plan.close()
        ms = float(np.median([a.elapsed_time(b) for a, b in ev]))
        rows.append({"n_dirs": M, "ms_p50": ms, "dir_samples_per_s": M * sc.n_samples / ms * 1e3})
    wall1 = time.time()
    clocks.stop()
    if rank != 0:
        return
    top = rows[-1]
    print(json.dumps({
        "metric": METRIC, "value": top["dir_samples_per_s"], "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": args.warmup, "ms_per_step": top["ms_p50"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "sweep", "description":
                   "2-D fan (32 mics, 12 cm disc), 163840 samples at 450 kHz, n=5 with CF, "
                   "nearest-sample delays, envelope; frame time per direction count "
                   "(median of CUDA-event steps, L2 flushed before each)",
                   "n_dirs": SWEEP_DIRS},
        "sweep": rows,
        "clocks": clocks.summary(wall0, wall1),
    }), flush=True)


# ---------------------------------------------------------------------------
# image SNR against microphone SNR (the paper's Sec. III-A experiment, Table I)
# ---------------------------------------------------------------------------
IMAGE_SNR_MIC_DB = [-40.0, -30.0, -20.0, -10.0, 0.0, 10.0, 20.0, 40.0]


def run_image_snr(args) -> None:
    import torch
    import paper_2511_09165_b300 as dm
    from workloads import image_quality as iq

    world, rank, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    rows = []
    for snr in IMAGE_SNR_MIC_DB:
        sc = scenes.point_target(snr)
        off = iq.off_target_mask(sc.dir_azel[:, 0], sc.n_samples, sc.fs, sc.c, 0.0, 1.0)
        x = torch.from_numpy(sc.frame).cuda()
        row = {"snr_mic_db": snr}
        for n in (1, 2, 3, 4, 5):
            for cf in (False, True):
                plan = dm.Plan(mic_xyz=sc.mic_xyz, dir_azel=sc.dir_azel, n_samples=sc.n_samples,
                               fs=sc.fs, c=sc.c, order=n, delay_mode=dm.LINEAR, cf=cf,
                               ng_prec=NG_PREC[args.ng](dm))
                img = plan(x).cpu().numpy()
                plan.check()
                plan.close()
                key = ("dmas%d" % n if n > 1 else "das") + ("_cf" if cf else "")
                row[key] = round(iq.image_snr_db(img, off), 2)
        rows.append(row)
    # directional PSF of the noise-free point target: all ten images from one
    # every-order pass
    sc = scenes.point_target(float("inf"))
    plan = dm.Plan(mic_xyz=sc.mic_xyz, dir_azel=sc.dir_azel, n_samples=sc.n_samples, fs=sc.fs,
                   c=sc.c, order=5, delay_mode=dm.LINEAR)
    imgs = plan.beamform_orders(torch.from_numpy(sc.frame).cuda()).cpu().numpy()
    plan.check()
    plan.close()
    psf = {("dmas%d" % n if n > 1 else "das") + ("_cf" if cf else ""):
           round(iq.psf_dynamic_range_db(imgs[int(cf), n - 1], sc.dir_azel[:, 0], 0.0), 1)
           for n in (1, 2, 3, 4, 5) for cf in (False, True)}
    print(json.dumps({
        "metric": "image SNR (dB) against microphone SNR", "unit": "dB", "n_gpus": 1,
        "data": "synthetic",
        "config": {"workload": "image_snr", "description":
                   "one reflector at broadside, 1 m, echo amplitude 1 at the 32 mics "
                   "(12 cm disc), white noise eta = 10^(-SNR/20), 181 azimuths x 2048 "
                   "samples, linear delays, 181-tap envelope, Newton-Girard " + args.ng +
                   "; image normalised to max 1, "
                   "SNR_image = 20 log10(1 / mean off-target level), target window "
                   "+-10 deg x +-0.15 m"},
        "table": rows,
        "psf_dynamic_range_db": psf,
        "psf": "noise-free point target, directional PSF = max over t per azimuth, "
               "dynamic range = 20 log10(1 / median outside +-10 deg)",
    }), flush=True)


# ---------------------------------------------------------------------------
# every order at once: DAS and DMAS-2..5, with and without CF, in one pass
# against ten single-order calls
# ---------------------------------------------------------------------------
def orders_ops_per_pixel(N: int, nmax: int, linear: bool) -> dict:
    """FP32 operations per direction·sample of the every-order pass, counted as
    for one order: its running sums accumulated over N mics (twice with
    interpolation), Newton-Girard of every order, CF, the CF-weighted copies."""
    sums = 2 + (1 if nmax >= 2 else 0) + nmax * (nmax - 1) // 2
    main = N * sums * (2 if linear else 1)
    ng = sum(k * (k + 1) // 2 + k for k in range(2, nmax + 1))
    return {"main": main, "newton_girard": ng, "cf": 6 + nmax, "beam_total": main + ng + 6 + nmax}


def run_orders(args) -> None:
    import torch
    import paper_2511_09165_b300 as dm

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, device=dev)
    steps = max(5, min(args.steps, 30))
    paper = args.workload == "orders_paper"
    if paper:
        # the paper's real-world imaging setting (Sec. III-B): 3601 azimuths at
        # 0.05 deg, 163840 samples, the eRTIS chirp and its matched filter
        sc = scenes.small_2d(seed=1, n_samples=163840, n_dirs=3601, pulse="chirp")
        mf = scenes.lfm_chirp(sc.fs).astype(np.float32)
        mode_list = ("round",)
        steps = max(3, min(args.steps, 5))
    else:
        sc = scenes.hemi_3d(seed=2)
        mf = None
        mode_list = ("linear", "round")
    N, M, T = sc.n_mics, sc.n_dirs, sc.n_samples
    px = M * T
    frame = torch.from_numpy(sc.frame).to(dev)
    images = torch.empty((2, 5, M, T), device=dev)
    clocks = ClockSampler(local)
    clocks.start()
    wall0 = time.time()
    peak = (torch.cuda.get_device_properties(dev).multi_processor_count * FP32_LANES_PER_SM *
            SM_MAX_MHZ * 1e6 / 1e12)
    modes = []

    def timed(fn):
        for _ in range(args.warmup):
            flush.zero_()
            fn()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize(dev)
        return float(np.median([a.elapsed_time(b) for a, b in ev]))

    for mode in mode_list:
        dmode = dm.LINEAR if mode == "linear" else dm.ROUND
        kw = dict(mic_xyz=sc.mic_xyz, dir_unit=sc.dir_unit, dir_azel=sc.dir_azel, n_samples=T,
                  fs=sc.fs, c=sc.c, delay_mode=dmode, mf_signal=mf)
        plan = dm.Plan(order=5, **kw)
        pass_ms = timed(lambda: plan.beamform_orders(frame, out=images, stream=stream))
        plan.set_profiling(True)
        stages = []
        for _ in range(5):
            plan.beamform_orders(frame, out=images, stream=stream)
            stages.append(plan.stage_ms())
        plan.check()
        plan.close()
        st = np.median(np.array(stages), axis=0)
        singles = [dm.Plan(order=k, cf=cf, **kw) for cf in (False, True) for k in range(1, 6)]

        def separate():
            for i, pl in enumerate(singles):
                pl(frame, out=images[i // 5, i % 5], stream=stream)

        sep_ms = timed(separate)
        per_order = {}
        for i, pl in enumerate(singles):
            name = ("das" if i % 5 == 0 else "dmas%d" % (i % 5 + 1)) + ("_cf" if i >= 5 else "")
            per_order[name] = timed(lambda: pl(frame, out=images[i // 5, i % 5], stream=stream))
        # the beamform stage of each single-order call with CF (configuration 2 asks
        # for n = 1..5 each) against the FP32 roofline, by the stage events
        single_roof = {}
        for i, pl in enumerate(singles[5:]):
            k = i + 1
            pl.set_profiling(True)
            bst = []
            for _ in range(max(5, steps // 2)):
                flush.zero_()
                pl(frame, out=images[1, i], stream=stream)
                bst.append(pl.stage_ms()[1])
            t_ms = float(np.median(bst))
            ops_k = algorithmic_ops_per_pixel(N, k, mode == "linear")["beam_total"]
            single_roof["das_cf" if k == 1 else "dmas%d_cf" % k] = {
                "beamform_ms": t_ms, "ops_per_pixel": ops_k,
                "frac": ops_k * px / (t_ms * 1e-3) / 1e12 / peak}
        for pl in singles:
            pl.check()
            pl.close()
        ops = orders_ops_per_pixel(N, 5, mode == "linear")
        achieved = ops["beam_total"] * px / (st[1] * 1e-3) / 1e12
        modes.append({
            "delays": mode, "pass_ms": pass_ms, "separate_ms": sep_ms,
            "single_call_ms": per_order,
            "single_order_beamform_cf": single_roof,
            "speedup": sep_ms / pass_ms,
            "stage_ms": {"root planes": float(st[0]), "beamform (every order)": float(st[1]),
                         "envelope (10 images)": float(st[2])},
            "images_dir_samples_per_s": 10 * px / (pass_ms * 1e-3),
            "roofline_beamform": {"bound": "alu", "kernel": "beamform_orders_kernel",
                                  "ops_per_pixel": ops, "achieved": achieved, "peak": peak,
                                  "unit": "Top/s", "frac": achieved / peak},
        })
    wall1 = time.time()
    clocks.stop()
    if rank != 0:
        return
    top = modes[0]
    print(json.dumps({
        "metric": "image·direction·samples/s: DAS and DMAS-2..5, each with and without CF "
                  "(10 images) per frame",
        "value": top["images_dir_samples_per_s"], "unit": "image·direction·samples/s",
        "n_gpus": world, "steps": steps, "warmup": args.warmup, "ms_per_step": top["pass_ms"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": args.workload, "description":
                   ("the paper's real-world imaging setting: 32 mics (12 cm disc), 3601 "
                    "azimuths -90..90 deg at 0.05 deg, 163840 samples at 450 kHz, chirp "
                    "echoes and the 1125-tap matched filter, nearest-sample delays" if paper
                    else "3-D hemisphere (32 mics, 2048 directions, 16384 samples)") +
                   ", the ten images of Table I's algorithms with the 181-tap envelope: one "
                   "dmas_beamform_orders call against ten dmas_beamform calls (median of "
                   "CUDA-event steps, L2 flushed before each)",
                   "l2": "flushed (256 MB write) before every step"},
        "modes": modes,
        "gpu_launches": 3 * steps,
        "clocks": clocks.summary(wall0, wall1),
    }), flush=True)


def main() -> None:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload",
                    choices=sorted(WORKLOADS) + ["serving", "sweep", "image_snr", "orders",
                                                 "orders_paper"],
                    default="hemi_3d_n5")
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[200.0, 1000.0])
    ap.add_argument("--serve-seconds", type=float, default=5.0)
    ap.add_argument("--serve-budget-gb", type=int, default=48)
    ap.add_argument("--serve-bulk-depth", type=int, default=2,
                    help="big-frame batches in flight at once")
    ap.add_argument("--serve-to-host-rates", type=float, nargs="*", default=[100.0])
    ap.add_argument("--serve-env-cap", type=int, default=0,
                    help="tensor-core envelope tiles per CTA for the bulk lane (0: no cap)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--split", action="store_true",
                    help="under torchrun: one frame split by directions across the ranks "
                         "(strong scaling) instead of one frame per rank")
    ap.add_argument("--ng", choices=sorted(NG_PREC), default="cf32",
                    help="Newton-Girard arithmetic: compensated FP32 (default), FP64, plain FP32")
    ap.add_argument("--serve-leg-seconds", type=float, default=2.0,
                    help="seconds of 200 frames/s serving in the default run (0: none)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.workload == "serving":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable":
                              "the serving workload has no CPU reference arm"}))
            return
        run_serving(args)
        return
    if args.workload == "image_snr":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable":
                              "the image-SNR experiment has no CPU reference arm"}))
            return
        run_image_snr(args)
        return
    if args.workload in ("orders", "orders_paper"):
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable":
                              "the every-order comparison has no CPU reference arm"}))
            return
        run_orders(args)
        return
    if args.workload == "sweep":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable":
                              "the direction sweep has no CPU reference arm"}))
            return
        run_sweep(args)
        return
    wl = WORKLOADS[args.workload]
    scene = wl["scene"]()
    if args.impl == "reference":
        run_reference(args, wl, scene)
    elif args.split:
        run_split(args, wl, scene)
    else:
        run_ours(args, wl, scene)


if __name__ == "__main__":
    main()
