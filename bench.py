#!/usr/bin/env python
"""Benchmark of the hot path of differentiable radio ray tracing on GB300.

Workload (street canyon, synthetic): 64 seeded boxes on a 500x500 m ground
(770 triangles), transmitter at 30 m, 4096 receivers on a 64x64 grid at 1.5 m,
10^6 Fibonacci rays, up to 3 specular reflections, CFR at 1024 subcarriers of
48.828125 kHz around 3.5 GHz.

One step = the whole hot path over this workload: trace_paths (SBR, dedup,
image method, visibility, path records) + eval_fields + CFR with power-MSE loss
and CFR adjoint (one fused launch) + eval_fields adjoint.  Metric: rays/s traced
= primary rays taken through the full step per second (whole job).

Also reported: the calibration step (fields + CFR + loss + adjoints) of the
indoor differentiation workload (1024 receivers, 1024 subcarriers) in ms, a
roofline line for the dominant kernel, the end-to-end number through host
buffers, and the FP64 CPU oracle on the same workload as the CPU baseline.

--impl reference times the FP64 CPU oracle (the only reference: the paper ships
no code) on the same workload and metric.
"""
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
sys.path.insert(0, ROOT)

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
# FP32 SIMT peak derived from unit counts and clocks: 152 SMs x 128 FP32 lanes x
# 2 flops (FMA) x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# algorithmic FP32 work of the BVH traversal (counted by the kernels):
# one node visit = two ray/box slab tests (12 flops each); one watertight
# ray/triangle test = 40 flops
FLOPS_PER_NODE_VISIT = 24
FLOPS_PER_TRI_TEST = 40


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return dict(PEAKS_FALLBACK), "fallback"


_MEASURED = {}


def measure_peaks(dev):
    """Peaks that MEASURED_PEAKS.json does not hold, measured here with cuBLAS through
    torch (best of 5 CUDA-event-timed products, after one untimed one):
      tf32_tflops  float32 matmul with TF32 tensor cores allowed (8192^3);
      fp32_tflops  float32 matmul with TF32 off, i.e. FP32 FMA on the SIMT units (8192^3);
      fp64_tflops  float64 matmul (4096^3).
    Each is 2 n^3 flops over the fastest run.  Measured once per process."""
    import torch
    if _MEASURED:
        return dict(_MEASURED)
    stream = torch.cuda.current_stream()

    def best(fn, flops, reps=5):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record(stream)
            fn()
            e.record(stream)
            e.synchronize()
            ts.append(s.elapsed_time(e))
        return flops / (min(ts) * 1e-3) / 1e12

    old_tf32 = torch.backends.cuda.matmul.allow_tf32
    try:
        n = 8192
        g = torch.Generator(device=dev).manual_seed(0)
        a = torch.randn((n, n), device=dev, generator=g)
        b = torch.randn((n, n), device=dev, generator=g)
        c = torch.empty((n, n), device=dev)
        torch.backends.cuda.matmul.allow_tf32 = True
        _MEASURED["tf32_tflops"] = best(lambda: torch.mm(a, b, out=c), 2.0 * n ** 3)
        torch.backends.cuda.matmul.allow_tf32 = False
        _MEASURED["fp32_tflops"] = best(lambda: torch.mm(a, b, out=c), 2.0 * n ** 3)
        del a, b, c
        n = 4096
        a = torch.randn((n, n), device=dev, dtype=torch.float64, generator=g)
        b = torch.randn((n, n), device=dev, dtype=torch.float64, generator=g)
        c = torch.empty((n, n), device=dev, dtype=torch.float64)
        _MEASURED["fp64_tflops"] = best(lambda: torch.mm(a, b, out=c), 2.0 * n ** 3, reps=3)
        del a, b, c
    finally:
        torch.backends.cuda.matmul.allow_tf32 = old_tf32
    torch.cuda.empty_cache()
    _MEASURED["how"] = ("cuBLAS via torch.mm, best of 5 CUDA-event-timed runs: float32 8192^3 with TF32 "
                        "allowed (tf32) and not allowed (fp32, SIMT FMA), float64 4096^3 (3 runs)")
    return dict(_MEASURED)


class ClockSampler:
    """SM clocks and clock-event (throttle) reasons sampled during the timed region.

    Reads NVML through ctypes every few milliseconds (the timed regions here are
    tens to hundreds of milliseconds, too short for nvidia-smi's 100 ms loop);
    falls back to `nvidia-smi -lms 100` when the NVML library cannot be loaded.
    Only reads; never changes a setting."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    # nvmlClocksEventReason* bits (nvml.h)
    REASON_BITS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
                   0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}
    NVML_CLOCK_SM = 1

    def __init__(self, torch_device, period_s=0.005):
        self.dev = torch_device
        self.period = period_s
        self.proc = None
        self.nvml = None
        self.lines = []
        self.samples = []
        self.stop_flag = threading.Event()

    def _nvml_handle(self):
        import ctypes

        import torch
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            return None
        h = ctypes.c_void_p()
        props = torch.cuda.get_device_properties(self.dev)
        uuid = getattr(props, "uuid", None)
        ok = False
        if uuid is not None:
            ok = lib.nvmlDeviceGetHandleByUUID(("GPU-" + str(uuid)).encode(), ctypes.byref(h)) == 0
        if not ok:
            ok = lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.dev), ctypes.byref(h)) == 0
        if not ok:
            return None
        self.max_mhz = ctypes.c_uint(0)
        lib.nvmlDeviceGetMaxClockInfo(h, self.NVML_CLOCK_SM, ctypes.byref(self.max_mhz))
        self.reason_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        return lib, h

    def _poll(self):
        import ctypes
        lib, h = self.nvml
        mhz = ctypes.c_uint(0)
        bits = ctypes.c_ulonglong(0)
        while not self.stop_flag.is_set():
            r0 = lib.nvmlDeviceGetClockInfo(h, self.NVML_CLOCK_SM, ctypes.byref(mhz))
            r1 = self.reason_fn(h, ctypes.byref(bits))
            if r0 == 0:
                self.samples.append((mhz.value, bits.value if r1 == 0 else 0))
            time.sleep(self.period)

    def start(self):
        try:
            self.nvml = self._nvml_handle()
        except (OSError, AttributeError):
            self.nvml = None
        if self.nvml is not None:
            self.thread = threading.Thread(target=self._poll, daemon=True)
            self.thread.start()
            return
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.nvml is not None:
            self.stop_flag.set()
            self.thread.join(timeout=5)
            sm = [m for m, _ in self.samples]
            reasons = sorted({name for _, b in self.samples for bit, name in self.REASON_BITS.items() if b & bit})
            return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": self.max_mhz.value,
                    "samples": len(sm), "source": "nvml", "reasons": reasons}
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "source": "nvidia-smi", "reasons": sorted(reasons)}


def dist_setup(n_gpus):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, x):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cpu" if dist.get_backend() == "gloo" else "cuda"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_step, steps, world, slowest_s):
    """Weak scaling: every rank processes units_per_step per step; the job's rate is
    all units of all ranks over the slowest rank's time."""
    return units_per_step * steps * world / slowest_s


# --------------------------------------------------------------------------- oracle (CPU)

def oracle_step(sc, n_sub):
    """The same step on the FP64 CPU oracle: trace, fields, CFR, loss, adjoints."""
    import oracle
    o = oracle.OracleScene(sc)
    tr = o.trace()
    a = o.fields(tr, eps_r=sc.eps_r * 1.2, sigma=sc.sigma * 0.7)
    H = oracle.cfr(a, tr["tau"], tr["rx_offsets"], sc.f_center_hz, sc.delta_f_hz, n_sub)
    T = np.abs(H) ** 2 * 1.05
    w = oracle.power_weights(T)
    L, gH = oracle.power_mse(H, T, w)
    ga = oracle.cfr_grad(tr["tau"], tr["rx_offsets"], sc.f_center_hz, sc.delta_f_hz, n_sub, gH)
    o.fields_grad(tr, ga, eps_r=sc.eps_r * 1.2, sigma=sc.sigma * 0.7)
    return len(tr["tau"])


def omp_threads():
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def run_reference(args):
    """--impl reference: the FP64 CPU oracle timed on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    import scenegen
    oracle.build()
    sc = scenegen.street_canyon()
    for _ in range(args.warmup):
        oracle_step(sc, args.n_sub)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle_step(sc, args.n_sub)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * statistics.mean(times)
    value = sc.n_rays * len(times) / sum(times)
    line = {
        "impl": "reference", "metric": "rays/s traced", "value": value, "unit": "rays/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        # the same config as the GPU arm, so the two lines compare like for like
        "config": workload_config(sc, args.n_sub, L2_NOTE),
        "cpu_baseline": {"value": value, "unit": "rays/s", "cores": omp_threads(), "kind": "oracle",
                         "sample": "full street-canyon step per timed step (trace, fields, CFR, loss, adjoints)"},
        "e2e": {"value": value, "unit": "rays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


L2_NOTE = "flushed: 256 MiB written between timed steps"


def workload_config(sc, n_sub, l2):
    return {"workload": "street_canyon", "n_tris": sc.n_tris, "n_rays": sc.n_rays, "max_depth": sc.max_depth,
            "n_rx": sc.n_rx, "n_sub": n_sub, "f_center_hz": sc.f_center_hz, "delta_f_hz": sc.delta_f_hz,
            "l2": l2}


# --------------------------------------------------------------------------- GPU

def run_ours(args):
    import torch

    import paper_2311_18558_gb300 as rt
    import scenegen

    world, rank, local = dist_setup(args.gpus)
    dev = torch.device("cuda", torch.cuda.current_device())
    peaks, peak_src = load_peaks()
    peaks.update(measure_peaks(dev))
    sc = scenegen.street_canyon()
    N = args.n_sub
    fc, df = sc.f_center_hz, sc.delta_f_hz
    ctx = rt.Context(torch.cuda.current_device())
    scene = rt.Scene.from_synthetic(ctx, sc)
    rx_dev = torch.tensor(sc.rx, dtype=torch.float64, device=dev)
    eps_gt = torch.tensor(sc.eps_r, device=dev)
    sig_gt = torch.tensor(sc.sigma, device=dev)
    # synthetic "measurement": CFR power of the ground-truth materials
    p0 = rt.trace_paths(ctx, scene, sc.tx, rx_dev, sc.n_rays, sc.max_depth)
    a0 = rt.eval_fields(ctx, p0, eps_gt, sig_gt, sc.freq_hz)
    H0 = rt.cfr(ctx, p0.rx_offsets, a0, p0.tau, fc, df, N)
    target = (H0.abs() ** 2).float().contiguous()
    mean = target.mean(dim=1)
    weight = torch.where(mean > 0, 1.0 / torch.where(mean > 0, mean, torch.ones_like(mean)),
                         torch.zeros_like(mean)).float().contiguous()
    eps = (eps_gt * 1.2).contiguous()
    sig = (sig_gt * 0.7).contiguous()
    M = sc.n_materials
    g_eps = torch.zeros(M, device=dev)
    g_sig = torch.zeros(M, device=dev)
    g_gain = torch.zeros(2, device=dev)
    loss_buf = torch.zeros(1, device=dev)
    n_paths = p0.n_paths
    del p0, a0, H0

    def step(rx_in, target_in, eps_in, sig_in, before_calibration=None):
        p = rt.trace_paths(ctx, scene, sc.tx, rx_in, sc.n_rays, sc.max_depth)
        if before_calibration is not None:
            before_calibration()
        a = rt.eval_fields(ctx, p, eps_in, sig_in, sc.freq_hz)
        _, ga, _ = rt.cfr_power_mse_fused(ctx, p.rx_offsets, a, p.tau, fc, df, N, target_in, weight, loss=loss_buf)
        g_eps.zero_()
        g_sig.zero_()
        g_gain.zero_()
        rt.eval_fields_backward(ctx, p, eps_in, sig_in, sc.freq_hz, ga, g_eps, g_sig, g_gain)
        return p

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 129 MB L2
    for _ in range(args.warmup):
        step(rx_dev, target, eps, sig)
    torch.cuda.synchronize()
    # the timed steps trace without host waits (rt_set_trace_async: capacities from
    # the warm-up traces, counts on the device, an overflow reported in the status
    # word, which is checked after the timed region)
    rt.set_trace_async(ctx, True)
    step(rx_dev, target, eps, sig)
    torch.cuda.synchronize()

    # ---------------- timed region (device-resident inputs)
    ctx.set_profiling(1)
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stage_acc = np.zeros(8)
    launches0, _, _ = ctx.profile()
    clocks = ClockSampler(torch.cuda.current_device())
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        step(rx_dev, target, eps, sig)
        ev[k][1].record(stream)
        _, stage_ms, _ = ctx.profile()
        stage_acc += np.array(stage_ms)
    torch.cuda.synchronize()
    barrier(world)
    clock_info = clocks.stop()
    launches1, _, _ = ctx.profile()
    step_ms = [s.elapsed_time(e) for s, e in ev]
    total_s = max_over_ranks(world, sum(step_ms) / 1e3)
    ms_per_step = 1e3 * total_s / args.steps
    value = whole_job_rate(sc.n_rays, args.steps, world, total_s)
    gpu_launches = launches1 - launches0
    stage_mean = stage_acc / args.steps
    status_after = ctx.status_word()
    if status_after != 0:
        raise RuntimeError(f"device status {status_after} after the timed steps")
    rt.set_trace_async(ctx, False)

    # ---------------- calibration kernels alone on the same paths (roofline inputs)
    ctx.set_profiling(0)
    p = rt.trace_paths(ctx, scene, sc.tx, rx_dev, sc.n_rays, sc.max_depth)
    a = rt.eval_fields(ctx, p, eps, sig, sc.freq_hz)
    cal = time_calibration(rt, ctx, p, eps, sig, target, weight, sc.freq_hz, fc, df, N, flush, args.steps)

    # ---------------- first-order diffraction on the same workload
    diffraction = time_diffraction(rt, ctx, scene, sc, p, rx_dev, eps, sig, flush, args.steps, peaks, peak_src)

    # ---------------- traversal counters (separate, untimed pass)
    ctx.set_profiling(2)
    rt.trace_paths(ctx, scene, sc.tx, rx_dev, sc.n_rays, sc.max_depth)
    _, _, counters = ctx.profile()
    ctx.set_profiling(0)

    # ---------------- end to end through host buffers
    rt.set_trace_async(ctx, True)
    e2e = time_e2e(rt, ctx, sc, step, target, eps, sig, g_eps, g_sig, g_gain, loss_buf, flush, args.steps, world)
    rt.set_trace_async(ctx, False)
    if ctx.status_word() != 0:
        raise RuntimeError("device status set during the end-to-end steps")

    # ---------------- indoor calibration step (the second metric), graph-captured
    calib_indoor = time_indoor_calibration(rt, ctx, flush, args)

    # ---------------- eval_fields / adjoint at an HBM-bound size
    fields_hbm = time_fields_hbm(rt, ctx, scene, sc, flush)

    # ---------------- diffuse reflection: trace, calibration step, field kernels
    diffuse = time_diffuse(rt, ctx, flush, args)

    # ---------------- learned form (neural materials) vs the plain per-object form
    learned = time_learned(rt, ctx, args)

    # ---------------- batched form: 16 cities in one pipeline vs a per-scene loop
    batch = time_batch(rt, ctx, args) if not args.no_batch else None

    # ---------------- the street-canyon step captured once in a CUDA graph and replayed
    # (the trace inside a capture runs from the capacities of the steps above; every
    # replay does the whole step's work).  Last, so that its graph memory does not
    # sit under the measurements above.  When it works it is the line's value; the
    # eagerly issued steps stay in "eager".
    rt.set_trace_async(ctx, True)
    try:
        e2e_graph = time_e2e_graph(rt, ctx, sc, step, target, eps, sig, g_eps, g_sig, g_gain, loss_buf, flush,
                                   args.steps, world)
    except Exception as e:
        e2e_graph = {"error": f"{type(e).__name__}: {e}"[:300]}
        torch.cuda.synchronize()
    rt.set_trace_async(ctx, False)
    e2e_eager = e2e
    if "ms_per_step" in e2e_graph:
        e2e = dict(e2e_graph)
        e2e["eager"] = {k: e2e_eager[k] for k in ("value", "ms_per_step")}
    eager = {"value": value, "ms_per_step": ms_per_step, "clocks": clock_info,
             "step_ms_spread": {"min": round(min(step_ms), 4), "median": round(float(np.median(step_ms)), 4),
                                "max": round(max(step_ms), 4)}}
    rt.set_trace_async(ctx, True)
    try:
        step_graph = time_step_graph(rt, ctx, step, rx_dev, target, eps, sig, flush, args.steps, sc.n_rays, world)
    except Exception as e:   # reported, not fatal: the eager steps then give the value
        step_graph = {"error": f"{type(e).__name__}: {e}"[:300]}
        torch.cuda.synchronize()
    rt.set_trace_async(ctx, False)
    if "ms_per_step" in step_graph:
        ms_per_step = step_graph["ms_per_step"]
        value = step_graph["value"]
        clock_info = step_graph["clocks"]
        timing = "CUDA graph replay of the whole step (trace + fields + fused CFR/loss/adjoint + fields adjoint)"
    else:
        timing = "eagerly issued steps"

    # ---------------- roofline of the dominant kernel
    stages = {"sbr": stage_mean[0], "dedup_sort": stage_mean[1], "image_method": stage_mean[2],
              "visibility": stage_mean[3], "emission_records": stage_mean[4],
              "sbr_kernel": stage_mean[6], "sbr_fp64_redo": stage_mean[7]}
    # the dominant single kernel (the shoot-and-bounce kernel alone, not its stage)
    kernels = {"sbr": stage_mean[6], "sbr_fp64_redo": stage_mean[7], "image_method": stage_mean[2],
               "visibility": stage_mean[3], "fields_fwd": cal["fields_fwd_ms"], "cfr_fused": cal["cfr_fused_ms"],
               "fields_bwd": cal["fields_bwd_ms"]}
    dominant = max(kernels, key=kernels.get)
    roofline = roofline_for(dominant, kernels[dominant], counters, cal, n_paths, sc, N, peaks, peak_src)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(sc, N)

    if rank == 0:
        line = {
            "metric": "rays/s traced", "value": value, "unit": "rays/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(sc, N, L2_NOTE),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": gpu_launches,
            "clocks": clock_info,
            # the metric's second half: the indoor calibration step (eval_fields, CFR, loss,
            # CFR adjoint, eval_fields adjoint; one CUDA graph), and the same math as plain
            # PyTorch complex64 ops on this GPU
            "calibration_step_ms": calib_indoor["ms_per_step_median"],
            "calibration_plain_ms": calib_indoor.get("plain_pytorch", {}).get("ms_per_step_median"),
            "paths_per_step": n_paths, "paths_per_s": n_paths * world / (ms_per_step * 1e-3),
            "timing": timing,
            "step_ms_spread": step_graph.get("step_ms_spread", eager["step_ms_spread"]),
            "eager": eager,
            "step_graph": {k: v for k, v in step_graph.items() if k != "clocks"},
            "stage_ms": {k: round(v, 4) for k, v in stages.items()},
            "calibration_ms": {k: round(v, 4) for k, v in cal.items()},
            "calibration_indoor": calib_indoor,
            "fields_hbm": fields_hbm,
            "diffuse": diffuse,
            "learned": learned,
            "diffraction": diffraction,
            "batch": batch,
            "peaks_measured": {k: (round(v, 2) if isinstance(v, float) else v) for k, v in measure_peaks(dev).items()},
            "counters": {"sbr_node_visits": counters[0], "sbr_tri_tests": counters[1], "sbr_queries": counters[2],
                         "fp64_retraced_rays": counters[3], "vis_node_visits": counters[4],
                         "vis_tri_tests": counters[5], "vis_segments": counters[6], "pairs_tested": counters[7]},
        }
        line["summary"] = summary(line)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def summary(line):
    """The headline figures of the nested records, repeated last on the line so that
    a reader of its end sees them."""
    def g(d, *ks):
        for k in ks:
            if not isinstance(d, dict) or k not in d:
                return None
            d = d[k]
        return round(d, 4) if isinstance(d, float) else d
    ci, df_, fh, lr, bt = (line.get(k) for k in ("calibration_indoor", "diffuse", "fields_hbm", "learned", "batch"))
    return {
        "rays_per_s": g(line, "value"), "ms_per_step": g(line, "ms_per_step"), "e2e_rays_per_s": g(line, "e2e", "value"),
        "eager_ms_per_step": g(line, "eager", "ms_per_step"),
        "calibration_step_ms": g(line, "calibration_step_ms"), "calibration_plain_ms": g(line, "calibration_plain_ms"),
        "frac": {"k_sbr": g(line, "roofline", "frac"), "k_cfr_tc": g(ci, "roofline_cfr", "frac"),
                 "k_fields_fwd": g(fh, "fields_fwd", "frac"), "k_fields_bwd": g(fh, "fields_bwd", "frac"),
                 "k_df_fwd": g(df_, "roofline_fields_diffuse", "frac"),
                 "k_df_bwd": g(df_, "roofline_fields_diffuse_bwd", "frac"),
                 "k_dif_fwd": g(line.get("diffraction"), "roofline_fields_diffraction", "frac"),
                 "k_dif_bwd": g(line.get("diffraction"), "roofline_fields_diffraction_bwd", "frac")},
        "learned": {"train_rx": g(lr, "train_rx"), "neural_step_ms": g(lr, "neural_step_ms"),
                    "plain_step_ms": g(lr, "plain_step_ms"), "heldout_loss_neural": g(lr, "heldout_loss_neural"),
                    "heldout_loss_plain": g(lr, "heldout_loss_plain"),
                    "eps_r_err_neural": g(lr, "per_triangle_error", "neural", "seen", "eps_r_mean_rel"),
                    "eps_r_err_plain": g(lr, "per_triangle_error", "plain", "seen", "eps_r_mean_rel")},
        "diffraction": {"n_paths": g(line.get("diffraction"), "n_paths"),
                        "trace_ms": g(line.get("diffraction"), "trace_ms"),
                        "fields_fwd_ms": g(line.get("diffraction"), "fields_fwd_ms"),
                        "fields_bwd_ms": g(line.get("diffraction"), "fields_bwd_ms")},
        "batch": {"trace_batched_ms": g(bt, "trace_batched_ms"), "trace_loop_ms": g(bt, "trace_loop_ms"),
                  "trace_cal_loop_ms": g(bt, "trace_and_calibration", "loop_ms"),
                  "trace_cal_graph_ms": g(bt, "trace_and_calibration", "graph_ms"),
                  "small_trace_cal_loop_ms": g(bt, "small_cities_trace_and_calibration", "loop_ms"),
                  "small_trace_cal_batched_ms": g(bt, "small_cities_trace_and_calibration", "batched_ms"),
                  "small_trace_cal_graph_ms": g(bt, "small_cities_trace_and_calibration", "graph_ms"),
                  "calibration_graph_ms": g(bt, "calibration_graph_ms"),
                  "calibration_loop_ms": g(bt, "calibration_loop_ms")},
    }


# algorithmic bytes per diffraction path: 14 FP32 records + the two faces (int2) +
# a out (complex64); the adjoint reads dL/da instead of writing a
DIF_BYTES_FWD = 14 * 4 + 8 + 8
DIF_BYTES_BWD = 14 * 4 + 8 + 8


def time_diffraction(rt, ctx, scene, sc, p_spec, rx_dev, eps, sig, flush, steps, peaks, peak_src):
    """First-order diffraction on the street canyon (every receiver; candidate
    wedges from the specular trace's first hits): the trace (wall time on the
    stream, host read-backs included), and the field kernel and its adjoint with
    their HBM roofline."""
    import torch
    stream = torch.cuda.current_stream()
    hbm = peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"])

    def timed(fn, n):
        ts = []
        for _ in range(n):
            flush.zero_()
            s0, e0 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            fn()
            e0.record(stream)
            e0.synchronize()
            ts.append(s0.elapsed_time(e0))
        return float(np.median(ts))

    for _ in range(3):
        d = rt.trace_diffraction(ctx, scene, p_spec, sc.tx, rx_dev)
    t_trace = timed(lambda: rt.trace_diffraction(ctx, scene, p_spec, sc.tx, rx_dev), max(steps, 10))
    d = rt.trace_diffraction(ctx, scene, p_spec, sc.tx, rx_dev)
    P = d.n_paths
    a = rt.eval_fields_diffraction(ctx, d, eps, sig, sc.freq_hz)
    g = torch.ones_like(a)
    ge = torch.zeros_like(eps)
    gs = torch.zeros_like(sig)
    t_f = timed(lambda: rt.eval_fields_diffraction(ctx, d, eps, sig, sc.freq_hz, out=a), max(steps, 20))
    t_b = timed(lambda: rt.eval_fields_diffraction_backward(ctx, d, eps, sig, sc.freq_hz, g, ge, gs), max(steps, 20))
    faces, n = rt.scene_wedges(ctx, scene)
    gf = DIF_BYTES_FWD * P / (t_f * 1e-3) / 1e9
    gb = DIF_BYTES_BWD * P / (t_b * 1e-3) / 1e9
    return {"workload": "street_canyon", "n_rx": sc.n_rx, "n_rays": sc.n_rays, "n_wedges": int(len(n)),
            "n_paths": P, "trace_ms": t_trace, "paths_per_s": P / (t_trace * 1e-3),
            "fields_fwd_ms": t_f, "fields_bwd_ms": t_b,
            "roofline_fields_diffraction": {"kernel": "k_dif_fwd", "bound": "hbm", "achieved": gf, "peak": hbm,
                                            "unit": "GB/s", "frac": gf / hbm, "traffic": None,
                                            "peak_source": peak_src,
                                            "algorithmic": f"{DIF_BYTES_FWD} B/path"},
            "roofline_fields_diffraction_bwd": {"kernel": "k_dif_bwd", "bound": "hbm", "achieved": gb, "peak": hbm,
                                                "unit": "GB/s", "frac": gb / hbm, "traffic": None,
                                                "peak_source": peak_src, "algorithmic": f"{DIF_BYTES_BWD} B/path"},
            "l2": "flushed: 256 MiB written between timed runs"}


def time_step_graph(rt, ctx, step, rx_dev, target, eps, sig, flush, steps, n_rays, world):
    """The street-canyon step (trace + fields + fused CFR/loss/adjoint + fields
    adjoint) captured in one CUDA graph and replayed: every replay does the whole
    step's work (a new trace, new fields, the loss and both adjoints); only the
    host's launch work is gone."""
    import torch
    ctx.set_profiling(0)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        step(rx_dev, target, eps, sig)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step(rx_dev, target, eps, sig)
    stream = torch.cuda.current_stream()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    clocks = ClockSampler(torch.cuda.current_device())
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        g.replay()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clock_info = clocks.stop()
    if ctx.status_word() != 0:
        raise RuntimeError("device status set during the graph-replayed steps")
    times = [a.elapsed_time(b) for a, b in ev]
    total_s = max_over_ranks(world, sum(times) / 1e3)
    del g
    return {"ms_per_step": 1e3 * total_s / steps, "value": whole_job_rate(n_rays, steps, world, total_s),
            "replays": steps, "warmup_replays": 3, "clocks": clock_info,
            "step_ms_spread": {"min": round(min(times), 4), "median": round(float(np.median(times)), 4),
                               "max": round(max(times), 4)},
            "l2": "flushed: 256 MiB written between replays"}


def time_calibration(rt, ctx, p, eps, sig, target, weight, freq, fc, df, N, flush, steps):
    """Per-kernel CUDA-event times of the calibration launches on traced paths."""
    import torch
    stream = torch.cuda.current_stream()
    ge = torch.zeros_like(eps)
    gs = torch.zeros_like(sig)
    gg = torch.zeros(2, device=eps.device)
    a = rt.eval_fields(ctx, p, eps, sig, freq)
    loss = torch.zeros(1, device=eps.device)
    _, ga, _ = rt.cfr_power_mse_fused(ctx, p.rx_offsets, a, p.tau, fc, df, N, target, weight, loss=loss)
    t = {"fields_fwd_ms": [], "cfr_fused_ms": [], "fields_bwd_ms": []}
    for _ in range(max(steps, 5)):
        flush.zero_()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record(stream)
        rt.eval_fields(ctx, p, eps, sig, freq, out=a)
        e[1].record(stream)
        rt.cfr_power_mse_fused(ctx, p.rx_offsets, a, p.tau, fc, df, N, target, weight, loss=loss, grad_a=ga)
        e[2].record(stream)
        rt.eval_fields_backward(ctx, p, eps, sig, freq, ga, ge, gs, gg)
        e[3].record(stream)
        torch.cuda.synchronize()
        t["fields_fwd_ms"].append(e[0].elapsed_time(e[1]))
        t["cfr_fused_ms"].append(e[1].elapsed_time(e[2]))
        t["fields_bwd_ms"].append(e[2].elapsed_time(e[3]))
    return {k: float(np.mean(v)) for k, v in t.items()}


def time_e2e(rt, ctx, sc, step, target, eps, sig, g_eps, g_sig, g_gain, loss_buf, flush, steps, world):
    """Same step through host buffers: H2D of the step's inputs from pinned memory
    and D2H of the loss and gradients inside the timed region.  The receivers go
    first (the trace needs them); the target power and the materials, needed only
    by the calibration, are copied on a second stream while the trace runs, and
    the calibration waits for that copy."""
    import torch
    rx_h = torch.tensor(sc.rx, dtype=torch.float64).pin_memory()
    tgt_h = target.cpu().pin_memory()
    eps_h = eps.cpu().pin_memory()
    sig_h = sig.cpu().pin_memory()
    out_h = torch.empty(1 + 2 * eps.numel() + 2, dtype=torch.float32).pin_memory()
    rx_d = torch.empty_like(rx_h, device="cuda")
    tgt_d = torch.empty_like(tgt_h, device="cuda")
    eps_d = torch.empty_like(eps_h, device="cuda")
    sig_d = torch.empty_like(sig_h, device="cuda")
    out_d = torch.empty_like(out_h, device="cuda")
    h2d = rx_h.numel() * 8 + tgt_h.numel() * 4 + eps_h.numel() * 4 + sig_h.numel() * 4
    d2h = out_h.numel() * 4
    stream = torch.cuda.current_stream()
    copy_stream = torch.cuda.Stream()
    times = []
    for _ in range(steps):
        flush.zero_()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        copied = torch.cuda.Event()
        s.record(stream)
        rx_d.copy_(rx_h, non_blocking=True)
        copy_stream.wait_event(s)
        with torch.cuda.stream(copy_stream):
            tgt_d.copy_(tgt_h, non_blocking=True)
            eps_d.copy_(eps_h, non_blocking=True)
            sig_d.copy_(sig_h, non_blocking=True)
            copied.record(copy_stream)
        step(rx_d, tgt_d, eps_d, sig_d, before_calibration=lambda: stream.wait_event(copied))
        torch.cat([loss_buf, g_eps, g_sig, g_gain], out=out_d)
        out_h.copy_(out_d, non_blocking=True)
        e.record(stream)
        e.synchronize()
        times.append(s.elapsed_time(e))
    total = max_over_ranks(world, sum(times) / 1e3)
    return {"value": sc.n_rays * steps * world / total, "unit": "rays/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * total / steps}


def time_e2e_graph(rt, ctx, sc, step, target, eps, sig, g_eps, g_sig, g_gain, loss_buf, flush, steps, world):
    """The end-to-end step of time_e2e (H2D of the receivers, target power and
    materials from pinned memory, the step, D2H of the loss and gradients) with the
    public-API calls captured once in a CUDA graph: every replay copies the pinned
    host inputs as they are at that moment, runs the whole step and copies the
    results back; the host waits for them after each replay."""
    import torch
    rx_h = torch.tensor(sc.rx, dtype=torch.float64).pin_memory()
    tgt_h = target.cpu().pin_memory()
    eps_h = eps.cpu().pin_memory()
    sig_h = sig.cpu().pin_memory()
    out_h = torch.empty(1 + 2 * eps.numel() + 2, dtype=torch.float32).pin_memory()
    rx_d = torch.empty_like(rx_h, device="cuda")
    tgt_d = torch.empty_like(tgt_h, device="cuda")
    eps_d = torch.empty_like(eps_h, device="cuda")
    sig_d = torch.empty_like(sig_h, device="cuda")
    out_d = torch.empty_like(out_h, device="cuda")
    h2d = rx_h.numel() * 8 + tgt_h.numel() * 4 + eps_h.numel() * 4 + sig_h.numel() * 4
    d2h = out_h.numel() * 4

    def body():
        cap = torch.cuda.current_stream()
        side = torch.cuda.Stream()
        rx_d.copy_(rx_h, non_blocking=True)
        side.wait_stream(cap)
        with torch.cuda.stream(side):   # the calibration's inputs while the trace runs
            tgt_d.copy_(tgt_h, non_blocking=True)
            eps_d.copy_(eps_h, non_blocking=True)
            sig_d.copy_(sig_h, non_blocking=True)
        step(rx_d, tgt_d, eps_d, sig_d, before_calibration=lambda: cap.wait_stream(side))
        torch.cat([loss_buf, g_eps, g_sig, g_gain], out=out_d)
        out_h.copy_(out_d, non_blocking=True)

    ctx.set_profiling(0)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        body()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        body()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    times = []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        g.replay()
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
    if ctx.status_word() != 0:
        raise RuntimeError("device status set during the graph-replayed end-to-end steps")
    expect = torch.cat([loss_buf, g_eps, g_sig, g_gain]).cpu()
    if not torch.equal(out_h, expect):
        raise RuntimeError("the replayed step's host results differ from the device results")
    del g
    total = max_over_ranks(world, sum(times) / 1e3)
    return {"value": sc.n_rays * steps * world / total, "unit": "rays/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * total / steps,
            "timing": "public-API step captured in a CUDA graph; every replay copies the inputs from pinned host "
                      "memory and the loss and gradients back, and the host waits for them"}


EPS0 = 8.8541878128e-12
C0 = 299792458.0


def plain_records(ex, sc, dev):
    """Frozen per-path geometry of the plain PyTorch arm, from the exported points
    (float64 torch ops, once, untimed, like the library's own record pass):
    per depth q the path indices, cos(theta_i) and material of every bounce, the
    q + 1 real 2x2 basis-change matrices (Tx theta/phi basis -> reflection bases
    -> Rx theta/phi basis along the AoA) and the path length."""
    import torch
    f64 = torch.float64
    verts = torch.tensor(sc.verts, dtype=torch.float32, device=dev).double()
    tris = torch.tensor(sc.tris, dtype=torch.int64, device=dev)
    v0, v1, v2 = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    nrm = torch.linalg.cross(v1 - v0, v2 - v0)
    nrm = nrm / nrm.norm(dim=1, keepdim=True)
    tri_mat = torch.tensor(sc.tri_material, dtype=torch.int64, device=dev)
    is_pec = torch.tensor(sc.is_pec, dtype=torch.bool, device=dev)

    def sph(k):
        th = torch.acos(k[:, 2].clamp(-1, 1))
        ph = torch.where((k[:, 0] == 0) & (k[:, 1] == 0), torch.zeros_like(th), torch.atan2(k[:, 1], k[:, 0]))
        t = torch.stack([th.cos() * ph.cos(), th.cos() * ph.sin(), -th.sin()], 1)
        p_ = torch.stack([-ph.sin(), ph.cos(), torch.zeros_like(ph)], 1)
        return t, p_

    def dots(a, b):
        return (a * b).sum(1)

    def dmat(ip, iq, op, oq):
        return torch.stack([torch.stack([dots(ip, op), dots(ip, oq)], 1),
                            torch.stack([dots(iq, op), dots(iq, oq)], 1)], 1)

    groups = []
    depth = ex["depth"].long()
    for q in range(int(depth.max().item()) + 1 if depth.numel() else 0):
        idx = torch.nonzero(depth == q).flatten()
        if idx.numel() == 0:
            continue
        pts = ex["pts"][idx, : q + 2]
        dv = pts[:, 1:] - pts[:, :-1]
        d = dv.norm(dim=2)
        k = dv / d[..., None]
        out_p, out_q = sph(k[:, 0])
        Ds, cos, mats, pec = [], [], [], []
        for j in range(1, q + 1):
            t = ex["seq"][idx, j - 1].long()
            n = nrm[t]
            kj = k[:, j - 1]
            n = torch.where((dots(kj, n) > 0)[:, None], -n, n)
            cos.append(-dots(kj, n))
            cr = torch.linalg.cross(kj, n)
            crn = cr.norm(dim=1, keepdim=True)
            alt = out_p - dots(out_p, kj)[:, None] * kj
            e_perp = torch.where(crn > 1e-12, cr / crn.clamp_min(1e-300), alt / alt.norm(dim=1, keepdim=True))
            in_q = torch.linalg.cross(e_perp, kj)
            Ds.append(dmat(e_perp, in_q, out_p, out_q))
            out_p, out_q = e_perp, torch.linalg.cross(e_perp, k[:, j])
            m = tri_mat[t]
            mats.append(m)
            pec.append(is_pec[m])
        rp, rq = sph(-k[:, q])
        Ds.append(dmat(rp, rq, out_p, out_q))
        groups.append({"idx": idx, "L": d.sum(1).float(), "D": torch.stack(Ds, 1).to(torch.complex64),
                       "cos": torch.stack(cos, 1).float() if q else None,
                       "mat": torch.stack(mats, 1) if q else None, "pec": torch.stack(pec, 1) if q else None})
    return groups


def plain_step(groups, rx, tau, n_rx, eps_r, sigma, freq, fc, df, N, target, w):
    """The calibration step as plain PyTorch complex64 ops: permittivity, Fresnel,
    2x2 chain, a = lambda / (4 pi L) [D_{q+1} G_q ... G_1 D_1 C_T]_0, the CFR as a
    dense P x N phasor matrix summed per receiver, and the weighted power MSE;
    autograd gives the adjoint."""
    import torch
    P = tau.shape[0]
    lam = C0 / freq
    eta = torch.complex(eps_r, -sigma / (EPS0 * 2 * np.pi * freq))
    a = torch.zeros(P, dtype=torch.complex64, device=tau.device)
    for g in groups:
        E = g["D"][:, 0, :, 0]                                   # D_1 C_T, C_T = [1, 0]
        for j in range(g["D"].shape[1] - 1):
            c = g["cos"][:, j].to(torch.complex64)
            e = eta[g["mat"][:, j]]
            s = torch.sqrt(e - (1 - c * c))
            r_perp = torch.where(g["pec"][:, j], torch.full_like(s, -1), (c - s) / (c + s))
            r_par = torch.where(g["pec"][:, j], torch.full_like(s, 1), (e * c - s) / (e * c + s))
            E = torch.stack([r_perp * E[:, 0], r_par * E[:, 1]], 1)
            E = torch.einsum("pab,pb->pa", g["D"][:, j + 1], E)
        a = a.index_put((g["idx"],), (lam / (4 * np.pi)) * E[:, 0] / g["L"])
    n = torch.arange(-N // 2, N // 2, device=tau.device, dtype=torch.float64)
    frac = torch.frac(tau[:, None] * (fc + n * df)[None, :])
    ang = (-2 * np.pi * frac).float()
    ph = torch.polar(torch.ones_like(ang), ang)
    H = torch.zeros((n_rx, N), dtype=torch.complex64, device=tau.device).index_add(0, rx, a[:, None] * ph)
    e_ = H.real ** 2 + H.imag ** 2 - target
    return ((w[:, None] * e_) ** 2).mean()


def time_plain_calibration(p, sc, eps, sig, target, w, flush, n_reps):
    """Times plain_step forward + autograd backward (eager, median of n_reps,
    L2 flushed between reps) and returns it with its loss and gradients."""
    import torch
    dev = eps.device
    ex = p.export()
    groups = plain_records(ex, sc, dev)
    rx = ex["rx"].long()
    e = eps.clone().requires_grad_(True)
    s_ = sig.clone().requires_grad_(True)
    args = (groups, rx, ex["tau"], sc.n_rx, e, s_, sc.freq_hz, sc.f_center_hz, sc.delta_f_hz, sc.n_sub, target, w)
    for _ in range(3):
        e.grad = s_.grad = None
        plain_step(*args).backward()
    stream = torch.cuda.current_stream()
    times = []
    for _ in range(n_reps):
        flush.zero_()
        e.grad = s_.grad = None
        s0, e0 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        L = plain_step(*args)
        L.backward()
        e0.record(stream)
        e0.synchronize()
        times.append(s0.elapsed_time(e0))
    return float(np.median(times)), float(L.item()), e.grad.detach(), s_.grad.detach()


def time_indoor_calibration(rt, ctx, flush, args, plain=True):
    """Calibration step of the indoor differentiation workload (1024 receivers,
    1024 subcarriers around 1.272 GHz): eval_fields -> CFR + power MSE + CFR
    adjoint -> eval_fields adjoint, captured in one CUDA graph."""
    import torch

    import scenegen
    sc = scenegen.indoor_diff()
    dev = torch.device("cuda", torch.cuda.current_device())
    scene = rt.Scene.from_synthetic(ctx, sc)
    rx = torch.tensor(sc.rx, dtype=torch.float64, device=dev)
    p = rt.trace_paths(ctx, scene, sc.tx, rx, sc.n_rays, sc.max_depth)
    fc, df, N = sc.f_center_hz, sc.delta_f_hz, sc.n_sub
    a = rt.eval_fields(ctx, p, torch.tensor(sc.eps_r, device=dev), torch.tensor(sc.sigma, device=dev), sc.freq_hz)
    H = rt.cfr(ctx, p.rx_offsets, a, p.tau, fc, df, N)
    target = (H.abs() ** 2).float().contiguous()
    m = target.mean(1)
    w = torch.where(m > 0, 1.0 / torch.where(m > 0, m, torch.ones_like(m)), torch.zeros_like(m)).float().contiguous()
    eps = torch.full((8,), 4.0, device=dev)
    sig = torch.full((8,), 0.05, device=dev)
    ge, gs, gg = torch.zeros(8, device=dev), torch.zeros(8, device=dev), torch.zeros(2, device=dev)
    loss = torch.zeros(1, device=dev)
    ga = torch.empty_like(a)

    def cal_step():
        rt.eval_fields(ctx, p, eps, sig, sc.freq_hz, out=a)
        rt.cfr_power_mse_fused(ctx, p.rx_offsets, a, p.tau, fc, df, N, target, w, loss=loss, grad_a=ga)
        ge.zero_()
        gs.zero_()
        gg.zero_()
        rt.eval_fields_backward(ctx, p, eps, sig, sc.freq_hz, ga, ge, gs, gg)

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(3):
            cal_step()
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        cal_step()
    stream = torch.cuda.current_stream()
    for _ in range(5):
        g.replay()
    times = []
    n = max(args.steps, 20)
    for _ in range(n):
        flush.zero_()
        s0, e0 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        g.replay()
        e0.record(stream)
        e0.synchronize()
        times.append(s0.elapsed_time(e0))
    # the fused CFR kernel alone (tensor cores), for its roofline
    kt = []
    for _ in range(20):
        flush.zero_()
        s0, e0 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        rt.cfr_power_mse_fused(ctx, p.rx_offsets, a, p.tau, fc, df, N, target, w, loss=loss, grad_a=ga)
        e0.record(stream)
        e0.synchronize()
        kt.append(s0.elapsed_time(e0))
    res = {"workload": "indoor_diff", "n_rx": sc.n_rx, "n_sub": N, "n_paths": p.n_paths,
           "ms_per_step_median": float(np.median(times)), "graph": True, "replays": n,
           "l2": "flushed: 256 MiB written between replays",
           "cfr_fused_ms": float(np.median(kt)),
           "roofline_cfr": roofline_cfr(float(np.median(kt)), p.n_paths, N)}
    if not plain:
        return res
    # the same step with the paper's loss (Eq. loss: SMAPE of the RMS delay spread
    # and of the scaled channel gain, power scale by its moving average), one graph
    res["paper_loss"] = time_paper_loss_step(rt, ctx, p, sc, eps, sig, flush, n)
    # the same step as plain PyTorch complex64 ops (eager, autograd), and how
    # closely its loss and gradients agree with the library's
    plain_ms, plain_loss, pe, ps = time_plain_calibration(p, sc, eps, sig, target, w, flush, min(n, 20))
    g.replay()
    torch.cuda.synchronize()

    def rel(x, ref):
        return float((x - ref).norm() / ref.norm().clamp_min(1e-30))
    res["plain_pytorch"] = {"ms_per_step_median": plain_ms, "eager": True, "dtype": "complex64",
                            "speedup": plain_ms / float(np.median(times)),
                            "loss_rel_diff": abs(plain_loss - loss.item()) / max(abs(loss.item()), 1e-30),
                            "grad_eps_rel_diff": rel(ge, pe), "grad_sigma_rel_diff": rel(gs, ps)}
    return res


def time_fields_hbm(rt, ctx, scene, sc, flush, reps=10, copies=1000):
    """eval_fields and its adjoint at a size where HBM binds: the street-canyon
    path set tiled `copies` times (each copy on its own receivers) through
    rt_paths_import.  Algorithmic bytes per path of depth q: forward 4 (depth) +
    4 (L) + 16 (D_1) + q (4 tri + 4 cos + 16 D) + 8 (a out); the adjoint reads the
    same records plus 8 (dL/da).  The material table is L2-resident."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    rx = torch.tensor(sc.rx, dtype=torch.float64, device=dev)
    p0 = rt.trace_paths(ctx, scene, sc.tx, rx, sc.n_rays, sc.max_depth)
    ex = p0.export()
    P0, R0 = p0.n_paths, sc.n_rx
    reps_rx = (ex["rx"].long()[None, :] + R0 * torch.arange(copies, device=dev)[:, None]).reshape(-1).int()
    p = rt.import_paths(ctx, scene, reps_rx, ex["depth"].repeat(copies), ex["seq"].repeat(copies, 1),
                        ex["pts"].repeat(copies, 1, 1), R0 * copies)
    del reps_rx
    q = ex["depth"].double()
    fwd_bytes = float(copies * (4 + 4 + 16 + 24 * q + 8).sum().item())
    bwd_bytes = fwd_bytes + 8.0 * copies * P0
    eps = torch.tensor(sc.eps_r, device=dev)
    sig = torch.tensor(sc.sigma, device=dev)
    a = rt.eval_fields(ctx, p, eps, sig, sc.freq_hz)
    ga = (a * 0.5).contiguous()
    ge, gs, gg = torch.zeros_like(eps), torch.zeros_like(sig), torch.zeros(2, device=dev)
    stream = torch.cuda.current_stream()

    def timed(fn):
        out = []
        for _ in range(reps):
            flush.zero_()
            s0, e0 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            fn()
            e0.record(stream)
            e0.synchronize()
            out.append(s0.elapsed_time(e0))
        return float(np.median(out))
    t_f = timed(lambda: rt.eval_fields(ctx, p, eps, sig, sc.freq_hz, out=a))
    t_b = timed(lambda: rt.eval_fields_backward(ctx, p, eps, sig, sc.freq_hz, ga, ge, gs, gg))
    peaks, src = load_peaks()
    hbm = peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"])
    gf, gb = fwd_bytes / (t_f * 1e-3) / 1e9, bwd_bytes / (t_b * 1e-3) / 1e9

    def line(ms, nbytes, g, kernel):
        # traffic: DRAM bytes per launch from the committed ncu counters (null once the
        # kernel's code changed); the records of a warp's paths have mixed depths, so a
        # slot's sectors are partly unused and DRAM traffic exceeds the algorithmic bytes
        tr = ncu_traffic(kernel) if copies == 1000 else None
        out = {"ms": ms, "bytes": nbytes, "achieved_gbs": g, "peak_gbs": hbm, "frac": g / hbm, "traffic": tr}
        if tr:
            out["dram_gbs"] = tr / (ms * 1e-3) / 1e9
            out["dram_frac"] = out["dram_gbs"] / hbm
        return out
    return {"workload": f"street_canyon paths x {copies} (rt_paths_import)", "n_paths": p.n_paths,
            "fields_fwd": line(t_f, fwd_bytes, gf, "k_fields_fwd"),
            "fields_bwd": line(t_b, bwd_bytes, gb, "k_fields_bwd"),
            "peak_source": src}


def time_diffuse(rt, ctx, flush, args, n_rx_step=4, n_rays_diffuse=20_000):
    """Diffuse reflection on the indoor scene (256 receivers): the diffuse trace
    (next-event estimation from every shoot-and-bounce hit), the calibration step
    over specular + diffuse paths captured in one CUDA graph (eval_fields ->
    specular share, eval_fields_diffuse -> per-receiver merge -> CFR + power MSE +
    CFR adjoint -> split -> adjoints of both), and the diffuse field kernels alone
    with their HBM roofline.  Algorithmic bytes per diffuse path of depth j:
    forward 4 (depth) + 8 j (material, cos) + 16 (j + 1) (basis changes) + 16
    (pattern cosines, 1/d) + 8 (a out) = 44 + 24 j; the adjoint reads the same
    records and dL/da instead of writing a."""
    import torch

    import scenegen
    sc = scenegen.indoor_diff()
    dev = torch.device("cuda", torch.cuda.current_device())
    scene = rt.Scene.from_synthetic(ctx, sc)
    rx = torch.tensor(sc.rx[::n_rx_step], dtype=torch.float64, device=dev)
    R = rx.shape[0]
    stream = torch.cuda.current_stream()

    def ev_time(fn, reps):
        out = []
        for _ in range(reps):
            flush.zero_()
            s0, e0 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            fn()
            e0.record(stream)
            e0.synchronize()
            out.append(s0.elapsed_time(e0))
        return float(np.median(out))
    ps = rt.trace_paths(ctx, scene, sc.tx, rx, sc.n_rays, sc.max_depth)
    pd = rt.trace_diffuse(ctx, scene, sc.tx, rx, n_rays_diffuse, sc.max_depth)
    trace_ms = ev_time(lambda: rt.trace_diffuse(ctx, scene, sc.tx, rx, n_rays_diffuse, sc.max_depth), 3)
    fc, df, N = sc.f_center_hz, sc.delta_f_hz, sc.n_sub
    eps = torch.tensor(sc.eps_r, device=dev)
    sig = torch.tensor(sc.sigma, device=dev)
    hidden = torch.tensor(scenegen.random_scattering(21, sc.n_materials), device=dev)
    tau, off = rt.rx_merge(ctx, ps.rx_offsets, pd.rx_offsets, ps.tau, pd.tau)
    a_s = rt.specular_reduction(ctx, ps, hidden, rt.eval_fields(ctx, ps, eps, sig, sc.freq_hz))
    a_d = rt.eval_fields_diffuse(ctx, pd, eps, sig, hidden, sc.freq_hz)
    a_m, _ = rt.rx_merge(ctx, ps.rx_offsets, pd.rx_offsets, a_s, a_d)
    T = (rt.cfr(ctx, off, a_m, tau, fc, df, N).abs() ** 2).float().contiguous()
    m = T.mean(1)
    w = torch.where(m > 0, 1.0 / torch.where(m > 0, m, torch.ones_like(m)), torch.zeros_like(m)).float().contiguous()
    scat = hidden.clone()
    scat[:, 0] *= 0.7
    scat[:, 1] = 0.25
    M = sc.n_materials
    ge, gs, gg = torch.zeros(M, device=dev), torch.zeros(M, device=dev), torch.zeros(2, device=dev)
    gc = torch.zeros_like(scat)
    loss = torch.zeros(1, device=dev)
    a_sp = torch.empty_like(a_s)
    a_sr = torch.empty_like(a_s)
    a_df = torch.empty_like(a_d)
    ga_m = torch.empty_like(a_m)
    Ps, Pd = ps.n_paths, pd.n_paths

    def cal_step():
        rt.eval_fields(ctx, ps, eps, sig, sc.freq_hz, out=a_sp)
        rt.specular_reduction(ctx, ps, scat, a_sp, out=a_sr)
        rt.eval_fields_diffuse(ctx, pd, eps, sig, scat, sc.freq_hz, out=a_df)
        am, _ = rt.rx_merge(ctx, ps.rx_offsets, pd.rx_offsets, a_sr, a_df)
        rt.cfr_power_mse_fused(ctx, off, am, tau, fc, df, N, T, w, loss=loss, grad_a=ga_m)
        g_s, g_d = rt.rx_split(ctx, ps.rx_offsets, pd.rx_offsets, ga_m, Ps, Pd)
        ge.zero_()
        gs.zero_()
        gg.zero_()
        gc.zero_()
        g_sp, _ = rt.specular_reduction_backward(ctx, ps, scat, a_sr, g_s, grad_scat=gc)
        rt.eval_fields_backward(ctx, ps, eps, sig, sc.freq_hz, g_sp, ge, gs, gg)
        rt.eval_fields_diffuse_backward(ctx, pd, eps, sig, scat, sc.freq_hz, g_d, ge, gs, gc)

    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        for _ in range(3):
            cal_step()
    stream.wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        cal_step()
    for _ in range(5):
        g.replay()
    n = max(args.steps, 20)
    step_ms = ev_time(g.replay, n)
    cfr_ms = ev_time(lambda: rt.cfr_power_mse_fused(ctx, off, a_m, tau, fc, df, N, T, w, loss=loss, grad_a=ga_m), 10)
    rt.set_cfr_tensor_cores(ctx, False)
    cfr_simt_ms = ev_time(lambda: rt.cfr_power_mse_fused(ctx, off, a_m, tau, fc, df, N, T, w, loss=loss,
                                                         grad_a=ga_m), 10)
    rt.set_cfr_tensor_cores(ctx, True)
    # receivers with more than 4096 paths take the non-uniform FFT (O(W) per path,
    # O(N log N) per receiver), the others the dense tensor-core product: the dense
    # flop count is then an equivalent-work rate, not a fraction of a roofline
    counts = (off[1:] - off[:-1]).cpu()
    heavy = counts > 4096
    p_nufft = int(counts[heavy].sum().item())
    cfr_split = {"kernel": "k_cfr_tc<8,3>", "kernel_ms": cfr_ms, "receivers_nufft": int(heavy.sum().item()),
                 "paths_nufft": p_nufft, "paths_dense": int(Ps + Pd) - p_nufft,
                 "dense_equivalent_tflops": 3 * 16.0 * N * (Ps + Pd) / (cfr_ms * 1e-3) / 1e12,
                 "roofline": None,
                 "note": "receivers above 4096 paths use the non-uniform FFT, latency-bound on the "
                         "shared-memory atomics of the spreading; the dense-equivalent rate counts "
                         "3 x 16 N P TF32 flops as if every path went through the dense product"}
    t_f = ev_time(lambda: rt.eval_fields_diffuse(ctx, pd, eps, sig, scat, sc.freq_hz, out=a_df), 20)
    gd = (a_df * 0.5).contiguous()
    t_b = ev_time(lambda: rt.eval_fields_diffuse_backward(ctx, pd, eps, sig, scat, sc.freq_hz, gd, ge, gs, gc), 20)
    j = pd.export()["depth"].double()
    fwd_bytes = float((44.0 + 24.0 * j).sum().item())
    peaks, src = load_peaks()
    hbm = peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"])
    gf, gb = fwd_bytes / (t_f * 1e-3) / 1e9, fwd_bytes / (t_b * 1e-3) / 1e9
    return {"workload": "indoor_diff, 256 receivers, specular 1e6 rays + diffuse 2e4 rays, depth 3",
            "n_rx": R, "n_rays_diffuse": n_rays_diffuse, "n_paths_specular": Ps, "n_paths_diffuse": Pd,
            "nee_pairs": n_rays_diffuse * sc.max_depth * R,
            "trace_diffuse_ms": trace_ms, "nee_pairs_per_s": n_rays_diffuse * sc.max_depth * R / (trace_ms * 1e-3),
            "calibration_step_ms": step_ms, "graph": True, "n_sub": N, "cfr_fused_ms": cfr_ms,
            "cfr_fused_simt_ms": cfr_simt_ms, "cfr_split": cfr_split,
            "l2": "flushed: 256 MiB written between timed runs",
            "roofline_fields_diffuse": {"kernel": "k_df_fwd", "bound": "hbm", "achieved": gf, "peak": hbm,
                                        "unit": "GB/s", "frac": gf / hbm, "ms": t_f, "bytes": fwd_bytes,
                                        "peak_source": src},
            "roofline_fields_diffuse_bwd": {"kernel": "k_df_bwd", "bound": "hbm", "achieved": gb, "peak": hbm,
                                            "unit": "GB/s", "frac": gb / hbm, "ms": t_b, "bytes": fwd_bytes,
                                            "peak_source": src}}


def time_paper_loss_step(rt, ctx, p, sc, eps, sig, flush, n):
    """Calibration step of Algorithm 1 with the paper's loss on traced paths:
    eval_fields -> CFR -> CIR statistics -> power scale (moving average) -> SMAPE
    loss and dL/dH -> CFR adjoint -> eval_fields adjoint, captured in one graph."""
    import torch
    dev = eps.device
    fc, df, N = sc.f_center_hz, sc.delta_f_hz, sc.n_sub
    a = rt.eval_fields(ctx, p, torch.tensor(sc.eps_r, device=dev), torch.tensor(sc.sigma, device=dev), sc.freq_hz)
    H = rt.cfr(ctx, p.rx_offsets, a, p.tau, fc, df, N)
    Pm, tm = rt.cir_stats(ctx, H, df)
    Pm = torch.where(Pm > 0, Pm * 0.25, torch.full_like(Pm, 1e-30)).contiguous()
    tm = torch.where(tm > 0, tm, torch.full_like(tm, 1e-9)).contiguous()
    R = sc.n_rx
    Pp = torch.empty(R, device=dev)
    state = torch.zeros(2, device=dev)
    loss = torch.zeros(1, device=dev)
    gH = torch.empty_like(H)
    ga = torch.empty_like(a)
    ge, gs, gg = torch.zeros_like(eps), torch.zeros_like(sig), torch.zeros(2, device=dev)

    def step():
        rt.eval_fields(ctx, p, eps, sig, sc.freq_hz, out=a)
        rt.cfr(ctx, p.rx_offsets, a, p.tau, fc, df, N, out=H)
        Pp_, _ = rt.cir_stats(ctx, H, df)
        Pp.copy_(Pp_)
        rt.power_scale_ema(ctx, Pm, Pp, 0.99, state)
        rt.delay_spread_power_loss(ctx, H, df, Pm, tm, state, loss=loss, grad_H=gH)
        rt.cfr_backward(ctx, p.rx_offsets, p.tau, fc, df, N, gH, out=ga)
        ge.zero_()
        gs.zero_()
        gg.zero_()
        rt.eval_fields_backward(ctx, p, eps, sig, sc.freq_hz, ga, ge, gs, gg)

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(3):
            step()
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    stream = torch.cuda.current_stream()
    for _ in range(3):
        g.replay()
    times = []
    for _ in range(n):
        flush.zero_()
        s0, e0 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        g.replay()
        e0.record(stream)
        e0.synchronize()
        times.append(s0.elapsed_time(e0))
    return {"ms_per_step_median": float(np.median(times)), "graph": True, "loss": float(loss.item()),
            "alpha": float(state[0].item()),
            "launches": "fields, CFR (tensor cores), CIR statistics, power scale, SMAPE loss + dL/dH, CFR adjoint "
                        "(tensor cores), fields adjoint"}


def time_batch(rt, ctx, args, reps=3):
    """16 procedural cities (1k-50k triangles, 65,536 receivers split unevenly,
    10^7 rays per scene, depth 4): rt_trace_batch against a loop of per-scene
    rt_trace_paths calls (both timed on the stream from the first launch to the
    last, host round trips included), then the calibration step over all scenes
    (fields + CFR at 256 subcarriers + loss + adjoints) as one CUDA graph against a
    per-scene loop.  The tracing launch shapes come from the autotuner run on the
    largest scene."""
    import torch

    import scenegen
    cities = scenegen.city_batch()
    dev = torch.device("cuda", torch.cuda.current_device())
    scenes = [rt.Scene.from_synthetic(ctx, c) for c in cities]
    rxs = [torch.tensor(c.rx, device=dev) for c in cities]
    txs = [c.tx for c in cities]
    n_rays, depth = cities[0].n_rays, cities[0].max_depth
    big = max(range(len(cities)), key=lambda i: cities[i].n_tris)
    tuned, tune_ms = rt.autotune_trace(ctx, scenes[big], txs[big], rxs[big], n_rays, depth)
    stream = torch.cuda.current_stream()

    def timed(fn):
        s0, e0 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        s0.record(stream)
        out = fn()
        e0.record(stream)
        e0.synchronize()
        return s0.elapsed_time(e0), out

    timed(lambda: rt.trace_batch(ctx, scenes, txs, rxs, n_rays, depth))
    t_batch, t_loop = [], []
    for _ in range(reps):
        t, pb = timed(lambda: rt.trace_batch(ctx, scenes, txs, rxs, n_rays, depth))
        t_batch.append(t)
        del pb
        t, pl = timed(lambda: [rt.trace_paths(ctx, scenes[i], txs[i], rxs[i], n_rays, depth)
                               for i in range(len(cities))])
        t_loop.append(t)
        del pl
    total_rays = n_rays * len(cities)
    # calibration over all scenes: one paths object (batch) vs per-scene objects
    pb = rt.trace_batch(ctx, scenes, txs, rxs, n_rays, depth)
    pl = [rt.trace_paths(ctx, scenes[i], txs[i], rxs[i], n_rays, depth) for i in range(len(cities))]
    c0 = cities[0]
    fc, df, N, f = c0.f_center_hz, c0.delta_f_hz, c0.n_sub, c0.freq_hz
    eps = torch.tensor(c0.eps_r, device=dev)
    sig = torch.tensor(c0.sigma, device=dev)
    eps_t, sig_t = (eps * 1.2).contiguous(), (sig * 0.7).contiguous()

    def target(p):
        a = rt.eval_fields(ctx, p, eps, sig, f)
        T = (rt.cfr(ctx, p.rx_offsets, a, p.tau, fc, df, N).abs() ** 2).float().contiguous()
        m = T.mean(1)
        w = torch.where(m > 0, 1 / torch.where(m > 0, m, torch.ones_like(m)), torch.zeros_like(m)).float()
        return T, w.contiguous()

    def make_step(p):
        T, w = target(p)
        a = torch.empty(max(p.n_paths, 1), dtype=torch.complex64, device=dev)[: p.n_paths]
        ga = torch.empty_like(a)
        loss = torch.zeros(1, device=dev)
        ge, gs, gg = torch.zeros_like(eps), torch.zeros_like(sig), torch.zeros(2, device=dev)

        def step():
            rt.eval_fields(ctx, p, eps_t, sig_t, f, out=a)
            rt.cfr_power_mse_fused(ctx, p.rx_offsets, a, p.tau, fc, df, N, T, w, loss=loss, grad_a=ga)
            rt.eval_fields_backward(ctx, p, eps_t, sig_t, f, ga, ge, gs, gg)
        return step

    step_b = make_step(pb)
    steps_l = [make_step(p) for p in pl]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(3):
            step_b()
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step_b()
    for _ in range(3):
        g.replay()
        for st in steps_l:
            st()
    cal_graph = [timed(g.replay)[0] for _ in range(10)]
    cal_loop = [timed(lambda: [st() for st in steps_l])[0] for _ in range(10)]
    n_paths_b, n_cand_b = pb.n_paths, pb.n_candidates
    del g, step_b, steps_l, pb, pl
    # trace + calibration of every scene: a per-scene loop, one batched pipeline,
    # and that pipeline replayed from one CUDA graph (the traces do not wait for
    # the host in any of the three)
    full = trace_calibration_forms(rt, ctx, scenes, txs, rxs, n_rays, depth, c0, dev, reps)
    small_idx = [i for i, c in enumerate(cities) if c.n_tris < 3500]
    small = trace_calibration_forms(rt, ctx, [scenes[i] for i in small_idx], [txs[i] for i in small_idx],
                                    [rxs[i] for i in small_idx], 100_000, depth, c0, dev, 20)
    small.update({"scenes": small_idx, "n_tris": [cities[i].n_tris for i in small_idx], "rays_per_scene": 100_000})
    return {"workload": "city_batch", "n_scenes": len(cities), "n_tris": [c.n_tris for c in cities],
            "n_rx": int(sum(c.n_rx for c in cities)), "rays_per_scene": n_rays, "max_depth": depth,
            "n_paths": n_paths_b, "n_candidates": n_cand_b,
            "trace_batched_ms": float(np.median(t_batch)), "trace_loop_ms": float(np.median(t_loop)),
            "rays_per_s_batched": total_rays / (np.median(t_batch) * 1e-3),
            "rays_per_s_loop": total_rays / (np.median(t_loop) * 1e-3),
            "calibration_graph_ms": float(np.median(cal_graph)), "calibration_loop_ms": float(np.median(cal_loop)),
            "trace_and_calibration": full, "small_cities_trace_and_calibration": small,
            "autotuned_blocks_per_sm": {"sbr": tuned[0], "pairs": tuned[1], "visibility": tuned[2]},
            "autotune_stage_ms": tune_ms}


def trace_calibration_forms(rt, ctx, scenes, txs, rxs, n_rays, depth, c0, dev, reps):
    """Trace + calibration step (fields, fused CFR + power MSE + adjoint at 256
    subcarriers, fields adjoint) of every scene, three ways: a loop of per-scene
    rt_trace_paths and calibration calls, one rt_trace_batch pipeline with one
    calibration over all receivers, and that pipeline captured in one CUDA graph
    and replayed.  Traces do not wait for the host (rt_set_trace_async; inside the
    graph they cannot); the median of `reps` timed runs on the stream, L2 not
    flushed (the scenes and paths are the step's working set)."""
    import torch
    stream = torch.cuda.current_stream()
    fc, df, N, f = c0.f_center_hz, c0.delta_f_hz, c0.n_sub, c0.freq_hz
    eps = torch.tensor(c0.eps_r, device=dev)
    sig = torch.tensor(c0.sigma, device=dev)
    eps_t, sig_t = (eps * 1.2).contiguous(), (sig * 0.7).contiguous()

    def target(p):
        a = rt.eval_fields(ctx, p, eps, sig, f)
        T = (rt.cfr(ctx, p.rx_offsets, a, p.tau, fc, df, N).abs() ** 2).float().contiguous()
        m = T.mean(1)
        return T, torch.where(m > 0, 1 / torch.where(m > 0, m, torch.ones_like(m)), torch.zeros_like(m)).float()

    pb = rt.trace_batch(ctx, scenes, txs, rxs, n_rays, depth)          # capacities, targets
    Tb, wb = target(pb)
    tl = [target(rt.trace_paths(ctx, scenes[i], txs[i], rxs[i], n_rays, depth)) for i in range(len(scenes))]
    loss = torch.zeros(1, device=dev)
    ge, gs, gg = torch.zeros_like(eps), torch.zeros_like(sig), torch.zeros(2, device=dev)

    def calibrate(p, T, w):
        a = rt.eval_fields(ctx, p, eps_t, sig_t, f)
        _, ga, _ = rt.cfr_power_mse_fused(ctx, p.rx_offsets, a, p.tau, fc, df, N, T, w, loss=loss)
        rt.eval_fields_backward(ctx, p, eps_t, sig_t, f, ga, ge, gs, gg)

    def step_batch():
        p = rt.trace_batch(ctx, scenes, txs, rxs, n_rays, depth)
        calibrate(p, Tb, wb)
        return p

    def step_loop():
        for i in range(len(scenes)):
            calibrate(rt.trace_paths(ctx, scenes[i], txs[i], rxs[i], n_rays, depth), *tl[i])

    def timed(fn, n):
        ts = []
        for _ in range(n):
            torch.cuda.synchronize()
            s0, e0 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            fn()
            e0.record(stream)
            e0.synchronize()
            ts.append(s0.elapsed_time(e0))
        return float(np.median(ts))

    rt.set_trace_async(ctx, True)
    try:
        for _ in range(2):
            step_loop()
            step_batch()
        t_loop = timed(step_loop, reps)
        t_batch = timed(step_batch, reps)
        side = torch.cuda.Stream()
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            step_batch()
        stream.wait_stream(side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            pg = step_batch()
        g.replay()
        t_graph = timed(g.replay, reps)
    finally:
        rt.set_trace_async(ctx, False)
    torch.cuda.synchronize()
    if ctx.status_word() != 0:
        raise RuntimeError("device status set during the batched trace measurement")
    pg.resolve()
    if pg.n_paths != pb.n_paths:
        raise RuntimeError("the graph-replayed batch found a different number of paths")
    del g, pg
    return {"n_scenes": len(scenes), "n_paths": pb.n_paths, "loop_ms": t_loop, "batched_ms": t_batch,
            "graph_ms": t_graph, "reps": reps}


def time_learned(rt, ctx, args, train_steps=150, timed_steps=20, warm_steps=3):
    """Room-and-corridor scene (19,626 triangles, per-triangle ground truth) at its
    stated size: 10^5 receivers at 256 subcarriers, 90,000 for training and 10,000
    held out, 10^6 rays at depth 3.  Both forms run full-batch Adam steps over all
    training receivers (one step = one epoch): the neural form (MLP -> per-triangle
    fields -> CFR loss -> adjoints -> MLP adjoint) and the plain per-object form
    (4 objects).  Both are warmed for the same steps, then the same number of steps
    of each is timed.  Reported: the step times, the held-out losses after the same
    number of steps, and the per-triangle eps_r / sigma errors of both against the
    hidden ground truth."""
    import torch

    import scenegen
    sc = scenegen.room_corridor()
    n_tr = 90_000
    dev = torch.device("cuda", torch.cuda.current_device())
    scene_tri = rt.Scene.from_synthetic(ctx, sc)
    scene_obj = rt.Scene(ctx, sc.verts, sc.tris, sc.tri_object, np.zeros(4, np.uint8))
    rx_tr = torch.tensor(sc.rx[:n_tr], device=dev)
    rx_te = torch.tensor(sc.rx[n_tr:], device=dev)
    fc, df, N, f = sc.f_center_hz, sc.delta_f_hz, sc.n_sub, sc.freq_hz
    eg, sg = torch.tensor(sc.eps_r, device=dev), torch.tensor(sc.sigma, device=dev)

    def target(p):
        a = rt.eval_fields(ctx, p, eg, sg, f, per_triangle=True)
        T = (rt.cfr(ctx, p.rx_offsets, a, p.tau, fc, df, N).abs() ** 2).float().contiguous()
        m = T.mean(1)
        w = torch.where(m > 0, 1 / torch.where(m > 0, m, torch.ones_like(m)), torch.zeros_like(m)).float()
        return T, w.contiguous()

    t0 = time.perf_counter()
    tri_tr = rt.trace_paths(ctx, scene_tri, sc.tx, rx_tr, sc.n_rays, sc.max_depth)
    torch.cuda.synchronize()
    trace_s = time.perf_counter() - t0
    tri_te = rt.trace_paths(ctx, scene_tri, sc.tx, rx_te, sc.n_rays, sc.max_depth)
    obj_tr = rt.trace_paths(ctx, scene_obj, sc.tx, rx_tr, sc.n_rays, sc.max_depth)
    obj_te = rt.trace_paths(ctx, scene_obj, sc.tx, rx_te, sc.n_rays, sc.max_depth)
    Ttr, wtr = target(tri_tr)
    Tte, wte = target(tri_te)
    seen = torch.unique(tri_tr.export()["seq"])
    seen = seen[seen >= 0]
    plain = rt.LogMaterials(np.full(4, 4.0), np.full(4, 0.05)).cuda()
    opt_p = torch.optim.Adam(plain.parameters(), lr=0.05)
    Ws, bs = scenegen.random_mlp_params(11)
    Ws = [w * 0.5 for w in Ws]
    bs[-1] = np.array([np.log(0.05), np.log(3.0)], np.float32)
    neural = rt.NeuralMaterials(Ws, bs)
    opt_n = torch.optim.Adam(neural.parameters(), lr=3e-3)

    def plain_step(p, T, w, train=True):
        e, s = plain()
        L = rt.calibration_loss(ctx, p, e.contiguous(), s.contiguous(), T, w, f, fc, df, N)
        if train:
            opt_p.zero_grad()
            L.backward()
            opt_p.step()
        return L

    def neural_step(p, T, w, train=True):
        e, s = neural(ctx, scene_tri)
        L = rt.calibration_loss(ctx, p, e, s, T, w, f, fc, df, N, per_triangle=True)
        if train:
            opt_n.zero_grad()
            L.backward()
            opt_n.step()
        return L

    stream = torch.cuda.current_stream()

    def timed(fn, n):
        s0, e0 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(n):
            fn()
        e0.record(stream)
        e0.synchronize()
        return s0.elapsed_time(e0) / n

    run_p = lambda: plain_step(obj_tr, Ttr, wtr)     # noqa: E731
    run_n = lambda: neural_step(tri_tr, Ttr, wtr)    # noqa: E731
    for _ in range(warm_steps):
        run_p()
        run_n()
    torch.cuda.synchronize()
    ms_plain = timed(run_p, timed_steps)
    ms_neural = timed(run_n, timed_steps)
    for _ in range(train_steps - warm_steps - timed_steps):
        run_p()
        run_n()
    with torch.no_grad():
        held_plain = plain_step(obj_te, Tte, wte, train=False).item()
        held_neural = neural_step(tri_te, Tte, wte, train=False).item()
        e_n, s_n = neural(ctx, scene_tri)
        e_o, s_o = plain()
        tob = torch.as_tensor(sc.tri_object, device=dev, dtype=torch.int64)
        e_p, s_p = e_o[tob], s_o[tob]

        def tri_err(e, s, idx):
            re = ((e[idx] - eg[idx]).abs() / eg[idx]).mean().item()
            ls = (torch.log10(s[idx]) - torch.log10(sg[idx])).abs().mean().item()
            return {"eps_r_mean_rel": re, "sigma_mean_abs_log10": ls}
        every = torch.arange(sc.n_tris, device=dev)
        errors = {"neural": {"seen": tri_err(e_n, s_n, seen), "all": tri_err(e_n, s_n, every)},
                  "plain": {"seen": tri_err(e_p, s_p, seen), "all": tri_err(e_p, s_p, every)},
                  "triangles_seen": int(seen.numel())}
    # MLP kernels alone (the a12 roofline inputs)
    w16 = neural.w.detach().to(torch.bfloat16)
    b = neural.b.detach()
    eps, sig, act = rt.mlp_forward(ctx, scene_tri, w16, b)
    g1 = torch.ones_like(eps)
    ms_fwd = timed(lambda: rt.mlp_forward(ctx, scene_tri, w16, b), 20)
    gw = torch.zeros(rt.MLP_NW, device=dev)
    gb = torch.zeros(rt.MLP_NB, device=dev)
    dz = torch.empty((sc.n_tris, 384), device=dev)
    ms_bwd = timed(lambda: rt.mlp_backward(ctx, scene_tri, w16, act, eps, sig, g1, g1, gw, gb, dz), 20)
    flops_fwd = 2.0 * sc.n_tris * (40 * 128 + 2 * 128 * 128 + 128 * 2)
    res = {"workload": "room_corridor", "n_tris": sc.n_tris, "train_rx": n_tr, "heldout_rx": sc.n_rx - n_tr,
           "n_sub": N, "n_rays": sc.n_rays, "train_paths": tri_tr.n_paths, "heldout_paths": tri_te.n_paths,
           "trace_train_s": trace_s, "adam_steps": train_steps,
           "step": "full batch over the training receivers (one Adam step = one epoch)",
           "warmup_steps_each": warm_steps, "timed_steps_each": timed_steps,
           "neural_step_ms": ms_neural, "plain_step_ms": ms_plain,
           "heldout_loss_neural": held_neural, "heldout_loss_plain": held_plain,
           "per_triangle_error": errors,
           "mlp_fwd_ms": ms_fwd, "mlp_bwd_ms": ms_bwd,
           "mlp_fwd_tflops": flops_fwd / (ms_fwd * 1e-3) / 1e12,
           "mlp_bwd_tflops": 2 * flops_fwd / (ms_bwd * 1e-3) / 1e12}
    del tri_tr, tri_te, obj_tr, obj_te, Ttr, Tte
    torch.cuda.empty_cache()
    return res


def code_sha256(path):
    """SHA-256 of a C/C++/CUDA source with its comments and layout removed: a
    change to the code changes it, a change to a comment or to whitespace does
    not.  String and character literals are kept as they are."""
    import hashlib
    with open(path, encoding="utf-8") as f:
        src = f.read()
    out = []
    i, n = 0, len(src)
    while i < n:
        ch = src[i]
        if src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        elif ch in "\"'":
            j = i + 1
            while j < n and src[j] != ch:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        else:
            out.append(ch)
            i += 1
    tokens = "".join(out).split()
    return hashlib.sha256(" ".join(tokens).encode()).hexdigest()


def ncu_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or None
    when the code of the kernel's source file changed since the counters were
    taken (comments aside)."""
    p = os.path.join(ROOT, "profiles", "ncu_counters.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f).get(kernel)
    if not d:
        return None
    src = os.path.join(ROOT, d["source"])
    if not os.path.exists(src):
        return None
    if code_sha256(src) != d["code_sha256"]:
        return None
    return d["dram_bytes_per_launch"] * d.get("scale_to_bench", 1.0)


def fp32_peak(peaks):
    """FP32 SIMT peak: the measured SGEMM rate when present, else unit counts x clock."""
    if peaks.get("fp32_tflops"):
        return peaks["fp32_tflops"], "measured: cuBLAS float32 matmul with TF32 off (SIMT FMA), 8192^3"
    return FP32_PEAK_TFLOPS, "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"


def roofline_for(name, ms, counters, cal, n_paths, sc, N, peaks, peak_src):
    hbm = peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"])
    fp32, fp32_src = fp32_peak(peaks)
    if name == "sbr":
        flops = FLOPS_PER_NODE_VISIT * counters[0] + FLOPS_PER_TRI_TEST * counters[1]
        ach = flops / (ms * 1e-3) / 1e12
        return {"kernel": "k_sbr", "bound": "alu", "achieved": ach, "peak": fp32,
                "unit": "TFLOP/s", "frac": ach / fp32, "traffic": ncu_traffic("k_sbr"),
                "kernel_ms": ms, "peak_source": fp32_src, "frac_of_derived": ach / FP32_PEAK_TFLOPS,
                "algorithmic": f"{FLOPS_PER_NODE_VISIT} flops/node visit + {FLOPS_PER_TRI_TEST} flops/triangle test"}
    if name == "visibility":
        flops = FLOPS_PER_NODE_VISIT * counters[4] + FLOPS_PER_TRI_TEST * counters[5]
        ach = flops / (ms * 1e-3) / 1e12
        return {"kernel": "k_visibility", "bound": "alu", "achieved": ach, "peak": fp32,
                "unit": "TFLOP/s", "frac": ach / fp32, "traffic": None, "peak_source": fp32_src}
    if name in ("fields_fwd", "fields_bwd"):
        # bytes per path of depth q: 4 (depth) + 4 (L) + 4q (tri) + 4q (cos) + 16(q+1) (D) + 8 (a)
        q = 2.0
        per = 4 + 4 + 8 * q + 16 * (q + 1) + 8 + (8 if name == "fields_bwd" else 0)
        gbs = per * n_paths / (ms * 1e-3) / 1e9
        return {"kernel": "k_" + name, "bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                "frac": gbs / hbm, "traffic": None, "peak_source": peak_src}
    # stage without a dedicated counter model: report time only against HBM with its bytes unknown
    return {"kernel": name, "bound": "alu", "achieved": None, "peak": fp32, "unit": "TFLOP/s",
            "frac": None, "traffic": None, "ms": ms}


def roofline_cfr(ms, n_paths, N):
    """Fused CFR + loss + adjoint on the tensor cores: 16 N P algorithmic FP32
    flops (8 per complex multiply-add, forward and adjoint), executed as three
    TF32 products each (hi.hi + hi.lo + lo.hi); peak = the TF32 dense rate measured
    with cuBLAS in this process (else the measured BF16 peak x the nominal TF32 /
    BF16 ratio 1.1 / 2.25)."""
    peaks, src = load_peaks()
    if _MEASURED.get("tf32_tflops"):
        tf32, psrc = _MEASURED["tf32_tflops"], "measured: cuBLAS float32 matmul with TF32 allowed, 8192^3"
    else:
        tf32 = peaks.get("bf16_tflops", PEAKS_FALLBACK["bf16_tflops"]) * (1.1 / 2.25)
        psrc = f"{src} bf16 x 1.1/2.25 (TF32)"
    ach = 3 * 16.0 * N * n_paths / (ms * 1e-3) / 1e12
    return {"kernel": "k_cfr_tc<8,3>", "bound": "tensor", "achieved": ach, "peak": tf32, "unit": "TFLOP/s",
            "frac": ach / tf32, "traffic": ncu_traffic("k_cfr_tc"), "kernel_ms": ms,
            "peak_source": psrc,
            "algorithmic": "3 x 16 N P TF32 flops (3xTF32 split of 8 N P complex MAC flops, forward and adjoint)"}


def cpu_baseline(sc, N):
    """The FP64 oracle as it stands on the host cores: the same step, full workload."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    oracle_step(sc, N)
    dt = time.perf_counter() - t0
    reps = 1
    if dt < 5.0:
        t0 = time.perf_counter()
        for _ in range(2):
            oracle_step(sc, N)
        dt = (time.perf_counter() - t0) / 2
        reps = 2
    return {"value": sc.n_rays / dt, "unit": "rays/s", "cores": omp_threads(), "kind": "oracle",
            "sample": f"full street-canyon step (trace + fields + CFR + loss + adjoints), mean of {reps}",
            "ms_per_step": 1e3 * dt}


def run_case(args):
    """One workload alone, for profiler captures (prints a short line, not the
    benchmark line): street_step = the street-canyon step (trace + fields +
    fused CFR loss + adjoints); indoor_calibration = the indoor calibration step
    (graph replays); fields_hbm = eval_fields and its adjoint on the tiled
    street-canyon paths; diffuse = the diffuse trace, calibration step and field
    kernels on the indoor scene; city_batch = one batched trace of the 16 cities."""
    import torch

    import paper_2311_18558_gb300 as rt
    import scenegen
    dev = torch.device("cuda", torch.cuda.current_device())
    ctx = rt.Context(torch.cuda.current_device())
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    out = {"case": args.case, "steps": args.steps, "warmup": args.warmup}
    if args.case == "street_step":
        sc = scenegen.street_canyon()
        scene = rt.Scene.from_synthetic(ctx, sc)
        rx = torch.tensor(sc.rx, dtype=torch.float64, device=dev)
        eps = torch.tensor(sc.eps_r, device=dev)
        sig = torch.tensor(sc.sigma, device=dev)
        N, fc, df = args.n_sub, sc.f_center_hz, sc.delta_f_hz
        p = rt.trace_paths(ctx, scene, sc.tx, rx, sc.n_rays, sc.max_depth)
        a = rt.eval_fields(ctx, p, eps, sig, sc.freq_hz)
        T = (rt.cfr(ctx, p.rx_offsets, a, p.tau, fc, df, N).abs() ** 2).float().contiguous()
        w = torch.ones(sc.n_rx, device=dev)
        for _ in range(args.warmup + args.steps):
            flush.zero_()
            p = rt.trace_paths(ctx, scene, sc.tx, rx, sc.n_rays, sc.max_depth)
            a = rt.eval_fields(ctx, p, eps * 1.2, sig * 0.7, sc.freq_hz)
            _, ga, _ = rt.cfr_power_mse_fused(ctx, p.rx_offsets, a, p.tau, fc, df, N, T, w)
            rt.eval_fields_backward(ctx, p, eps * 1.2, sig * 0.7, sc.freq_hz, ga)
        out["n_paths"] = p.n_paths
    elif args.case == "indoor_calibration":
        args.steps = max(args.steps, 1)
        out.update(time_indoor_calibration(rt, ctx, flush, args, plain=False))
    elif args.case == "fields_hbm":
        sc = scenegen.street_canyon()
        scene = rt.Scene.from_synthetic(ctx, sc)
        out.update(time_fields_hbm(rt, ctx, scene, sc, flush, reps=max(args.steps, 1)))
    elif args.case == "diffuse":
        args.steps = max(args.steps, 1)
        out.update(time_diffuse(rt, ctx, flush, args))
    elif args.case == "diffraction":
        sc = scenegen.street_canyon()
        scene = rt.Scene.from_synthetic(ctx, sc)
        rx = torch.tensor(sc.rx, dtype=torch.float64, device=dev)
        eps = torch.tensor(sc.eps_r, device=dev)
        sig = torch.tensor(sc.sigma, device=dev)
        spec = rt.trace_paths(ctx, scene, sc.tx, rx, sc.n_rays, sc.max_depth)
        stream = torch.cuda.current_stream()
        tt = []
        for it in range(args.warmup + args.steps):
            flush.zero_()
            s0, e0 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            d = rt.trace_diffraction(ctx, scene, spec, sc.tx, rx)
            e0.record(stream)
            a = rt.eval_fields_diffraction(ctx, d, eps, sig, sc.freq_hz)
            rt.eval_fields_diffraction_backward(ctx, d, eps, sig, sc.freq_hz, torch.ones_like(a))
            e0.synchronize()
            if it >= args.warmup:
                tt.append(s0.elapsed_time(e0))
        out["n_paths"] = d.n_paths
        out["trace_ms"] = float(np.median(tt))
    elif args.case == "city_batch":
        cities = scenegen.city_batch()
        scenes = [rt.Scene.from_synthetic(ctx, c) for c in cities]
        rxs = [torch.tensor(c.rx, device=dev) for c in cities]
        for _ in range(args.warmup + args.steps):
            pb = rt.trace_batch(ctx, scenes, [c.tx for c in cities], rxs, cities[0].n_rays, cities[0].max_depth)
        out["n_paths"] = pb.n_paths
    torch.cuda.synchronize()
    out["status_word"] = ctx.status_word()
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n-sub", type=int, default=1024)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 16-city batched measurement")
    ap.add_argument("--case", choices=["street_step", "indoor_calibration", "fields_hbm", "diffuse", "diffraction",
                                       "city_batch"],
                    default=None,
                    help="run one workload alone (for profiler captures) instead of the benchmark")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.case is not None:
        run_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
