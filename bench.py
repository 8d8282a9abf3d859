#!/usr/bin/env python3
"""Benchmark: solves/s to ||r||/||f|| <= 1e-10 on the 2048^2 periodic
pressure-Poisson workload, FP32 V-cycles in FP64 defect correction (the
headline) next to the plain FP64 V-cycle on the same GPU.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one complete solve of one right-hand side from x = 0 through the
C ABI (mg_solve).  Inputs are resident in HBM when a timed step starts; L2 is
flushed (a 512 MB write) and x reset between steps, outside the timed events.
Under torchrun (N > 1) every rank solves its own right-hand sides (replicas,
weak scaling, no collective on the data path); the time is the max over ranks.
`--impl reference` times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N = 2048
LEVELS = 9
KMAX = 256
TOL = 1e-10
METRIC = "solves/s to ||r||/||f||<=1e-10, mixed vs FP64 V-cycle; serve p50/p99 ms"
WORKLOAD = ("2048^2 periodic pressure-Poisson -Lap_h p = f (5-point, h = 2pi/2048), 9 levels to 8^2, "
            "V(2,2) red-black Gauss-Seidel, full weighting, periodic cubic-spline prolongation, exact "
            "8^2 coarse solve; FP32 V-cycles (1 to 3 per outer step, adaptive) in FP64 defect correction; "
            "tol ||r||/||f|| <= 1e-10; seeded k^-5/3 turbulent source, 1 <= k <= 256")
# kernels the library's probe can time (mg_probe_kernel kinds); the library
# credits each timed launch with its algorithmic bytes
PROBE_NAMES = {1: "k_down<float,2> (finest: 2 RB-GS sweeps + residual + FW)",
               2: "k_up<float,2> (finest: cubic prolongation + correction + 2 RB-GS sweeps)",
               3: "k_outer_residual (binary64 operands, exact integer stencil sum, one rounding to float, norms)",
               4: "k_update (FP64 x += e)",
               5: "coarse levels (1024^2 down to the bottom kernel and back, one span per V-cycle)",
               6: "k_update_residual (FP64 x + e into the other iterate buffer, fused with the next outer residual)"}
# FP32 finest-level stencils (V(2,2)): the per-point algorithmic bytes of the
# unfused steps a launch performs, 4 B x (2 sweeps x 3 words + 2.25 words of
# residual + restriction, or of prolongation + correction) = 33 B, against the
# fused kernel's compulsory 13 B the library's probe credits
SURVEY_BYTES_PER_POINT = 33
SURVEY_BYTES_RATIO = {1: 33 / 13, 2: 33 / 13}
CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def max_over_ranks_of(v, dist=None, device="cpu"):
    """Max of the local value v over the process group (v itself without one)."""
    if dist is None or not dist.is_initialized():
        return v
    import torch
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(local_seconds, units_per_rank, world, dist=None, device="cpu"):
    """Whole-job throughput of replicas: the units all ranks processed over the
    slowest rank's time (every rank does the same units on its own inputs)."""
    return world * units_per_rank / max_over_ranks_of(local_seconds, dist, device)


SIDE_REPS = 20  # repetitions of the secondary measurements (probe, FP64 leg, e2e x4, batched, SR)


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_sha():
    h = hashlib.sha1()
    for name in ("mg_kernels.cu", "mg_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2403_07936_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()



def kernel_roofline(kind, n_l, ms, nbytes, peak, peak_src, sms=None, sm_mhz=None):
    """Roofline of one probed kernel kind: launches n_l, total ms, algorithmic bytes.
    Every probed kernel is bounded by memory (HBM peak): the FP32 stencils, and
    the outer residual, whose exact stencil sum runs on the integer pipe.  With
    a committed capture of the kernel's shared-memory wavefronts, the line also
    carries its shared-memory roofline: one 128-byte wavefront per cycle per
    SM at the SM clock."""
    if not n_l:
        return None
    us = ms / n_l * 1e3
    cap = read_capture(kind)
    base = {"kernel": PROBE_NAMES[kind], "avg_launch_us": us, "launches": n_l,
            "algorithmic_bytes_per_launch": nbytes / n_l,
            "traffic": cap.get("dram_bytes_per_launch") if cap else None}
    wf = cap.get("smem_wavefronts_per_launch") if cap else None
    if wf and sms and sm_mhz:
        speak = sms * sm_mhz * 1e6
        base["smem"] = {"wavefronts_per_launch": wf, "achieved_per_s": wf / (us * 1e-6), "peak_per_s": speak,
                        "frac": wf / (us * 1e-6) / speak,
                        "note": f"128-byte shared-memory wavefronts (ncu, {cap.get('profile')}) per second of the "
                                f"live launch time, against one per cycle on each of {sms} SMs at {sm_mhz:.0f} MHz"}
    if kind == 5:
        base.update({"bound": "launch/latency", "achieved": (nbytes / n_l) / (us * 1e-6) / 1e9, "unit": "GB/s",
                     "peak": None, "frac": None,
                     "note": "a span of 9 launches per V-cycle on grids of 1024^2 and less; its bytes fit L2"})
        return base
    ach_c = (nbytes / n_l) / (us * 1e-6) / 1e9
    psrc = f"{peak_src} ({'MEASURED_PEAKS.json hbm_gbs' if peak_src == 'measured' else 'recipe fallback'})"
    if kind in SURVEY_BYTES_RATIO:
        # the per-point count of the unfused steps (each sweep reads x and b and
        # writes x; prolongation + correction and residual + restriction 2.25
        # words each), over the same points as the fused kernel's compulsory count
        sb = nbytes / n_l * SURVEY_BYTES_RATIO[kind]
        ach = sb / (us * 1e-6) / 1e9
        base.update({"bound": "hbm", "algorithmic_bytes_per_launch": sb,
                     "bytes_per_point": SURVEY_BYTES_PER_POINT,
                     "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak, "peak_source": psrc,
                     "compulsory": {"bytes_per_launch": nbytes / n_l, "bytes_per_point": 13, "achieved": ach_c,
                                    "frac": ach_c / peak,
                                    "note": "the fused kernel's own minimum traffic (read x, b and 1/4 of the "
                                            "coarse grid, write x): the stricter figure"}})
        return base
    base.update({"bound": "hbm", "achieved": ach_c, "peak": peak, "unit": "GB/s", "frac": ach_c / peak,
                 "peak_source": psrc})
    return base


def read_capture(kernel_kind):
    """Per-launch counters (DRAM bytes, shared-memory wavefronts) from a committed
    ncu capture, if it was taken of this kernel source."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    ent = d.get(str(kernel_kind))
    if not ent or ent.get("source_sha1") != kernel_source_sha():
        return None
    return ent


class ClockSampler:
    """nvidia-smi clock/throttle samples every 10 ms while the timed region runs
    (the region starts once the first sample is in, so start-up latency of
    nvidia-smi does not leave the region unsampled)."""

    def __init__(self, gpu_index):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.gpu = gpu_index

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={CLOCK_QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "10"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return self
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 5.0 and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.005)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax = float(parts[2])
                except ValueError:
                    continue
                for k, name in enumerate(names):
                    if parts[5 + k].lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle legs
# ---------------------------------------------------------------------------

def oracle_cycle_sample(f, cycles):
    """Time `cycles` iterations of the FP64 oracle solve loop (V-cycle + residual)."""
    from oracle import multigrid as omg
    h = omg.grid_h(f.shape[0])
    fz = f - f.mean()
    x = np.zeros_like(fz)
    t0 = time.perf_counter()
    rels = []
    for _ in range(cycles):
        x = omg.vcycle(x, fz, h)
        rels.append(omg.relative_residual(fz, x, h))
    return time.perf_counter() - t0, rels


ORACLE_CYCLES_PER_SOLVE = 7  # FP64 V(2,2) cycles the oracle needs on this workload (tests pin it)


def oracle_accuracy(f, x):
    """|x - x_exact|_inf / |x_exact|_inf and the relative residual of a GPU result,
    by the oracle (part of the CPU-baseline leg)."""
    from oracle import multigrid as omg
    xe = omg.exact_solve_fft(f - f.mean())
    return (float(np.abs(x - xe).max() / np.abs(xe).max()),
            float(omg.relative_residual(f - f.mean(), x, omg.grid_h(f.shape[0]))))


def cpu_baseline_leg(f, cycles=3):
    dt, rels = oracle_cycle_sample(f, cycles)
    per_cycle = dt / cycles
    value = 1.0 / (per_cycle * ORACLE_CYCLES_PER_SOLVE)
    return {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": f"{cycles} FP64 oracle V(2,2) cycles + residuals on the 2048^2 source "
                      f"({dt:.1f} s, {per_cycle:.2f} s/cycle), scaled by the oracle's "
                      f"{ORACLE_CYCLES_PER_SOLVE} cycles per solve; numpy, single thread, "
                      f"host {os.uname().machine} x{os.cpu_count()}",
            "all_cores": cpu_all_cores()}


# The multi-core CPU figure: independent solves, one per core (the oracle
# itself stays single-threaded), each process timing one oracle V-cycle on its
# own 2048^2 source; the processes start the cycle together at a barrier.
_THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
_CYCLE_BARRIER = None


def _cycle_pool_init(barrier):
    global _CYCLE_BARRIER
    _CYCLE_BARRIER = barrier


def _oracle_cycle_worker(seed):
    global np
    import numpy as np
    from synthetic.sources import turbulent_source
    f = turbulent_source(N, KMAX, seed)
    _CYCLE_BARRIER.wait(timeout=120)
    dt, _ = oracle_cycle_sample(f, 1)
    return dt


def _mem_available_bytes():
    try:
        with open("/proc/meminfo") as fh:
            for line in fh:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return None


def cpu_all_cores(per_process_bytes=1 << 30):
    """Aggregate oracle solves/s with one independent solve per core (spawned
    processes: this runs after the device has been used).  Processes are
    limited to what the available memory holds at about 1 GiB each."""
    import concurrent.futures as cf
    import multiprocessing as mp
    procs = os.cpu_count() or 1
    avail = _mem_available_bytes()
    if avail is not None:
        procs = max(1, min(procs, avail // (2 * per_process_bytes)))
    saved = {k: os.environ.get(k) for k in _THREAD_VARS}
    try:
        for k in _THREAD_VARS:
            os.environ[k] = "1"
        ctx = mp.get_context("spawn")
        barrier = ctx.Barrier(procs)
        with cf.ProcessPoolExecutor(max_workers=procs, mp_context=ctx, initializer=_cycle_pool_init,
                                    initargs=(barrier,)) as ex:
            futs = [ex.submit(_oracle_cycle_worker, 1000 + i) for i in range(procs)]
            dts = [fu.result(timeout=300) for fu in futs]
    except Exception as e:  # reported, never fatal to the benchmark
        return {"value": None, "error": f"{type(e).__name__}: {e}"}
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    value = sum(1.0 / (dt * ORACLE_CYCLES_PER_SOLVE) for dt in dts)
    return {"value": value, "unit": "solves/s", "cores": procs, "kind": "oracle",
            "sample": f"{procs} processes, each one FP64 oracle V(2,2) cycle + residual on its own "
                      f"2048^2 source, started together ({min(dts):.2f}-{max(dts):.2f} s per cycle); "
                      f"sum over processes of 1 / ({ORACLE_CYCLES_PER_SOLVE} x cycle time)"}


def bench_config(world):
    """The workload both arms time (the same dict in both JSON lines)."""
    return {"workload": WORKLOAD, "grid": N, "levels": LEVELS, "rhs_per_step": 1, "prolongation": "cubic",
            "l2": "GPU arm: flushed between steps (512 MB write), x reset to 0; CPU arm: n/a",
            "initial_guess": "x = 0 (cold start); the GPU arm declares it to the library (mg_set_zero_guess), "
                             "whose mixed solves then take x = 0 in their first residual and first update "
                             "without reading x",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}


def run_reference(args, rank):
    if rank != 0:
        return
    from synthetic.sources import config_seed, turbulent_source
    f = turbulent_source(N, KMAX, config_seed(1, 0))
    for _ in range(args.warmup):
        oracle_cycle_sample(f, 1)
    times = []
    for _ in range(args.steps):
        dt, _ = oracle_cycle_sample(f, 1)
        times.append(dt)
    per_cycle = sum(times) / len(times)
    value = 1.0 / (per_cycle * ORACLE_CYCLES_PER_SOLVE)
    sample = (f"each step = 1 FP64 oracle V(2,2) cycle + residual on the 2048^2 source "
              f"({per_cycle:.2f} s); solves/s = 1 / (step time x {ORACLE_CYCLES_PER_SOLVE} cycles "
              f"per solve); numpy, single thread")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": per_cycle * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(args.gpus),
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)



# ---------------------------------------------------------------------------
# Secondary legs: batched mixed-size solves and the SR prolongation
# ---------------------------------------------------------------------------
BATCH_SIZES = [256] * 128 + [512] * 96 + [1024] * 32
SR_TENSOR_FLOP_PER_COARSE_PX = 2 * 64 * 576 * (16 + 4)  # 16 convs 64->64 and conv 64->256 (as 4 x 64)


def _levels(n, coarsest=8):
    return (n // coarsest).bit_length()  # log2(n / coarsest) + 1 for powers of two


def _events_time(stream, fn, reps):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3 / reps


def batched_leg(mg, dev, stream, flush, args, rank, prolong="cubic"):
    import torch
    from synthetic.sources import config_seed, turbulent_source
    sizes = BATCH_SIZES
    fts = [torch.tensor(turbulent_source(n, n // 8, config_seed(3, rank * 1000 + i)), device=dev)
           for i, n in enumerate(sizes)]
    blob = open(SR_WEIGHTS, "rb").read() if prolong == "sr" else None
    ctxs = []
    for n in sizes:
        c = mg.Context(_levels(n), n)
        c.set_options(stream=stream)
        if blob is not None:
            c.load_weights(blob)
        ctxs.append(c)
    xs = [torch.zeros_like(f) for f in fts]
    for _ in range(args.warmup if prolong == "cubic" else 2):
        for x in xs:
            x.zero_()
        infos = mg.solve_batched(ctxs, fts, xs, prolong=prolong)
    times = []
    for _ in range(min(args.steps, SIDE_REPS if prolong == "cubic" else 3)):
        for x in xs:
            x.zero_()
        flush.zero_()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos = mg.solve_batched(ctxs, fts, xs, prolong=prolong)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        times.append(e0.elapsed_time(e1) / 1e3)
    t = sum(times) / len(times)
    pts = sum(n * n for n in sizes)
    vc = max(i["vcycles"] for i in infos)
    outer = max(i["outer_iters"] for i in infos)
    # algorithmic bytes of one batch solve: per inner V-cycle ~35 B per finest point (fused
    # down + up passes, 13 B each, over the 4/3 hierarchy), per outer step 40 B (FP64 residual
    # 20 B + update 20 B), plus the first residual, the source sum and the projection (44 B)
    bytes_alg = pts * (vc * 13 * 2 * 4 / 3 + outer * 40 + 44)
    if prolong == "sr":
        coarse_px = sum((n // 2) ** 2 for n in sizes)
        sr_cyc = [i["sr_cycles"] for i in infos]
        return {"workload": "256 right-hand sides: 128 x 256^2, 96 x 512^2, 32 x 1024^2, independent k^-5/3 "
                            "sources, FP32 V(2,2) in FP64 defect correction (2 V-cycles per outer step), SR "
                            "prolongation at every right-hand side's finest transition on every V-cycle "
                            "(trained generator; one launch per layer and grid size for the whole batch), tol 1e-10",
                "value": len(sizes) / t, "unit": "solves/s", "ms_per_batch": t * 1e3,
                "vcycles_max": max(i["vcycles"] for i in infos), "outer_max": outer,
                "sr_vcycles_min": min(sr_cyc), "sr_vcycles_max": max(sr_cyc),
                "sr_fallbacks": sum(i["sr_fallback"] for i in infos),
                "rel_residual_max": max(i["rel_residual"] for i in infos),
                "generator_tflop_per_vcycle": SR_TENSOR_FLOP_PER_COARSE_PX * coarse_px / 1e12,
                "reps": len(times), "l2": "flushed between steps (512 MB write)"}
    return {"workload": "256 right-hand sides: 128 x 256^2, 96 x 512^2, 32 x 1024^2 (67.1 M points), "
                        "independent k^-5/3 sources, FP32 V(2,2) cubic in FP64 defect correction, tol 1e-10, "
                        "one CUDA graph per batch (one launch per grid size and direction per V-cycle)",
            "value": len(sizes) / t, "unit": "solves/s", "ms_per_batch": t * 1e3,
            "vcycles_max": vc, "outer_max": outer,
            "rel_residual_max": max(i["rel_residual"] for i in infos),
            "effective_gbs": bytes_alg / t / 1e9,
            "l2": "flushed between steps (512 MB write); working set 2.2 GB > L2"}


SR_WEIGHTS = os.path.join(ROOT, "paper_2403_07936_gb300", "weights", "sr_generator.mgsrw")


def sr_leg(mg, dev, stream, flush, f_dev, x, args):
    """SR prolongation (C3): generator throughput, and whole solves at 2048^2
    and 1024^2 with cubic, SR on every V-cycle, and SR alternated with cubic
    (N_GAN = 1), using the generator trained by train_sr.py."""
    import torch
    from paper_2403_07936_gb300 import sr
    from synthetic.sources import config_seed, turbulent_source
    from synthetic.weights import random_weights
    if os.path.exists(SR_WEIGHTS):
        blob, wdesc = open(SR_WEIGHTS, "rb").read(), "trained (weights/sr_generator.mgsrw)"
    else:
        w = random_weights(11, gain=0.5)
        w["out.w"] = w["out.w"] * 0.1
        blob, wdesc = sr.pack_weights(w), "seeded random (trained weights not found)"
    ctx = mg.Context(LEVELS, N)
    ctx.set_options(stream=stream)
    ctx.load_weights(blob)
    nc = N // 2
    ec = torch.tensor(turbulent_source(nc, nc // 8, 4242) * 1e-3, dtype=torch.float32, device=dev)
    out = torch.empty((N, N), dtype=torch.float32, device=dev)
    for _ in range(2):
        mg.op_sr_generator(ctx, ec, out)
    t_gen = _events_time(stream, lambda: mg.op_sr_generator(ctx, ec, out), SIDE_REPS)
    tflop = SR_TENSOR_FLOP_PER_COARSE_PX * nc * nc / 1e12
    peak_tf = read_bf16_peak()
    # the windowed form (Sec. 3.1, Fig. 2): 6 x 6 windows at stride 2 with
    # symmetric-log normalisation, on the same coarse field, as a mosaic of
    # 7 x 7 cells (6 x 6 values and a zero separator), 128 windows per row
    for _ in range(2):
        mg.op_sr_windowed(ctx, ec, out)
    t_win = _events_time(stream, lambda: mg.op_sr_windowed(ctx, ec, out), 5)
    mosaic_px = (nc // 2) ** 2 // 128 * 7 * 896
    windowed = {"ms_2048": t_win * 1e3, "ratio_to_whole_grid": t_win / t_gen,
                "mosaic_coarse_px": mosaic_px, "whole_grid_coarse_px": nc * nc,
                "tensor_tflops": SR_TENSOR_FLOP_PER_COARSE_PX * mosaic_px / 1e12 / t_win,
                "note": "windows of 36 values in 49-cell mosaic cells; each coarse value is in 9 windows"}
    reps = 3
    solves = {}
    for n in (N, N // 2):
        c = ctx if n == N else mg.Context(LEVELS - 1, n)
        if n != N:
            c.set_options(stream=stream)
            c.load_weights(blob)
        f = torch.tensor(turbulent_source(n, n // 8, config_seed(3, 900)), device=dev)
        xx = torch.zeros_like(f)
        res = {}
        for name, prolong, n_gan in (("cubic", "cubic", float("inf")), ("sr", "sr", float("inf")),
                                     ("alternate", "sr", 1.0)):
            c.set_prolong_policy(n_gan, 0.0)
            for _ in range(2):
                xx.zero_()
                c.solve(f, xx, prolong=prolong)
            times, info = [], None
            for _ in range(reps):
                xx.zero_()
                flush.zero_()
                torch.cuda.synchronize(dev)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                info = c.solve(f, xx, prolong=prolong)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                times.append(e0.elapsed_time(e1) / 1e3)
            t = sum(times) / len(times)
            res[name] = {"solves_per_s": 1.0 / t, "ms_per_solve": t * 1e3, "vcycles": info["vcycles"],
                         "sr_vcycles": info["sr_cycles"], "outer_iters": info["outer_iters"],
                         "rel_residual": info["rel_residual"], "sr_fallback": info["sr_fallback"]}
        c.set_prolong_policy(float("inf"), 0.0)
        solves[f"{n}^2"] = res
    return {"workload": "SR prolongation at the finest transition of the 2048^2 and 1024^2 mixed solves "
                        "(generator on the coarse error: conv 1->64, 8 residual blocks, conv 64->256 + pixel "
                        "shuffle, conv 64->1; bf16 operands, fp32 accumulate); weights: " + wdesc +
                        "; policies: cubic only, SR every V-cycle, SR alternated with cubic (N_GAN = 1)",
            "generator_ms_2048": t_gen * 1e3,
            "tensor_roofline": {"bound": "tensor", "kernel": "k_conv_tc (tcgen05 implicit GEMM)",
                                "achieved": tflop / t_gen, "peak": peak_tf[0], "unit": "TFLOP/s",
                                "frac": tflop / t_gen / peak_tf[0], "peak_source": peak_tf[1],
                                "note": "achieved counts the tensor-core FLOPs of the whole generator call "
                                        "(which also includes the CUDA-core first/last layers and s = max|e|)"},
            "windowed": windowed,
            "solves": solves}


SERVE_SIZES = (128, 256, 512, 1024, 2048)
SERVE_STREAMS = 16
SERVE_BUDGET = 160 * (1 << 30)
SERVE_CHAIN = 4


def _serve_sources(dev, rank):
    """Per stream a chain of SERVE_CHAIN sources, each a 1% perturbation of the last.

    Stream s has grid size SERVE_SIZES[s % 5]; the perturbation fields are
    drawn once per size and shared by that size's streams.  A stream's
    requests walk its chain forwards and back (0, 1, 2, 3, 2, 1, 0, 1, ...),
    so consecutive requests of a stream always differ by one 1% step.
    """
    import torch
    from synthetic.sources import config_seed, default_kmax, perturb_with, turbulent_source
    gs = {n: [turbulent_source(n, default_kmax(n), config_seed(6, rank * 100000 + 1000 * n + k))
              for k in range(SERVE_CHAIN - 1)] for n in SERVE_SIZES}
    chains, sizes = [], []
    for st in range(SERVE_STREAMS):
        n = SERVE_SIZES[st % len(SERVE_SIZES)]
        f = [turbulent_source(n, default_kmax(n), config_seed(5, rank * 100000 + st))]
        for g in gs[n]:
            f.append(perturb_with(f[-1], g))
        chains.append([torch.tensor(a, device=dev) for a in f])
        sizes.append(n)
    return chains, sizes


def _chain_index(k):
    period = 2 * (SERVE_CHAIN - 1)
    k %= period
    return k if k < SERVE_CHAIN else period - k


def serve_leg(mg, dev, stream, args, rank):
    """Poisson arrivals at each rate against the continuous-batching server.

    Each request draws N uniformly from SERVE_SIZES and one of that size's
    streams uniformly; its source is the stream's next chain entry and its
    warm start the stream's last solution (kept by the server).  Latency is
    the time from the scheduled arrival to the end of the tick that retired
    the request; requests arriving during the first `warm` seconds of a rate
    are not counted.  solves/s counts requests retired inside the window.
    """
    import torch
    chains, sizes = _serve_sources(dev, rank)
    by_size = {n: [s for s in range(SERVE_STREAMS) if sizes[s] == n] for n in SERVE_SIZES}
    outs = [torch.zeros_like(c[0]) for c in chains]
    # buffers of earlier legs are released here, not by the collector in the middle of a
    # timed arrival process (a release synchronises the device)
    gc.collect()
    torch.cuda.synchronize(dev)
    srv = mg.Server(SERVE_BUDGET, stream=stream)
    step = [0] * SERVE_STREAMS
    rng = np.random.default_rng(12345 + rank)

    def submit(st):
        f = chains[st][_chain_index(step[st])]
        step[st] += 1
        return srv.submit(f, outs[st], stream_id=st)

    # untimed warm-up: one request per stream, drained
    for st in range(SERVE_STREAMS):
        submit(st)
    while True:
        a, q, _ = srv.tick()
        srv.poll()
        if a == 0 and q == 0:
            break
    results = []
    warm = args.serve_warmup
    for lam in args.serve_rates:
        # long enough for serve_min_completions requests (p99 from >= 2000 samples)
        dur = max(args.serve_seconds, args.serve_min_completions / lam)
        t_arr = np.cumsum(rng.exponential(1.0 / lam, size=int(lam * (warm + dur) * 1.5) + 16))
        t_arr = t_arr[t_arr < warm + dur]
        req_n = rng.integers(0, len(SERVE_SIZES), size=t_arr.size)
        req_s = [by_size[SERVE_SIZES[k]][rng.integers(0, len(by_size[SERVE_SIZES[k]]))] for k in req_n]
        pending = {}
        lat, lat_n, cyc, bad, done_in_window = [], {n: [] for n in SERVE_SIZES}, [], 0, 0
        gc.collect()
        gc.disable()  # no collector pauses inside the arrival process (re-enabled after it)
        ticks, max_inflight = 0, 0
        i = 0
        t0 = time.perf_counter()
        deadline = warm + dur + 10.0
        while True:
            now = time.perf_counter() - t0
            while i < t_arr.size and t_arr[i] <= now:
                rid = submit(req_s[i])
                pending[rid] = (t_arr[i], sizes[req_s[i]])
                i += 1
            if not pending:
                if i == t_arr.size:
                    break
                time.sleep(max(0.0, min(t_arr[i] - now, 0.002)))
                continue
            a, q, _ = srv.tick()
            ticks += 1
            max_inflight = max(max_inflight, a + q)
            t_done = time.perf_counter() - t0
            for r in srv.poll():
                t_a, n = pending.pop(r["request_id"])
                if r["status"] != 0:
                    bad += 1
                if warm <= t_done < warm + dur:
                    done_in_window += 1
                if t_a >= warm:
                    lat.append(t_done - t_a)
                    lat_n[n].append(t_done - t_a)
                    cyc.append(r["vcycles"])
            if t_done > deadline:
                break
        gc.enable()
        unfinished = len(pending) + (t_arr.size - i)
        while pending:  # drain what is left before the next rate
            srv.tick()
            for r in srv.poll():
                pending.pop(r["request_id"], None)
        lat_ms = np.array(lat) * 1e3
        results.append({
            "lambda_req_s": lam, "window_s": dur, "offered": int(np.sum((t_arr >= warm))), "completed": len(lat),
            "p99_samples": len(lat),
            "solves_per_s": done_in_window / dur,
            "p50_ms": float(np.percentile(lat_ms, 50)) if lat else None,
            "p99_ms": float(np.percentile(lat_ms, 99)) if lat else None,
            "p50_ms_by_N": {str(n): float(np.percentile(v, 50) * 1e3) for n, v in lat_n.items() if v},
            "mean_vcycles": float(np.mean(cyc)) if cyc else None,
            "ticks": ticks, "max_in_flight": max_inflight, "failed": bad,
            "saturated": unfinished > 0})
    srv.close()
    return {"workload": f"Poisson arrivals; N uniform in {list(SERVE_SIZES)}; {SERVE_STREAMS} streams "
                        f"(stream s has N = sizes[s mod 5]); each request a 1% perturbation of its stream's "
                        f"previous source, warm-started from the stream's previous solution; memory budget "
                        f"160 GiB; tol 1e-10; per rate max({args.serve_seconds:g} s, "
                        f"{args.serve_min_completions} / rate) measured after {warm:g} s warm-up",
            "rates": results}


def read_bf16_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["bf16_tflops"]), "measured (MEASURED_PEAKS.json bf16_tflops, burst)"
    return 1900.0, "fallback"

# ---------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skip-batched", action="store_true")
    ap.add_argument("--skip-sr", action="store_true")
    ap.add_argument("--skip-serve", action="store_true")
    ap.add_argument("--skip-smoothing", action="store_true")
    ap.add_argument("--skip-two-level", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    ap.add_argument("--serve-min-completions", type=int, default=2000)
    ap.add_argument("--serve-warmup", type=float, default=0.5)
    ap.add_argument("--serve-rates", type=lambda v: [float(t) for t in v.split(",")],
                    default=[50.0, 100.0, 200.0, 500.0, 1000.0, 2000.0])
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local_rank = _env_int("LOCAL_RANK", 0)

    global np
    import numpy as np

    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)

    import __graft_entry__
    __graft_entry__.build()
    from paper_2403_07936_gb300 import mg
    from synthetic.sources import config_seed, turbulent_source

    stream = torch.cuda.current_stream(dev)
    srcs = [turbulent_source(N, KMAX, config_seed(1, rank * 100 + i)) for i in range(2)]
    f_dev = [torch.tensor(s, device=dev) for s in srcs]
    x = torch.zeros_like(f_dev[0])
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def make_ctx(precision):
        c = mg.Context(LEVELS, N)
        c.set_options(precision=precision, stream=stream)
        return c

    def timed_solves(ctx, k_steps, f_list, xbuf, host=False):
        times, infos = [], []
        for k in range(k_steps):
            f = f_list[k % len(f_list)]
            xbuf.zero_()
            flush.zero_()
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            infos.append(ctx.solve(f, xbuf, tol=TOL))
            e1.record(stream)
            torch.cuda.synchronize(dev)
            times.append(e0.elapsed_time(e1) / 1e3)
        return times, infos

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    # ---- mixed precision (headline): each solve is one CUDA graph launch -----
    # (every solve starts from x = 0, and the context is told so)
    ctx = make_ctx("mixed")
    ctx.set_zero_guess(True)
    timed_solves(ctx, args.warmup, f_dev, x)
    barrier()
    l0 = mg.kernel_launches()
    with ClockSampler(local_rank) as clk:
        t_wall0 = time.perf_counter()
        times, infos = timed_solves(ctx, args.steps, f_dev, x)
        t_wall = time.perf_counter() - t_wall0
    launches = mg.kernel_launches() - l0
    barrier()
    value = weak_scaling_value(sum(times), args.steps, world, dist, dev)
    clocks = clk.summary()
    x_keep = x.clone()

    # ---- roofline probe: the same solves with CUDA events around one kernel
    # kind (the probe runs the host-loop execution mode, whose kernels are the
    # graph's).  First pick the kernel kind with the largest time per solve.
    kernel_ms = {}
    for kind in (1, 2, 3, 4, 5, 6):
        ctx.probe(kind, 256)
        timed_solves(ctx, 1, f_dev, x)
        n_l, ms, by = ctx.probe_read()
        kernel_ms[kind] = (n_l, ms, by)
    dom = max((k for k in kernel_ms if k != 5), key=lambda k: kernel_ms[k][1])  # 5 is a span of kernels
    n_probe = min(args.steps, SIDE_REPS)
    ctx.probe(dom, 64 * n_probe)
    tprobe, _ = timed_solves(ctx, n_probe, f_dev, x)
    n_l, probe_ms, probe_bytes = ctx.probe_read()
    ctx.probe(0, 0)
    x.copy_(x_keep)

    # the last solve's result, checked by the oracle in the CPU-baseline leg
    f_last = srcs[(args.steps - 1) % len(srcs)]
    x_last = x.cpu().numpy()

    # ---- plain FP64 V-cycle on the same GPU ------------------------------
    ctx64 = make_ctx("fp64")
    timed_solves(ctx64, args.warmup, f_dev, x)
    k64 = min(max(3, args.steps // 2), SIDE_REPS)
    t64, info64 = timed_solves(ctx64, k64, f_dev, x)
    value64 = weak_scaling_value(sum(t64), k64, world, dist, dev)
    f64_last, x64_last = srcs[(k64 - 1) % 2], x.cpu().numpy()

    # ---- end to end through host (pinned) buffers --------------------------
    # (the workload starts from x = 0: the context is told so, and x is then
    # output only, so a solve copies f in and x out)
    f_host = [torch.tensor(s).pin_memory() for s in srcs]
    x_host = torch.zeros_like(f_host[0]).pin_memory()
    timed_solves(ctx, 2, f_host, x_host)
    n_e2e = min(args.steps, 4 * SIDE_REPS)
    te2e, _ = timed_solves(ctx, n_e2e, f_host, x_host)
    value_e2e = weak_scaling_value(sum(te2e), n_e2e, world, dist, dev)
    bytes_grid = N * N * 8

    # the host link's copy bandwidth, for the end-to-end bound: a cold-start
    # solve from host buffers copies f in and x out around the device solve
    # (the rate of the host-to-device copies is measured on f and x together)
    def link_ms(fn, reps=10):
        with torch.cuda.stream(stream):
            fn()
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / reps

    def h2d():
        f_dev[0].copy_(f_host[0], non_blocking=True)
        x.copy_(x_host, non_blocking=True)

    def d2h():
        x_host.copy_(x, non_blocking=True)

    h2d_gbs = 2 * bytes_grid / (link_ms(h2d) * 1e-3) / 1e9
    d2h_gbs = bytes_grid / (link_ms(d2h) * 1e-3) / 1e9  # (f_host[0] holds f_dev[0]'s source)

    # ---- roofline of the dominant kernel -----------------------------------
    peak, peak_src = read_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = (clocks or {}).get("sm_max_mhz")
    roofline = kernel_roofline(dom, n_l, probe_ms, probe_bytes, peak, peak_src, sms, sm_mhz)
    mean_step = sum(times) / len(times)
    mean_probe_step = sum(tprobe) / len(tprobe)
    roofline["share_of_solve"] = (probe_ms / n_probe / 1e3) / mean_probe_step
    roofline["measured_over"] = (f"{n_probe} solves of the same workload with CUDA events on the "
                                 f"launching stream around each launch of this kernel (host-loop "
                                 f"execution, {mean_probe_step * 1e3:.3f} ms per solve)")
    kernels = {PROBE_NAMES[k]: {"launches_per_solve": v[0], "ms_per_solve": v[1],
                                "gbs": (v[2] / (v[1] / 1e3) / 1e9) if v[1] else None,
                                "roofline": kernel_roofline(k, v[0], v[1], v[2], peak, peak_src, sms, sm_mhz)}
               for k, v in kernel_ms.items()}

    # ---- batched: 256 right-hand sides of mixed sizes in one graph ----------
    batched = batched_leg(mg, dev, stream, flush, args, rank) if not args.skip_batched else None
    batched_sr = (batched_leg(mg, dev, stream, flush, args, rank, prolong="sr")
                  if not args.skip_batched and os.path.exists(SR_WEIGHTS) else None)

    # ---- SR prolongation at 2048^2 (tensor-core generator) ------------------
    sr_info = sr_leg(mg, dev, stream, flush, f_dev, x, args) if not args.skip_sr else None

    # ---- serving: Poisson arrivals into the continuous-batching server -----
    serving = serve_leg(mg, dev, stream, args, rank) if not args.skip_serve else None

    # ---- smoothing-count sweep: V(nu, nu) for nu = 1..4 on the same workload --
    smoothing = None
    if not args.skip_smoothing:
        smoothing = {"workload": "the 2048^2 headline solve with V(nu, nu), nu = 1..4 (cubic, mixed, adaptive "
                                 "V-cycles per outer step with the contraction estimate 0.06 of V(2,2))",
                     "runs": []}
        for nu in (1, 2, 3, 4):
            cs = make_ctx("mixed")
            cs.set_options(nu_pre=nu, nu_post=nu)
            timed_solves(cs, 3, f_dev, x)  # warm-up (records the graph)
            ts, inf = timed_solves(cs, SIDE_REPS, f_dev, x)
            ms = sum(ts) / len(ts) * 1e3
            vc = inf[-1]["vcycles"]
            smoothing["runs"].append({
                "nu": nu, "vcycles": vc, "outer_iters": inf[-1]["outer_iters"], "ms_per_solve": ms,
                "solves_per_s": 1e3 / ms, "rel_residual": inf[-1]["rel_residual"],
                # smoothing sweeps per V-cycle on the finest level, times V-cycles: the paper's
                # iteration count weighted by the smoothing work it carries
                "finest_sweeps_per_solve": 2 * nu * vc})
            cs.close()

    cpu, err, rel, err64 = None, None, None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_leg(srcs[0])
        err, rel = oracle_accuracy(f_last, x_last)
        err64, _ = oracle_accuracy(f64_last, x64_last)

    # ---- the paper's two-level x16 configuration (cubic spline prolongation) --
    two_level = None
    if not args.skip_two_level:
        two_level = {"workload": "two-level cycles (Sec. 4.1): one coarse level 16x coarser, N_smooth red-black "
                                 "sweeps on the finest grid, 10 coarse sweeps, cubic spline prolongation by 16 in "
                                 "one step (runs with 'prolong': SR by 16 as four stages of the cubic spline by 2 "
                                 "plus the trained generator's correction, every cycle or alternated with cubic), "
                                 "FP32 cycles in FP64 defect correction, tol 1e-10, x from 0",
                     "runs": []}
        for n2, lev2 in ((1024, 8), (2048, 9)):
            f2 = torch.tensor(turbulent_source(n2, n2 // 8, config_seed(1, rank * 100 + 50)), device=dev)
            x2 = torch.zeros_like(f2)
            c2 = mg.Context(lev2, n2)
            c2.set_options(stream=stream)
            for nus in (15, 20):
                c2.two_level_solve(f2, x2, max_cycles=400, nu_smooth=nus, check=False)  # warm-up
                ts2, inf2 = [], None
                for _ in range(3):
                    x2.zero_()
                    torch.cuda.synchronize(dev)
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    inf2 = c2.two_level_solve(f2, x2, max_cycles=400, nu_smooth=nus, check=False)
                    e1.record(stream)
                    torch.cuda.synchronize(dev)
                    ts2.append(e0.elapsed_time(e1))
                xm = torch.zeros_like(f2)
                vm = c2.solve(f2, xm)["vcycles"]
                two_level["runs"].append({"n": n2, "nu_smooth": nus, "coarse_sweeps": 10, "status": inf2["status"],
                                          "cycles": inf2["vcycles"], "rel_residual": inf2["rel_residual"],
                                          "ms_per_solve": sum(ts2) / len(ts2),
                                          "multilevel_vcycles_same_source": vm})
            if n2 == 2048 and os.path.exists(SR_WEIGHTS):
                # SR x16: four stages of (cubic by 2 + the trained generator's correction)
                with open(SR_WEIGHTS, "rb") as fh:
                    c2.load_weights(fh.read())
                for label, n_gan in (("sr", float("inf")), ("alternate", 1.0)):
                    c2.set_prolong_policy(n_gan, 0.0)
                    c2.two_level_solve(f2, x2, max_cycles=2, nu_smooth=20, prolong="sr", check=False)  # buffers
                    x2.zero_()
                    torch.cuda.synchronize(dev)
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    inf2 = c2.two_level_solve(f2, x2, max_cycles=400, nu_smooth=20, prolong="sr", check=False)
                    e1.record(stream)
                    torch.cuda.synchronize(dev)
                    two_level["runs"].append({"n": n2, "nu_smooth": 20, "coarse_sweeps": 10, "prolong": label,
                                              "status": inf2["status"], "cycles": inf2["vcycles"],
                                              "sr_cycles": inf2["sr_cycles"], "sr_fallback": inf2["sr_fallback"],
                                              "rel_residual": inf2["rel_residual"],
                                              "ms_per_solve": e0.elapsed_time(e1)})
                c2.set_prolong_policy(float("inf"), 0.0)
            c2.close()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean_step * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (V-cycles) + f64 (outer residual, update, norms)", "data": "synthetic",
            "config": bench_config(world),
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": value_e2e, "unit": "solves/s", "h2d_bytes_per_step": bytes_grid,
                    "d2h_bytes_per_step": bytes_grid,
                    "path": "mg_solve with pinned host f and x (copies inside the call); the context is set "
                            "to a zero initial guess (mg_set_zero_guess), the workload's cold start, so x "
                            "is output only: f is copied in, x out",
                    "link_gbs": {"h2d": h2d_gbs, "d2h": d2h_gbs},
                    "bound": 1.0 / (mean_step + bytes_grid / (h2d_gbs * 1e9) + bytes_grid / (d2h_gbs * 1e9)),
                    "bound_note": "1 / (device solve time + copies at the measured host-link bandwidths): "
                                  "the copies cannot overlap the solve, which needs all of f first"},
            "gpu_launches": launches,
            "clocks": clocks,
            "wall_s_timed_region": t_wall,
            "solve": {"vcycles": infos[-1]["vcycles"], "outer_iters": infos[-1]["outer_iters"],
                      "rel_residual": infos[-1]["rel_residual"], "rel_residual_by_oracle": rel,
                      "err_inf_vs_exact_fft": err,
                      "accuracy_check": "by the oracle in the CPU-baseline leg (null when that leg is skipped)"},
            "fp64_vcycle": {"value": value64, "unit": "solves/s", "steps": k64,
                            "ms_per_step": sum(t64) / k64 * 1e3,
                            "roofline": {"bound": "fp64 pipe",
                                         "kernel": "k_up<double> (53 % of an FP64 solve) after k_refine_rows "
                                                   "(10 %), the prolongation's pass along x once per level",
                                         "fp64_pipe_active_pct": {"k_up<double>": 66.5, "k_refine_rows": 83.3},
                                         "dram_throughput_pct": {"k_up<double>": 2.1, "k_refine_rows": 0.9},
                                         "source": "ncu captures of the 2048^2 launches, "
                                                   "profiles/k_up_k_down_fp64_2048.md (k_up<double> taken at one "
                                                   "block per SM, before its tile dropped the unused coarse-tile "
                                                   "space for two)",
                                         "note": "the FP64 V-cycle's stencils are bound by the FP64 pipe (1/64 of "
                                                 "the FP32 rate on GB300), not by HBM"},
                            "vcycles": info64[-1]["vcycles"], "err_inf_vs_exact_fft": err64},
            "mixed_over_fp64": value / value64,
            "kernels_per_solve": kernels,
            "batched": batched,
            "batched_sr": batched_sr,
            "sr": sr_info,
            "serving": serving,
            "smoothing_sweep": smoothing,
            "two_level_x16": two_level,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
