#!/usr/bin/env python
"""Throughput of the FP64 Taylor-Couette step on GB300: grid-point-steps/s.

Workload: the 64 x 128 x 128 run with Boussinesq temperature and the dynamic
CFL step (eta = 0.71, Re_i = 3000, Re_o = -1000, Ra = 1e4, Pr = 0.7), seeded
divergence-free perturbation.  One step = one predictor-corrector step (two
nonlinear evaluations, two radial stages, the dt policy and any refactoring).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

N > 1 runs N independent replicas (the path has no exchange step), one rank
per GPU under torchrun; value = all ranks' grid-point-steps / max rank time.
Prints one JSON line on rank 0.
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
sys.path.insert(0, ROOT)

from inputs import WORKLOADS, psi_coefficients, temperature_coefficients  # noqa: E402

WORKLOAD = "tc_fp64T_nr64_n128"
METRIC = "grid-point-steps/s"
# FP64 peak of the ALU roofline: 152 SMs x 2.07 GHz x 4 FP64 flop/clk/SM
# (2 DFMA/clk/SM); tc_measure_fp64_rate measures 1.257 TFLOP/s sustained at 2070 MHz.
FP64_PEAK_TFLOPS = 152 * 2.07e9 * 4 / 1e12
# FP32 peak for the mixed form's transform kernels: 128 FP32 FMA/clk/SM
FP32_PEAK_TFLOPS = 152 * 2.07e9 * 256 / 1e12
L2_FLUSH_BYTES = 512 << 20
KERNEL_TIMING_STEPS = 50      # steps of the per-kernel timing pass


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--precision", type=int, default=None, choices=[0, 1],
                    help="override the workload's precision (0 FP64, 1 mixed)")
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true",
                    help="skip the differentiation-form measurement")
    ap.add_argument("--ensemble", type=int, default=0,
                    help="benchmark the batched form: N uneven runs replayed as one graph")
    ap.add_argument("--config", default=None,
                    help="MB,LB,MBF,TT,TZ: fixed nonlinear-stage tiles and tensor-core paths "
                         "(tensor_theta, tensor_z) instead of the autotuner's choice, so that "
                         "a profiler run launches the same kernels as the timed one")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the mixed-precision and ensemble forms (N = 1 only)")
    return ap.parse_args()


def max_over_ranks(dist, value, device):
    """The largest of each rank's value (all ranks get it); value itself alone."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(points, steps, world, slowest_ms):
    """Whole-job grid-point-steps/s: every rank's points and steps over the
    slowest rank's time (replicas run the same workload)."""
    return points * steps * world / (slowest_ms * 1e-3)


def measured_bf16_peak():
    """Dense BF16 tensor rate measured on the GB300s (TFLOP/s, burst)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        return 1900.0


def measured_hbm_peak():
    """Copy bandwidth measured on the GB300s (GB/s), else the fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


def config_of(wl, extra=None):
    cfg = {"workload": f"{wl.name}: Nr={wl.Nr} Ntheta={wl.Ntheta} Nz={wl.Nz} eta={wl.eta} "
                       f"Re_i={wl.Re_i} Re_o={wl.Re_o} Ra={wl.Ra} Pr={wl.Pr} "
                       f"dt={'CFL dynamic' if wl.dt <= 0 else wl.dt}",
           "grid_points": wl.points, "fields": 4 if wl.Ra else 3,
           "precision": "mixed: FP32 transforms of u', FP64 mean-flow products and solves"
           if getattr(wl, "precision", 0) else "fp64"}
    if extra:
        cfg.update(extra)
    return cfg


# ----------------------------------------------------------------- clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------ oracle timing
def oracle_throughput(wl, budget_s=20.0, max_steps=None, warmup=0):
    """Time the FP64 oracle (scipy.fft transform mode) on this host's cores,
    after `warmup` untimed steps (the timed steps continue from them).

    Returns (pt-steps/s, steps timed, seconds, cores, sample description).
    """
    from oracle import Model
    t0 = time.perf_counter()
    mdl = Model(wl, "fft")
    X = mdl.initial_state(psi_coefficients(wl.seed, wl.mp, wl.kp),
                          temperature_coefficients(wl.seed, wl.mp, wl.kp) if wl.Ra else None)
    setup = time.perf_counter() - t0
    dt_prev = 0.0
    for _ in range(warmup):
        X, _, dt_prev, _ = mdl.step(X, wl.dt, dt_prev)
    n = 0
    t0 = time.perf_counter()
    while True:
        X, _, dt_prev, _ = mdl.step(X, wl.dt, dt_prev)
        n += 1
        el = time.perf_counter() - t0
        if el >= budget_s or (max_steps and n >= max_steps):
            break
    cores = os.cpu_count()
    start = (f"after {warmup} untimed steps from its seeded initial state" if warmup
             else "from its seeded initial state")
    sample = (f"{n} full steps of {wl.name} {start} "
              f"(oracle, scipy.fft transforms, LAPACK radial solves; set-up {setup:.1f} s excluded)")
    return wl.points * n / el, n, el, cores, sample


# ------------------------------------------------------- algorithmic flops
def fft_flops(n):
    """Nominal flops of a complex FFT of length n (5 n log2 n)."""
    return 5.0 * n * math.log2(n)


def kernel_flops(name, wl):
    """Algorithmic FP64 flops of one launch of a hot kernel (None if not modelled)."""
    nf = 4 if wl.Ra else 3
    M, K = (wl.Ntheta - 1) // 3, (wl.Nz - 1) // 3
    NM, NK = M + 1, 2 * K + 1
    if name == "k_theta":
        # per z-row: 2 nf inverse + 2 forward complex FFTs along theta (two real
        # fields each), ~30 flops of products and curvature terms per point
        return wl.Nr * wl.Nz * ((2 * nf + 2) * fft_flops(wl.Ntheta) + 30 * wl.Ntheta)
    if name == "k_theta_tc":
        # the part of the same stage that runs on the FP64 pipe: the 2 forward
        # complex FFTs and the products per z-row (the inverse transforms run
        # as BF16 slice products on the tensor cores: tensor_flops)
        return wl.Nr * wl.Nz * (2 * fft_flops(wl.Ntheta) + 30 * wl.Ntheta)
    if name == "k_zinv":
        # 3 fields per component and m column, plus the 9-point d/dr (72 flops/coeff)
        return wl.Nr * nf * NM * (3 * fft_flops(wl.Nz) + 72 * NK)
    if name == "k_zinv_tc":
        # the part of the same stage that runs on the FP64 pipe: the 9-point
        # d/dr (the transforms run as BF16 slice products: tensor_flops)
        return wl.Nr * nf * NM * 72 * NK
    if name == "k_zfwd":
        return wl.Nr * nf * NM * fft_flops(wl.Nz)
    return None


def tensor_flops(name, wl):
    """BF16 tensor flops one launch of a tensor-core transform kernel issues:
    per CTA (32 data columns, 128 rows of the DFT matrix, 96 coefficients)
    the products of matrix slice i with data slices 0..6-i, 28 slice pairs of
    128 x 32 x 96.  k_theta_tc: a CTA per 2 z rows of a radius; k_zinv_tc: a
    CTA per 5 m columns of a radius and field."""
    if name == "k_theta_tc":
        ctas = wl.Nr * ((wl.Nz + 1) // 2)
    else:
        nf = 4 if wl.Ra else 3
        NM = (wl.Ntheta - 1) // 3 + 1
        ctas = wl.Nr * nf * ((NM + 4) // 5)
    return ctas * 28 * 2.0 * 128 * 32 * 96


# tensor-core kernel -> the FFT kernel of the same stage (same algorithmic count)
TENSOR_STAGE = {"k_theta_tc": "k_theta", "k_zinv_tc": "k_zinv"}


def step_flops(wl):
    """Algorithmic FP64 flops of one predictor-corrector step (two stages).

    Nonlinear stage: the three transform kernels' counts above.  Linear
    stage per stage, per stored coefficient S: the explicit part's
    Laplacian stencils (nf fields x 9 taps x 4 flops, once per step), the
    divergence and gradient stencils (2 x 9 x 4), the banded sweeps (2 nf + 2
    real systems, forward and backward, 4 off-diagonal FMAs per row) and the
    influence correction (about 50).  A count of the method's arithmetic, not
    of this implementation's instructions."""
    nf = 4 if wl.Ra else 3
    M, K = (wl.Ntheta - 1) // 3, (wl.Nz - 1) // 3
    S = wl.Nr * (M + 1) * (2 * K + 1)
    nonlinear, linear = stage_flops(wl)
    return 2 * (nonlinear + linear)


def stage_flops(wl):
    """(nonlinear, linear) algorithmic flops of one stage (see step_flops)."""
    nf = 4 if wl.Ra else 3
    M, K = (wl.Ntheta - 1) // 3, (wl.Nz - 1) // 3
    S = wl.Nr * (M + 1) * (2 * K + 1)
    nonlinear = sum(kernel_flops(k, wl) for k in ("k_theta", "k_zinv", "k_zfwd"))
    linear = nf * 9 * 4 * S / 2 + (2 * 9 * 4 + (2 * nf + 2) * 2 * 10 + 50) * S
    return nonlinear, linear


def source_hash(names):
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_1908_00587_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_for(kernel, workload, precision):
    """Per-launch DRAM bytes from the committed ncu summary, if it was taken on
    this workload and precision and the kernel's sources have not changed."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f)
    ent = rec.get(kernel)
    if not ent or ent.get("workload") != workload or ent.get("precision") != precision:
        return None
    if ent.get("source_hash") != source_hash(ent.get("sources", [])):
        return None
    return ent.get("dram_bytes_per_launch")


# ------------------------------------------------------------------ arms
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    wl = WORKLOADS[args.workload]
    # bounded sample: about a minute of oracle steps whatever K is
    value, n, el, cores, sample = oracle_throughput(wl, budget_s=60.0, max_steps=args.steps,
                                                    warmup=args.warmup)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC,
            "n_gpus": args.gpus, "steps": n, "warmup": args.warmup, "ms_per_step": 1e3 * el / n,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(wl, {"sample_of_requested_steps": args.steps}),
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_gb300(args):
    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__ as g
    if rank == 0:
        g.build()
    if dist:
        dist.barrier()
    from paper_1908_00587_gb300 import tc

    wl = WORKLOADS[args.workload]
    if args.precision is not None:
        wl = wl.scaled(precision=args.precision)
    run = tc.Run.from_workload(wl)
    stream = torch.cuda.current_stream()
    run.set_stream(stream.cuda_stream)
    psi = psi_coefficients(wl.seed, wl.mp, wl.kp)
    tco = temperature_coefficients(wl.seed, wl.mp, wl.kp) if wl.Ra else None
    run.init_perturbation(psi, wl.amp, tco, wl.amp_T)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    if args.config:                         # a fixed configuration (profiler runs)
        mb, lb, mbf, tt, tz = (int(v) for v in args.config.split(","))
        for key, val in (("tile_mb", mb), ("tile_lb", lb), ("tile_mbf", mbf),
                         ("tensor_theta", tt), ("tensor_z", tz)):
            tc.tc_set_option(run.ctx, key, val)
    else:
        tc.tc_autotune(run.ctx)             # tile shapes of the nonlinear stage
    info = tc.tc_get_info(run.ctx)
    tiles = (info.tile_mb, info.tile_lb, info.tile_mbf)
    azimuthal = ("tensor cores: DFT-matrix products of 7 BF16 slices (k_theta_tc)"
                 if info.tensor_theta else "FP64 FFT (k_theta)")
    axial = ("tensor cores: folded DFT-matrix products of 7 BF16 slices (k_zinv_tc)"
             if info.tensor_z else "FP64 FFT (k_zinv)")

    for _ in range(args.warmup):
        run.step(1, wl.dt)                  # the first one also captures the step graph
    torch.cuda.synchronize()

    launches0 = tc.tc_get_info(run.ctx).launches
    clocks = Clocks(local)
    clocks.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.fill_(i & 0xFF)               # evict L2 between timed steps
        starts[i].record(stream)
        run.step(1, wl.dt)
        ends[i].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    clk = clocks.stop()
    launches = tc.tc_get_info(run.ctx).launches - launches0
    total_ms = sum(step_ms)

    # kernel durations: a second timed pass of the same steps (L2 flushed the
    # same way) with CUDA events around every launch on the context's stream.
    # Events between kernels cost time, so this pass is not the one `value`
    # comes from; the kernels themselves run the same.
    kt_steps = min(args.steps, KERNEL_TIMING_STEPS)
    tc.tc_set_option(run.ctx, "timing", 1)
    tc.tc_reset_timing(run.ctx)
    ks = [torch.cuda.Event(enable_timing=True) for _ in range(kt_steps)]
    ke = [torch.cuda.Event(enable_timing=True) for _ in range(kt_steps)]
    torch.cuda.synchronize()
    for i in range(kt_steps):
        flush.fill_(i & 0xFF)
        ks[i].record(stream)
        run.step(1, wl.dt)
        ke[i].record(stream)
    torch.cuda.synchronize()
    kt_total_ms = sum(a.elapsed_time(b) for a, b in zip(ks, ke))
    timing = tc.tc_get_timing(run.ctx)
    tc.tc_set_option(run.ctx, "timing", 0)
    # production form of the same steps: one tc_step call of K steps (the
    # graph replayed back to back, one host round trip per call; no L2 flush
    # can sit between the steps of one call, and the 15 MB state fits in L2)
    ms_a = torch.cuda.Event(enable_timing=True)
    ms_b = torch.cuda.Event(enable_timing=True)
    flush.fill_(7)
    torch.cuda.synchronize()
    ms_a.record(stream)
    run.step(args.steps, wl.dt)
    ms_b.record(stream)
    torch.cuda.synchronize()
    multi_ms = ms_a.elapsed_time(ms_b) / args.steps
    total_ms = max_over_ranks(dist, total_ms, "cuda")
    value = replica_throughput(wl.points, args.steps, world, total_ms)

    # end to end through the public API with host buffers: state in from pinned
    # host memory, one step, state out to pinned host memory (--e2e-steps 0
    # skips it, for states too large to pin on the host).  Each step is a
    # restart from host memory: the state and its clock go back in, so the
    # dynamic step continues the run as it would on the device
    e2e = None
    ne = min(args.e2e_steps, args.steps)
    if ne > 0:
        host = torch.empty(run.shape, dtype=torch.complex128, pin_memory=True).numpy()
        run.get_state(host)
        t_sim, dt_prev = run.get_clock()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(ne):
            run.set_state(host)
            run.set_clock(t_sim, dt_prev)
            dt_prev = float(run.step(1, wl.dt)[-1])
            t_sim += dt_prev
            run.get_state(host)
        torch.cuda.synchronize()
        e2e_s = max_over_ranks(dist, time.perf_counter() - t0, "cuda")
        state_bytes = int(np.prod(run.shape)) * 16
        e2e = {"value": replica_throughput(wl.points, ne, world, e2e_s * 1e3), "unit": METRIC,
               "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": state_bytes,
               "steps": ne}

    # roofline of the dominant kernel: the FP64 step is bound by the FP64 pipe
    # (about 1.7e3 flop against 157 algorithmic bytes per grid-point-step)
    # (the mixed form's transform kernels compute in FP32: FP32 peak)
    mixed = int(getattr(wl, "precision", 0))
    dom = max(timing, key=lambda k: timing[k][1])
    nl, ms = timing[dom]
    tensor_dom = dom in TENSOR_STAGE
    # algorithmic flops of the dominant kernel's stage (nominal count: the
    # transforms as 5 n log2 n FFTs plus the products); for the tensor-core
    # transform kernels that is the same count as for their FFT kernels
    fl = kernel_flops(TENSOR_STAGE.get(dom, dom), wl)
    fp32_dom = mixed and dom in ("k_theta", "k_zinv", "k_zfwd")
    peak = FP32_PEAK_TFLOPS if fp32_dom else FP64_PEAK_TFLOPS
    roof = {"kernel": dom, "bound": "alu", "unit": "TFLOP/s", "peak": peak,
            "peak_source": ("derived: 152 SMs x 2.07 GHz x 256 FP32 flop/clk/SM" if fp32_dom
                            else "derived: 152 SMs x 2.07 GHz x 4 FP64 flop/clk/SM"),
            "share_of_step": ms / kt_total_ms,
            "ms_per_launch": ms / nl,
            "timed": f"{kt_steps} steps with per-launch CUDA events after the main timed region"}
    if fl is not None:
        ach = fl / (ms / nl * 1e-3) / 1e12
        roof.update({"achieved": ach, "frac": ach / peak,
                     "flops_per_launch": fl})
    else:
        roof.update({"achieved": None, "frac": None})
    if tensor_dom:
        # a stage with its inverse transforms on the tensor cores: achieved is
        # the stage's algorithmic count over the kernel's time, so frac may
        # exceed 1 (the FP64 FFT kernels cannot): the FP64 pipe runs only the
        # rest of the stage (fp64_pipe: forward FFTs and products, or the
        # d/dr stencil), the inverse transforms run as BF16 slice products
        # (tensor)
        tf = tensor_flops(dom, wl)
        bf16 = measured_bf16_peak()
        f64 = kernel_flops(dom, wl)
        roof["how"] = (f"algorithmic flops of the stage (FFT count, as for {TENSOR_STAGE[dom]}) "
                       "over the tensor-core kernel's time; its inverse transforms run on the "
                       "tensor cores, so the FP64 peak does not cap it")
        roof["fp64_pipe"] = {
            "flops_per_launch": f64, "achieved_tflops": f64 / (ms / nl * 1e-3) / 1e12,
            "frac": f64 / (ms / nl * 1e-3) / 1e12 / peak,
            "how": ("the flops run on the FP64 pipe (forward FFTs and products, or the "
                    "d/dr stencil) over the kernel's time")}
        roof["tensor"] = {"bf16_flops_per_launch": tf,
                          "achieved_tflops": tf / (ms / nl * 1e-3) / 1e12,
                          "peak_tflops": bf16,
                          "frac": (tf / (ms / nl * 1e-3) / 1e12 / bf16) if bf16 else None,
                          "peak_source": "MEASURED_PEAKS.json bf16_tflops (cuBLAS bf16, burst)"}
    # the FP64 FMA rate this GPU sustains, measured after the timed regions
    # (the derived peak above counts 4 flop/clk/SM; the FP64 units deliver less)
    fp64_meas = None
    try:
        fp64_meas = tc.tc_measure_fp64_rate(250.0, torch.cuda.current_stream().cuda_stream)
    except Exception:   # a measurement aid: its absence only drops the extra fields
        fp64_meas = None
    if fp64_meas and not fp32_dom:
        roof["measured_peak"] = fp64_meas
        roof["measured_peak_source"] = ("tc_measure_fp64_rate: 4 FMA chains per thread, "
                                        "32 warps per SM, 0.25 s after the timed regions")
        if roof.get("achieved") is not None:
            roof["frac_of_measured"] = roof["achieved"] / fp64_meas
    tr = traffic_for(dom, args.workload, mixed)
    roof["traffic"] = tr
    # the whole step against HBM: algorithmic bytes per grid-point-step (every
    # spectral field pass read or written once: 44 passes with T, 33 without,
    # of 16 B per stored coefficient, S/P coefficients per grid point)
    S = wl.Nr * ((wl.Ntheta - 1) // 3 + 1) * (2 * ((wl.Nz - 1) // 3) + 1)
    passes = 44 if wl.Ra else 33
    alg_b = passes * 16.0 * S / wl.points
    hbm_peak = measured_hbm_peak()
    hbm = {"alg_bytes_per_point_step": alg_b, "achieved_GBs": alg_b * value / 1e9,
           "peak_GBs": hbm_peak,
           "frac": alg_b * value / 1e9 / hbm_peak if hbm_peak else None,
           "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy bandwidth)"}
    fl_step = step_flops(wl)
    # whole step against the FP64 peak (FP64 form only: the mixed form's
    # transforms are FP32)
    fp64 = None if mixed else {"flops_per_point_step": fl_step / wl.points,
            "achieved_tflops": fl_step * value / wl.points / 1e12,
            "peak_tflops": FP64_PEAK_TFLOPS,
            "frac": fl_step * value / wl.points / 1e12 / FP64_PEAK_TFLOPS,
            "peak_source": "derived: 152 SMs x 2.07 GHz x 4 FP64 flop/clk/SM"}
    if fp64 is not None and fp64_meas:
        fp64["measured_peak_tflops"] = fp64_meas
        fp64["frac_of_measured"] = fp64["achieved_tflops"] / fp64_meas
    kernels = {k: {"launches": v[0], "ms": round(v[1], 4)} for k, v in sorted(timing.items())}
    kernels["_pass"] = {"steps": kt_steps, "ms": round(kt_total_ms, 4)}

    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if getattr(wl, "precision", 0) else "f64",
            "data": "synthetic",
            "config": config_of(wl, {"l2": "flushed between timed steps (512 MiB write)",
                                     "parallelism": f"replicas x{world}",
                                     "tiles_mb_lb_mbf": list(tiles),
                                     "azimuthal_transforms": azimuthal,
                                     "axial_inverse_transforms": axial,
                                     "launch": "one step captured as a CUDA graph, replayed per step",
                                     "stated_error": (
                                         "rel L2 <= 1.3e-11 vs the FP64 path after 50 steps at "
                                         "256x512x512 (<= 2e-6 of max|N| on a random O(1) state)"
                                         if mixed else "rel L2 <= 1e-10 vs FP64 oracle")}),
            "multistep": {"value": wl.points / (multi_ms * 1e-3), "unit": METRIC,
                          "ms_per_step": multi_ms,
                          "how": f"one tc_step call of {args.steps} steps, CUDA events around "
                                 "it; L2 flushed once before the call, not between its steps"},
            "e2e": e2e, "gpu_launches": launches, "roofline": roof, "hbm_of_step": hbm,
            "fp64_of_step": fp64,
            "clocks": clk,
            "kernels": kernels}
    run.close()
    if not args.no_adjoint:
        line["adjoint"] = adjoint_throughput(tc, torch, flush)
    if world == 1 and not args.no_forms:
        del flush
        torch.cuda.empty_cache()
        line["forms"] = {"mixed": forms_mixed(tc, torch),
                         "ensemble": ensemble_form(tc, torch, 64, 20, 3)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, n, el, cores, sample = oracle_throughput(wl, budget_s=15.0)
        line["cpu_baseline"] = {"value": v, "unit": METRIC, "cores": cores, "kind": "oracle",
                                "sample": sample}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def adjoint_throughput(tc, torch, flush, steps=200, checkpoint=20, timed_adj=50):
    """Differentiation form on its own workload (64^3, FP64, fixed dt).

    (1) the discrete adjoint step alone: tc_adjoint_step from a stored state,
    CUDA events per step on the context's stream, L2 flushed between steps;
    (2) one whole gradient of J = E_pert(T) over `steps` steps: forward with
    a checkpoint every `checkpoint` steps, then per segment recompute and
    adjoint steps back (the autograd.Function path), wall clock with a device
    synchronisation at both ends.  Both in grid-point-steps/s, the second
    counting the `steps` steps of the differentiated window."""
    from paper_1908_00587_gb300.autograd import perturbation_energy

    wl = WORKLOADS["tc_adjoint_nr64_n64"]
    run = tc.Run.from_workload(wl)
    stream = torch.cuda.current_stream()
    run.set_stream(stream.cuda_stream)
    run.init_perturbation(psi_coefficients(wl.seed, wl.mp, wl.kp), wl.amp)
    X = torch.empty(run.shape, dtype=torch.complex128, device="cuda")
    tc.tc_get_state(run.ctx, X)
    lam = torch.empty_like(X)
    tc.tc_objective(run.ctx, lam)
    for _ in range(3):
        tc.tc_adjoint_step(run.ctx, X, wl.dt, lam)
    ks = [torch.cuda.Event(enable_timing=True) for _ in range(timed_adj)]
    ke = [torch.cuda.Event(enable_timing=True) for _ in range(timed_adj)]
    torch.cuda.synchronize()
    for i in range(timed_adj):
        flush.fill_(i & 0xFF)
        ks[i].record(stream)
        tc.tc_adjoint_step(run.ctx, X, wl.dt, lam)
        ke[i].record(stream)
    torch.cuda.synchronize()
    adj_ms = sum(a.elapsed_time(b) for a, b in zip(ks, ke)) / timed_adj
    # the reverse sweep over recorded steps (no forward stage recomputed)
    nrec = checkpoint
    rec = torch.empty(nrec * tc.tc_record_bytes_per_step(run.ctx), dtype=torch.uint8,
                      device="cuda")
    tc.tc_step_record(run.ctx, nrec, wl.dt, rec)
    tc.tc_adjoint_steps(run.ctx, nrec, rec, wl.dt, lam)          # warm-up
    ra = torch.cuda.Event(enable_timing=True)
    rb = torch.cuda.Event(enable_timing=True)
    flush.fill_(1)
    torch.cuda.synchronize()
    ra.record(stream)
    tc.tc_adjoint_steps(run.ctx, nrec, rec, wl.dt, lam)
    rb.record(stream)
    torch.cuda.synchronize()
    rec_ms = ra.elapsed_time(rb) / nrec
    del rec
    # whole gradient through the autograd.Function
    psi = torch.from_numpy(psi_coefficients(wl.seed, wl.mp, wl.kp)).requires_grad_(True)
    J = perturbation_energy(run, psi, 2, wl.dt, wl.amp, checkpoint=checkpoint)
    J.backward()                          # warm-up of the whole path
    psi.grad = None
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J = perturbation_energy(run, psi, steps, wl.dt, wl.amp, checkpoint=checkpoint)
    J.backward()
    torch.cuda.synchronize()
    grad_s = time.perf_counter() - t0
    run.close()
    return {"workload": f"{wl.name}: Nr={wl.Nr} Ntheta={wl.Ntheta} Nz={wl.Nz} eta={wl.eta} "
                        f"Re_i={wl.Re_i} dt={wl.dt}",
            "adjoint_step": {"value": wl.points / (adj_ms * 1e-3), "unit": METRIC,
                             "ms_per_step": adj_ms, "steps": timed_adj,
                             "l2": "flushed between timed steps",
                             "includes": "recomputation of the step's forward stages"},
            "adjoint_step_recorded": {"value": wl.points / (rec_ms * 1e-3), "unit": METRIC,
                                      "ms_per_step": rec_ms, "steps": nrec,
                                      "includes": "reverse sweep over tc_step_record records"},
            "gradient": {"value": wl.points * steps / grad_s, "unit": METRIC,
                         "seconds": grad_s, "steps": steps, "checkpoint_every": checkpoint,
                         "includes": "forward with checkpoints, per segment a recorded "
                                     "re-run and the adjoint sweep over its records, "
                                     "host-side psi marshalling"}}


def cc_radial_weights(Nr):
    """Clenshaw-Curtis weights of the Nr Chebyshev-Gauss-Lobatto nodes mapped
    to a gap of width 1 (the quadrature of the S14 parity norm; a measurement
    helper, checked against the oracle's weights by the tests)."""
    import numpy as np
    n = Nr - 1
    theta = np.pi * np.arange(Nr) / n
    w = np.zeros(Nr)
    for j in range(Nr):
        s = 0.0
        for k in range(1, n // 2 + 1):
            b = 1.0 if 2 * k == n else 2.0
            s += b * np.cos(2 * k * theta[j]) / (4 * k * k - 1)
        c = 1.0 if j in (0, n) else 2.0
        w[j] = c / n * (1.0 - s)
    return 0.5 * w


def weighted_rel_l2(a, b, r, w):
    """Per-field relative L2 of a against b (torch complex tensors of the state
    layout), weights c_m w_j r_j with c_0 = 1, c_m>0 = 2."""
    import torch
    nf, Nr, NM, _ = b.shape
    wr = torch.as_tensor(w * r, dtype=torch.float64, device=b.device).view(Nr, 1, 1)
    cm = torch.full((NM,), 2.0, dtype=torch.float64, device=b.device)
    cm[0] = 1.0
    wt = wr * cm.view(1, NM, 1)
    out = []
    for f in range(nf):
        num = torch.sum(wt * (a[f] - b[f]).abs() ** 2)
        den = torch.sum(wt * b[f].abs() ** 2)
        out.append(float(torch.sqrt(num / den)))
    return out


def forms_mixed(tc, torch, steps=10, total=50):
    """Mixed precision against FP64 on the same GPU at 256 x 512 x 512 (eta =
    0.875, Re_i = 1e4, amplitude 0.1, dt = 2e-6): both forms run `total`
    steps from the same seeded state; `steps` of them (after 3 untimed) are
    timed with CUDA events on the context's stream (the 717 MB state exceeds
    L2), and the per-field relative L2 of the mixed state against the FP64
    state after `total` steps is the mixed form's stated error."""
    import numpy as np
    wl = WORKLOADS["tc_mixed_nr256_n512"]
    psi = psi_coefficients(wl.seed, wl.mp, wl.kp)
    stream = torch.cuda.current_stream()
    res, final = {}, {}
    for prec in (1, 0):
        w = wl.scaled(precision=prec)
        run = tc.Run.from_workload(w)
        run.set_stream(stream.cuda_stream)
        run.init_perturbation(psi, w.amp)
        tc.tc_autotune(run.ctx)
        info = tc.tc_get_info(run.ctx)
        run.step(3, w.dt)
        clocks = Clocks(torch.cuda.current_device())
        clocks.start()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        ev[0].record(stream)
        run.step(steps, w.dt)
        ev[1].record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        ms = ev[0].elapsed_time(ev[1]) / steps
        run.step(total - 3 - steps, w.dt)
        X = torch.empty(run.shape, dtype=torch.complex128, device="cuda")
        tc.tc_get_state(run.ctx, X)
        final[prec] = X
        res[prec] = {"value": w.points / (ms * 1e-3), "unit": METRIC, "ms_per_step": ms,
                     "steps_timed": steps, "clocks": clk,
                     "tiles_mb_lb_mbf": [info.tile_mb, info.tile_lb, info.tile_mbf]}
        run.close()
    g = 0.5 * (1.0 - np.cos(np.pi * np.arange(wl.Nr) / (wl.Nr - 1)))
    r = wl.eta / (1.0 - wl.eta) + g
    err = weighted_rel_l2(final[1], final[0], r, cc_radial_weights(wl.Nr))
    del final
    torch.cuda.empty_cache()
    return {"workload": f"{wl.name}: Nr={wl.Nr} Ntheta={wl.Ntheta} Nz={wl.Nz} eta={wl.eta} "
                        f"Re_i={wl.Re_i} amp={wl.amp} dt={wl.dt}",
            "mixed": res[1], "fp64": res[0],
            "speedup_vs_fp64": res[1]["value"] / res[0]["value"],
            "stated_error": {"rel_l2_vs_fp64_per_field": dict(zip(("u_r", "u_theta", "u_z"), err)),
                             "after_steps": total,
                             "norm": "c_m w_j r_j weighted (Clenshaw-Curtis w_j)"}}


def ensemble_form(tc, torch, n=64, steps=20, warmup=3):
    """Batched form: n uneven runs (every other one mixed precision), one step
    of all of them captured into one CUDA graph and replayed, against the same
    runs stepped one after another (each replaying its own step graph)."""
    import numpy as np
    from inputs import ensemble_members
    members = [w.scaled(precision=i % 2) for i, w in enumerate(ensemble_members(n))]
    t0 = time.perf_counter()
    ens = tc.tc_ensemble_create(members, autotune_tiles=True)
    setup_s = time.perf_counter() - t0
    dts = []
    for i, wl in enumerate(members):
        ctx = tc.tc_ensemble_member(ens, i)
        tc.tc_init_perturbation(ctx, psi_coefficients(wl.seed, wl.mp, wl.kp), wl.amp)
        info = tc.tc_get_info(ctx)
        X = torch.empty((info.nfields, info.Nr, info.M + 1, 2 * info.K + 1),
                        dtype=torch.complex128, device="cuda")
        tc.tc_get_state(ctx, X)
        out = torch.zeros_like(X)
        rate = tc.tc_nonlinear(ctx, X, out)
        dts.append(min(1e-3, 0.25 / rate))
    pts = sum(w.points for w in members)

    def timed(mode):
        tc.tc_ensemble_set_mode(ens, mode)
        tc.tc_ensemble_step(ens, warmup, dts)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tc.tc_ensemble_step(ens, steps, dts)
        torch.cuda.synchronize()
        return time.perf_counter() - t0, tc.tc_ensemble_kernels_per_step(ens)

    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    graph_s, kps = timed(0)            # default: one CUDA graph of per-member kernels per step
    clk = clocks.stop()
    persist_s, kps_persist = timed(1)  # one persistent launch per call
    tc.tc_ensemble_set_mode(ens, 0)
    seq_s = 0.0
    for i, wl in enumerate(members):
        ctx = tc.tc_ensemble_member(ens, i)
        tc.tc_step(ctx, 1, dts[i])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tc.tc_step(ctx, steps, dts[i])
        seq_s += time.perf_counter() - t0
    tc.tc_ensemble_destroy(ens)
    # how much of the FP64 unit one ensemble step keeps busy: the FP64
    # members' whole steps and the mixed members' FP64 linear stages
    fp64_flops = 0.0
    fp32_flops = 0.0
    for wl in members:
        nl, lin = stage_flops(wl)
        if wl.precision:
            fp64_flops += 2 * lin
            fp32_flops += 2 * nl
        else:
            fp64_flops += 2 * (nl + lin)
    step_s = graph_s / steps
    try:
        fp64_peak = tc.tc_measure_fp64_rate(250.0, torch.cuda.current_stream().cuda_stream)
    except Exception:
        fp64_peak = FP64_PEAK_TFLOPS
    fp64_use = {"fp64_flops_per_step": fp64_flops, "fp32_flops_per_step": fp32_flops,
                "achieved_fp64_tflops": fp64_flops / step_s / 1e12,
                "fp64_peak_tflops": fp64_peak,
                "frac": fp64_flops / step_s / 1e12 / fp64_peak,
                "peak_source": "tc_measure_fp64_rate (measured FP64 FMA rate of this GPU)"}
    return {"workload": f"ensemble of {len(members)} uneven runs (Nr in 32/48/64, "
                        f"N in 32/64/96, eta in 0.5/0.71/0.875, Re_i in [80, 400], "
                        f"every other member mixed precision), fixed dt per member",
            "grid_points_total": pts, "steps": steps, "warmup": warmup,
            "value": pts * steps / graph_s, "unit": METRIC,
            "ms_per_step": 1e3 * graph_s / steps,
            "launch": "default mode 0: one step of every member captured as one CUDA graph "
                      "(members are independent branches), replayed per step",
            "persistent": {"value": pts * steps / persist_s,
                           "ms_per_step": 1e3 * persist_s / steps,
                           "launches_per_call": kps_persist,
                           "how": f"mode 1: one persistent kernel launch for all {steps} steps "
                                  "of every member; CTA tiles claimed from per-member stage "
                                  "counters"},
            "sequential": {"value": pts * steps / seq_s, "ms_per_step": 1e3 * seq_s / steps},
            "speedup_vs_sequential": seq_s / graph_s,
            "persistent_vs_graph": graph_s / persist_s,
            "kernels_per_step": kps, "tile_autotune_s": setup_s,
            "fp64_of_step": fp64_use,
            "timing": "wall clock around tc_ensemble_step with a device synchronisation "
                      "at both ends", "clocks": clk}


def run_ensemble(args):
    """Batched form on its own line (--ensemble N)."""
    import torch

    import __graft_entry__ as g
    g.build()
    from paper_1908_00587_gb300 import tc
    torch.cuda.set_device(0)
    f = ensemble_form(tc, torch, args.ensemble, args.steps, args.warmup)
    line = {"metric": METRIC, "value": f["value"], "unit": METRIC, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": f["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 and f32+f64 members", "data": "synthetic",
            "config": {"workload": f["workload"], "grid_points_total": f["grid_points_total"],
                       "tile_autotune_s": f["tile_autotune_s"],
                       "l2": "working set of all members exceeds L2"},
            "sequential": f["sequential"], "speedup_vs_sequential": f["speedup_vs_sequential"],
            "persistent": f["persistent"],
            "gpu_launches": f["kernels_per_step"] * args.steps, "clocks": f["clocks"]}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.ensemble:
        return run_ensemble(args)
    return run_gb300(args)


if __name__ == "__main__":
    sys.exit(main())
