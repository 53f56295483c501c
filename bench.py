"""Benchmark of the Fourier-Galerkin hot path on one GB300 (or N replicas under torchrun).

Workload: 3-D scalar conductivity on the 243^3 grid (3^5), FP64, GaNi (trapezoidal
integration), centred cubic inclusion of volume fraction 0.2 (143^3 nodes, 0.2038 realised),
contrast 1e3, E = (1, 0, 0). One step is one conjugate-gradient iteration (Algorithm 2):
the fused pre-pass p = r + beta p with A p, the forward 3-D DFT, the projection Gamma^, the
inverse DFT with the (C p, p) partials, and the x/r update with (r, r). `value` counts
G A matvecs per second (one per step). The 243^3 fields (344 MB each) exceed the 129 MB L2,
so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Profiling helpers (not bench lines): --quick skips the end-to-end, CG-to-tolerance and CPU
legs; --precision fp32 (with --quick) times the FP32 inner CG step instead; --grid n runs the
same step on an n^3 grid (used for ncu captures on a smaller case).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import microstructure as ms  # noqa: E402

N_GRID = (243, 243, 243)  # may be overridden by --grid for profiling captures
VF = 0.2
CONTRAST = 1000.0
E_MACRO = np.array([1.0, 0.0, 0.0])
METRIC = "G·A matvecs/s at 243^3 (FP64 CG step)"
UNIT = "matvec/s"
D = 3


def workload():
    h = ms.inclusion_side_for_fraction(VF, D)
    ph = ms.box_phase(N_GRID, h)
    table = ms.isotropic_table([1.0, CONTRAST], D)
    return ph, table


def measured_peaks():
    """HBM copy bandwidth measured on the GB300s (generated file), else the
    recipe's fallback figure."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured (MEASURED_PEAKS.json hbm_gbs)"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "source": "fallback 6.8 TB/s"}


def config(extra=None):
    c = {"workload": "GaNi 243^3 FP64 CG step, centred cube vf 0.2, contrast 1e3, E=(1,0,0)",
         "grid": list(N_GRID), "d": D, "integration": "approx (GaNi)", "solver": "cg",
         "l2": "inputs larger than L2 (344 MB per field)"}
    if extra:
        c.update(extra)
    return c


# ------------------------------------------------------------------------------------------
# distributed helpers (replicas: each rank solves its own copy, no data-path collective)
# ------------------------------------------------------------------------------------------

def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world):
    """The largest of the ranks' values (the timed region of a replica run ends when the slowest
    rank ends); on the process group's own device (NCCL: the GPU, gloo: the host)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(ms_step_local, world):
    """Whole-job matvecs/s of N replicas: every rank runs one step per ms_step of its own, the
    job's step time is the slowest rank's, and N steps complete per job step."""
    ms = max_over_ranks(ms_step_local, world)
    return ms, world * 1000.0 / ms


# ------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.strip().split(",") for r in self.file.read().splitlines() if r.strip()]
        self.file.close()
        os.unlink(self.file.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for i, nm in enumerate(names):
                if len(r) > 5 + i and "Active" in r[5 + i] and "Not" not in r[5 + i]:
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------
# CPU oracle leg (test infrastructure, timed as it stands)
# ------------------------------------------------------------------------------------------

def cufft_matvec(ph, table, x_dev, dtype, steps):
    """The same G A x on the same grid with PyTorch's FFTs (cuFFT), as a timed comparison only:
    A x pointwise, rfftn over the three axes, Gamma^ = k k^T / |k|^2 (k = 0 zeroed), irfftn.
    torch's rfftn is unscaled and irfftn carries 1/|N|, the normalisation of eq. (DFT) up to
    where the factor sits. Returns (ms per matvec, result)."""
    import torch
    dev = x_dev.device
    n0, n1, n2 = N_GRID
    a = torch.as_tensor(np.asarray(table)[:, 0, 0], device=dev, dtype=dtype)[
        torch.as_tensor(ph.astype(np.int64), device=dev)]
    k0 = torch.fft.fftfreq(n0, 1.0 / n0, device=dev, dtype=dtype).view(n0, 1, 1)
    k1 = torch.fft.fftfreq(n1, 1.0 / n1, device=dev, dtype=dtype).view(1, n1, 1)
    k2 = torch.fft.rfftfreq(n2, 1.0 / n2, device=dev, dtype=dtype).view(1, 1, -1)
    kk = k0 * k0 + k1 * k1 + k2 * k2
    inv = torch.where(kk > 0, 1.0 / torch.where(kk > 0, kk, torch.ones_like(kk)), torch.zeros_like(kk))
    x = x_dev.to(dtype)

    def matvec(xx):
        vh = torch.fft.rfftn(a * xx, dim=(1, 2, 3))
        s = (k0 * vh[0] + k1 * vh[1] + k2 * vh[2]) * inv
        yh = torch.stack((k0 * s, k1 * s, k2 * s))
        return torch.fft.irfftn(yh, s=(n0, n1, n2), dim=(1, 2, 3))

    for _ in range(2):
        y = matvec(x)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        y = matvec(x)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, y


def host_cpu() -> str:
    """The host CPU as the kernel reports it: model name (x86) or implementer/part (Arm)."""
    model, impl, part = "", "", ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k, _, v = line.partition(":")
                k, v = k.strip(), v.strip()
                if k == "model name" and not model:
                    model = v
                elif k == "CPU implementer" and not impl:
                    impl = v
                elif k == "CPU part" and not part:
                    part = v
    except OSError:
        pass
    if model:
        return model
    if impl or part:
        # 0x41 = Arm Ltd; part 0xd4f = Neoverse V2 (the Grace core)
        names = {("0x41", "0xd4f"): "Arm Neoverse V2"}
        return names.get((impl, part), f"Arm implementer {impl} part {part}")
    import platform
    return platform.machine()


def cpu_oracle_cg_steps(nsteps=1):
    """Time CG iterations of the FP64 NumPy oracle on this host at the bench workload."""
    import oracle as O
    ph, table = workload()
    a = O.expand_phase(ph, table)[0, 0]
    sysn = O.GaNi(a, D)
    t0 = time.perf_counter()
    res = O.cg(sysn, E_MACRO, fixed_iters=nsteps)
    dt = time.perf_counter() - t0
    # fixed_iters=k costs k matvecs plus the two of the set-up (b and r_0)
    matvecs = nsteps + 2
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    del res
    return {"value": matvecs / dt, "unit": UNIT, "cores": cores, "cpu": host_cpu(),
            "kind": "oracle",
            "sample": f"{nsteps} oracle CG iteration(s) + set-up at 243^3 ({matvecs} matvecs, "
                      f"{dt:.1f} s, NumPy FP64 dense-matrix DFT, BLAS threads = host cores)"}


# ------------------------------------------------------------------------------------------
# roofline bookkeeping of the dominant kernel
# ------------------------------------------------------------------------------------------

def plan_radices(n, rmax):
    """The library's radix plan of an axis (first-fit grouping of the prime factors, largest
    first, into register radices <= rmax; stages in decreasing radix order)."""
    primes = []
    m = n
    for R in (31, 29, 23, 19, 17, 13, 11, 7, 5, 3):
        while m % R == 0:
            primes.append(R)
            m //= R
    groups = []
    for f in primes:
        best = None
        for gi, g in enumerate(groups):
            if g * f <= rmax and (best is None or g > groups[best]):
                best = gi
        if best is None:
            groups.append(f)
        else:
            groups[best] *= f
    return sorted(groups, reverse=True)


def _smallest_factor(R):
    for p in (3, 5, 7, 11, 13, 17, 19, 23, 29, 31):
        if R % p == 0:
            return p
    return R


def reg_dft_flops(R):
    """Flops of the in-register DFT of R points (FMA = 2): prime R by the pairing method
    (8H^2 + 8H, H = (R-1)/2), composite R = A B as B A-point and A B-point DFTs plus the
    non-trivial internal twiddles (6 flops each)."""
    A = _smallest_factor(R)
    if A == R:
        H = (R - 1) // 2
        return 8 * H * H + 8 * H
    B = R // A
    tw = sum(1 for j2 in range(B) for k1 in range(A) if (j2 * k1) % R)
    return B * reg_dft_flops(A) + A * reg_dft_flops(B) + 6 * tw


def fft_flops_per_point(n, rmax):
    """Flops per complex point of one transform of length n with the library's plan: per stage
    of radix R, one R-point register DFT per R points plus R - 1 twiddle products (6 flops) when
    earlier stages exist."""
    total, p = 0.0, 1
    for R in plan_radices(n, rmax):
        total += (reg_dft_flops(R) + (6 * (R - 1) if p > 1 else 0)) / R
        p *= R
    return total


def pass_flops(rmax):
    """Algorithmic flops of one launch of each pass kind (d = 3, FP64 CG step)."""
    n = N_GRID[0]
    nh = (n + 1) // 2
    lines_c = n * n * D / 2.0                 # complex lines of the packed real transforms
    f1 = fft_flops_per_point(n, rmax)
    spec = n * n * nh * D                     # half-spectrum points per transform pass
    return {
        "line_fwd": lines_c * n * f1 + n * n * n * D * 2 + n * n * nh * D * 6,
        "strided": spec * f1,
        "proj": 2 * spec * f1 + n * n * nh * (4 * D + 2 + 2 * D),
        "line_inv": lines_c * n * f1 + n * n * n * D * 2,
    }


def pass_flops_model(n=None):
    """Algorithmic flops of one launch of each pass kind by the standard model of an FFT,
    2.5 n log2 n per real transform of length n along each axis: a pass that transforms one
    axis of the d components counts d x 2.5 |N| log2(n_axis); the projection pass transforms
    axis 0 forward and inverse. One matvec sums to 2 d x 2.5 |N| log2 |N| (5.1 GFLOP at
    243^3)."""
    import math
    n0, n1, n2 = N_GRID if n is None else n
    nodes = n0 * n1 * n2
    per_axis = lambda m: D * 2.5 * nodes * math.log2(m)  # noqa: E731
    return {"line_fwd": per_axis(n2), "strided": per_axis(n1), "proj": 2 * per_axis(n0),
            "line_inv": per_axis(n2)}


def measure_fp64_peak(H, local):
    """FP64 rate of this GPU, measured with the library's DFMA / DADD chain kernel
    (hom_measure_fp64): best of three timed waves each, SM clock sampled meanwhile."""
    import torch
    clocks = ClockSampler(local)
    clocks.start()
    best_fma, best_add = 0.0, 0.0
    for _ in range(3):
        ms_, ops = H.hom_measure_fp64(0, 1500)
        best_fma = max(best_fma, ops / ms_ / 1e9)
        ms_, ops = H.hom_measure_fp64(1, 1500)
        best_add = max(best_add, ops / ms_ / 1e9)
    torch.cuda.synchronize()
    clk = clocks.stop()
    return {"dfma_tflops": round(best_fma, 4), "dadd_tinstr_per_s": round(best_add, 4),
            "sm_mhz": clk.get("sm_mhz"), "reasons": clk.get("reasons"),
            "how": "hom_measure_fp64: 8 independent FP64 FMA (or add) chains per thread, one "
                   "full wave of resident CTAs on every SM, CUDA events, best of 3"}


# DRAM bytes read + written per launch of the dominant kernels of the 243^3 CG steps (ncu
# dram__bytes_read.sum + dram__bytes_write.sum on GB300 of the kernels as they are now;
# profiles/ gives the commands); other kernels and grids have no capture (null)
NCU_TRAFFIC = {("fp64", "strided"): 634.6e6, ("fp32", "line_fwd"): 644.0e6,
               ("fp32", "line_inv"): 984.8e6, ("fp32", "pot_inv"): 342.6e6,
               ("fp32", "pot_line"): 300.9e6, ("fp32", "pot_fwd"): 199.0e6}


def ncu_traffic(precision, kind):
    if tuple(N_GRID) != (243, 243, 243):
        return None
    return NCU_TRAFFIC.get((precision, kind))


# FP64 thread instructions (DADD + DFMA + DMUL) per launch of the FP64 CG step's pass kernels at
# 243^3 (ncu smsp__sass_thread_inst_executed_op_{dadd,dfma,dmul}_pred_on.sum on GB300 of the
# kernels as they are now; profiles/ gives the command). The strided pass runs 27.11 a complex
# point: 84/9 + 106/9 + 18/3 for the [9, 9, 3] plan with cosine-factored twiddles.
NCU_FP64_INST = {"line_fwd": 808.7e6, "strided": 585.9e6, "proj": 882.1e6, "line_inv": 765.1e6}


def fp64_issue(pk, ms_step, steps, probe):
    """The FP64 step against its instruction bound: the FP64 instructions ncu counts in each
    pass kernel, over its measured time, as a fraction of the FP64 instruction rate the probe
    measured on this GPU (the larger of DFMA and DADD instructions per second)."""
    if tuple(N_GRID) != (243, 243, 243) or not probe:
        return None
    rate = max(probe["dfma_tflops"] / 2.0, probe["dadd_tinstr_per_s"]) * 1e12
    out = {"rate_tinst_per_s": round(rate / 1e12, 4), "source": "ncu FP64 instruction counts "
           "(NCU_FP64_INST) over the measured pass times and the probe's instruction rate"}
    step_inst = 0.0
    for k, v in pk.items():
        if k in NCU_FP64_INST:
            inst = NCU_FP64_INST[k]
            step_inst += inst * v["launches"] / steps
            out[k] = round(inst / (v["ms_avg"] * 1e-3) / rate, 4)
    out["step_inst"] = step_inst
    out["step_frac"] = round(step_inst / (ms_step * 1e-3) / rate, 4)
    return out


def pass_bytes(word=8, two_line=False, fused_cg=False):
    """Compulsory DRAM bytes of one launch of each pass kind in a CG step (word = 8 for FP64,
    4 for FP32). two_line: the 3-D scalar projection keeps two spectrum lines between its column
    passes (the axis-1 passes read or write two components of three, the projection two and
    two). fused_cg: the fused CG step of both precisions, whose inverse pass reads the spectrum
    and x, r, p and writes x, r (no separate vector update); otherwise line_inv reads the
    spectrum and p and writes C p, and the vector update reads x, p, r, C p and writes x, r."""
    n = N_GRID[0]
    nh = (n + 1) // 2
    spec = n * n * nh * D * 2 * word  # all D components of the half spectrum
    field = n * n * n * D * word
    out = {"line_fwd": 2 * field + field + n ** 3 + spec,  # r, p read; p written; phase; spectrum
           "strided": 2 * spec, "proj": 2 * spec}
    if two_line:
        out["strided"] = spec * 5 // 3   # forward 3 read + 2 written, inverse 2 read + 3 written
        out["proj"] = spec * 4 // 3
    if fused_cg:
        out["line_inv"] = spec + 3 * field + 2 * field
    else:
        out["line_inv"] = spec + 2 * field                # spectrum; p read; C p written
        out["vector"] = 6 * field
    return out


def pot_bytes(word=4):
    """Compulsory DRAM bytes of one launch of each pass of the CG step in potential coordinates
    (the FP32 inner solver): u, r, p are one complex component on the half spectrum (c bytes
    each); pot_inv reads r, p, u and writes p, u (the deferred u += alpha p) and two spectrum
    lines; the axis-1 passes move two and three lines; pot_line reads and writes three lines
    and reads the phase image; pot_fwd reads two lines and r and writes r."""
    n = N_GRID[0]
    nh = (n + 1) // 2
    c = n * n * nh * 2 * word
    return {"pot_inv": 7 * c, "strided": 5 * c, "pot_line": 6 * c + n ** 3, "pot_fwd": 4 * c}


# ------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------

def run_ours(args, rank, world, local):
    """Everything on a stream of its own: the library launches its pass kernels there with a
    programmatic dependency on the kernel before them (on the legacy default stream it cannot),
    so each pass's launch overlaps the previous pass's drain."""
    import torch
    torch.cuda.set_device(local)
    with torch.cuda.stream(torch.cuda.Stream()):
        return _run_ours(args, rank, world, local)


def _run_ours(args, rank, world, local):
    import torch
    import paper_1508_02045_gb300 as H

    global N_GRID
    if args.grid:
        N_GRID = (args.grid,) * 3

    torch.cuda.set_device(local)
    if args.quick and args.precision == "elastic":  # profiling helper: the elasticity step alone
        line = elastic_step(args.steps, args.warmup, N_GRID[0])
        if rank == 0:
            print(json.dumps({"quick": True, "precision": "elastic", **line}), flush=True)
        return None
    ph, table = workload()
    fp32_only = args.quick and args.precision == "fp32"
    prob = H.Problem(D, N_GRID, H.phase_material(ph, table),
                     precision=H.HOM_FP32_REFINED if fp32_only else H.HOM_FP64)
    # the launch plan a user gets from the autotuner (--no-tune: the default plan, for
    # profiler captures that should not see the candidates' launches)
    tune = H.hom_autotune(prob.h, reps=2) if not args.no_tune else {"rmax64": 15, "smem_kb64": 110}
    fp64_peak = None if args.quick else measure_fp64_peak(H, local)
    stream = torch.cuda.current_stream()
    total = args.warmup + args.steps
    if fp32_only:  # the FP32 inner CG step of the refinement (profiling helper)
        opts = H.make_opts(maxit=2, inner_tol=1e-30, inner_form=args.inner_form)
        H.hom_solve_begin(prob.h, E_MACRO, H.HOM_CG, 1e-30, opts)
    else:
        opts = H.make_opts(fixed_iters=total + 1)
        H.hom_solve_begin(prob.h, E_MACRO, H.HOM_CG, 0.0, opts)
    H.hom_solve_iterate(prob.h, args.warmup)
    torch.cuda.synchronize()

    # ---- timed region: K CG steps, inputs resident in HBM ----
    clocks = ClockSampler(local)
    clocks.start()
    H.hom_profile_enable(True)
    barrier(world)
    torch.cuda.synchronize()
    launches0 = H.hom_kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    H.hom_solve_iterate(prob.h, args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    launches = H.hom_kernel_launches() - launches0
    H.hom_profile_enable(False)
    clk = clocks.stop()
    passes = H.hom_profile_read()
    ms_total = max_over_ranks(e0.elapsed_time(e1), world)
    ms_step = ms_total / args.steps
    H.hom_solve_end(prob.h, D, allow_not_converged=True)
    if args.quick:
        prob.close()
        if rank == 0:
            print(json.dumps({"quick": True, "precision": args.precision, "grid": list(N_GRID),
                              "ms_per_step": ms_step,
                              "passes": passes, "gpu_launches": int(launches)}), flush=True)
        return None

    # ---- the same CG step in FP32 (the inner solver of HOM_FP32_REFINED): in potential
    # coordinates (the default inner form of refined CG) and in the field form ----
    p32 = H.Problem(D, N_GRID, H.phase_material(ph, table), precision=H.HOM_FP32_REFINED)
    tune32 = H.hom_autotune(p32.h, reps=2)
    fp32_forms = {}
    for form in (0, 1):
        H.hom_solve_begin(p32.h, E_MACRO, H.HOM_CG, 1e-30,
                          H.make_opts(maxit=2, inner_tol=1e-30, inner_form=form))
        H.hom_solve_iterate(p32.h, args.warmup)
        torch.cuda.synchronize()
        H.hom_profile_enable(True)
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        H.hom_solve_iterate(p32.h, args.steps)
        f1.record(stream)
        torch.cuda.synchronize()
        H.hom_profile_enable(False)
        fp32_forms[form] = (f0.elapsed_time(f1) / args.steps, H.hom_profile_read())
        H.hom_solve_end(p32.h, D, allow_not_converged=True)
    # a refined CG solve of the same problem to 1e-8 in either inner form (outside the timed
    # region): in potential coordinates the FP32 iterates stay exact gradients
    refined_solves = {}
    for solver, sname in ((H.HOM_CG, "cg"), (H.HOM_CHEBYSHEV, "chebyshev")):
        for form, name in ((0, "potential"), (1, "field")):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            AHr, _, str_, _ = H.hom_solve(p32.h, E_MACRO, solver, 1e-8,
                                          H.make_opts(maxit=50, inner_form=form))
            torch.cuda.synchronize()
            refined_solves[f"{sname}_{name}"] = {
                "seconds": round(time.perf_counter() - t0, 4), "A_H": AHr,
                "outer": str_["iterations"], "inner": str_["inner_iterations"],
                "converged": bool(str_["converged"])}
    p32.close()

    # ---- end to end through the C ABI: every step hom_apply reads the field from pinned host
    # memory and writes the result back to pinned host memory (HOM_OP_X_HOST | HOM_OP_Y_HOST:
    # the pass kernels load and store the host buffers through their device mapping), and the
    # call returns once the result is in host memory ----
    nfield = D * int(np.prod(N_GRID))
    xh = torch.from_numpy(ms.random_field((D,) + tuple(N_GRID), 11)).pin_memory()
    yh = torch.empty((D,) + tuple(N_GRID), dtype=torch.float64).pin_memory()
    for _ in range(args.warmup):
        H.hom_apply(prob.h, H.HOM_OP_LINEAR, None, xh, yh)
    torch.cuda.synchronize()
    barrier(world)
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    t_e2e = time.perf_counter()
    f0.record(stream)
    for _ in range(args.steps):
        H.hom_apply(prob.h, H.HOM_OP_LINEAR, None, xh, yh)
    f1.record(stream)
    torch.cuda.synchronize()
    e2e_wall_ms = (time.perf_counter() - t_e2e) * 1e3 / args.steps
    e2e_ms = max_over_ranks(f0.elapsed_time(f1), world) / args.steps
    # the same application on device-resident fields, for the cost of the host traffic
    xdev = xh.cuda()
    ydev = torch.empty_like(xdev)
    H.hom_apply(prob.h, H.HOM_OP_LINEAR, None, xdev, ydev)
    torch.cuda.synchronize()
    d0 = torch.cuda.Event(enable_timing=True)
    d1 = torch.cuda.Event(enable_timing=True)
    d0.record(stream)
    for _ in range(args.steps):
        H.hom_apply(prob.h, H.HOM_OP_LINEAR, None, xdev, ydev)
    d1.record(stream)
    torch.cuda.synchronize()
    dev_apply_ms = d0.elapsed_time(d1) / args.steps
    e2e_equal = bool(torch.equal(ydev.cpu(), yh))
    del xdev, ydev

    # ---- the same matvec with cuFFT (torch.fft), a timed comparison only ----
    xr = torch.from_numpy(ms.random_field((D,) + tuple(N_GRID), 12)).cuda()
    ours = prob.field()
    H.hom_apply(prob.h, H.HOM_OP_LINEAR, None, xr, ours)
    cmp_steps = max(3, min(args.steps, 10))
    cu64_ms, cu64_y = cufft_matvec(ph, table, xr, torch.float64, cmp_steps)
    cu_rel = float(torch.linalg.vector_norm(cu64_y - ours) / torch.linalg.vector_norm(ours))
    del cu64_y
    cu32_ms, cu32_y = cufft_matvec(ph, table, xr, torch.float32, cmp_steps)
    del cu32_y, xr, ours
    torch.cuda.synchronize()

    # ---- CG time to 1e-6 (outside the timed region) ----
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    AH, flux, stats, st = H.hom_solve(prob.h, E_MACRO, H.HOM_CG, 1e-6,
                                      H.make_opts(maxit=2000, check_every=16), None,
                                      allow_not_converged=True)
    cg_wall = time.perf_counter() - t0
    prob.close()

    if rank != 0:
        return None
    flops = pass_flops_model()
    flops_radix = pass_flops(tune["rmax64"])
    byts = pass_bytes(8, fused_cg=True)
    byts32 = pass_bytes(4, two_line=bool(tune32.get("two_line32")), fused_cg=True)
    peaks = measured_peaks()

    def per_kind(pr):
        out = {}
        for k, (ms_k, cnt) in pr.items():
            if cnt:
                out[k] = {"ms_avg": round(ms_k / cnt, 4), "launches": cnt}
        tot = sum(v["ms_avg"] * v["launches"] for v in out.values())
        for v in out.values():
            v["share"] = round(v["ms_avg"] * v["launches"] / tot, 4) if tot else None
        return out

    pk = per_kind(passes)
    dom = max((k for k in pk if k in flops), key=lambda k: pk[k]["ms_avg"] * pk[k]["launches"])
    dom_ms = pk[dom]["ms_avg"]
    achieved = flops[dom] / (dom_ms * 1e-3) / 1e12
    peak = fp64_peak["dfma_tflops"]  # measured on this GPU before the timed region
    # compulsory bytes of one step: per kind, bytes per launch x launches per step (measured)
    step_bytes = sum(byts[k] * pk[k]["launches"] / args.steps for k in pk if k in byts)
    fp32 = {}
    for form, bb in ((0, pot_bytes(4)), (1, byts32)):
        ms32, pr32 = fp32_forms[form]
        pk32 = per_kind(pr32)
        dom32 = max((k for k in pk32 if k in bb), key=lambda k: pk32[k]["ms_avg"] * pk32[k]["launches"])
        ach32 = bb[dom32] / (pk32[dom32]["ms_avg"] * 1e-3) / 1e9
        sb32 = sum(bb[k] * pk32[k]["launches"] / args.steps for k in pk32 if k in bb)
        fp32[form] = {"value": round(1000.0 / ms32, 3), "unit": UNIT, "ms_per_step": round(ms32, 4),
                      "step_bytes": int(sb32), "hbm_gbs": round(sb32 / (ms32 * 1e-3) / 1e9, 1),
                      "roofline": {"bound": "hbm", "kernel": f"k_{dom32}", "achieved": round(ach32, 1),
                                   "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                   "frac": round(ach32 / peaks["hbm_gbs"], 4),
                                   "traffic": ncu_traffic("fp32", dom32),
                                   "peak_source": peaks["source"]},
                      "passes": pk32}
    value = world * 1000.0 / ms_step
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded centred-cube phase image)",
        "config": config({"parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                          "plan": {"fp64_rmax": tune["rmax64"], "fp64_smem_kb": tune["smem_kb64"]}}),
        "e2e": {"value": round(world * 1000.0 / e2e_ms, 3), "unit": UNIT,
                "h2d_bytes_per_step": nfield * 8, "d2h_bytes_per_step": nfield * 8,
                "ms_per_step": round(e2e_ms, 4), "host_wall_ms_per_step": round(e2e_wall_ms, 4),
                "device_fields_ms_per_matvec": round(dev_apply_ms, 4),
                "result_equals_device_path": e2e_equal,
                "path": "C ABI hom_apply(HOM_OP_LINEAR | HOM_OP_X_HOST | HOM_OP_Y_HOST) on pinned "
                        "host buffers, every step: the first pass reads x from host memory and "
                        "the last writes y to host memory (over the GPU's host link), the call "
                        "returns with y in host memory; K steps between CUDA events"},
        "gpu_launches": int(launches),
        "hbm_gbs": round(step_bytes / (ms_step * 1e-3) / 1e9, 1),
        "roofline": {"bound": "alu", "kernel": f"k_{dom}", "achieved": round(achieved, 4),
                     "peak": peak, "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                     "traffic": ncu_traffic("fp64", dom),
                     "peak_source": "measured FP64 FMA rate of this GPU (hom_measure_fp64, burst)",
                     "peak_nominal": 1.25, "flop_model": "2.5 n log2 n per real transform and axis",
                     "flops_per_launch": round(flops[dom]),
                     "achieved_radix_model": round(flops_radix[dom] / (dom_ms * 1e-3) / 1e12, 4),
                     "fp64_probe": fp64_peak,
                     "fp64_issue_frac": fp64_issue(pk, ms_step, args.steps, fp64_peak),
                     "hbm_gbs_of_dominant": round(byts[dom] / (dom_ms * 1e-3) / 1e9, 1)},
        "passes": pk,
        "fp32_step": {"metric": "G·A matvecs/s at 243^3 (FP32 CG step, inner solver of the refinement, "
                                "in potential coordinates)",
                      **fp32[0],
                      "plan": {"rmax": tune32["rmax32"], "smem_kb": tune32["smem_kb32"],
                               "two_line": bool(tune32.get("two_line32"))},
                      "field_form": fp32[1],
                      "refined_to_1e-8": refined_solves},
        "clocks": clk,
        "cufft_comparison": {
            "what": "G A x with torch.fft (cuFFT rfftn/irfftn) + elementwise torch ops, same grid "
                    "and coefficients; timed comparison, not the product path",
            "fp64_ms": round(cu64_ms, 4), "fp64_matvec_per_s": round(1000.0 / cu64_ms, 3),
            "fp32_ms": round(cu32_ms, 4), "fp32_matvec_per_s": round(1000.0 / cu32_ms, 3),
            "fp64_rel_diff_vs_ours": cu_rel},
        "cg_to_1e-6": {"iterations": stats["iterations"], "seconds": round(cg_wall, 3),
                       "device_ms": round(stats["time_ms"], 2), "A_H": AH,
                       "converged": bool(stats["converged"])},
    }
    # the studies after the timed step run at one GPU only: a replica run (N > 1) would hold
    # every GPU while rank 0 repeats them, and the oracle's host timing belongs to N = 1
    single = world == 1
    if single and not args.no_elastic:
        line["elastic"] = elastic_step(min(args.steps, 10), 3, solves=True)
    if single and not args.no_kappa:
        # Section 4.6 in 3-D, reduced: 63^3 and its double grid 125^3, kappa 10, 100, 1000, all
        # four solvers (Richardson where its O(kappa) count stays within 8000 iterations)
        line["kappa_63"] = kappa_sweep(63, (10.0, 100.0, 1000.0),
                                       ("richardson", "cg", "chebyshev", "eyre_milton"), 8000)
    if single and not args.no_served:
        # a short served run (driver-visible): 12 requests over 0.5 s, Richardson capped at
        # 2000 iterations (--serve runs longer mixes with the cap at 1e5)
        sv = served_mix(12, 0.5, 64.0, 2000)
        line["served"] = {k: sv[k] for k in ("value", "unit", "p50_ms", "p99_ms", "fp32_refined",
                                             "fp64", "speedup_vs_fp64",
                                             "AH_max_rel_diff_fp32_refined_vs_fp64",
                                             "AH_compared_requests", "config")}
    if single and not args.no_c4:
        line["c4_405_refined"] = c4_check()
    if single and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_oracle_cg_steps(1)
    if not single:
        line["studies"] = "elastic, kappa_63, served, c4_405_refined and cpu_baseline run at N = 1 only"
    return line


# ------------------------------------------------------------------------------------------
# served mix (continuous batching): FP32 inner solves with FP64 refinement vs plain FP64
# ------------------------------------------------------------------------------------------

def served_requests(n_req, seed=2024):
    """Seeded heterogeneous requests: odd grids from {45, 81, 135, 243}^3, periodic random
    spheres (volume fraction U[0.1, 0.4], radii U[0.02, 0.06] of the cell but at least 1.5
    nodes, so that a sphere on the 45^3 grid covers more than one node), contrast
    logU[10, 1e4], anisotropic SPD phase tensors R diag(lambda) R^T (Haar R,
    lambda = scale x logU[1, 3], scale 1 for the matrix and the contrast for every sphere),
    random unit E, solver uniform over Richardson, CG, Chebyshev and Eyre-Milton, tolerance
    1e-6."""
    rng = np.random.default_rng(seed)
    reqs = []
    grids = [45, 81, 135, 243]
    probs = [0.35, 0.35, 0.2, 0.1]
    solvers = ["richardson", "cg", "chebyshev", "eyre_milton"]
    for i in range(n_req):
        n = int(rng.choice(grids, p=probs))
        vf = rng.uniform(0.1, 0.4)
        contrast = float(np.exp(rng.uniform(np.log(10.0), np.log(1e4))))
        rmin = max(0.02, 1.5 / n)
        rmax = max(0.06, rmin + 0.02)
        ph, _, radii = ms.rsa_spheres((n,) * 3, seed + i, rmin=rmin, rmax=rmax, vf=vf)
        scales = np.concatenate([[1.0], np.full(len(radii), contrast)])
        table = ms.random_spd_table(len(scales), 3, seed + 1000 + i, scales)
        E = ms.random_unit_vector(3, seed + 2000 + i)
        solver = solvers[int(rng.integers(0, 4))]
        reqs.append({"n": n, "phase": ph, "table": table, "E": E, "solver": solver,
                     "contrast": contrast, "vf": float((ph > 0).mean())})
    return reqs


# the FP32-refined arm runs the two solvers it has inner FP32 kernels for: CG for requests
# drawn as CG or Richardson, Chebyshev for Chebyshev or Eyre-Milton
REFINED_SOLVER = {"richardson": "cg", "cg": "cg", "chebyshev": "chebyshev",
                  "eyre_milton": "chebyshev"}


def serve_arm(reqs, mats, arrivals, prec, budget_gb, rich_maxit):
    """Serve `reqs` through hom_server with the given arrival times (seconds from the start), in
    plain FP64 with the drawn solvers or FP32-refined; per-request latency, throughput from the
    first arrival to the last completion, converged and non-converged requests, A_H."""
    import torch
    import paper_1508_02045_gb300 as H

    S = H.hom_server_create(int(budget_gb * (1 << 30)), max_batch=8)
    submitted, results = {}, {}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nxt = 0
    steps = 0
    while len(results) < len(reqs):
        now = time.perf_counter() - t0
        while nxt < len(reqs) and arrivals[nxt] <= now:
            r = reqs[nxt]
            if prec == H.HOM_FP64:
                solver = r["solver"]
                maxit = rich_maxit if solver == "richardson" else 20000
            else:
                solver = REFINED_SOLVER[r["solver"]]
                maxit = 50
            q = H.make_request(3, (r["n"],) * 3, mats[nxt], r["E"], H.SOLVERS[solver], 1e-6,
                               precision=prec, opts=H.make_opts(maxit=maxit))
            submitted[H.hom_server_submit(S, q)] = nxt
            nxt += 1
        active, queued, _ = H.hom_server_status(S)
        if active == 0 and queued == 0:
            if nxt < len(reqs):
                time.sleep(max(0.0, arrivals[nxt] - (time.perf_counter() - t0)))
            continue
        H.hom_server_step(S, 8)
        steps += 1
        for res in H.hom_server_poll(S):
            results[submitted[res["id"]]] = res
    wall = time.perf_counter() - t0
    H.hom_server_destroy(S)
    lat = np.array([results[i]["latency_ms"] for i in range(len(reqs))])
    conv = [bool(results[i]["stats"]["converged"]) for i in range(len(reqs))]
    by_solver = {}
    for i, r in enumerate(reqs):
        sv = r["solver"] if prec == H.HOM_FP64 else REFINED_SOLVER[r["solver"]]
        e = by_solver.setdefault(sv, {"requests": 0, "converged": 0})
        e["requests"] += 1
        e["converged"] += int(conv[i])
    return {"solves_per_s": round(len(reqs) / (wall - arrivals[0]), 3),
            "p50_ms": round(float(np.percentile(lat, 50)), 1),
            "p99_ms": round(float(np.percentile(lat, 99)), 1),
            "wall_s": round(wall, 2), "steps": steps,
            "converged": int(sum(conv)), "not_converged": int(len(conv) - sum(conv)),
            "by_solver": by_solver,
            "AH": [results[i]["AH_EE"] for i in range(len(reqs))], "conv": conv}


SERVE_WORKLOAD = ("served mix: grids {45,81,135,243}^3, RSA spheres vf 0.1-0.4, radii 0.02-0.06 "
                  "(>= 1.5 nodes), contrast logU[10,1e4], anisotropic SPD phases, solver uniform "
                  "over the four (FP64 arm; the refined arm runs CG for CG/Richardson and "
                  "Chebyshev for Chebyshev/Eyre-Milton), tol 1e-6")


def served_mix(n_req, window, budget_gb, rich_maxit, seed=2024):
    """Serve the seeded mix through hom_server (Poisson arrivals over `window` seconds), once
    in plain FP64 with the drawn solvers and once FP32-refined; solves/s, p50/p99 latency,
    converged and non-converged requests, and the A_H agreement of the two arms."""
    import paper_1508_02045_gb300 as H

    reqs = served_requests(n_req, seed)
    rng = np.random.default_rng(seed + 7)
    arrivals = np.cumsum(rng.exponential(window / len(reqs), size=len(reqs)))
    mats = [H.phase_material(r["phase"], r["table"]) for r in reqs]
    out = {label: serve_arm(reqs, mats, arrivals, prec, budget_gb, rich_maxit)
           for label, prec in (("fp64", H.HOM_FP64), ("fp32_refined", H.HOM_FP32_REFINED))}
    a64 = np.array(out["fp64"].pop("AH"))
    a32 = np.array(out["fp32_refined"].pop("AH"))
    c64 = out["fp64"].pop("conv")
    c32 = out["fp32_refined"].pop("conv")
    both = [i for i in range(len(reqs)) if c64[i] and c32[i]]
    diff = float(np.max(np.abs(a32[both] - a64[both]) / np.abs(a64[both]))) if both else None
    return {"metric": "served solves/s (continuous batching, FP32 inner + FP64 refinement)",
            "value": out["fp32_refined"]["solves_per_s"], "unit": "solves/s",
            "higher_is_better": True, "n_gpus": 1, "dtype": "f32 inner / f64 outer",
            "data": "synthetic (seeded random-sphere microstructures)",
            "config": {"workload": SERVE_WORKLOAD,
                       "requests": len(reqs), "arrival_window_s": window,
                       "hbm_budget_gb": budget_gb, "max_batch": 8,
                       "richardson_maxit": rich_maxit,
                       "grid_counts": {str(g): int(sum(r["n"] == g for r in reqs)) for g in (45, 81, 135, 243)}},
            "p50_ms": out["fp32_refined"]["p50_ms"], "p99_ms": out["fp32_refined"]["p99_ms"],
            "fp32_refined": out["fp32_refined"], "fp64": out["fp64"],
            "speedup_vs_fp64": round(out["fp32_refined"]["solves_per_s"] / out["fp64"]["solves_per_s"], 2),
            "AH_max_rel_diff_fp32_refined_vs_fp64": diff,
            "AH_compared_requests": len(both)}


def serve_load(n_req, factors, budget_gb, rich_maxit, seed=2024):
    """The served mix at fixed offered loads: each arm's capacity is measured with every request
    queued at t = 0, then the FP32-refined arm serves the same requests with Poisson arrivals at
    factor x its capacity (seeded); throughput, p50 and p99 per load."""
    import paper_1508_02045_gb300 as H

    reqs = served_requests(n_req, seed)
    mats = [H.phase_material(r["phase"], r["table"]) for r in reqs]
    at_once = np.zeros(len(reqs))
    cap = {}
    ah = {}
    for label, prec in (("fp32_refined", H.HOM_FP32_REFINED), ("fp64", H.HOM_FP64)):
        res = serve_arm(reqs, mats, at_once, prec, budget_gb, rich_maxit)
        ah[label] = (np.array(res.pop("AH")), res.pop("conv"))
        cap[label] = res
    both = [i for i in range(len(reqs)) if ah["fp64"][1][i] and ah["fp32_refined"][1][i]]
    diff = (float(np.max(np.abs(ah["fp32_refined"][0][both] - ah["fp64"][0][both])
                         / np.abs(ah["fp64"][0][both]))) if both else None)
    c = cap["fp32_refined"]["solves_per_s"]
    rows = []
    for k, f in enumerate(factors):
        rng = np.random.default_rng(seed + 100 + k)
        arrivals = np.cumsum(rng.exponential(1.0 / (f * c), size=len(reqs)))
        res = serve_arm(reqs, mats, arrivals, H.HOM_FP32_REFINED, budget_gb, rich_maxit)
        res.pop("AH"), res.pop("conv")
        rows.append({"load": f, "offered_per_s": round(f * c, 3), **res})
    return {"metric": "served solves/s at offered loads (FP32 inner + FP64 refinement)",
            "unit": "solves/s", "n_gpus": 1, "data": "synthetic (seeded random-sphere microstructures)",
            "config": {"workload": SERVE_WORKLOAD, "requests": len(reqs), "hbm_budget_gb": budget_gb,
                       "max_batch": 8, "richardson_maxit": rich_maxit,
                       "grid_counts": {str(g): int(sum(r["n"] == g for r in reqs)) for g in (45, 81, 135, 243)}},
            "capacity": cap, "capacity_speedup_vs_fp64": round(c / cap["fp64"]["solves_per_s"], 2),
            "AH_max_rel_diff_fp32_refined_vs_fp64": diff, "AH_compared_requests": len(both),
            "loads": rows}


def elastic_step(steps, warmup, n=243, solves=False):
    """Linear elasticity (the strain form, six Mandel components) on the bench geometry: the
    243^3 cube of volume fraction 0.2, isotropic phases (lambda, mu) = (1, 1) and (1000, 1000),
    E = e_11; `steps` FP64 CG steps timed with CUDA events (inputs larger than L2: 688 MB a
    field), the operator's passes by kind; with `solves`, CG to 1e-8 in FP64 and FP32-refined."""
    import torch
    import paper_1508_02045_gb300 as H
    N = (n,) * 3
    ph = ms.box_phase(N, ms.inclusion_side_for_fraction(VF, D))
    table = np.array([elastic_stiffness(1.0, 1.0), elastic_stiffness(CONTRAST, CONTRAST)])
    P = H.Problem(3, N, H.stiffness_material(ph, table))
    E = np.array([1.0, 0, 0, 0, 0, 0])
    H.hom_solve_begin(P.h, E, H.HOM_CG, 0.0, H.make_opts(fixed_iters=steps + warmup + 1))
    H.hom_solve_iterate(P.h, warmup)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    H.hom_profile_enable(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    H.hom_solve_iterate(P.h, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    H.hom_profile_enable(False)
    passes = H.hom_profile_read()
    ms_step = e0.elapsed_time(e1) / steps
    H.hom_solve_end(P.h, 6, allow_not_converged=True)
    out = {"metric": "G·C matvecs/s at 243^3, linear elasticity (FP64 CG step, 6 components)",
           "value": round(1000.0 / ms_step, 3), "unit": UNIT, "ms_per_step": round(ms_step, 4),
           "steps": steps, "grid": list(N),
           "passes": {k: {"ms_avg": round(v[0] / v[1], 4), "launches": v[1]}
                      for k, v in passes.items() if v[1]}}
    if solves:
        # CG to 1e-8 in FP64 and with FP32 inner solves in FP64 refinement (outside the timed
        # region of the step)
        res = {}
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        AH, _, st, _ = H.hom_solve(P.h, E, H.HOM_CG, 1e-8, H.make_opts(maxit=5000))
        torch.cuda.synchronize()
        res["fp64"] = {"seconds": round(time.perf_counter() - t0, 3), "A_H": AH,
                       "iterations": st["iterations"], "converged": bool(st["converged"])}
        P.close()
        P = H.Problem(3, N, H.stiffness_material(ph, table), precision=H.HOM_FP32_REFINED)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        AH32, _, st, _ = H.hom_solve(P.h, E, H.HOM_CG, 1e-8, H.make_opts(maxit=50))
        torch.cuda.synchronize()
        res["fp32_refined"] = {"seconds": round(time.perf_counter() - t0, 3), "A_H": AH32,
                               "iterations": st["iterations"],
                               "inner_iterations": st["inner_iterations"],
                               "converged": bool(st["converged"])}
        res["A_H_rel_diff"] = abs(AH32 - AH) / AH
        res["speedup"] = round(res["fp64"]["seconds"] / res["fp32_refined"]["seconds"], 2)
        out["cg_to_1e-8"] = res
    P.close()
    return out


def elastic_stiffness(lam, mu):
    """Mandel matrix (3-D) of the isotropic stiffness lam tr(e) I + 2 mu e (an input table)."""
    C = np.zeros((6, 6))
    C[:3, :3] = lam
    for a in range(3):
        C[a, a] += 2 * mu
    for m in range(3, 6):
        C[m, m] = 2 * mu
    return C


def run_served(args):
    if args.serve_load:
        print(json.dumps(serve_load(args.serve, (0.5, 0.8, 1.0, 1.2), args.serve_budget_gb,
                                    args.serve_rich_maxit)), flush=True)
        return
    print(json.dumps(served_mix(args.serve, args.serve_window, args.serve_budget_gb,
                                args.serve_rich_maxit)), flush=True)


def c4_check():
    """Configuration 4 (405^3 random spheres, FP32 inner CG in FP64 refinement, tolerance 1e-8)
    with its error stated against the FP64 oracle: the oracle evaluates, at the refined
    solution x, the residual ||C x - b|| (one oracle matvec) and the energy. Since C is SPD on
    the conforming space with smallest eigenvalue >= c_A and x - x* lies in that space, the
    A_H of x exceeds the exact discrete A_H by (C(x - x*), x - x*) <= ||C x - b||^2 / c_A, a
    bound computed by the oracle alone. The plain FP64 solve runs beside it."""
    import torch
    import oracle as O
    import paper_1508_02045_gb300 as H

    N = (405,) * 3
    E = np.array([1.0, 0.0, 0.0])
    ph, _, radii = ms.rsa_spheres(N, 1, vf=0.3)
    rng = np.random.default_rng(101)
    table = ms.isotropic_table(np.concatenate(
        [[1.0], np.exp(rng.uniform(np.log(10), np.log(1000), len(radii)))]), 3)
    out = {"grid": list(N), "spheres": int(len(radii)), "vf": float((ph > 0).mean()), "tol": 1e-8}
    for label, prec, maxit in (("fp32_refined", H.HOM_FP32_REFINED, 50), ("fp64", H.HOM_FP64, 3000)):
        P = H.Problem(3, N, H.phase_material(ph, table), precision=prec)
        x = P.field() if label == "fp32_refined" else None
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        AH, _, st, _ = H.hom_solve(P.h, E, H.HOM_CG, 1e-8, H.make_opts(maxit=maxit), x,
                                   allow_not_converged=True)
        torch.cuda.synchronize()
        out[label] = {"A_H": AH, "seconds": round(time.perf_counter() - t0, 3),
                      "iterations": st["iterations"], "inner_iterations": st["inner_iterations"],
                      "converged": bool(st["converged"]), "true_residual": st["true_residual"]}
        if x is not None:
            xh = x.cpu().numpy()
        del x
        P.close()
    t0 = time.perf_counter()
    A = O.expand_phase(ph, table)[0, 0]
    sysn = O.GaNi(A, 3)
    v = sysn.const(E) + xh
    res = sysn.matvec(v)                       # C x - b = G A (E + x)
    rn = float(np.sqrt(np.mean(np.sum(res * res, axis=0))))
    en = O.energy(A, v)
    cA = float(A.min())
    AH32 = out["fp32_refined"]["A_H"]
    out["oracle_check"] = {
        "residual_norm": rn, "energy_at_x": en,
        "A_H_minus_oracle_energy_rel": abs(AH32 - en) / en,
        "A_H_error_bound_rel": rn * rn / cA / en,
        "seconds": round(time.perf_counter() - t0, 1),
        "what": "FP64 NumPy oracle at the refined solution x: ||C x - b|| (one matvec), its "
                "energy, and the bound ||C x - b||^2 / c_A on A_H(x) - A_H(x*)"}
    out["A_H_rel_diff_fp32_refined_vs_fp64"] = abs(AH32 - out["fp64"]["A_H"]) / out["fp64"]["A_H"]
    out["speedup"] = round(out["fp64"]["seconds"] / out["fp32_refined"]["seconds"], 2)
    return out


# ------------------------------------------------------------------------------------------
# configurations 1-4 end to end (solver results and times; not the bench line)
# ------------------------------------------------------------------------------------------

def run_configs(args):
    import torch
    import paper_1508_02045_gb300 as H

    out = {}
    sync = torch.cuda.synchronize

    def solve(P, E, solver, tol, opts=None, x=None):
        sync()
        t0 = time.perf_counter()
        AH, flux, st, status = H.hom_solve(P.h, E, solver, tol, opts, x, allow_not_converged=True)
        sync()
        return {"A_H": AH, "iterations": st["iterations"], "inner_iterations": st["inner_iterations"],
                "converged": bool(st["converged"]), "true_residual": st["true_residual"],
                "seconds": round(time.perf_counter() - t0, 4)}

    # config 1: 2-D 63^2, square of side 0.6, contrast 10, E = (1, 0), Richardson and CG to 1e-8
    N = (63, 63)
    P = H.Problem(2, N, H.phase_material(ms.box_phase(N, 0.6), ms.isotropic_table([1.0, 10.0], 2)))
    E = np.array([1.0, 0.0])
    out["c1_63sq"] = {s: solve(P, E, H.SOLVERS[s], 1e-8) for s in ("richardson", "cg")}
    P.close()
    # config 2: 243^3 cube vf 0.2, contrast 1e3, all four solvers to 1e-6
    N = (243,) * 3
    P = H.Problem(3, N, H.phase_material(ms.box_phase(N, ms.inclusion_side_for_fraction(0.2, 3)),
                                        ms.isotropic_table([1.0, 1000.0], 3)))
    E = np.array([1.0, 0.0, 0.0])
    out["c2_243cube"] = {}
    for s in ("cg", "chebyshev", "eyre_milton", "richardson"):
        out["c2_243cube"][s] = solve(P, E, H.SOLVERS[s], 1e-6, H.make_opts(maxit=args.configs_maxit))
        r = out["c2_243cube"][s]
        r["matvecs_per_s"] = round(r["iterations"] / r["seconds"], 2)
    P.close()
    # config 3: Ga, N = 81^3 on the double grid 161^3, cube vf 0.3, contrast 100, CG to 1e-8,
    # with the GaNi guaranteed bound via prolongation and the Hashin-Shtrikman lower bound
    N = (81,) * 3
    h = ms.inclusion_side_for_fraction(0.3, 3)
    Pn = H.Problem(3, N, H.phase_material(ms.box_phase(N, h), ms.isotropic_table([1.0, 100.0], 3)))
    xn = Pn.field()
    gani = solve(Pn, E, H.HOM_CG, 1e-8, None, xn)
    M = (161,) * 3
    Pg = H.Problem(3, N, H.fourier_material(ms.box_fourier_coefficients(M, h, 1.0, 100.0).astype(np.complex128),
                                            1.0, 100.0), H.HOM_EXACT)
    bound = H.hom_bound(Pn.h, Pg.h, E, xn)
    gar = solve(Pg, E, H.HOM_CG, 1e-8)
    hs = 1.0 + 0.3 / (1.0 / 99.0 + 0.7 / 3.0)
    out["c3_ga_81_on_161"] = {"gani": gani, "gani_bound": bound, "ga": gar, "hashin_shtrikman_lower": hs,
                              "ordering_holds": bool(hs < gar["A_H"] < bound)}
    Pn.close()
    Pg.close()
    # the same study on an image (Section 2.2 for voxel-wise constant coefficients): 81^3 random
    # spheres (vf 0.3, contrast 100), GaNi, its guaranteed bound via prolongation to 161^3 and
    # the exact-integration value of the image on 161^3
    ph, _, radii = ms.rsa_spheres(N, 2, vf=0.3)
    table = ms.isotropic_table(np.concatenate([[1.0], np.full(len(radii), 100.0)]), 3)
    Pn = H.Problem(3, N, H.phase_material(ph, table))
    Pg = H.Problem(3, N, H.phase_material(ph, table), H.HOM_EXACT)
    xn = Pn.field()
    gani = solve(Pn, E, H.HOM_CG, 1e-8, None, xn)
    bound = H.hom_bound(Pn.h, Pg.h, E, xn)
    gar = solve(Pg, E, H.HOM_CG, 1e-8)
    out["c3_voxel_ga_spheres_81_on_161"] = {
        "spheres": int(len(radii)), "gani": gani, "gani_bound": bound, "ga": gar,
        "bound_gap_rel": (bound - gar["A_H"]) / gar["A_H"], "ordering_holds": bool(gar["A_H"] < bound)}
    Pn.close()
    Pg.close()
    # config 4: 405^3 random spheres, log-uniform conductivities, CG in FP64 vs FP32 + refinement
    N = (405,) * 3
    ph, _, radii = ms.rsa_spheres(N, 1, vf=0.3)
    rng = np.random.default_rng(101)
    table = ms.isotropic_table(np.concatenate([[1.0], np.exp(rng.uniform(np.log(10), np.log(1000), len(radii)))]), 3)
    res = {}
    for label, prec in (("fp32_refined", H.HOM_FP32_REFINED), ("fp64", H.HOM_FP64)):
        P = H.Problem(3, N, H.phase_material(ph, table), precision=prec)
        res[label] = solve(P, E, H.HOM_CG, 1e-8, H.make_opts(maxit=3000 if prec == H.HOM_FP64 else 50))
        P.close()
    res["A_H_rel_diff"] = abs(res["fp32_refined"]["A_H"] - res["fp64"]["A_H"]) / res["fp64"]["A_H"]
    res["speedup"] = round(res["fp64"]["seconds"] / res["fp32_refined"]["seconds"], 2)
    res["spheres"] = int(len(radii))
    out["c4_405_spheres"] = res
    print(json.dumps({"configs": out}), flush=True)


def kappa_sweep(n, kappas, solvers, maxit):
    """Iterations to the relative residual 1e-6 against the contrast (Section 4.6) for the cube
    of volume fraction 0.2 on n^3 (GaNi) and its double grid (Ga); returns rows and the growth
    of the count from the first to the last contrast."""
    import torch
    import paper_1508_02045_gb300 as H

    N = (n,) * 3
    M = tuple(2 * k - 1 for k in N)
    E = np.array([1.0, 0.0, 0.0])
    h = ms.inclusion_side_for_fraction(0.2, 3)
    rows = []
    for kappa in kappas:
        probs = {"gani": H.Problem(3, N, H.phase_material(ms.box_phase(N, h),
                                                          ms.isotropic_table([1.0, kappa], 3))),
                 "ga": H.Problem(3, N, H.fourier_material(
                     ms.box_fourier_coefficients(M, h, 1.0, kappa).astype(np.complex128), 1.0, kappa),
                     H.HOM_EXACT)}
        for disc, P in probs.items():
            for s in solvers:
                if disc == "ga" and s == "eyre_milton":
                    continue  # not defined for Ga (Section 3.4)
                if s == "richardson" and 0.5 * kappa * np.log(1e6) > maxit:
                    continue
                stop = H.HOM_STOP_INCREMENT if s == "eyre_milton" else H.HOM_STOP_RESIDUAL
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                AH, _, st, _ = H.hom_solve(P.h, E, H.SOLVERS[s], 1e-6,
                                           H.make_opts(maxit=maxit, stop=stop),
                                           allow_not_converged=True)
                torch.cuda.synchronize()
                rows.append({"kappa": kappa, "discretization": disc, "solver": s,
                             "iterations": st["iterations"], "converged": bool(st["converged"]),
                             "A_H": AH, "seconds": round(time.perf_counter() - t0, 4)})
        for P in probs.values():
            P.close()
    lo, hi = kappas[0], kappas[-1]
    growth = {}
    for r in rows:
        if r["kappa"] in (lo, hi):
            growth.setdefault((r["discretization"], r["solver"]), {})[r["kappa"]] = r["iterations"]
    ratio = {f"{d}/{s}": round(v[hi] / v[lo], 2) for (d, s), v in growth.items() if len(v) == 2}
    return {"grid": list(N), "double_grid": list(M), "tol": 1e-6, "rows": rows,
            f"iterations_ratio_{int(hi)}_over_{int(lo)}": ratio}


def run_kappa(args):
    """Section 4.6 rerun in 3-D: iterations to the relative residual 1e-6 against the contrast
    kappa (inclusion coefficient, matrix 1) for the cubic inclusion of volume fraction 0.2, GaNi
    on N^3 with all four solvers and Ga on the double grid (2N-1)^3 with Richardson, CG and
    Chebyshev; every solver stops on the relative residual, as in the paper's study (Eyre-Milton,
    which has no residual of its own, on its increment). Richardson is run where its O(kappa)
    iteration count stays within --kappa-maxit."""
    out = kappa_sweep(args.kappa, (10.0, 100.0, 1000.0, 10000.0),
                      ("richardson", "cg", "chebyshev", "eyre_milton"), args.kappa_maxit)
    print(json.dumps({"kappa_study": out}), flush=True)


def run_reference(args, rank, world):
    if rank != 0:
        return None
    # the oracle as it stands, on this host's cores, same workload and unit: Algorithm 2 step by
    # step on the oracle's operator (set-up matvec untimed), W warm-up steps, then K timed steps
    import oracle as O
    ph, table = workload()
    sysn = O.GaNi(O.expand_phase(ph, table)[0, 0], D)
    b = sysn.rhs(E_MACRO)
    state = {"x": np.zeros_like(b), "r": b.copy(), "p": b.copy()}

    def dot(u, v):
        return float(np.mean(np.sum(u * v, axis=0)))

    state["rr"] = dot(b, b)

    def step():
        Cp = sysn.matvec(state["p"])
        alpha = state["rr"] / dot(Cp, state["p"])
        state["x"] = state["x"] + alpha * state["p"]
        state["r"] = state["r"] - alpha * Cp
        rr_new = dot(state["r"], state["r"])
        state["p"] = state["r"] + (rr_new / state["rr"]) * state["p"]
        state["rr"] = rr_new

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    v = args.steps / dt
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    sample = (f"{args.steps} timed oracle CG iterations after {args.warmup} warm-up ones at 243^3 "
              f"(one matvec each, {dt:.1f} s, NumPy FP64 dense-matrix DFT, BLAS threads = host cores)")
    return {
        "impl": "reference", "metric": METRIC, "value": round(v, 5), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1000.0 / v, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded centred-cube phase image)", "config": config(),
        "cpu_baseline": {"value": round(v, 5), "unit": UNIT, "cores": cores, "cpu": host_cpu(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(v, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true")
    ap.add_argument("--grid", type=int, default=0)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "elastic"],
                    help="with --quick: time the FP64 CG step, the FP32 inner CG step or the "
                         "elasticity CG step")
    ap.add_argument("--serve", type=int, default=0, help="run the served mix with this many requests")
    ap.add_argument("--serve-window", type=float, default=1.0)
    ap.add_argument("--serve-load", action="store_true",
                    help="with --serve N: capacity of both arms, then the refined arm at 0.5, 0.8, "
                         "1.0 and 1.2 x its capacity")
    ap.add_argument("--serve-budget-gb", type=float, default=64.0)
    ap.add_argument("--serve-rich-maxit", type=int, default=100000)
    ap.add_argument("--no-served", action="store_true", help="skip the short served run")
    ap.add_argument("--no-c4", action="store_true", help="skip the 405^3 refinement check")
    ap.add_argument("--no-elastic", action="store_true", help="skip the elasticity step")
    ap.add_argument("--no-kappa", action="store_true", help="skip the reduced contrast study")
    ap.add_argument("--inner-form", type=int, default=0, choices=[0, 1],
                    help="--quick --precision fp32: 0 potential coordinates, 1 field form")
    ap.add_argument("--no-tune", action="store_true",
                    help="with --quick: keep the default launch plan (profiler captures)")
    ap.add_argument("--configs", action="store_true", help="run configurations 1-4 end to end")
    ap.add_argument("--configs-maxit", type=int, default=20000)
    ap.add_argument("--kappa", type=int, default=0,
                    help="iterations against the contrast (Section 4.6) on this odd N^3")
    ap.add_argument("--kappa-maxit", type=int, default=20000)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.serve:
        run_served(args)
        return
    if args.configs:
        run_configs(args)
        return
    if args.kappa:
        run_kappa(args)
        return
    if args.impl == "reference":
        rank = int(os.environ.get("RANK", "0"))
        world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
        line = run_reference(args, rank, world)
    else:
        rank, world, local = dist_init()
        line = run_ours(args, rank, world, local)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
