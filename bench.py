"""Benchmark: FFT-accelerated matvecs/s at N = 16384 on the deep corrugation (TM/Neumann, period 10
wavelengths, depth/period 2, 128 x 257 cells), mixed precision (FP32 complex projection/FFT/
interpolation, float-float near field) beside the FP64 path.

The workload uses the periodic Green function without shifts (j = 0, n_per = 2048), as the paper
does for its deep non-Wood gratings (Section 6, Table deep_gratings); the same geometry with the
shifted kernel (j = 8) is timed beside it, and the headline FP64 and mixed solves are timed too.

One step = one application of the accelerated operator (Algorithm 3) to one density vector,
inputs resident on the device. L2 is flushed (256 MiB write) before every timed step; each step is
timed with CUDA events on the stream the library launches on, the flush outside the events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank builds its own replica (independent problems, no collective) and the
slowest rank's time is reported. `--impl reference` times the CPU oracle: the exact operator,
assembled as dense rows of the same workload, applied by ZGEMV on all host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1707_04950_gb300 import inputs  # noqa: E402

WORKLOAD = "deep_corrugation_tm_d10_depth20_n16384_cells128x257"
METRIC = "FFT-accel shifted-Green matvecs/s at N=16384; mixed vs FP64 at 1e-6 rel err"


def workload():
    return inputs.wl_deep_corrugation_neumann(N=16384, nx=128)


def job_times(local, device=None):
    """Per-quantity maximum over the ranks of this rank's times (the job is as slow as its slowest
    replica); the local values when running alone."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return list(local)
    t = torch.tensor(list(local), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def whole_job_rate(world_size, ms_per_step):
    """Applications per second of the whole job: every rank applies its own replica once per step."""
    return world_size * 1000.0 / ms_per_step


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons while the GPU is under the benchmark's
    load. nvidia-smi writes its samples straight to a file (-f), so nothing is lost in a pipe buffer
    when it is stopped; start() returns once the first sample is on disk."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # the raw samples go to SGF_CLOCKS_DIR (default: the system's temporary directory); the JSON
        # line carries their summary
        out_dir = os.environ.get("SGF_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"clocks_gpu{index}_{os.getpid()}.csv")

    def _lines(self):
        try:
            with open(self.path) as f:
                return [ln for ln in f.read().splitlines() if ln.strip()]
        except OSError:
            return []

    def start(self, wait_s=5.0):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            if os.path.exists(self.path):
                os.remove(self.path)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        t0 = time.time()
        while time.time() - t0 < wait_s and not self._lines():
            time.sleep(0.05)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.send_signal(2)  # SIGINT: nvidia-smi closes its file
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self._lines():
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm), "window": "nvidia-smi every 100 ms across the load window that holds the "
                                              "timed steps (at least 1 s of back-to-back applications)"}


STAGES = ["project", "fft_x", "conv_y", "ifft_x", "near", "interp"]


def stage_bytes(info, s):
    """Algorithmic bytes per stage of the forward map (compulsory traffic) for far-field complex size
    s (8 mixed, 16 FP64); the near field is float-float (16 bytes per entry) or FP64 either way."""
    N, nnz, neq, nfit = info["N"], info["nnz"], info["neq"], info["nfit"]
    gH, gV = info["PxH"] * info["nrowH"], info["PxV"] * info["nrowV"]
    kH, kV = info["PxH"] * info["PyH"], info["PxV"] * info["PyV"]
    return {
        "project": s * 4 * neq * N + 16 * N + s * 2 * (gH + gV) * 2,
        "fft_x": s * 2 * 2 * (gH + gV),
        "conv_y": s * ((2 * gH + 2 * kH + gH) + (2 * gV + 2 * kV + gV)),
        "ifft_x": s * 2 * (gH + gV),
        "near": 16 * nnz + 32 * N,
        "interp": s * nfit * N + s * info["n_occ"] * nfit + 32 * N,
    }


# launches per stage of one application (two orientations where a stage has two)
LAUNCHES = {"project": 1, "fft_x": 2, "conv_y": 2, "ifft_x": 2, "near": 1, "interp": 1}
# DRAM bytes (read + write) per launch of the current mixed-path kernels at the benchmark workload,
# from one ncu capture of the first mixed application (graph capture off, so that ncu sees the
# launches): `SGF_NO_GRAPH=1 ncu --set full --clock-control none -k regex:"k_(near_rows|conv_y|fft_x|
# project|interp_far)" -s 89 -c 9 -o prof_mixed python bench.py --steps 3 --warmup 3 --batch 0
# --gradient 0 --field 0 --solve 0 --shifted 0 --sweep 0 --multi 0 --no-cpu-baseline`. Two-launch
# stages give the mean of their H and V launches. Each kernel's writes stay in the 129 MB L2 while it
# runs (ncu reports 0 bytes written), so these are the reads. None where no capture of the current
# kernel exists.
DRAM_BYTES_PER_LAUNCH = {"project": 12.708e6, "fft_x": 4.274e6, "conv_y": 13.743e6, "ifft_x": 2.163e6,
                         "near": 36.591e6, "interp": 5.438e6}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def time_applies(sgf, op, mu, out, stream, flush, steps, warmup):
    """Mean CUDA-event time (ms) of one application, L2 flushed before every step (outside the
    events), after `warmup` untimed applications."""
    import torch

    for _ in range(warmup):
        sgf.sgf_apply(op.ctx, mu.data_ptr(), out.data_ptr())
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        sgf.sgf_apply(op.ctx, mu.data_ptr(), out.data_ptr())
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    return float(np.mean([a.elapsed_time(b) for a, b in ev]))


def stage_times(sgf, op, mu, out, flush, n):
    """Per-stage device times (ms) of `n` applications with profiling on: the stages then run one
    after another on the context stream, each bracketed by CUDA events on that stream."""
    sgf.sgf_set_profiling(op.ctx, 1)
    st = np.zeros(8)
    for _ in range(n):
        flush.zero_()
        sgf.sgf_apply(op.ctx, mu.data_ptr(), out.data_ptr())
        st += sgf.sgf_stage_times(op.ctx)
    sgf.sgf_set_profiling(op.ctx, 0)
    st /= n
    return dict(zip(STAGES, st[:6].tolist()))


def run_solves(sgf, par, dev, stream, tol, maxit):
    """Headline solves (Algorithm 1, zero initial guess): FP64 GMRES and the mixed path (FP32 far
    field, FP64 residual refinement), each timed end to end (one untimed solve first), with the
    energy error of its solution and the distance between the two solutions."""
    import torch

    out = {}
    sols = {}
    for prec in (64, 32):
        op = sgf.Operator(par, device=dev.index, stream=stream.cuda_stream, precision=prec)
        x = torch.zeros(par["N"], dtype=torch.complex128, device=dev)
        sgf.sgf_solve(op.ctx, tol, maxit, x.data_ptr())  # warm-up
        x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, its, rr = sgf.sgf_solve(op.ctx, tol, maxit, x.data_ptr())
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        _, _, eps = sgf.sgf_rayleigh(op.ctx, x.data_ptr(), -40, 40)
        op.close()
        sols[prec] = x
        out["fp64" if prec == 64 else "mixed"] = {
            "value": 1.0 / t, "unit": "solves/s", "s": t, "tol": tol, "status": st, "applications": its,
            "relres": rr, "energy_error": eps}
    out["mixed_vs_fp64_solution_rel"] = float(torch.linalg.norm(sols[32] - sols[64]) / torch.linalg.norm(sols[64]))
    return out


def run_ours(args):
    import torch

    from paper_1707_04950_gb300 import sgf

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    par = workload()
    stream = torch.cuda.current_stream(dev)
    mu_h = inputs.random_density(par["N"], 7 + rank)
    mu = torch.from_numpy(mu_h).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    res = {}
    ops = {}
    for prec in (64, 32):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        op = sgf.Operator(par, device=local, stream=stream.cuda_stream, precision=prec)
        torch.cuda.synchronize()
        t_build = time.perf_counter() - t0
        ops[prec] = op
        out = torch.empty_like(mu)
        clocks = Clocks(local)
        if prec == 32:
            clocks.start()
            # back-to-back load before the timed steps, so that the sampler sees the clocks under it
            t0 = time.perf_counter()
            while time.perf_counter() - t0 < 0.5:
                for _ in range(50):
                    sgf.sgf_apply(op.ctx, mu.data_ptr(), out.data_ptr())
                torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        ms = time_applies(sgf, op, mu, out, stream, flush, args.steps, args.warmup)
        if ws > 1:
            torch.distributed.barrier()
        ck = None
        if prec == 32:
            t0 = time.perf_counter()
            while time.perf_counter() - t0 < 0.5:
                for _ in range(50):
                    sgf.sgf_apply(op.ctx, mu.data_ptr(), out.data_ptr())
                torch.cuda.synchronize()
            ck = clocks.stop()
        stg = stage_times(sgf, op, mu, out, flush, max(3, min(args.steps, 20)))
        info = op.info
        res[prec] = {"ms": ms, "stages_ms": stg, "clocks": ck, "out": out.clone(), "info": info,
                     "init": {"s": t_build, "build_ms": info["build_ms"], "tables_ms": info["build_tables_ms"],
                              "least_squares_ms": info["build_ls_ms"], "near_operator_ms": info["build_near_ms"]}}
    # accuracy of the mixed path against the FP64 path on the benchmark input
    y64, y32 = res[64]["out"], res[32]["out"]
    mixed_err = float(torch.linalg.norm(y32 - y64) / torch.linalg.norm(y64))
    # end to end through the C ABI with host buffers (copies inside the timed region)
    op32 = ops[32]
    mu_pin = torch.from_numpy(mu_h).pin_memory()
    y_pin = torch.empty_like(mu_pin).pin_memory()
    for _ in range(max(1, args.warmup)):
        sgf.sgf_apply_host_ptr(op32.ctx, mu_pin.data_ptr(), y_pin.data_ptr())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sgf.sgf_apply_host_ptr(op32.ctx, mu_pin.data_ptr(), y_pin.data_ptr())
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / args.steps
    for op in ops.values():
        op.close()
    solves = run_solves(sgf, par, dev, stream, 1e-12, 4000) if args.solve and rank == 0 else None
    shifted = run_shifted(sgf, dev, stream, flush, args) if args.shifted and rank == 0 else None
    multi = run_multi_rhs(sgf, dev, stream, flush, args) if args.multi and rank == 0 else None
    periods = run_periods(sgf, dev, stream, flush, args.periods) if args.periods > 1 and rank == 0 else None
    sweep = run_sweep(sgf, dev, stream, flush, args) if args.sweep and rank == 0 else None
    batch = run_batch(args, dev, stream, flush) if args.batch > 0 and rank == 0 else None
    grad = run_gradient(dev, stream) if args.gradient and rank == 0 else None
    tune = run_autotune(dev, stream) if args.gradient and rank == 0 else None
    field = run_field(dev, stream) if args.field and rank == 0 else None
    exact = run_exact(dev, stream, flush, max(3, min(args.steps, 50))) if args.field and rank == 0 else None
    tables = run_tables(dev, stream) if args.tables and rank == 0 else None
    st32 = res[32]["stages_ms"]
    cufft = run_cufft_reference(res[32]["info"], st32["fft_x"] + st32["conv_y"] + st32["ifft_x"], dev, stream, flush,
                                max(3, min(args.steps, 50))) if rank == 0 else None

    ms32, ms64, e2e_s = job_times([res[32]["ms"], res[64]["ms"], e2e_s], dev)
    if rank != 0:
        return
    info = res[32]["info"]
    # roofline of the dominant kernel of the headline (mixed) path, from its own CUDA-event time
    hbm, kind = peaks()
    sb = stage_bytes(info, 8)
    stg = res[32]["stages_ms"]
    dom = max(STAGES, key=lambda k: stg[k])
    per_launch_ms = stg[dom] / LAUNCHES[dom]
    ach = sb[dom] / LAUNCHES[dom] / (per_launch_ms * 1e-3) / 1e9
    kernel_names = {"project": "k_project", "fft_x": "k_fft_x (forward)", "conv_y": "k_conv_y",
                    "ifft_x": "k_fft_x (inverse)", "near": "k_near_rows<float>", "interp": "k_interp_far<float>"}
    line = {
        "metric": METRIC,
        "value": whole_job_rate(ws, ms32),
        "unit": "matvecs/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms32,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "c64 far field (projection, FFT, interpolation); float-float (FP32 hi/lo pairs, compensated "
                 "FP32 arithmetic) near field and modes; c128 in and out",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": int(par["N"]), "cells": f"{par['nx']}x{par['ny']}", "k": "2pi",
                   "theta_deg": 45, "bc": "neumann", "shifts_j": int(par["j"]), "n_per": int(par["n_per"]),
                   "eq_sources_per_orientation": int(info["neq"]),
                   "fft_grids": f"H {int(info['PxH'])}x{int(info['PyH'])}, V {int(info['PxV'])}x{int(info['PyV'])}",
                   "near_field_entries": int(info["nnz"]), "l2": "flushed (256 MiB write) before each timed step",
                   "parallelism": f"replicas x{ws}"},
        "fp64": {"value": ws * 1000.0 / ms64, "unit": "matvecs/s", "ms_per_step": ms64,
                 "stages_ms": res[64]["stages_ms"],
                 "whole_step_hbm_frac": res[64]["info"]["bytes64"] / (ms64 * 1e-3) / 1e9 / hbm},
        "whole_step_hbm_frac": info["bytes32"] / (ms32 * 1e-3) / 1e9 / hbm,
        "mixed_rel_err_vs_fp64": mixed_err,
        "stages_ms": stg,
        "stage_hbm_frac": {k: sb[k] / (stg[k] * 1e-3) / 1e9 / hbm for k in STAGES if stg[k] > 0},
        "init": {"mixed": res[32]["init"], "fp64": res[64]["init"]},
        "roofline": {"bound": "hbm", "kernel": kernel_names[dom], "stage": dom, "achieved": ach, "peak": hbm,
                     "unit": "GB/s", "frac": ach / hbm, "traffic": DRAM_BYTES_PER_LAUNCH.get(dom), "peak_kind": kind,
                     "algorithmic_bytes_per_launch": sb[dom] / LAUNCHES[dom],
                     "time": "CUDA events around the stage's launches on the library's stream (stages serialised)"},
        "e2e": {"value": ws / e2e_s, "unit": "matvecs/s", "h2d_bytes_per_step": 16 * int(par["N"]),
                "d2h_bytes_per_step": 16 * int(par["N"])},
        "gpu_launches": int(info["launches"]) * args.steps,
        "clocks": res[32]["clocks"],
    }
    if solves is not None:
        line["solve"] = solves
    if shifted is not None:
        line["shifted_j8"] = shifted
    if periods is not None:
        line["periods"] = periods
    if multi is not None:
        line["multi_rhs"] = multi
    if sweep is not None:
        line["sweep_batch"] = sweep
    if batch is not None:
        line["batch"] = batch
    if grad is not None:
        line["gradient"] = grad
    if tune is not None:
        line["autotune"] = tune
    if field is not None:
        line["field"] = field
    if exact is not None:
        line["exact_dense"] = exact
    if tables is not None:
        line["sinusoid_tables"] = tables
    if cufft is not None:
        line["cufft_reference"] = cufft
    if not args.no_cpu_baseline and ws >= 1:
        line["cpu_baseline"] = cpu_baseline(rows=args.cpu_rows)
    print(json.dumps(line), flush=True)


def run_sweep(sgf, dev, stream, flush, args):
    """The batched sweep, bounded to one surface per period: Gaussian rough surfaces of periods 10,
    25, 50, 100 (N = 2048 ... 16384), each at 16 of the 64 incidence angles (every 4th) and at 4 of
    the 16 Wood wavenumbers (w = 1, 5, 9, 13), mixed precision: 80 problems. Timed two ways: one
    batch over all 80 (one graph launch per application of every problem) and one batch per surface
    and wavenumber (where the angles of a surface may take the multi-column form). Solves: lockstep
    GMRES of every batch to 1e-8."""
    import torch

    t0 = time.perf_counter()
    groups = []
    for pi in range(len(inputs.SWEEP_SURFACES)):
        ang = [sgf.Operator(inputs.wl_sweep_angle(pi, 0, i), device=dev.index, stream=stream.cuda_stream,
                            precision=32) for i in range(0, 64, 4)]
        wood = [sgf.Operator(inputs.wl_sweep_wood(pi, 0, w), device=dev.index, stream=stream.cuda_stream,
                             precision=32) for w in (1, 5, 9, 13)]
        groups.append((ang, wood))
    torch.cuda.synchronize()
    t_init = time.perf_counter() - t0
    ops = [op for a, w in groups for op in a + w]
    xs = [torch.from_numpy(inputs.random_density(op.par["N"], 90 + p)).to(dev) for p, op in enumerate(ops)]
    ys = [torch.empty_like(x) for x in xs]
    steps = max(3, min(args.steps, 20))

    def timed(batches):
        def once():
            for b, idx in batches:
                sgf.sgf_batch_apply(b, [xs[i].data_ptr() for i in idx], [ys[i].data_ptr() for i in idx])
        for _ in range(3):
            once()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            flush.zero_()
            ev[k][0].record(stream)
            once()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        return float(np.mean([a.elapsed_time(b) for a, b in ev]))

    b_all = sgf.sgf_batch_create([op.ctx for op in ops], stream.cuda_stream)
    ms_all = timed([(b_all, list(range(len(ops))))])
    sgf.sgf_batch_destroy(b_all)
    per = []
    forms = []
    p0 = 0
    for ang, wood in groups:
        for grp in (ang, wood):
            idx = list(range(p0, p0 + len(grp)))
            b = sgf.sgf_batch_create([op.ctx for op in grp], stream.cuda_stream)
            per.append((b, idx))
            forms.append(int(sgf.sgf_batch_shared_near(b)))
            p0 += len(grp)
    ms_per = timed(per)
    mus = [torch.zeros_like(x) for x in xs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    its_all, rr_max, st_all = [], 0.0, 0
    for b, idx in per:
        st, its, rr = sgf.sgf_batch_solve(b, 1e-8, 2000, [mus[i].data_ptr() for i in idx])
        st_all = st_all or st
        its_all += list(its)
        rr_max = max(rr_max, float(np.max(rr)))
    torch.cuda.synchronize()
    t_solve = time.perf_counter() - t0
    for b, _ in per:
        sgf.sgf_batch_destroy(b)
    for op in ops:
        op.close()
    n = len(ops)
    return {"workload": "gaussian rms 0.5 lc 2, periods 10/25/50/100 with N 2048/4096/8192/16384, one surface each, "
                        "16 angles (every 4th of 64) + 4 Wood wavenumbers (w = 1, 5, 9, 13) per surface",
            "problems": n, "precision": "mixed", "init_s": t_init,
            "apply_one_batch": {"value": n * 1000.0 / ms_all, "unit": "matvecs/s", "ms_per_step": ms_all},
            "apply_per_surface": {"value": n * 1000.0 / ms_per, "unit": "matvecs/s", "ms_per_step": ms_per,
                                  "forms": forms, "form_legend": "0 child graphs, 1 shared near pass, 2 multi-column"},
            "solve": {"value": n / t_solve, "unit": "solves/s", "s": t_solve, "tol": 1e-8, "status": st_all,
                      "applications": its_all, "max_relres": rr_max},
            "l2": "flushed (256 MiB write) before each timed step"}


def run_periods(sgf, dev, stream, flush, r):
    """The headline forward map on r repetitions of the same corrugation (N = 16384 r): what the
    kernels reach when the application is r times longer than the latency-bound N = 16384 case."""
    import torch

    par = inputs.wl_deep_corrugation_neumann_periods(r)
    op = sgf.Operator(par, device=dev.index, stream=stream.cuda_stream, precision=32)
    info = op.info
    hbm, kind = peaks()
    mu = torch.from_numpy(inputs.random_density(par["N"], 7)).to(dev)
    out = torch.empty_like(mu)
    ms = time_applies(sgf, op, mu, out, stream, flush, 100, 10)
    sb = stage_bytes(info, 8)
    stg = stage_times(sgf, op, mu, out, flush, 20)
    op.close()
    return {"workload": f"deep corrugation repeated {r} times, period {10 * r}, N = {par['N']}, {128 * r} cell columns",
            "N": int(par["N"]), "ms_per_step": ms, "value": 1000.0 / ms, "unit": "matvecs/s",
            "unknowns_per_s": par["N"] * 1000.0 / ms, "algorithmic_bytes": sum(sb.values()),
            "stages_ms": stg, "stage_hbm_frac": {k: sb[k] / (stg[k] * 1e-3) / 1e9 / hbm for k in STAGES if stg[k] > 0},
            "peak_kind": kind}


def run_multi_rhs(sgf, dev, stream, flush, args):
    """Several densities through the headline operator per call (sgf_apply with nrhs columns): the
    operator data (P, the near rows, the reconstruction rows) is read once per pass of up to 8
    columns. Applications per second for nrhs = 1, 8, 64, both precisions."""
    import torch

    par = workload()
    out = {}
    for prec in (32, 64):
        op = sgf.Operator(par, device=dev.index, stream=stream.cuda_stream, precision=prec)
        res = {}
        for nrhs in (1, 8, 64):
            X = torch.from_numpy(np.concatenate([inputs.random_density(par["N"], 60 + r) for r in range(nrhs)])).to(dev)
            Y = torch.empty_like(X)
            for _ in range(3):
                sgf.sgf_apply(op.ctx, X.data_ptr(), Y.data_ptr(), nrhs, 0)
            torch.cuda.synchronize()
            steps = max(3, min(args.steps, 20))
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            for k in range(steps):
                flush.zero_()
                ev[k][0].record(stream)
                sgf.sgf_apply(op.ctx, X.data_ptr(), Y.data_ptr(), nrhs, 0)
                ev[k][1].record(stream)
            torch.cuda.synchronize()
            ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
            res[str(nrhs)] = {"value": nrhs * 1000.0 / ms, "unit": "matvecs/s", "ms_per_call": ms}
        op.close()
        out["mixed" if prec == 32 else "fp64"] = res
    out["note"] = ("nrhs = 1 is the single-density path (captured graph); nrhs > 1 the multi-column path "
                   "(direct launches, 8 columns per pass)")
    return out


def run_shifted(sgf, dev, stream, flush, args):
    """The same geometry with the shifted kernel (j = 8, n_per = 40, h ~ lambda/2): applications per
    second of both precisions. The shifted system is nearly singular on this 20-wavelength-deep
    profile (condition ~4^j growth), so no solve is timed for it."""
    import torch

    par = inputs.wl_deep_corrugation_neumann(j=8, n_per=40)
    mu = torch.from_numpy(inputs.random_density(par["N"], 7)).to(dev)
    out = {}
    for prec in (32, 64):
        op = sgf.Operator(par, device=dev.index, stream=stream.cuda_stream, precision=prec)
        y = torch.empty_like(mu)
        ms = time_applies(sgf, op, mu, y, stream, flush, max(3, min(args.steps, 100)), args.warmup)
        info = op.info
        op.close()
        out["mixed" if prec == 32 else "fp64"] = {"value": 1000.0 / ms, "unit": "matvecs/s", "ms_per_step": ms,
                                                   "near_field_entries": int(info["nnz"])}
    return out


def run_cufft_reference(info, ours_ms, dev, stream, flush, steps):
    """Reference point for the grid convolution stage (X passes, Y convolution, inverse X passes of
    both orientations): the same zero-padded 2D convolutions done with torch.fft (cuFFT) in complex64
    on random data of the same shapes, launched one orientation after the other like the profiled
    stages. cuFFT is not on the library's path; this only calibrates the hand-written FFT stage."""
    import torch

    g = torch.Generator(device=dev).manual_seed(3)
    shapes = [(int(info["PxH"]), int(info["nrowH"]), int(info["PyH"])),
              (int(info["PxV"]), int(info["nrowV"]), int(info["PyV"]))]
    data = []
    for Px, nr, Py in shapes:
        def rnd(*sh):
            return torch.complex(torch.randn(*sh, generator=g, device=dev), torch.randn(*sh, generator=g, device=dev))
        data.append((rnd(Px, nr), rnd(Px, nr), rnd(Px, Py), rnd(Px, Py), Py, nr))

    def conv():
        for xi, ze, km, kd, Py, nr in data:
            xp = torch.zeros(xi.shape[0], Py, dtype=torch.complex64, device=dev)
            zp = torch.zeros_like(xp)
            xp[:, :nr] = xi
            zp[:, :nr] = ze
            y = torch.fft.ifft2(km * torch.fft.fft2(xp) + kd * torch.fft.fft2(zp))
            xi.copy_(y[:, :nr])

    for _ in range(3):
        conv()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        conv()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    ms = float(np.mean([x.elapsed_time(y) for x, y in ev]))
    return {"cufft_ms": ms, "ours_ms": ours_ms, "what": "fft_x + conv_y + ifft_x of both orientations, "
            "complex64, sequential launches (ours: profiled stage events)"}


def run_gradient(dev, stream):
    """The 128-coefficient gradient workload (N = 4096): one forward solve, then sgf_gradient (adjoint
    solve + node-local rebuilds), against the 2 x 128 solves a difference quotient would need."""
    import torch

    from paper_1707_04950_gb300 import sgf

    par = inputs.wl_harmonic_gradient()
    op = sgf.Operator(par, device=dev.index, stream=stream.cuda_stream, precision=64)
    mu = torch.zeros(par["N"], dtype=torch.complex128, device=dev)
    sgf.sgf_solve(op.ctx, 1e-12, 3000, mu.data_ptr())  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st, its, rr = sgf.sgf_solve(op.ctx, 1e-12, 3000, mu.data_ptr())
    torch.cuda.synchronize()
    t_solve = time.perf_counter() - t0
    M = len(par["a"]) - 1
    t0 = time.perf_counter()
    ga, gb, Bn, en, adj_its = sgf.sgf_gradient(op.ctx, mu.data_ptr(), 0, M)
    torch.cuda.synchronize()
    t_grad = time.perf_counter() - t0
    op.close()
    return {"workload": "harmonic64_d20_n4096_theta20_dirichlet", "coefficients": 2 * M, "e0": en,
            "forward_solve_s": t_solve, "forward_iters": its, "gradient_s": t_grad, "adjoint_iters": adj_its,
            "grad_norm": float(np.sqrt(np.sum(ga**2) + np.sum(gb**2))),
            "difference_quotient_equivalent_s": 2 * (2 * M) * t_solve}


def run_field(dev, stream, n_side=256):
    """Scattered field image of the deep corrugation (N = 16384, mixed operator; the field itself is
    FP64): an n_side x n_side grid over one period, from the bottom of the cell box to one period
    above its top, keeping the targets at least three node spacings above the surface. One
    sgf_field call = host binning + copies of the targets + kernels + synchronisation."""
    import torch

    from paper_1707_04950_gb300 import sgf

    par = inputs.wl_deep_corrugation_neumann()
    op = sgf.Operator(par, device=dev.index, stream=stream.cuda_stream, precision=32)
    mu = torch.from_numpy(inputs.random_density(par["N"], 21)).to(dev)
    top = par["hmin"] + par["ny"] * par["L"]
    xs = np.arange(n_side) * par["d"] / n_side
    ys = par["hmin"] + np.arange(n_side) * (top + par["d"] - par["hmin"]) / n_side
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    fx = inputs.profile_eval_host({"d": par["d"], "a": par["a"], "b": par["b"]}, X.ravel())
    keep = Y.ravel() > fx + 3 * par["d"] / par["N"]
    xy = np.stack([X.ravel()[keep], Y.ravel()[keep]], 1)
    u = torch.empty(len(xy), dtype=torch.complex128, device=dev)
    sgf.sgf_field(op.ctx, mu.data_ptr(), xy, u.data_ptr())  # warm-up
    torch.cuda.synchronize()
    reps = 3
    t0 = time.perf_counter()
    for _ in range(reps):
        sgf.sgf_field(op.ctx, mu.data_ptr(), xy, u.data_ptr())
    torch.cuda.synchronize()
    t = (time.perf_counter() - t0) / reps
    n_box = int(np.sum(xy[:, 1] < top))
    op.close()
    return {"workload": f"deep corrugation N=16384, {n_side}x{n_side} image over one period",
            "targets": len(xy), "targets_in_box": n_box, "targets_above_box": len(xy) - n_box,
            "s_per_call": t, "value": len(xy) / t, "unit": "targets/s", "precision": "fp64"}


def _table_rows():
    """The paper's table rows (golden fixtures the tests use): sinusoid tables of Section 6.2 and the
    composite-surface convergence table of Section 6.1, as (label, profile, k, theta_deg, N, j, h,
    n_per, lambda, max|f'|, paper eps, paper s/iter or None, paper iters or None)."""
    root = os.path.dirname(os.path.abspath(__file__))
    rows = []
    for ln in open(os.path.join(root, "tests", "golden", "sinusoid_littrow_energy_error.txt")):
        if not ln.strip() or ln.startswith("#"):
            continue
        r = ln.split()
        Hd, dl, N, hl, n_per = float(r[0]), float(r[2]), int(r[3]), float(r[4]), int(r[5])
        d = 2 * math.pi
        lam = d / dl
        H = Hd * d
        prof = {"d": d, "a": np.zeros(2), "b": np.array([0.0, H / 2])}
        shifted = hl > 0
        rows.append((f"sinusoid H/d={Hd} d/lambda={dl}", prof, dl, math.degrees(math.asin(1 / 3)), N,
                     8 if shifted else 0, hl * lam if shifted else 0.5, n_per, lam, math.pi * Hd,
                     float(r[8]), float(r[6]), int(r[7])))
    comp = {"d": 2 * math.pi, "a": np.zeros(5), "b": -0.25 * np.array([0.0, 1.0, 1 / 2, 1 / 3, 1 / 4])}
    slope = 0.25 * (1 + 1 + 1 + 1)
    for ln in open(os.path.join(root, "tests", "golden", "composite_surface_energy_error.txt")):
        if not ln.strip() or ln.startswith("#"):
            continue
        r = ln.split()
        N, n_per = int(r[0]), int(r[1])
        kw = 6.0 / (1.0 - math.sin(math.radians(45.0)))
        rows.append((f"composite k=20 N={N}", comp, 20.0, 45.0, N, 0, 0.5, n_per, 2 * math.pi / 20.0, slope,
                     float(r[2]), None, None))
        rows.append((f"composite Wood N={N}", comp, kw, 45.0, N, 8, 0.16, n_per, 2 * math.pi / kw, slope,
                     float(r[3]), None, None))
    return rows


def run_tables(dev, stream):
    """The paper's tables (Section 6.1 composite-surface convergence, Section 6.2 sinusoid gratings)
    with the accelerated operator (cells L <= 0.45 lambda, N rounded up to a multiple of the cell
    columns, FP64, GMRES to 1e-12, twice the paper's n_per) and, for the sinusoids, with the dense
    unaccelerated operator at the paper's N: energy error, iterations and time per iteration beside
    the paper's single-core values."""
    import torch

    from paper_1707_04950_gb300 import sgf

    out = []
    for (label, prof, k, th, N, j, h, n_per, lam, slope, peps, pit_s, pits) in _table_rows():
        row = {"row": label, "paper_eps": peps, "paper_s_per_iter": pit_s, "paper_iters": pits}
        try:
            par = inputs.accel_table_params(prof, k, th, N, j, h, 2 * n_per, lam, slope)
        except ValueError as e:
            row["accelerated"] = {"skipped": str(e)}
            par = None
        try:
            if par is None:
                raise LookupError
            op = sgf.Operator(par, device=dev.index, stream=stream.cuda_stream, precision=64)
            mu = torch.zeros(par["N"], dtype=torch.complex128, device=dev)
            sgf.sgf_solve(op.ctx, 1e-12, 2000, mu.data_ptr())
            mu.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, its, rr = sgf.sgf_solve(op.ctx, 1e-12, 2000, mu.data_ptr())
            torch.cuda.synchronize()
            t = time.perf_counter() - t0
            _, _, eps = sgf.sgf_rayleigh(op.ctx, mu.data_ptr(), -60, 60)
            op.close()
            row["accelerated"] = {"N": par["N"], "cells": par["nx"], "eps": abs(eps), "iters": its, "relres": rr,
                                  "status": st, "s_per_iter": t / max(1, its)}
        except LookupError:
            pass
        except sgf.SgfError as e:
            row["accelerated"] = {"N": par["N"], "error": str(e)}
        if label.startswith("sinusoid"):
            dl = k
            Hd = 2 * prof["b"][1] / prof["d"]
            parx = inputs.wl_littrow(Hd, dl, N, h / lam if j else 0.0, 2 * n_per)
            ctx = sgf.sgf_create(dev.index, stream.cuda_stream)
            sgf.sgf_set_profile_fourier(ctx, parx["d"], parx["a"], parx["b"])
            sgf.sgf_set_wave(ctx, parx["k"], parx["theta"], parx["bc"])
            sgf.sgf_set_params(ctx, sgf.params_from(parx, 64))
            sgf.sgf_build_exact(ctx)
            sgf.sgf_select_operator(ctx, 1)
            mu = torch.zeros(N, dtype=torch.complex128, device=dev)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, its, rr = sgf.sgf_solve(ctx, 1e-12, 2000, mu.data_ptr())
            torch.cuda.synchronize()
            t = time.perf_counter() - t0
            _, _, eps = sgf.sgf_rayleigh(ctx, mu.data_ptr(), -60, 60)
            sgf.sgf_destroy(ctx)
            row["dense"] = {"N": N, "eps": abs(eps), "iters": its, "relres": rr, "status": st,
                            "s_per_iter": t / max(1, its)}
        out.append(row)
    return out


FP64_TFLOPS = 1.25  # GB300 FP64 (vector) rate, nominal


def run_exact(dev, stream, flush, steps):
    """The unaccelerated operator as a dense matrix on the 128-coefficient gradient workload
    (N = 4096): assembly time, and one application (a bandwidth-bound GEMV over the 16 N^2-byte
    matrix, larger than L2) against one FP64 application of the accelerated operator."""
    import torch

    from paper_1707_04950_gb300 import sgf

    par = inputs.wl_harmonic_gradient()
    N = par["N"]
    op = sgf.Operator(par, device=dev.index, stream=stream.cuda_stream, precision=64)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sgf.sgf_build_exact(op.ctx)
    t_build = time.perf_counter() - t0
    x = torch.from_numpy(inputs.random_density(N, 5)).to(dev)
    y = torch.empty_like(x)

    def timed(exact):
        sgf.sgf_select_operator(op.ctx, exact)
        for _ in range(3):
            sgf.sgf_apply(op.ctx, x.data_ptr(), y.data_ptr())
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            flush.zero_()
            ev[k][0].record(stream)
            sgf.sgf_apply(op.ctx, x.data_ptr(), y.data_ptr())
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        return float(np.mean([a.elapsed_time(b) for a, b in ev]))

    ms_dense = timed(True)
    y_dense = y.clone()
    ms_acc = timed(False)
    rel = float(torch.linalg.norm(y - y_dense) / torch.linalg.norm(y_dense))
    op.close()
    hbm, kind = peaks()
    gbs = (16.0 * N * N + 32.0 * N) / (ms_dense * 1e-3) / 1e9
    # 8 flops (four FP64 FMAs) per 16-byte entry: above the FP64 ridge (1.25 TFLOP/s nominal for
    # GB300, against the measured HBM bandwidth), so the FP64 pipes bound the GEMV
    tflops = 8.0 * N * N / (ms_dense * 1e-3) / 1e12
    return {"workload": "harmonic64_d20_n4096_theta20_dirichlet", "N": N, "assembly_s": t_build,
            "dense_apply_ms": ms_dense, "accelerated_fp64_apply_ms": ms_acc,
            "dense_gemv": {"bound": "alu", "achieved": tflops, "peak": FP64_TFLOPS, "unit": "TFLOP/s",
                           "frac": tflops / FP64_TFLOPS, "peak_kind": "nominal FP64 of GB300",
                           "hbm_gbs": gbs, "hbm_frac": gbs / hbm, "hbm_peak_kind": kind,
                           "algorithmic_flops_per_launch": 8.0 * N * N,
                           "algorithmic_bytes_per_launch": 16.0 * N * N + 32.0 * N},
            "accelerated_vs_dense_rel_diff": rel}


def run_autotune(dev, stream):
    """Cell-size candidates for the deep corrugation (the benchmark fixes 128 cell columns, the
    configured 128 x 256 cells): time per mixed application and energy error of each candidate; the
    fastest one below 1e-8 is kept, and its solve is reported."""
    from paper_1707_04950_gb300 import sgf

    import torch

    par = inputs.wl_deep_corrugation_neumann()
    op = sgf.Operator(par, device=dev.index, stream=stream.cuda_stream, precision=32)
    cands = [32, 64, 128]
    st, best, ms, eps = sgf.sgf_autotune(op.ctx, cands, 1e-8, reps=50)
    # the chosen cells' accuracy: the headline solve and its energy error
    x = torch.zeros(par["N"], dtype=torch.complex128, device=dev)
    sst, its, rr = sgf.sgf_solve(op.ctx, 1e-12, 4000, x.data_ptr())
    _, _, e = sgf.sgf_rayleigh(op.ctx, x.data_ptr(), -40, 40)
    op.close()
    return {"workload": "deep corrugation N=16384 (j = 0), mixed", "candidates_nx": cands,
            "ms_per_application": [float(x) if x > 0 else None for x in ms],
            "energy_error": [float(x) for x in eps], "eps_tol": 1e-8, "status": st, "best_nx": best,
            "best_solve": {"status": sst, "applications": its, "relres": rr, "energy_error": e}}


# GMRES tolerance of the batched solves: the FP64 operator of these rough-surface problems reaches a
# relative residual of about 5e-12 at best (rounding of the far-field/local-subtraction cancellation
# in each application), so 1e-12 is not attainable for all 16 angles.
BATCH_TOL = 1e-10


def run_batch(args, dev, stream, flush):
    """Independent problems side by side: the multi-angle Gaussian-surface workload (N = 2048, one
    surface, every 4th of the 64 incidence angles), mixed precision. One batched graph launch per
    step against the same problems launched one after another; one lockstep batched solve against
    sequential solves."""
    import torch

    from paper_1707_04950_gb300 import sgf

    idx = list(range(0, 64, 64 // args.batch))[: args.batch]
    pars = [inputs.wl_gaussian_angles(i) for i in idx]
    ops = [sgf.Operator(p, device=dev.index, stream=stream.cuda_stream, precision=32) for p in pars]
    infos = [op.info for op in ops]
    mus = [torch.from_numpy(inputs.random_density(p["N"], 30 + q)).to(dev) for q, p in enumerate(pars)]
    outs = [torch.empty_like(m) for m in mus]
    b = sgf.sgf_batch_create([op.ctx for op in ops], stream.cuda_stream)
    shared = bool(sgf.sgf_batch_shared_near(b))
    mp, op_ = [m.data_ptr() for m in mus], [o.data_ptr() for o in outs]
    steps = max(3, min(args.steps, 50))

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            flush.zero_()
            ev[k][0].record(stream)
            fn()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        return float(np.mean([x.elapsed_time(y) for x, y in ev]))

    ms_b = timed(lambda: sgf.sgf_batch_apply(b, mp, op_))
    y_b = [o.clone() for o in outs]

    def seq():
        for op, m, o in zip(ops, mus, outs):
            sgf.sgf_apply(op.ctx, m.data_ptr(), o.data_ptr())

    ms_s = timed(seq)
    diff = max(float(torch.linalg.norm(x - y) / torch.linalg.norm(y)) for x, y in zip(y_b, outs))
    sol = [torch.zeros_like(m) for m in mus]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st, its, rr = sgf.sgf_batch_solve(b, BATCH_TOL, 2000, [x.data_ptr() for x in sol])
    torch.cuda.synchronize()
    t_b = time.perf_counter() - t0
    sol_s = [torch.zeros_like(m) for m in mus]
    t0 = time.perf_counter()
    its_s = []
    for op, x in zip(ops, sol_s):
        st_s, it1, _ = sgf.sgf_solve(op.ctx, BATCH_TOL, 2000, x.data_ptr())
        its_s.append(it1)
    torch.cuda.synchronize()
    t_s = time.perf_counter() - t0
    sol_diff = max(float(torch.linalg.norm(x - y) / torch.linalg.norm(y)) for x, y in zip(sol, sol_s))
    sgf.sgf_batch_destroy(b)
    for op in ops:
        op.close()
    n = len(ops)
    bytes_step = sum(op_info["bytes32"] for op_info in infos)
    hbm, _ = peaks()
    return {
        "workload": f"gaussian_rms0.5_lc2_d10_n2048_{n}angles_of_64", "problems": n, "precision": "mixed",
        "shared_near": shared,
        "apply": {"value": n * 1000.0 / ms_b, "unit": "matvecs/s", "ms_per_step": ms_b,
                  "hbm_frac": bytes_step / (ms_b * 1e-3) / 1e9 / hbm},
        "apply_sequential": {"value": n * 1000.0 / ms_s, "unit": "matvecs/s", "ms_per_step": ms_s},
        "batch_vs_sequential_rel_diff": diff,
        "solve": {"value": n / t_b, "unit": "solves/s", "s": t_b, "tol": BATCH_TOL, "status": st, "iters": its,
                  "max_relres": float(np.max(rr))},
        "solve_sequential": {"value": n / t_s, "unit": "solves/s", "s": t_s, "iters": its_s},
        "solution_rel_diff": sol_diff,
        "l2": "flushed (256 MiB write) before each timed apply step",
    }


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def assemble_oracle_rows(par, rows):
    """Oracle rows of the exact operator (the assembly cost, timed on its own) and the dense
    row block the ZGEMV is timed on: the assembled rows tiled to GEMV_BLOCK rows."""
    from oracle import direct

    N = par["N"]
    idx = np.linspace(0, N - 1, rows).astype(int)
    t0 = time.perf_counter()
    R = direct.assemble_rows(par, idx)
    t_asm = time.perf_counter() - t0
    blk = np.ascontiguousarray(np.tile(R, (GEMV_BLOCK // rows, 1)))
    return blk, t_asm


GEMV_BLOCK = 512


def gemv_times(blk, mu, threads, reps_min_s=1.0, steps=None):
    """Seconds per ZGEMV (blk @ mu) with `threads` BLAS threads, in a child process (the BLAS thread
    count is fixed when numpy loads). steps: time exactly that many GEMVs and return each one's time;
    otherwise repeat for at least reps_min_s and return the mean."""
    d = tempfile.mkdtemp(prefix="sgf_gemv_")
    fa, fm = os.path.join(d, "blk.npy"), os.path.join(d, "mu.npy")
    np.save(fa, blk)
    np.save(fm, mu)
    env = dict(os.environ)
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = str(threads)
    cmd = [sys.executable, os.path.abspath(__file__), "--gemv-worker", fa, fm, str(reps_min_s),
           str(steps if steps else 0)]
    r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=600)
    for f in (fa, fm):
        os.remove(f)
    os.rmdir(d)
    if r.returncode != 0:
        raise RuntimeError("ZGEMV worker failed: " + r.stderr[-500:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def gemv_worker(fa, fm, reps_min_s, steps):
    blk = np.load(fa)
    mu = np.load(fm)
    for _ in range(3):
        blk @ mu
    if steps > 0:
        ts = []
        for _ in range(steps):
            t0 = time.perf_counter()
            blk @ mu
            ts.append(time.perf_counter() - t0)
        print(json.dumps(ts))
        return
    n, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < reps_min_s:
        blk @ mu
        n += 1
    print(json.dumps((time.perf_counter() - t0) / n))


def cpu_baseline(rows=4):
    """The CPU oracle's matvec: the exact operator assembled as dense rows (assembly timed on its own)
    and applied by ZGEMV, on all host cores and on one. `rows` rows of the benchmark workload are
    assembled and tiled to a GEMV_BLOCK x N block; the block's GEMV time is scaled by N / GEMV_BLOCK
    to one full matvec (extrapolated: the N x N matrix, 4.3 GB at N = 16384, is not assembled)."""
    par = workload()
    N = par["N"]
    blk, t_asm = assemble_oracle_rows(par, rows)
    mu = inputs.random_density(N, 7)
    cores = host_cores()
    t_all = gemv_times(blk, mu, cores)
    t_one = gemv_times(blk, mu, 1)
    scale = N / GEMV_BLOCK
    return {"value": 1.0 / (t_all * scale), "unit": "matvecs/s", "cores": cores, "kind": "oracle",
            "sample": f"dense ZGEMV (numpy/OpenBLAS, {cores} threads) of a {GEMV_BLOCK} x {N} row block of the exact "
                      f"operator ({rows} assembled rows tiled), {t_all * 1e3:.2f} ms, scaled by N/{GEMV_BLOCK} "
                      f"(extrapolated); assembly of the {rows} rows {t_asm:.1f} s on one core",
            "one_core": {"value": 1.0 / (t_one * scale), "unit": "matvecs/s", "cores": 1},
            "assembly_s_per_row": t_asm / rows, "assembly_s_extrapolated": t_asm / rows * N,
            "extrapolated": True}


def run_reference(args):
    """The CPU oracle as the reference arm, on the benchmark workload: `--cpu-rows` rows of the exact
    operator are assembled once (timed and reported; scaled to the full matrix), then every step is one
    dense ZGEMV of a GEMV_BLOCK x N row block on all host cores, scaled by N / GEMV_BLOCK to one matvec."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    par = workload()
    N = par["N"]
    blk, t_asm = assemble_oracle_rows(par, args.cpu_rows)
    mu = inputs.random_density(N, 7)
    cores = host_cores()
    steps = args.steps
    ts = gemv_times(blk, mu, cores, steps=args.warmup + steps)[args.warmup:]
    scale = N / GEMV_BLOCK
    ms = float(np.mean(ts)) * scale * 1e3
    v = 1000.0 / ms
    sample = (f"dense ZGEMV (numpy/OpenBLAS, {cores} threads) of a {GEMV_BLOCK} x {N} row block of the exact operator "
              f"({args.cpu_rows} assembled rows tiled) per step, scaled by N/{GEMV_BLOCK} (extrapolated); "
              f"assembly {t_asm / args.cpu_rows * N:.0f} s extrapolated to all N rows (one core)")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "matvecs/s", "n_gpus": ws,
            "steps": steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": N, "cells": "128x257", "shifts_j": int(par["j"]),
                       "n_per": int(par["n_per"]), "parallelism": f"cpu oracle, {cores} cores"},
            "cpu_baseline": {"value": v, "unit": "matvecs/s", "cores": cores, "kind": "oracle", "sample": sample,
                             "assembly_s_extrapolated": t_asm / args.cpu_rows * N},
            "e2e": {"value": v, "unit": "matvecs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-rows", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch", type=int, default=16, help="problems of the batched block (0: skip)")
    ap.add_argument("--solve", type=int, default=1, help="1: time the headline FP64 and mixed solves")
    ap.add_argument("--shifted", type=int, default=1, help="1: time the j = 8 shifted kernel on the same geometry")
    ap.add_argument("--multi", type=int, default=1, help="1: time several densities per call (nrhs 1, 8, 64)")
    ap.add_argument("--periods", type=int, default=0,
                    help="R > 1: also time the forward map on the corrugation repeated R times (N = 16384 R; R <= 4)")
    ap.add_argument("--sweep", type=int, default=1, help="1: the batched angle/Wood sweep over four surfaces")
    ap.add_argument("--gradient", type=int, default=1, help="1: time the 128-coefficient gradient block")
    ap.add_argument("--tables", type=int, default=0,
                    help="1: the paper's composite and sinusoid tables, accelerated and dense operators")
    ap.add_argument("--field", type=int, default=1,
                    help="1: time the scattered-field image and the dense unaccelerated operator blocks")
    ap.add_argument("--gemv-worker", nargs=4, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.gemv_worker:
        fa, fm, rs, st = args.gemv_worker
        gemv_worker(fa, fm, float(rs), int(st))
        return
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        run_reference(args)
    else:
        from paper_1707_04950_gb300 import build

        build.build()
        run_ours(args)


if __name__ == "__main__":
    main()
