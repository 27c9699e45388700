#!/usr/bin/env python3
"""Throughput benchmark of the pseudo-time residual sweep.

Metric: cell pseudo-iterations per second = sum over tanks of (interior
cells x pseudo-iterations completed) / time of the ac_physical_step calls.
One pseudo-iteration = s_max = 3 fused stage sweeps + the residual test.

Default workload: the hydrostatic two-fluid tank, 256 x 256 cells, FP64,
each step one physical step (dt = 1e-3 s) iterated to a 1e-8 residual drop
or 500 pseudo-iterations.  The state stays resident in HBM; L2 is flushed
(256 MiB write) between timed steps, outside the event pairs.

Extra objects on the JSON line:
  roofline      the stage sweep's own event-timed duration against its
                arithmetic roof (FP64 is ALU-bound on this part)
  e2e           the same metric through the public API with host buffers:
                ac_set_state from pinned host memory + the step +
                ac_get_state into pinned host memory, every step
  cpu_baseline  the FP64 oracle on the host cores, bounded sample

``--impl reference`` times the FP64 oracle itself on the host cores (the
project's reference implementation), on the same workload and metric.
Under torchrun every rank runs its own replica of the workload (replicas
only: one tank does not shard across GPUs here); rank 0 prints.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell pseudo-iterations/sec"
UNIT = "cell-iter/s"
# FP64 peak of the part (recipe's nominal dense FP64 rate, FLOP/s); the
# stage sweep is bound by it, not by HBM
FP64_PEAK_TFLOPS = 1.25


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="hydrostatic_256")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-large", action="store_true", help="skip the 2048x8192 mixed-form leg")
    ap.add_argument("--no-checks", action="store_true",
                    help="skip the configurations' own checks (GPU against GPU, outside the timed region)")
    ap.add_argument("--configs", action="store_true",
                    help="instead of the benchmark line: one line per test configuration at its stated length "
                         "(FP64, mixed, errors, the configuration's own checks)")
    ap.add_argument("--config4-steps", type=int, default=20,
                    help="physical steps of the 2048x8192 Rayleigh-Taylor configuration in --configs (stated: 200)")
    return ap.parse_args()


def make_case(name):
    from paper_2108_08769_gb300 import workloads as W
    if name == "hydrostatic_256":
        c = W.hydrostatic_tank(256)
        desc = ("hydrostatic two-fluid tank 256x256, closed 1x1 m box, water 1000 below y=0.5, air 1 above, "
                "at rest, discrete hydrostatic p, g=-9.81, c0=20 m/s (beta=4e5 Pa), dt=1e-3 s, "
                "pseudo-iterations to a 1e-8 residual drop or 500, FP64")
        return c, desc
    raise SystemExit(f"unknown workload {name}")


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("AC_BENCH_BACKEND", "nccl") == "nccl" else "gloo")
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        # raw samples beside the run (AC_BENCH_CLOCKS_DIR), else in the temporary directory
        self.path = os.path.join(os.environ.get("AC_BENCH_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"ac_bench_clocks_{os.getpid()}.csv")
        self.proc = None

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "samples": len(sm), "reasons": sorted(reasons)}


def host_cpu():
    """Host CPU model and core count, as lscpu reports them."""
    import platform
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for l in out.splitlines():
            if l.startswith("Model name:"):
                model = l.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return f"{model or platform.processor() or 'unknown'} ({platform.machine()}, {os.cpu_count()} cores)"


def cpu_baseline_sample(case, iters=10):
    """The FP64 oracle as it stands, single-threaded, on a bounded sample:
    one physical step of the same tank with a fixed number of iterations."""
    import oracle
    oracle.build()
    state = case.state()
    t0 = time.perf_counter()
    _, st, its, _, _ = oracle.physical_step(case, state, tol=-1.0, max_iters=iters)
    dt = time.perf_counter() - t0
    return {"value": case.cells * its / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_cpu(),
            "sample": f"1 physical step x {its} pseudo-iterations on the full {case.nx}x{case.ny} tank "
                      f"({dt:.1f} s, FP64 C oracle, 1 thread)"}


def _oracle_worker(workload, iters, barrier):
    """One copy of the oracle in its own process (all-core baseline)."""
    case, _ = make_case(workload)
    import oracle
    oracle.build()
    state = case.state()
    barrier.wait()
    t0 = time.perf_counter()
    _, _, its, _, _ = oracle.physical_step(case, state, tol=-1.0, max_iters=iters)
    return t0, time.perf_counter(), case.cells * its


def cpu_baseline_all_cores(workload, iters=10):
    """The same oracle sample run as one copy per host core, in processes
    started with spawn (no GPU context is inherited): all copies' cell
    pseudo-iterations over the span from the first start to the last
    finish."""
    import multiprocessing as mp
    n = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        barrier = mgr.Barrier(n)
        with ctx.Pool(n) as pool:
            res = pool.starmap(_oracle_worker, [(workload, iters, barrier)] * n)
    span = max(r[1] for r in res) - min(r[0] for r in res)
    work = sum(r[2] for r in res)
    case, _ = make_case(workload)
    return {"value": work / span, "unit": UNIT, "cores": n, "kind": "oracle", "host": host_cpu(),
            "sample": f"{n} processes, each 1 physical step x {iters} pseudo-iterations on the full "
                      f"{case.nx}x{case.ny} tank ({span:.1f} s wall, FP64 C oracle, 1 thread each)"}


def run_reference(args, ws, rank):
    if rank != 0:
        return
    case, desc = make_case(args.workload)
    import oracle
    oracle.build()
    iters = 3
    for _ in range(args.warmup):
        oracle.physical_step(case, case.state(), tol=-1.0, max_iters=iters)
    tot, cells_iters = 0.0, 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        _, st, its, _, _ = oracle.physical_step(case, case.state(), tol=-1.0, max_iters=iters)
        tot += time.perf_counter() - t0
        cells_iters += case.cells * its
    v = cells_iters / tot
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": desc, "cells": case.cells,
                                            "pseudo_iters_per_step": iters,
                                            "note": f"each timed step is one physical step of {iters} pseudo-iterations "
                                                    "of the full tank (the GPU arm's steps run to the stopping test, "
                                                    "500 here); the metric is a rate, so the two compare"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_cpu(),
                             "sample": f"each step: 1 physical step x {iters} pseudo-iterations of the full "
                                       f"{case.nx}x{case.ny} tank, FP64 C oracle, 1 thread"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def timed_steps(tank, case, steps, stream, flush, barrier, tol=None, max_iters=None):
    """K physical steps, each bracketed by CUDA events on the library's
    stream, L2 flushed before each (outside the events)."""
    import torch
    tol = case.tol if tol is None else tol
    max_iters = case.max_iters if max_iters is None else max_iters
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    iters = []
    launches0 = tank.kernel_launches()
    barrier()
    for k in range(steps):
        flush.zero_()
        evs[k][0].record(stream)
        rc, its = tank.physical_step(case.dt, tol, max_iters)
        evs[k][1].record(stream)
        iters.append(its)
    barrier()
    ms = sum(a.elapsed_time(b) for a, b in evs)
    return ms, iters, tank.kernel_launches() - launches0


def stage_launch_ms(tank, case, steps, tol=None, max_iters=None):
    """Average event-timed duration of one stage-sweep launch, measured on
    the same physical steps (profiling mode brackets every launch)."""
    tank.set_profiling(True)
    for _ in range(steps):
        tank.physical_step(case.dt, case.tol if tol is None else tol,
                           case.max_iters if max_iters is None else max_iters)
    ms, n = tank.stage_kernel_time()
    tank.set_profiling(False)
    return ms / max(n, 1)


def field_errors(a, b):
    """Relative L-inf and L1 error per field, every field (each momentum
    component separately) against its own largest magnitude; the momentum
    scales floored at max(rho) * 1e-3 m/s in the main figures and unfloored
    in the `*_unfloored` ones."""
    import numpy as np
    rho = float(np.abs(b[0]).max())
    names = ("rho", "rhou", "rhov", "p")
    raw = [rho, float(np.abs(b[1]).max()), float(np.abs(b[2]).max()), max(float(np.abs(b[3]).max()), 1e-12)]
    floored = [raw[0], max(raw[1], 1e-3 * rho), max(raw[2], 1e-3 * rho), raw[3]]
    out = {}
    for k, x, y, s, su in zip(names, a, b, floored, raw):
        d = np.abs(np.asarray(x) - np.asarray(y))
        out[k] = float(d.max() / s)
        out[k + "_unfloored"] = float(d.max() / max(su, 1e-300))
        out[k + "_l1"] = float(d.mean() / max(float(np.abs(y).mean()), 1e-300))
    return out


def run_ours(args, ws, rank, local):
    import numpy as np
    import torch
    from paper_2108_08769_gb300 import ac, workloads as W

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    case, desc = make_case(args.workload)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    # ---- primary: the FP64 tank, state resident in HBM ----
    tank = ac.Tank.from_case(case)
    tank.set_stream(stream.cuda_stream)
    for _ in range(args.warmup):
        tank.physical_step(case.dt, case.tol, case.max_iters)
    tank.set_state(*case.state())
    with Clocks(local) as clk:
        wall0 = time.perf_counter()
        dev_ms, iters, launches = timed_steps(tank, case, args.steps, stream, flush, barrier)
        wall = time.perf_counter() - wall0
    f64_state = tank.get_state()
    from paper_2108_08769_gb300.replicas import aggregate
    _, t_max, value = aggregate(case.cells * sum(iters), dev_ms, device=dev)

    # ---- e2e: host buffers through the public API ----
    pinned = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in case.state()]
    outs = [torch.empty(case.cells, dtype=torch.float64).pin_memory() for _ in range(4)]
    host_in = [p.numpy().reshape(-1) for p in pinned]
    host_out = [o.numpy() for o in outs]
    e_iters = []
    barrier()
    e0 = time.perf_counter()
    for k in range(args.steps):
        tank.set_state(*host_in)
        rc, its = tank.physical_step(case.dt, case.tol, case.max_iters)
        tank.get_state_into(*host_out)
        e_iters.append(its)
    barrier()
    e_wall = time.perf_counter() - e0
    e2e = {"value": ws * case.cells * sum(e_iters) / e_wall, "unit": UNIT,
           "h2d_bytes_per_step": 4 * case.cells * 8, "d2h_bytes_per_step": 4 * case.cells * 8}

    # ---- roofline of the FP64 stage sweep ----
    # the stage launch's duration inside the timed steps: each step's time
    # over its stage launches (the end-of-iteration kernel's few per cent
    # included, so the rate is a lower bound); the same launch timed alone
    # with events on either side is reported beside it
    s_max = case.options.s_max
    per_launch_s = dev_ms * 1e-3 / (s_max * sum(iters))
    tank.set_state(*case.state())
    isolated_s = stage_launch_ms(tank, case, min(args.steps, 3)) * 1e-3
    ftx, fty, _, fv = tank.tile_shape()
    achieved = FP64_ALG_FLOPS_PER_CELL_STAGE * case.cells / per_launch_s / 1e12
    # the part's FP64 FMA rate measured here (independent FMA chains), as a
    # check of the nominal peak the fraction is taken against
    probe = ac.ac_probe_fp64_fma_tflops()
    roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS,
                "traffic": FP64_TRAFFIC_PER_CELL_STAGE * case.cells,
                "kernel": f"stage_kernel<double,{ftx},{fty}>", "tile_variant": fv,
                "launch_ms": per_launch_s * 1e3, "launch_ms_timed_alone": isolated_s * 1e3,
                "flops_per_cell_stage": FP64_ALG_FLOPS_PER_CELL_STAGE,
                "flops_note": "algorithmic FP64 flops of one stage per cell, fixed (derivation in the design notes)",
                "executed_flops_per_cell_stage": FP64_EXEC_FLOPS_PER_CELL_STAGE,
                "executed_frac": FP64_EXEC_FLOPS_PER_CELL_STAGE * case.cells / per_launch_s / 1e12 / FP64_PEAK_TFLOPS,
                "peak_source": "nominal FP64 rate of the part (profiling recipe: 2 FP64 FMA lanes/SM)",
                "peak_probe_tflops": probe, "frac_of_probe": achieved / probe,
                # the same launch counted in FP64 instructions against the pipe's
                # issue rate (2 per SM per clock): DADD and DMUL take a pipe slot
                # for one flop
                "dp_instructions_per_cell_stage": FP64_INSTR_PER_CELL_STAGE,
                "dp_pipe_frac": FP64_INSTR_PER_CELL_STAGE * case.cells / per_launch_s / FP64_PIPE_INSTR_PER_S,
                "hbm_frac_of_measured": BYTES_PER_CELL_ITER_F64 / 3.0 * case.cells / per_launch_s / 1e9
                / measured_hbm_gbs()}
    tank.close()

    # ---- the same tank in the mixed form ----
    # Same work as the FP64 leg: the pseudo-iteration count is fixed at the
    # FP64 leg's (with the stopping test on, the mixed form stops after one
    # iteration here: the reference split makes the rest state exact, R = 0).
    n_fixed = int(round(statistics.mean(iters)))
    mt = ac.Tank.from_case(case, precision="mixed")
    mt.set_stream(stream.cuda_stream)
    for _ in range(args.warmup):
        mt.physical_step(case.dt, -1.0, n_fixed)
    mt.set_state(*case.state())
    m_ms, m_iters, m_launches = timed_steps(mt, case, args.steps, stream, flush, barrier, tol=-1.0,
                                            max_iters=n_fixed)
    m_state = mt.get_state()
    mt.set_state(*case.state())
    m_launch_ms = stage_launch_ms(mt, case, min(args.steps, 3), tol=-1.0, max_iters=n_fixed)
    mt.set_state(*case.state())
    rc, conv_iters = mt.physical_step(case.dt, case.tol, case.max_iters)
    mt.close()
    m_value = ws * case.cells * sum(m_iters) / (m_ms * 1e-3)
    mixed = {"value": m_value, "unit": UNIT, "speedup_vs_fp64": m_value / value,
             "ms_per_step": m_ms / args.steps, "pseudo_iters_per_step": n_fixed, "launch_ms": m_launch_ms,
             "gpu_launches": m_launches, "error_vs_fp64": field_errors(m_state, f64_state),
             "error_note": f"after {args.steps} physical steps of {n_fixed} pseudo-iterations from the same state, "
                           "relative L-inf per field against its own max (momentum scales floored at max(rho) x 1e-3 m/s; "
                           "unfloored beside), relative L1 against the field's mean magnitude",
             "iters_with_stopping_test": conv_iters}

    # ---- large grid in the mixed form: HBM-sized workload ----
    large = None
    if not args.no_large:
        lc = W.rayleigh_taylor(2048, 8192)
        lt = ac.Tank.from_case(lc, precision="mixed")
        lt.set_stream(stream.cuda_stream)
        lt.physical_step(lc.dt, lc.tol, lc.max_iters)
        lt.set_state(*lc.state())
        lk = min(args.steps, 3)
        l_ms, l_iters, l_launches = timed_steps(lt, lc, lk, stream, flush, barrier)
        lt.set_state(*lc.state())
        l_launch_s = stage_launch_ms(lt, lc, 1, tol=-1.0, max_iters=30) * 1e-3
        ltx, lty, lnt, lv = lt.tile_shape()
        # error against the FP64 GPU path after one step of 20 iterations
        lt.set_state(*lc.state())
        lt.physical_step(lc.dt, -1.0, 20)
        lm_state = lt.get_state()
        lt.close()
        ft = ac.Tank.from_case(lc)
        ft.physical_step(lc.dt, -1.0, 20)
        lf_state = ft.get_state()
        ft.close()
        l_value = ws * lc.cells * sum(l_iters) / (l_ms * 1e-3)
        gbs = MIXED_BYTES_PER_CELL_ITER / 3.0 * lc.cells / l_launch_s / 1e9
        l_traffic, l_ops = MIXED_COUNTS_BY_VARIANT.get(lv, (None, None))
        ops = None if l_ops is None else l_ops * lc.cells / l_launch_s / 1e12
        large = {"workload": "Rayleigh-Taylor tank 2048x8192 (1x4 m, rho 3 over 1, cosine interface, slip walls, "
                             "c0=10 m/s, dt=5e-4 s, 1e-8 drop or 500 pseudo-iterations), mixed form",
                 "value": l_value, "unit": UNIT, "steps": lk, "ms_per_step": l_ms / lk,
                 "pseudo_iters_per_step": statistics.mean(l_iters), "gpu_launches": l_launches,
                 "roofline": {"bound": "hbm", "achieved": gbs, "peak": measured_hbm_gbs(), "unit": "GB/s",
                              "frac": gbs / measured_hbm_gbs(), "frac_of_nominal_8tbs": gbs / 8000.0,
                              "kernel": (f"sweep_kernel_mixed<{lty},{lnt // 32}> (28-column strips)" if ltx == 28
                                         else f"stage_kernel_mixed<{ltx},{lty},{lnt}>"), "tile_variant": lv,
                              "launch_ms": l_launch_s * 1e3,
                              "launch_ms_in_step": l_ms * 1e-3 / (3 * sum(l_iters)) * 1e3,
                              "bytes_per_cell_iter": MIXED_BYTES_PER_CELL_ITER,
                              "traffic": None if l_traffic is None else l_traffic * lc.cells,
                              "alu_frac": None if ops is None else ops / FP32_PEAK_TOPS,
                              "alu_note": (f"{l_ops:.0f} FP32 arithmetic operations per cell-stage (ncu) against "
                                           f"{FP32_PEAK_TOPS:.1f} T/s (128 lanes/SM x 152 SMs x 2.07 GHz)"
                                           if l_ops is not None else "no ncu count for this variant")},
                 "error_vs_fp64_gpu": field_errors(lm_state, lf_state)}

    # ---- many tanks in one batch vs the same tanks run one after another ----
    batched = None
    if not args.no_large:
        batched = run_batched(args, stream, flush, barrier)
    checks = None
    if not args.no_checks and rank == 0:
        checks = run_checks(stream)

    if rank != 0:
        return
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "cells": case.cells, "rk_stages": case.options.s_max,
                       "pseudo_iters_per_step": statistics.mean(iters), "tol": case.tol,
                       "max_iters": case.max_iters,
                       "l2": "flushed between timed steps (256 MiB write outside the event pairs)",
                       "parallelism": f"replicas x{ws}"},
            "wall_s": wall, "gpu_launches": launches, "roofline": roofline, "e2e": e2e,
            "clocks": clk.summary(), "mixed": mixed}
    if large is not None:
        line["mixed_large"] = large
    if batched is not None:
        line["batched"] = batched
    if checks is not None:
        line["checks"] = checks
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline_sample(case)
        line["cpu_baseline_all_cores"] = cpu_baseline_all_cores(args.workload)
    print(json.dumps(line), flush=True)


BATCH_ABS_TOL = (0.03, 0.3, 0.3, 100.0)


def run_checks(stream):
    """The single-tank configurations' own checks, GPU against GPU, after the
    timed legs: the hydrostatic tank 256x256 at its stated 100 physical steps in
    both forms (at rest to 1e-10 m/s, the pressure kink held: slope ratio water
    / air = 1000); the collapsing water column 1024x512 while it moves, mixed
    against FP64 after 10 physical steps of 100 pseudo-iterations, every field
    and momentum component against its own maximum (the regime where the
    pressure increment is largest); and the Riemann tank 200x4 at its stated 20
    physical steps, mixed against FP64.  The stopping test is on (1e-8 drop or
    500 pseudo-iterations) except for the fixed-length water column."""
    import numpy as np
    from paper_2108_08769_gb300 import ac, workloads as W

    def run(case, prec, steps, tol, iters):
        t = ac.Tank.from_case(case, precision=prec)
        t.set_stream(stream.cuda_stream)
        its = []
        for _ in range(steps):
            its.append(t.physical_step(case.dt, tol, iters)[1])
        state = t.get_state()
        t.close()
        return state, {"pseudo_iters_min": min(its), "pseudo_iters_max": max(its)}

    def max_velocity(q):
        return float(max(np.abs(q[1] / q[0]).max(), np.abs(q[2] / q[0]).max()))

    t0 = time.perf_counter()
    out = {}
    hc = W.hydrostatic_tank(256)
    f64, f_it = run(hc, "fp64", hc.steps, hc.tol, hc.max_iters)
    mx, m_it = run(hc, "mixed", hc.steps, hc.tol, hc.max_iters)
    col = f64[3][:, hc.nx // 2]
    sl = np.diff(col) / hc.dy
    out["hydrostatic_256_100_steps"] = {
        "fp64": {"max_velocity": max_velocity(f64), "kink_slope_ratio": float(sl[hc.ny // 4] / sl[3 * hc.ny // 4]),
                 **f_it},
        "mixed": {"max_velocity": max_velocity(mx), **m_it, "error_vs_fp64": field_errors(mx, f64)},
        "pass": bool(max_velocity(f64) < 1e-10 and max_velocity(mx) < 1e-10
                     and abs(sl[hc.ny // 4] / sl[3 * hc.ny // 4] - 1000.0) < 1e-6)}
    wc = W.water_column(1024, 512)
    f64, _ = run(wc, "fp64", 10, -1.0, 100)
    mx, _ = run(wc, "mixed", 10, -1.0, 100)
    err = field_errors(mx, f64)
    out["water_column_1024x512_10x100"] = {
        "max_velocity_fp64": max_velocity(f64), "error_vs_fp64": err,
        "pass": bool(max(err["rho_unfloored"], err["rhou_unfloored"], err["rhov_unfloored"], err["p_unfloored"])
                     <= 1e-5)}
    rc = W.riemann_tank()
    f64, f_it = run(rc, "fp64", rc.steps, rc.tol, rc.max_iters)
    mx, m_it = run(rc, "mixed", rc.steps, rc.tol, rc.max_iters)
    err = field_errors(mx, f64)
    out["riemann_200x4_20_steps"] = {"fp64": f_it, "mixed": {**m_it, "error_vs_fp64": err},
                                     "pass": bool(max(err["rho"], err["rhou"], err["rhov"], err["p"]) <= 1e-5)}
    out["wall_s"] = time.perf_counter() - t0
    out["note"] = ("FP64 against the FP64 oracle (1e-11 per physical step) and the Riemann tank against the exact "
                   "solution are the GPU tests' (tests/test_gpu_configs.py, tests/test_gpu_riemann.py)")
    return out


def run_batched(args, stream, flush, barrier):
    """64 closed tanks (sizes 64^2..1024^2, density ratio 2..1000, own beta)
    advanced as one batch, against the same tanks run one after another as
    single mixed-form contexts; same stopping rule (absolute residual
    floors), same iteration cap."""
    import torch
    from paper_2108_08769_gb300 import ac, workloads as W
    cases = W.batched_tanks(count=64, nmin=64, nmax=1024)
    for c in cases:
        c.options.abs_tol = BATCH_ABS_TOL
    max_iters = 500
    b = ac.Batch.from_cases(cases)
    b.set_stream(stream.cuda_stream)
    b.physical_step(1e-3, 0.0, max_iters)           # warm-up (and tile-shape tuning)
    for k, c in enumerate(cases):
        b.set_state(k, *c.state())
    steps = min(args.steps, 2)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    its_all = []
    launches0 = b.kernel_launches()
    barrier()
    for s_ in range(steps):
        flush.zero_()
        ev[s_][0].record(stream)
        rc, its, st = b.physical_step(1e-3, 0.0, max_iters)
        ev[s_][1].record(stream)
        its_all.append(its)
    barrier()
    b_ms = sum(x.elapsed_time(y) for x, y in ev)
    b_launches = b.kernel_launches() - launches0
    for k, c in enumerate(cases):
        b.set_state(k, *c.state())
    b.set_profiling(True)
    b.physical_step(1e-3, -1.0, 20)     # every tank active in every launch
    st_ms, st_n = b.stage_kernel_time()
    b.set_profiling(False)
    shape = b.tile_shape()
    b.close()
    cell_iters = sum(c.cells * it for its in its_all for c, it in zip(cases, its))
    # the same tanks one after another
    q_ms, q_cell_iters = 0.0, 0
    for c in cases:
        t = ac.Tank.from_case(c, precision="mixed")
        t.set_stream(stream.cuda_stream)
        t.physical_step(1e-3, 0.0, max_iters)
        for s_ in range(steps):
            t.set_state(*c.state())
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.zero_()
            e0.record(stream)
            rc, n = t.physical_step(1e-3, 0.0, max_iters)
            e1.record(stream)
            e1.synchronize()
            q_ms += e0.elapsed_time(e1)
            q_cell_iters += c.cells * n
        t.close()
    total_cells = sum(c.cells for c in cases)
    value = cell_iters / (b_ms * 1e-3)
    seq = q_cell_iters / (q_ms * 1e-3)
    per_launch_s = st_ms * 1e-3 / max(st_n, 1)
    gbs = MIXED_BYTES_PER_CELL_ITER / 3.0 * total_cells / per_launch_s / 1e9
    return {"workload": "64 closed tanks, square sizes uniform 64^2..1024^2 (seeded), density ratio log-uniform "
                        "[2,1000], water column w, h uniform [0.2,0.6], beta = rho_heavy (10 sqrt(g h))^2, mixed "
                        f"form, dt=1e-3 s, each tank stops on its own absolute residual floors {BATCH_ABS_TOL} "
                        f"or {max_iters} pseudo-iterations",
            "tanks": len(cases), "cells": total_cells, "steps": steps, "value": value, "unit": UNIT,
            "ms_per_step": b_ms / steps, "iters_per_tank_min_max": [min(its_all[-1]), max(its_all[-1])],
            "tanks_converged_early": sum(1 for x in its_all[-1] if x < max_iters),
            "sequential_single_tank_value": seq, "speedup_vs_sequential": value / seq,
            "gpu_launches": b_launches, "tile_shape": {"tx": shape[0], "ty": shape[1], "threads": shape[2]},
            "stage_launch_ms_all_tanks_active": per_launch_s * 1e3,
            "roofline_all_tanks_active": {"bound": "hbm", "achieved": gbs, "peak": measured_hbm_gbs(),
                                          "unit": "GB/s", "frac": gbs / measured_hbm_gbs()}}


# FP64 flops of one stage per cell that the method itself needs (the
# rank-2 Osher flux of one x- and one y-face, 178 flops each, in the form
# whose acoustic terms carry no density; W, the limited slopes'
# differences, the pressure gradient of Eq. new_gradp, the face states, the
# divergence, sources and the point-implicit update; the real-time terms,
# local dtau and residual squares of stage 1 averaged over the three
# stages), counted with an FMA as 2 flops and a reciprocal, square root or
# reciprocal square root as 1; limiting, comparisons and sign handling
# count 0.  The derivation is tabulated with the design notes.  It does not
# move when the kernel executes fewer or more operations (recomputation on
# a tile's ring, stage-1 values read back), only with the formulation.
FP64_ALG_FLOPS_PER_CELL_STAGE = 483.0
# what stage_kernel<double,32,14> executes on this 256x256 tank (ncu: DFMA x 2
# + DADD + DMUL, mean of stages 1-3: 721.2, 639.2, 639.2; the tile's ring
# recomputes slopes and pressure gradients, and stage 1 forms the values
# stages 2 and 3 read back), and the FP64 instructions behind them
FP64_EXEC_FLOPS_PER_CELL_STAGE = 666.5
FP64_INSTR_PER_CELL_STAGE = 455.3
FP64_PIPE_INSTR_PER_S = 2 * 152 * 2.07e9
# DRAM bytes per cell of one FP64 stage launch, same capture, averaged over
# the three stages (3.74, 6.36, 6.36 MB read; the output stays in L2)
FP64_TRAFFIC_PER_CELL_STAGE = 83.7
# algorithmic HBM bytes per cell-iteration of the FP64 sweep (s_max = 3):
# stage 1 reads Q^{m} (32 B) and Q^n (24 B), writes Q^1 (32 B) and the four
# per-cell values kept for the later stages (32 B); stages 2 and 3 read
# Q^{s-1}, Q^{m} and those values and write Q^s (4 x 32 B each)
BYTES_PER_CELL_ITER_F64 = 376.0
# mixed form: stage 1 reads the (Q^n, rho_ref) and (dQ^{m}, dp^{m}) records
# (2 x 16 B) and the level-jump record (8 B) and writes 16 B; stages 2 and 3
# also read the (dQ^{s-1}, dp^{s-1}) record (16 B).  The column-strip sweep
# moves 4 B per cell and stage more (stage 1 stores the local pseudo-time
# step, stages 2 and 3 read it): 212 B, a choice of the kernel, not counted here
MIXED_BYTES_PER_CELL_ITER = 56.0 + 2 * 72.0
# measured (ncu, stages 1 and 2 of a pseudo-iteration on this 2048x8192
# tank, summarised under profiles/) for the strip variant the autotuner
# picks there: DRAM bytes and FP32 arithmetic operations (FFMA, FADD, FMUL;
# packed FP32x2 forms counted as two) per cell of one stage launch, the
# mean over the three stages (stage 3 as stage 2).  A variant without a
# capture of its current code reports null.
MIXED_COUNTS_BY_VARIANT = {
    16: ((61.5 + 2 * 79.7) / 3, (449.7 + 2 * 405.6) / 3),   # sweep_kernel_mixed<64,4,4,1>, <64,4,4,2>
    17: ((60.0 + 2 * 77.5) / 3, (446.5 + 2 * 402.4) / 3),   # sweep_kernel_mixed<128,4,4,1>, <128,4,4,2>
}
FP32_PEAK_TOPS = 128 * 152 * 2.07e9 / 1e12


def measured_hbm_gbs():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except Exception:
        return 6800.0


def run_configs(args, rank, local):
    """Every single-tank configuration of the test set at its stated length,
    in both forms, one JSON line each: throughput (CUDA events around every
    physical step, the stopping test on: 1e-8 residual drop or 500
    pseudo-iterations), the HBM fraction from the algorithmic bytes, per-field
    relative L-inf and L1 errors of the mixed form against FP64, the
    configuration's own checks, and the clocks seen.  The Rayleigh-Taylor tank
    runs --config4-steps of its 200 physical steps (the FP64 form alone takes
    ~23 s per step there).  The Riemann tank against the FP64 oracle over its
    20 steps and against the exact solution are GPU tests
    (tests/test_gpu_configs.py, tests/test_gpu_riemann.py)."""
    import numpy as np
    import torch
    from paper_2108_08769_gb300 import ac, workloads as W
    if rank != 0:
        return
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def run(case, prec, steps):
        t = ac.Tank.from_case(case, precision=prec)
        t.set_stream(stream.cuda_stream)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        its, rcs = [], []
        with Clocks(local) as clk:
            for k in range(steps):
                flush.zero_()
                evs[k][0].record(stream)
                rc, n = t.physical_step(case.dt, case.tol, case.max_iters)
                evs[k][1].record(stream)
                its.append(n)
                rcs.append(rc)
            torch.cuda.synchronize(dev)
        ms = sum(a.elapsed_time(b) for a, b in evs)
        state = t.get_state()
        tx, ty, nt, v = t.tile_shape()
        t.close()
        val = case.cells * sum(its) / (ms * 1e-3)
        bpc = BYTES_PER_CELL_ITER_F64 if prec == "fp64" else MIXED_BYTES_PER_CELL_ITER
        return state, {"value": val, "unit": UNIT, "ms_per_step": ms / steps,
                       "hbm_frac_of_measured": val * bpc / 1e9 / measured_hbm_gbs(),
                       "pseudo_iters": {"min": min(its), "max": max(its), "total": sum(its)},
                       "converged_steps": sum(1 for r in rcs if r == ac.AC_OK),
                       "tile": [tx, ty, nt], "tile_variant": v, "clocks": clk.summary()}

    configs = [("riemann_200x4", W.riemann_tank, None), ("hydrostatic_256", lambda: W.hydrostatic_tank(256), None),
               ("water_column_1024x512", lambda: W.water_column(1024, 512), None),
               ("rayleigh_taylor_2048x8192", lambda: W.rayleigh_taylor(2048, 8192), args.config4_steps)]
    for name, fn, nsteps in configs:
        case = fn()
        steps = nsteps or case.steps
        line = {"config": name, "cells": case.cells, "physical_steps": steps, "of_stated": case.steps,
                "dt": case.dt, "t_end": steps * case.dt, "tol": case.tol, "max_iters": case.max_iters}
        f64, line["fp64"] = run(case, "fp64", steps)
        mixed, line["mixed"] = run(case, "mixed", steps)
        line["mixed"]["speedup_vs_fp64"] = line["mixed"]["value"] / line["fp64"]["value"]
        line["mixed"]["error_vs_fp64_gpu"] = field_errors(mixed, f64)
        if name == "hydrostatic_256":
            # at rest to 1e-10, the pressure kink held: slope ratio water/air = density ratio
            u = np.abs(f64[1] / f64[0]).max()
            v = np.abs(f64[2] / f64[0]).max()
            col = f64[3][:, case.nx // 2]
            sl = np.diff(col) / case.dy
            line["fp64"]["max_velocity"] = float(max(u, v))
            line["fp64"]["kink_slope_ratio"] = float(sl[case.ny // 4] / sl[3 * case.ny // 4])
            line["mixed"]["max_velocity"] = float(max(np.abs(mixed[1] / mixed[0]).max(), np.abs(mixed[2] / mixed[0]).max()))
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    ws, rank, local = dist_init()
    if args.configs:
        run_configs(args, rank, local)
    elif args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
