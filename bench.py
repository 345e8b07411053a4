#!/usr/bin/env python3
"""Benchmark of the localized Newton solver (Algorithm 1) on the 400x400 + DFN model.

One step = one whole simulation case: the 40 timesteps (0.01 d growing to 30 d, 365 d in
total) of the 400x400-cell matrix with a 300-segment natural fracture network and four
80-cell hydraulic fractures on a producer at 1500 psi (166,659 cells), started from the
initial state.  Residual, Jacobian assembly, convergence checks and the Newton update are
FP64; the BiCGStab solve and its preconditioner run in FP32 as an inexact Newton (the default,
--krylov fp64 for FP64 throughout).  The headline value is cell-Newton-updates per second (the
sum over Newton iterations of the active-set size n_A, divided by the case time).  Beside it:
the same case with the other Krylov precision and with standard (full-domain) Newton on the
same GPU, the final fields' error against the FP64 CPU oracle, the end-to-end figure through
the C ABI with host buffers, the roofline of the dominant kernel, the CPU oracle on a bounded
sample of the same workload, and the SM clocks.

Multi-GPU: the path does not shard (one model per process), so N GPUs run N independent
replicas ("weak" scaling); rank 0 prints the aggregate.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-Newton-updates/s & case time, localized vs full Newton; p99 req latency"
UNIT = "cell-Newton-updates/s"
FALLBACK_HBM_GBS = 6800.0
FP64_PEAK_TFLOPS = 1.25  # GB300 nominal FP64 rate (vector and tensor alike)
# FP64 instructions the GPU retires per cycle (ncu sm__sass_thread_inst_executed_op_dfma_pred_on
# .sum.peak_sustained on GB300: 2 per SM per cycle) at the maximum SM clock
FP64_INSTR_PEAK_G = 304 * 2.07
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mode", choices=["local", "full", "dd"], default="local",
                    help="solver whose case is the headline (default: Algorithm 1)")
    ap.add_argument("--case", choices=["config1", "config0", "config2"], default="config1",
                    help="config1: 400x400 + DFN (the headline); config0: 50x50 + one fracture; config2: the 3D "
                         "200x200x20 + 2000-fracture oil-water model")
    ap.add_argument("--krylov", choices=["fp32", "fp64"], default="fp32",
                    help="BiCGStab and preconditioner precision: FP32 (inexact Newton, the default) or FP64; "
                         "residual, Jacobian assembly, convergence checks and updates are FP64 in both")
    ap.add_argument("--fp32-krylov", action="store_true", help="same as --krylov fp32")
    ap.add_argument("--precond", choices=["lines", "cells"], default="lines",
                    help="block Jacobi with fracture-segment blocks (default) or single-cell blocks")
    ap.add_argument("--headline-only", action="store_true",
                    help="run only the headline case (for profiler launch lists)")
    ap.add_argument("--ensemble-only", action="store_true",
                    help="run only the batched-ensemble run (--ensemble realizations) and print its record")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the CPU-oracle sample")
    ap.add_argument("--serve-seconds", type=float, default=20.0,
                    help="each measured window of the serving run (Poisson arrivals); 0 skips it")
    ap.add_argument("--serve-runs", type=int, default=3, help="measured serving windows (their spread is reported)")
    ap.add_argument("--serve-warmup", type=float, default=10.0, help="serving warm-up before the windows (s)")
    ap.add_argument("--serve-models", type=int, default=64, help="resident models of the serving run")
    ap.add_argument("--serve-rate", type=float, default=200.0, help="request arrival rate (1/s)")
    ap.add_argument("--serve-workers", type=int, default=8, help="requests run at once")
    ap.add_argument("--ensemble", type=int, default=256,
                    help="realizations in the batched-ensemble run (N ~ U{150..500} grids; 0 skips it)")
    ap.add_argument("--large-3d", type=int, default=1,
                    help="1: also run the 3D 200x200x20 + 2000-fracture oil-water case once per Krylov precision")
    ap.add_argument("--iteration-log", default=None,
                    help="after the run, write one JSON line per Newton iteration of one more (untimed) case "
                         "(n_A, Krylov iterations, per kernel class: ms and algorithmic bytes)")
    ap.add_argument("--write-traffic", default=None, metavar="NCU_RAW_CSV",
                    help="no GPU work: write profiles/traffic.json from an ncu raw-page CSV of one launch "
                         "(--kernel-class, its 0-based --launch-index) and the --iteration-log of the same case")
    ap.add_argument("--kernel-class", default="bicgstab", help="kernel class of --write-traffic")
    ap.add_argument("--launch-index", type=int, default=0, help="launch of the class captured (ncu -s)")
    ap.add_argument("--solver", choices=["grid", "cluster"], default=None,
                    help="--write-traffic: the solver the captured launch ran (checked against the log)")
    ap.add_argument("--krylov-rtol", type=float, default=None,
                    help="BiCGStab relative tolerance (default: the library's)")
    return ap.parse_args()


def make_case(name):
    from paper_2008_01539_gb300 import casegen as cg

    return {"config1": cg.config1, "config0": cg.config0, "config2": cg.config2}[name]()


def workload_name(case, args):
    if "nz" in case.meta or "nx" not in case.meta:
        return f"{case.name}, n={case.n} cells, {len(case.dt_schedule)} timesteps"
    mode = {"local": "localized Newton (Algorithm 1, m=2, eps=0.3 psi)", "full": "standard Newton",
            "dd": "adaptive nonlinear DD (Algorithm 2, m=2)"}[args.mode]
    meta = case.meta
    return (f"{meta['nx']}x{meta['ny']} matrix ({meta['dx']:.0f} m cells) + {meta['n_segments'] - meta['n_hf']}-segment "
            f"DFN + {meta['n_hf']} hydraulic fractures, n={case.n} cells, {len(case.dt_schedule)} timesteps to "
            f"{case.dt_schedule.sum() / 86400:.0f} d, {mode}, "
            f"{'FP64 residual/Jacobian + FP32 BiCGStab' if args.fp32_krylov else 'FP64 throughout'}")


# ---------------------------------------------------------------------------------------
# distributed plumbing (replicas only)
# ---------------------------------------------------------------------------------------
def dist_setup(args):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def reduce_max(x, world):
    return _reduce(x, world, "max")


def reduce_sum(x, world):
    return _reduce(x, world, "sum")


def _reduce(x, world, op):
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if torch.cuda.is_available() and dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.idx)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in out.strip().splitlines():
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------------------
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("k_krylov.cu", "k_assemble.cu", "k_sets.cu", "lns_internal.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2008_01539_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_class, alg_bytes_per_launch):
    """DRAM bytes per launch: the ncu capture's DRAM/algorithmic byte ratio (profiles/
    traffic.json) applied to this launch's algorithmic bytes, i.e. scaled by the rows and
    iterations the launch processes.  None when absent or when the kernel sources changed
    since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return None
    k = d.get("kernels", {}).get(kernel_class)
    if not k or d.get("source_hash") != kernel_source_hash():
        return None
    return k["dram_over_algorithmic"] * alg_bytes_per_launch


def run_case(model, case):
    """All timesteps of the case from the model's current state; returns the step stats."""
    out = []
    for dt in case.dt_schedule:
        st = model.lns_timestep(float(dt))
        out.append(st)
    return out


# ---------------------------------------------------------------------------------------
# CPU oracle: bounded sample of the same workload
# ---------------------------------------------------------------------------------------
def oracle_sample(case, mode, budget_s, max_steps=None):
    import oracle as O

    mode_id = {"local": 1, "full": 0, "dd": 2}[mode]
    sim = O.Sim(case, O.Options(mode=mode_id))
    updates = 0
    steps = 0
    t0 = time.perf_counter()
    for dt in case.dt_schedule:
        st = sim.timestep(float(dt))
        updates += st["cell_updates"]
        steps += 1
        if time.perf_counter() - t0 >= budget_s or (max_steps and steps >= max_steps):
            break
    el = time.perf_counter() - t0
    return updates, el, steps


# ---------------------------------------------------------------------------------------
# reference arm: the CPU oracle, timed on the host cores
# ---------------------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    case = make_case(args.case)
    # one step = the first `steps_per_sample` timesteps of the case, sized to a few seconds
    probe_u, probe_t, probe_steps = oracle_sample(case, args.mode, 4.0)
    n_ts = max(1, probe_steps)
    for _ in range(args.warmup):
        oracle_sample(case, args.mode, 1e9, max_steps=n_ts)
    times, ups = [], []
    for _ in range(args.steps):
        u, t, _ = oracle_sample(case, args.mode, 1e9, max_steps=n_ts)
        times.append(t)
        ups.append(u)
    value = sum(ups) / sum(times)
    sample = f"first {n_ts} of {len(case.dt_schedule)} timesteps of the case, oracle mode {args.mode}"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(case, args) + "; CPU oracle (plain C, hand-written sparse LU)",
                       "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------------
def time_case(model, case, steps, flush, stream):
    """Run the case `steps` times from the initial state; CUDA-event times (s) and stats."""
    import torch

    ev, stats_all = [], []
    for _ in range(steps):
        flush.zero_()
        model.lns_reset()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        stats_all.append(run_case(model, case))
        e1.record(stream)
        ev.append((e0, e1))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) / 1e3 for a, b in ev], stats_all


def field_error(p, sw, p_ref, sw_ref):
    """Difference of final fields from the FP64 oracle's."""
    import numpy as np

    from paper_2008_01539_gb300 import lns

    dp = np.abs(p - p_ref)
    return {"max_abs_dp_psi": float(dp.max()) / lns.PSI,
            "max_rel_dp": float((dp / np.abs(p_ref)).max()),
            "max_abs_dsw": float(np.abs(sw - sw_ref).max())}


def oracle_case(case, mode):
    """The FP64 oracle's final fields for the whole case (the accuracy reference)."""
    import oracle as O

    mode_id = {"local": 1, "full": 0, "dd": 2}[mode]
    sim = O.Sim(case, O.Options(mode=mode_id))
    t0 = time.perf_counter()
    for dt in case.dt_schedule:
        sim.timestep(float(dt))
    return sim.p.copy(), sim.sw.copy(), time.perf_counter() - t0


def tight_errors(case, opts):
    """The whole case at a tight Newton tolerance (tol_dp = 1 Pa, CNV < 1e-10) on both sides:
    Algorithm 1 with the FP64 Krylov (1e-12) and with the FP32 Krylov (the headline's 1e-5), final
    fields against the oracle's."""
    import oracle as O
    from paper_2008_01539_gb300 import lns

    tight = dict(tol_dp=1.0, tol_cnv=1e-10, max_newton=40)
    sim = O.Sim(case, O.Options(mode=1, **tight))
    its_ref = [sim.timestep(float(dt))["iterations"] for dt in case.dt_schedule]
    out = {"tolerance": "tol_dp 1 Pa, CNV 1e-10", "oracle_newton_iterations": sum(its_ref)}
    for tag, kw in (("fp64_krylov", dict(krylov_fp32=0, krylov_rtol=1e-12, krylov_maxit=20000)),
                    ("fp32_krylov", dict(krylov_fp32=1, krylov_rtol=1e-5))):
        m = lns.Model(case, lns.Options(**{**opts.__dict__, **tight, **kw}))
        its = [m.lns_timestep(float(dt))["iterations"] for dt in case.dt_schedule]
        p, sw = m.lns_get_state()
        m.close()
        e = field_error(p, sw, sim.p, sim.sw)
        e["newton_iterations"] = sum(its)
        e["max_per_step_iteration_difference"] = max(abs(a - b) for a, b in zip(its, its_ref))
        out[tag] = e
    return out


def large_3d_run(opts, flush, stream):
    """config2-shaped 3D case, once with FP32 and once with FP64 BiCGStab, kernel classes timed."""
    import numpy as np

    from paper_2008_01539_gb300 import casegen as cg
    from paper_2008_01539_gb300 import lns

    hbm, _ = measured_peaks()
    t0 = time.perf_counter()
    case = cg.config2()
    out = {"workload": f"{case.name}: 200x200x20 matrix (5x5x2 m cells) + 10 hydraulic-fracture stages "
                       f"(40x12 cells) + 2000 natural-fracture panels, n={case.n} cells, "
                       f"{len(case.dt_schedule)} timesteps to {case.dt_schedule.sum() / 86400:.0f} d, oil-water "
                       f"(the three-phase black-oil variant is not built), localized Newton",
           "cells": case.n, "generate_s": time.perf_counter() - t0}
    states = {}
    for tag, fp32 in (("fp32_krylov", 1), ("fp64_krylov", 0)):
        o = lns.Options(**{**opts.__dict__, "krylov_fp32": fp32, "krylov_rtol": 1e-5 if fp32 else 1e-6,
                           "profile": 1})
        m = lns.Model(case, o)
        for dt in case.dt_schedule[:2]:  # warm-up: first two timesteps
            m.lns_timestep(float(dt))
        m.lns_reset_kernel_times()
        t, st = time_case(m, case, 1, flush, stream)
        kt = m.lns_kernel_times()
        states[tag] = m.lns_get_state()
        m.close()
        st = st[0]
        r = {"case_time_s": t[0], "value": sum(x["cell_updates"] for x in st) / t[0], "unit": UNIT,
             "newton_iterations": sum(x["iterations"] for x in st),
             "krylov_iterations": sum(x["krylov_iters"] for x in st),
             "fp64_retries": sum(x["fp64_retries"] for x in st),
             "M_A_per_case": sum(x["cell_updates"] for x in st) / case.n,
             "kernels": {k["name"]: {"launches": k["launches"], "ms": round(k["total_ms"], 2),
                                     "GBps": k["bytes"] / (k["total_ms"] / 1e3) / 1e9 if k["total_ms"] > 0 else None,
                                     "frac_of_measured_hbm": k["bytes"] / (k["total_ms"] / 1e3) / 1e9 / hbm
                                     if k["total_ms"] > 0 else None}
                         for k in kt if k["launches"] > 0}}
        out[tag] = r
    out["fp32_krylov"]["error_vs_fp64_krylov_gpu"] = field_error(*states["fp32_krylov"], *states["fp64_krylov"])
    if os.environ.get("RANK", "0") == "0":
        out["cpu_baseline"] = oracle_ilu0_iteration(case)
    return out


def oracle_ilu0_iteration(case):
    """The oracle's per-Newton-iteration time on the 3D model: one Algorithm 1 iteration (the first
    timestep's first, on its initial active set) with the block ILU(0)-preconditioned BiCGStab
    linear step; the sparse LU is infeasible at this size."""
    import numpy as np

    import oracle as O

    m = O.Model(case)
    opts = O.Options(mode=1, linear=1, lin_rtol=1e-8)
    va = O.initial_set(m, opts, np.zeros(case.n, np.uint8), False)
    t0 = time.perf_counter()
    O.local_solve(m, opts, case.p0, case.sw0, case.p0, case.sw0, float(case.dt_schedule[0]), va)
    t = time.perf_counter() - t0
    n_a = int(va.sum())
    return {"value": n_a / t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one Newton iteration of Algorithm 1 (the first timestep's first, n_A = {n_a} rows) with "
                      f"the oracle's block ILU(0)-BiCGStab linear step (rtol 1e-8), single thread, {t:.1f} s; the "
                      f"oracle's sparse LU is infeasible at a million cells"}


ENSEMBLE_SPAN_DAYS = 30.0
ENSEMBLE_CTL = dict(dt_init=0.01 * 86400.0, dt_min=0.01 * 86400.0 / 64, dt_max=10.0 * 86400.0, grow=2.0, cut=0.5,
                    easy_iters=4)


def _oracle_realization(r):
    """One realization advanced by the oracle with the ensemble's controller (a worker process)."""
    sys.path.insert(0, ROOT)
    import oracle as O
    from paper_2008_01539_gb300 import casegen as cg

    case = cg.realization(r)
    sim = O.Sim(case, O.Options(mode=1))
    t0 = time.perf_counter()
    c = ENSEMBLE_CTL
    out = sim.advance(ENSEMBLE_SPAN_DAYS * 86400.0, c["dt_init"], c["dt_min"], c["dt_max"], c["grow"], c["cut"],
                      c["easy_iters"])
    return out["cell_updates"], time.perf_counter() - t0, case.n


def ensemble_cpu_baseline(cores):
    """The oracle on the host cores, one realization per core (realizations 0..cores-1)."""
    import multiprocessing as mp

    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_realization, range(cores), chunksize=1)
    wall = time.perf_counter() - t0
    upd = sum(r[0] for r in res)
    return {"value": upd / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"realizations 0-{cores - 1} ({sum(r[2] for r in res)} cells), one per host core in its own "
                      f"process, each advanced {ENSEMBLE_SPAN_DAYS:.0f} d by the oracle's Algorithm 1 with the same "
                      f"controller; wall {wall:.1f} s (slowest realization {max(r[1] for r in res):.1f} s)"}


def ensemble_run(args, opts, stream, cpu_baseline=True):
    """K independent realizations advanced together by lns_batch_advance (each member its own model,
    stream, active sets and time-step controller), localized and standard Newton; device time with
    CUDA events across the members' streams."""
    import torch

    from paper_2008_01539_gb300 import casegen as cg
    from paper_2008_01539_gb300 import lns

    t0 = time.perf_counter()
    cases = [cg.realization(r) for r in range(args.ensemble)]
    t_gen = time.perf_counter() - t0
    streams = [torch.cuda.Stream() for _ in cases]
    t0 = time.perf_counter()
    models = [lns.Model(c, opts, stream=s) for c, s in zip(cases, streams)]
    torch.cuda.synchronize()
    t_create = time.perf_counter() - t0
    span = ENSEMBLE_SPAN_DAYS * cg.DAY
    out = {"realizations": len(cases), "cells": int(sum(c.n for c in cases)),
           "workload": f"{len(cases)} seeded realizations (N x N matrix, N ~ U{{150..500}}, U{{50..400}} natural "
                       f"fractures, 2 hydraulic fractures on a producer each), each its own model advanced "
                       f"{ENSEMBLE_SPAN_DAYS:.0f} d by its own time-step controller (dt 0.01 d growing x2 after easy "
                       f"steps, at most 10 d, cut x0.5 on failure), all members together (lns_batch_advance)",
           "generate_s": t_gen, "create_s": t_create}
    try:
        for tag, mode in (("localized", lns.LNS_MODE_LOCAL), ("full_newton", lns.LNS_MODE_FULL)):
            mopts = lns.Options(**{**opts.__dict__, "mode": mode})
            for m in models:
                m.set_options(mopts)
                m.lns_reset()
            lns.lns_batch_advance(models, 0.05 * cg.DAY, **ENSEMBLE_CTL, allow_noconv=True)  # warm-up
            for m in models:
                m.lns_reset()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for s_ in streams:
                s_.wait_event(e0)
            outs, bst = lns.lns_batch_advance(models, span, **ENSEMBLE_CTL, allow_noconv=True)
            for s_ in streams:
                stream.wait_stream(s_)
            e1.record(stream)
            torch.cuda.synchronize()
            et = e0.elapsed_time(e1) / 1e3
            upd = sum(o["cell_updates"] for o in outs)
            out[tag] = {"time_s": et, "value": upd / et, "unit": UNIT, "cell_updates": upd,
                        "newton_iterations": sum(o["iterations"] for o in outs),
                        "krylov_iterations": sum(o["krylov_iters"] for o in outs),
                        "accepted_steps": sum(o["steps"] for o in outs), "step_cuts": sum(o["cuts"] for o in outs),
                        "failed_members": sum(1 for o in outs if o["status"] != 0),
                        "batch_rounds": bst["rounds"], "cluster_solves": bst["cluster_solves"],
                        "grid_solves": bst["grid_solves"]}
        out["speedup_vs_full_newton"] = out["full_newton"]["time_s"] / out["localized"]["time_s"]
    finally:
        for m in models:
            m.close()
    if cpu_baseline and os.environ.get("RANK", "0") == "0" and int(os.environ.get("WORLD_SIZE", "1")) == 1:
        out["cpu_baseline"] = ensemble_cpu_baseline(min(os.cpu_count() or 1, len(cases)))
    return out


def _serve_window(srv, ids, rng, rate, seconds, warmup):
    """Poisson arrivals of 'advance model k by dt' requests for warmup + seconds; the requests
    submitted after the warm-up are measured (latency = completion - submission, server clock)."""
    import numpy as np

    from paper_2008_01539_gb300 import casegen as cg

    start = srv.now()
    total = warmup + seconds
    t_next, sub, done = start, 0, []
    rid0 = _serve_window.rid
    while True:
        now = srv.now()
        while t_next <= now and t_next - start < total:
            mid = int(rng.integers(len(ids)))
            dt = float(np.exp(rng.uniform(np.log(0.1), np.log(30.0)))) * cg.DAY
            srv.submit(ids[mid], dt, _serve_window.rid)
            _serve_window.rid += 1
            sub += 1
            t_next += float(rng.exponential(1.0 / rate))
        done += srv.poll(512, 0.0)
        if t_next - start >= total:
            break
        time.sleep(max(0.0, min(t_next - srv.now(), 0.002)))
    srv.drain(600.0)
    while True:
        got = srv.poll(512, 0.0)
        if not got:
            break
        done += got
    done = [c for c in done if c["request_id"] >= rid0]
    meas = [c for c in done if c["t_submit"] - start >= warmup]
    ok = [c for c in meas if c["status"] == 0]
    lat = np.array([c["t_done"] - c["t_submit"] for c in ok])
    t_first = min(c["t_submit"] for c in meas) if meas else 0.0
    t_last = max(c["t_done"] for c in meas) if meas else 1.0
    upd = sum(c["stats"]["cell_updates"] for c in ok)
    return {"requests": len(meas), "failed": len(meas) - len(ok),
            "p50_latency_ms": float(np.percentile(lat, 50)) * 1e3 if len(lat) else None,
            "p99_latency_ms": float(np.percentile(lat, 99)) * 1e3 if len(lat) else None,
            "mean_latency_ms": float(lat.mean()) * 1e3 if len(lat) else None,
            "value": upd / max(t_last - t_first, 1e-9),
            "timestep_cuts": int(sum(c["stats"]["dd_outer"] for c in ok))}


_serve_window.rid = 0


def serving_run(args, opts):
    """Requests 'advance model k by dt' with Poisson arrivals over resident models of log-uniform
    size, half of them 2D (N x N matrix + DFN) and half 3D (N x N x 10 layers + fracture planes and
    panels); one warm-up window, then args.serve_runs measured windows on the same server."""
    import numpy as np

    from paper_2008_01539_gb300 import casegen as cg
    from paper_2008_01539_gb300 import lns

    rng = np.random.default_rng(4)
    sizes = np.exp(rng.uniform(np.log(1e4), np.log(1e6), args.serve_models)).astype(int)
    t0 = time.perf_counter()
    cases = [(cg.serving_model if k % 2 == 0 else cg.serving_model_3d)(k, int(c)) for k, c in enumerate(sizes)]
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    srv = lns.Server(workers=args.serve_workers, hbm_budget_bytes=150 << 30)
    ids = [srv.add_model(c, opts) for c in cases]
    t_setup = time.perf_counter() - t0
    _serve_window(srv, ids, rng, args.serve_rate, 0.0, args.serve_warmup)  # warm-up: models admitted
    runs = [_serve_window(srv, ids, rng, args.serve_rate, args.serve_seconds, 0.0) for _ in range(args.serve_runs)]
    st = srv.stats()
    srv.close()

    def spread(key):
        v = [r[key] for r in runs if r[key] is not None]
        return {"median": float(np.median(v)), "min": float(min(v)), "max": float(max(v))} if v else None

    return {
        "workload": f"{len(ids)} resident models ({sum(1 for k in range(len(ids)) if k % 2 == 0)} 2D N x N matrix + "
                    f"DFN, {sum(1 for k in range(len(ids)) if k % 2)} 3D N x N x 10 + fracture planes and panels; "
                    f"{int(min(c.n for c in cases))}-{int(max(c.n for c in cases))} cells, log-uniform), Poisson "
                    f"arrivals at {args.serve_rate:.0f}/s, dt log-uniform 0.1-30 d, model uniform, "
                    f"{args.serve_workers} workers, HBM budget 150 GB; each request through the time-step "
                    f"controller (cut down to dt/65536)",
        "window_s": args.serve_seconds, "windows": len(runs), "warmup_s": args.serve_warmup,
        "requests": sum(r["requests"] for r in runs), "failed": sum(r["failed"] for r in runs),
        "p50_latency_ms": spread("p50_latency_ms"), "p99_latency_ms": spread("p99_latency_ms"),
        "mean_latency_ms": spread("mean_latency_ms"),
        "value": float(np.median([r["value"] for r in runs])), "unit": UNIT,
        "per_window": runs,
        "timestep_cuts": sum(r["timestep_cuts"] for r in runs),
        "resident_models": st["resident_models"], "resident_gb": st["resident_bytes"] / 2 ** 30,
        "evictions": st["evictions"], "total_cells": int(sum(c.n for c in cases)), "generate_s": t_gen,
        "setup_s": t_setup}


def write_traffic(args):
    """profiles/traffic.json: DRAM bytes of one captured launch over its algorithmic bytes, tagged
    with the hash of the kernel sources (bench.py reports traffic only while they are unchanged)."""
    import csv

    rows = list(csv.reader(open(args.write_traffic)))
    hdr, data = rows[0], rows[2:]
    assert len(data) == 1, "the CSV must hold exactly one captured launch"
    col = {h: i for i, h in enumerate(hdr)}
    unit = rows[1]
    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}

    def val(name):
        return float(data[0][col[name]].replace(",", "")) * scale.get(unit[col[name]], 1.0)

    dram = val("dram__bytes_read.sum") + val("dram__bytes_write.sum")
    its = [json.loads(x) for x in open(args.iteration_log)]
    launches = [r for r in its if r["kernels"].get(args.kernel_class, {}).get("launches", 0) > 0]
    rec = launches[args.launch_index]
    if args.solver and rec.get("krylov_solver") != {"cluster": 1, "grid": 2}[args.solver]:
        raise SystemExit(f"iteration {args.launch_index} was not solved by the {args.solver} solver")
    alg = rec["kernels"][args.kernel_class]["bytes"]
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        out = json.load(open(path))
    except (OSError, ValueError):
        out = {}
    if out.get("source_hash") != kernel_source_hash():
        out = {"source_hash": kernel_source_hash(), "kernels": {}}
    out["kernels"][args.kernel_class] = {
        "dram_bytes": dram, "algorithmic_bytes": alg, "dram_over_algorithmic": dram / alg,
        "launch_index": args.launch_index, "n_active": rec["n_active"], "krylov_iters": rec["krylov_iters"],
        "case": args.case}
    json.dump(out, open(path, "w"), indent=1)
    print(json.dumps(out["kernels"][args.kernel_class]))
    return 0


def iteration_log(model, case, opts, path):
    """One more case with every kernel class timed, one Newton iteration at a time."""
    from paper_2008_01539_gb300 import lns

    model.set_options(lns.Options(**{**opts.__dict__, "profile": 1}))
    model.lns_reset()
    with open(path, "w") as f:
        for step, dt in enumerate(case.dt_schedule):
            while True:
                model.lns_reset_kernel_times()
                st = model.lns_newton_iter(float(dt))
                kt = {k["name"]: {"launches": k["launches"], "ms": k["total_ms"], "bytes": k["bytes"]}
                      for k in model.lns_kernel_times()}
                f.write(json.dumps({"step": step, "n_active": st["n_active"], "krylov_iters": st["krylov_iters"],
                                    "krylov_solver": st["krylov_solver"], "kernels": kt}) + "\n")
                if st["step_done"]:
                    break
    model.set_options(opts)


def main():
    args = parse()
    args.fp32_krylov = args.fp32_krylov or args.krylov == "fp32"
    if args.write_traffic:
        return write_traffic(args)
    if args.impl == "reference":
        return run_reference(args)
    import numpy as np
    import torch

    from paper_2008_01539_gb300 import lns

    rank, world, local = dist_setup(args)
    lns.load(build_if_missing=True)
    # the models run on a stream of their own (a captured Newton iteration cannot use the legacy
    # default stream)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        return bench_ours(args, rank, world, local)


def bench_ours(args, rank, world, local):
    import numpy as np
    import torch

    from paper_2008_01539_gb300 import lns

    if args.ensemble_only:
        eopts = lns.Options(mode=lns.LNS_MODE_LOCAL, krylov_fp32=int(args.fp32_krylov),
                            krylov_rtol=1e-5 if args.fp32_krylov else lns.Options().krylov_rtol)
        rec = ensemble_run(args, eopts, torch.cuda.current_stream(), cpu_baseline=False)
        print(json.dumps(rec), flush=True)
        return 0
    case = make_case(args.case)
    mode_id = {"local": lns.LNS_MODE_LOCAL, "full": lns.LNS_MODE_FULL, "dd": lns.LNS_MODE_DD}[args.mode]
    rtol = args.krylov_rtol if args.krylov_rtol is not None else (1e-5 if args.fp32_krylov else lns.Options().krylov_rtol)
    opts = lns.Options(mode=mode_id, krylov_fp32=int(args.fp32_krylov), krylov_rtol=rtol,
                       precond=lns.LNS_PRECOND_BJAC if args.precond == "lines" else lns.LNS_PRECOND_BJAC_CELL)
    stream = torch.cuda.current_stream()
    model = lns.Model(case, opts)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    # warm-up
    for _ in range(max(args.warmup, 0)):
        model.lns_reset()
        run_case(model, case)
    torch.cuda.synchronize()

    # timed region: K cases, inputs resident, L2 flushed before each case; the BiCGStab solves are
    # timed live with CUDA events (profile level 2: one event pair per Newton iteration)
    model.set_options(lns.Options(**{**opts.__dict__, "profile": 2}))
    model.lns_reset_kernel_times()
    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    launches0 = lns.lns_launch_count()
    ev = []
    updates = 0
    iters = 0
    kry = 0
    for _ in range(args.steps):
        flush.zero_()
        model.lns_reset()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        stats = run_case(model, case)
        e1.record(stream)
        ev.append((e0, e1))
        updates += sum(s["cell_updates"] for s in stats)
        iters += sum(s["iterations"] for s in stats)
        kry += sum(s["krylov_iters"] for s in stats)
    torch.cuda.synchronize()
    launches = lns.lns_launch_count() - launches0
    clk = clocks.stop()
    barrier(world)
    t_rank = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    t_max = reduce_max(t_rank, world)
    updates_all = reduce_sum(updates, world)
    value = updates_all / t_max
    ktimes_live = model.lns_kernel_times()
    p_final, sw_final = model.lns_get_state()
    # per-kernel split from one more (untimed) case with every kernel class timed
    model.set_options(lns.Options(**{**opts.__dict__, "profile": 1}))
    model.lns_reset_kernel_times()
    model.lns_reset()
    run_case(model, case)
    torch.cuda.synchronize()
    ktimes = model.lns_kernel_times()
    model.set_options(opts)
    if args.iteration_log and rank == 0:
        iteration_log(model, case, opts, args.iteration_log)

    # roofline of the dominant kernel (live CUDA-event timing inside the timed region)
    hbm, hbm_src = measured_peaks()
    dom = max(ktimes_live, key=lambda k: k["total_ms"])
    per_launch_s = dom["total_ms"] / 1e3 / max(dom["launches"], 1)
    bytes_per_launch = dom["bytes"] / max(dom["launches"], 1)
    achieved = bytes_per_launch / per_launch_s / 1e9 if per_launch_s > 0 else 0.0
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": ncu_traffic(dom["name"], bytes_per_launch), "kernel": dom["name"],
            "peak_source": f"{hbm_src} (MEASURED_PEAKS.json hbm_gbs)" if hbm_src == "measured" else "fallback",
            "share_of_case": dom["total_ms"] / 1e3 / max(t_rank, 1e-12)}
    # the assembly is bound by the FP64 pipe, not by bytes: its roof is the FP64 rate
    asm = [k for k in ktimes if k["name"] == "assemble" and k["total_ms"] > 0]
    asm_roof = None
    if asm:
        a = asm[0]
        gi = a["flops"] / (a["total_ms"] / 1e3) / 1e9  # FP64 instructions (per thread) per second, G
        asm_roof = {"bound": "alu", "kernel": "assemble", "achieved": gi, "peak": FP64_INSTR_PEAK_G,
                    "unit": "G FP64 instructions/s", "frac": gi / FP64_INSTR_PEAK_G,
                    "peak_source": "the FP64 pipe's 2 instructions per SM per cycle (ncu peak_sustained) x "
                                   "152 SMs x 2.07 GHz; MEASURED_PEAKS.json has no FP64 figure",
                    "instructions_per_row": "2 x (70 + 19 x degree), the ncu count on this case",
                    "ms_per_launch": a["total_ms"] / max(a["launches"], 1),
                    "GBps": a["bytes"] / (a["total_ms"] / 1e3) / 1e9}
    kernels = {k["name"]: {"launches": k["launches"], "ms": round(k["total_ms"], 3),
                           "GBps": (k["bytes"] / (k["total_ms"] / 1e3) / 1e9) if k["total_ms"] > 0 else None}
               for k in ktimes}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32" if args.fp32_krylov else "f64",
            "data": "synthetic (seeded generator shaped like the paper's DFN models)",
            "config": {"workload": workload_name(case, args), "cells": case.n, "timesteps": len(case.dt_schedule),
                       "l2": "flushed (256 MB write) before every timed case", "parallelism": f"replicas x{world}"},
            "case_time_s": t_max / max(args.steps, 1),
            "newton_iterations_per_case": iters / max(args.steps, 1),
            "krylov_iterations_per_case": kry / max(args.steps, 1),
            "M_A_per_case": updates / max(args.steps, 1) / case.n,
            "gpu_launches": launches, "kernels": kernels,
            "kernels_note": "split from one more (untimed) case with every kernel class timed by CUDA events",
            "roofline": roof, "assembly_roofline": asm_roof, "clocks": clk,
            "autotune": model.lns_get_tuning()}

    if not args.headline_only:
        # the other Krylov precision and standard Newton on the same GPU, same case
        def variant(vopts):
            vm = lns.Model(case, vopts)
            vm.lns_reset()
            run_case(vm, case)  # warm-up
            vt, vst = time_case(vm, case, max(1, min(args.steps, 3)), flush, stream)
            vp, vsw = vm.lns_get_state()
            vm.close()
            return vt, vst, vp, vsw

        other = "fp64" if args.fp32_krylov else "fp32"
        oopts = lns.Options(**{**opts.__dict__, "krylov_fp32": int(not args.fp32_krylov),
                               "krylov_rtol": lns.Options().krylov_rtol if args.fp32_krylov else 1e-5})
        vt, vst, vp, vsw = variant(oopts)
        line[f"{other}_krylov"] = {
            "case_time_s": statistics.mean(vt), "unit": UNIT,
            "value": sum(s["cell_updates"] for st in vst for s in st) / sum(vt),
            "newton_iterations_per_case": sum(s["iterations"] for st in vst for s in st) / len(vt),
            "krylov_iterations_per_case": sum(s["krylov_iters"] for st in vst for s in st) / len(vt),
            "krylov_rtol": oopts.krylov_rtol}
        other_state = (vp, vsw)
        if args.mode != "full":
            ft, fst, pf, _ = variant(lns.Options(**{**opts.__dict__, "mode": lns.LNS_MODE_FULL}))
            tf = statistics.mean(ft)
            line["full_newton"] = {"case_time_s": tf, "value": sum(s["cell_updates"] for st in fst for s in st) / sum(ft),
                                   "unit": UNIT,
                                   "newton_iterations_per_case": sum(s["iterations"] for st in fst for s in st) / len(ft),
                                   "max_abs_dp_vs_localized_psi": float(np.max(np.abs(pf - p_final))) / lns.PSI}
            line["speedup_vs_full_newton"] = tf / line["case_time_s"]
            # Algorithm 2 (adaptive nonlinear domain decomposition) on the same case
            try:
                dt_, dst, pd, _ = variant(lns.Options(**{**opts.__dict__, "mode": lns.LNS_MODE_DD}))
                line["algorithm2_dd"] = {
                    "case_time_s": statistics.mean(dt_), "unit": UNIT,
                    "value": sum(s["cell_updates"] for st in dst for s in st) / sum(dt_),
                    "local_solves_per_case": sum(s["iterations"] for st in dst for s in st) / len(dt_),
                    "outer_passes_per_case": sum(s["dd_outer"] for st in dst for s in st) / len(dt_),
                    "krylov_iterations_per_case": sum(s["krylov_iters"] for st in dst for s in st) / len(dt_),
                    "M_A_per_case": sum(s["cell_updates"] for st in dst for s in st) / len(dt_) / case.n,
                    "max_abs_dp_vs_localized_psi": float(np.max(np.abs(pd - p_final))) / lns.PSI}
            except lns.LnsError as err:
                line["algorithm2_dd"] = {"failed": str(err)}
            # its variants: subdomain visits to local convergence (up to 4 steps), with localization
            # inside the subdomain (later steps solve the previous step's support)
            try:
                dt_, dst, pd, _ = variant(lns.Options(**{**opts.__dict__, "mode": lns.LNS_MODE_DD,
                                                         "dd_local_newton": 4, "dd_local_shrink": 1}))
                line["algorithm2_dd_local"] = {
                    "case_time_s": statistics.mean(dt_), "unit": UNIT,
                    "value": sum(s["cell_updates"] for st in dst for s in st) / sum(dt_),
                    "local_solves_per_case": sum(s["iterations"] for st in dst for s in st) / len(dt_),
                    "outer_passes_per_case": sum(s["dd_outer"] for st in dst for s in st) / len(dt_),
                    "M_A_per_case": sum(s["cell_updates"] for st in dst for s in st) / len(dt_) / case.n,
                    "max_abs_dp_vs_localized_psi": float(np.max(np.abs(pd - p_final))) / lns.PSI,
                    "variant": "dd_local_newton 4, dd_local_shrink 1"}
            except lns.LnsError as err:
                line["algorithm2_dd_local"] = {"failed": str(err)}
            # the residual-based estimate the paper compares against (unconverged cells + 1 layer);
            # it grows the set one layer per iteration, so long steps take many more iterations
            try:
                rm = lns.Model(case, lns.Options(**{**opts.__dict__, "mode": lns.LNS_MODE_RESIDUAL, "m_layers": 1,
                                                    "max_newton": 3000}))
                for dt in case.dt_schedule[:2]:  # warm-up
                    rm.lns_timestep(float(dt))
                rt, rst = time_case(rm, case, 1, flush, stream)
                pr, swr = rm.lns_get_state()
                rm.close()
            except lns.LnsError as err:
                rt = None
                line["residual_sets"] = {"failed": str(err)}
        if args.mode != "full" and rt is not None:
            line["residual_sets"] = {
                "case_time_s": statistics.mean(rt), "unit": UNIT,
                "value": sum(s["cell_updates"] for st in rst for s in st) / sum(rt),
                "newton_iterations_per_case": sum(s["iterations"] for st in rst for s in st) / len(rt),
                "krylov_iterations_per_case": sum(s["krylov_iters"] for st in rst for s in st) / len(rt),
                "M_A_per_case": sum(s["cell_updates"] for st in rst for s in st) / len(rt) / case.n,
                "max_abs_dp_vs_localized_psi": float(np.max(np.abs(pr - p_final))) / lns.PSI,
                "note": "active set = cells with CNV >= tol_cnv on the full-domain residual, plus 1 layer "
                        "(the estimate the paper compares against); same Krylov settings as the headline, "
                        "max_newton 3000, one timed case"}
        # end to end through the C ABI with host buffers
        p_h = torch.from_numpy(np.ascontiguousarray(case.p0)).pin_memory()
        s_h = torch.from_numpy(np.ascontiguousarray(case.sw0)).pin_memory()
        po = torch.empty(case.n, dtype=torch.float64).pin_memory()
        so = torch.empty(case.n, dtype=torch.float64).pin_memory()
        e2e_t, e2e_u = [], 0
        barrier(world)
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            model.lns_set_state_ptrs(p_h.data_ptr(), s_h.data_ptr())
            st = run_case(model, case)
            model.lns_get_state_ptrs(po.data_ptr(), so.data_ptr())
            e2e_t.append(time.perf_counter() - t0)
            e2e_u += sum(s["cell_updates"] for s in st)
        te = reduce_max(sum(e2e_t), world)
        line["e2e"] = {"value": reduce_sum(e2e_u, world) / te, "unit": UNIT,
                       "h2d_bytes_per_step": 2 * 8 * case.n, "d2h_bytes_per_step": 2 * 8 * case.n,
                       "case_time_s": te / max(args.steps, 1)}
        # batched ensemble: independent realizations of uneven size advanced together
        if args.ensemble > 0:
            try:
                line["ensemble"] = ensemble_run(args, opts, stream)
            except lns.LnsError as err:
                line["ensemble"] = {"realizations": args.ensemble, "failed": str(err)}
            torch.cuda.empty_cache()
        # the 3D 200x200x20 matrix + 10 hydraulic-fracture stages + 2000 natural fractures (oil-water):
        # one case per Krylov precision with every kernel class timed (large active sets, where the
        # kernels run at HBM rates); the FP32 run's error is taken against the FP64 GPU run (the
        # oracle's sparse LU is far too slow at a million cells)
        if args.large_3d and rank == 0:
            line["large_3d"] = large_3d_run(opts, flush, stream)
        # serving: requests over many resident models (continuous batching on worker streams)
        if args.serve_seconds > 0:
            # long requested steps on large models need many expansion iterations (the active set
            # grows by m layers per iteration), hence a larger Newton budget per step
            line["serving"] = serving_run(args, lns.Options(**{**opts.__dict__, "max_newton": 60}))
        # accuracy: final fields against the FP64 oracle's whole case (rank 0, N = 1)
        if rank == 0 and world == 1:
            p_ref, sw_ref, t_ref = oracle_case(case, args.mode)
            line["error_vs_fp64_oracle"] = {
                "headline": field_error(p_final, sw_final, p_ref, sw_ref),
                f"{other}_krylov": field_error(other_state[0], other_state[1], p_ref, sw_ref),
                "oracle_case_time_s": t_ref,
                "note": "operating point: both sides stop at max|dp| < 0.3 psi per step, so differences below "
                        "that cutoff accumulate over the case"}
            if args.mode == "local":
                line["error_vs_fp64_oracle"]["tight_tolerance"] = tight_errors(case, opts)
        # CPU oracle on the host cores, bounded sample (rank 0, N = 1)
        if rank == 0 and world == 1:
            u, t, n_ts = oracle_sample(case, args.mode, args.cpu_seconds)
            line["cpu_baseline"] = {"value": u / t, "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": f"first {n_ts} of {len(case.dt_schedule)} timesteps of the same case, "
                                              f"oracle mode {args.mode} (plain C, single thread), {t:.1f} s"}
    model.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
