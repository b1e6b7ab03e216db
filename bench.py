"""Benchmark: cell-updates/s of the EGLM-MHD block-pool step on one GB300.

Workload: the 3D uniform linear Alfven wave, 256^3 cells as 4096 blocks of 16^3 (+2 ghost
layers), TVD-LF with the van Leer limiter, EGLM sources, gamma = 5/3 (synthetic input,
closed-form initial condition).  A step is one pass of the whole hot path: ghost fill,
CFL reduction (dt, c_h, c_p), the scheme update with sources and psi damping, and the FP64
conservation sums.  `value` is the FP32 + FP64-fix batched form (graph-replayed
map_advance); the plain FP64 form (per-level launches, host-synchronised dt) is reported
beside it.  The state (1.2 GB in FP32, 2.4 GB in FP64) is larger than the 129 MB L2, so
no flush is needed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""

from __future__ import annotations

import argparse
import json
import math
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

METRIC = "cell-updates/s"
WORKLOAD = "alfven3d_256^3_lf_vanleer_eglm"
BYTES_PER_CELL_F32 = 72.0     # read 9 x 4 B + write 9 x 4 B per cell-update
BYTES_PER_CELL_F64 = 144.0
# Floating-point operations per cell-update of this workload's step (TVD-LF, van Leer,
# EGLM, 3D), counted by the flop-counting build of the oracle on the 256^3 initial state
# with every face counted once (1651.9; the van Leer branch makes it data-dependent, by
# under 1% between 32^3 and 256^3).
FLOPS_PER_CELL = 1652.0
# FP32 peak of the CUDA cores: 152 SMs x 128 FP32 lanes x 2 flop per FMA x SM clock.
SMS, FP32_LANES_PER_SM = 152, 128
# DRAM bytes (read + write) of one step-kernel launch on the 128^3 case (512 blocks),
# from an ncu capture of the current kernel; traffic grows with the block count.
STEP_KERNEL_DRAM_BYTES_512_BLOCKS = 162.622464e6 + 107.649024e6


NAMES = ("rho", "mx", "my", "mz", "bx", "by", "bz", "e", "psi")


def error_table(A, B):
    """Per variable: L1 of A - B over the mean |B|, Linf over the max |B| (each scale floored
    at 1e-3 of the largest variable's)."""
    big1 = max(float(np.abs(B[:, v]).mean()) for v in range(9))
    bigi = max(float(np.abs(B[:, v]).max()) for v in range(9))
    l1, li = {}, {}
    for v, nm in enumerate(NAMES):
        d = np.abs(A[:, v] - B[:, v])
        l1[nm] = float(d.mean() / max(float(np.abs(B[:, v]).mean()), 1e-3 * big1))
        li[nm] = float(d.max() / max(float(np.abs(B[:, v]).max()), 1e-3 * bigi))
    return {"l1_rel": l1, "linf_rel": li}


def max_over_ranks(ms: float, dist=None, device: str = "cuda") -> float:
    """The job's time: the slowest rank's (every rank times the same number of steps).
    dist is torch.distributed (initialised) or None for one process."""
    if dist is None:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, cells: int, steps: int, ms: float) -> float:
    """Whole-job cell-updates/s: every rank runs its own replica of the workload (weak
    scaling, no collective on the data path), so the job updates world x cells per step."""
    return world * cells * steps / (ms * 1e-3)


def prints_line(rank: int) -> bool:
    """Only rank 0 prints the JSON line."""
    return rank == 0


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def sm_max_mhz():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return float(json.load(open(path)).get("sm_max_mhz", 2070.0)), "measured sm_max_mhz"
    return 2070.0, "nominal maximum SM clock"


class ClockSampler:
    """nvidia-smi samples during the timed region (clocks and throttle reasons)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def build_workload(size: int = 256):
    import workloads as w
    from workloads.problems import config_alfven3d
    cfg = config_alfven3d()
    if size != 256:
        cfg["mesh"] = w.uniform_mesh(3, 16, (size // 16,) * 3)
    mesh = cfg["mesh"]
    U0 = w.evaluate_on_mesh(mesh, w.alfven_wave, ndim=3)
    params = dict(cfg["params"], fp64_fix_tau=1e-2)
    return cfg, mesh, U0, params


def cpu_baseline(params, seconds: float = 10.0):
    """The oracle as it stands on the host cores, on a bounded sample of the same workload:
    a periodic 64^3 box (4^3 blocks of 16^3) of the same wave, stepped until ~seconds."""
    import workloads as w
    from oracle import Oracle
    mesh = w.uniform_mesh(3, 16, (4, 4, 4))
    U = w.evaluate_on_mesh(mesh, w.alfven_wave, ndim=3)
    orc = Oracle(mesh, U)
    orc.advance(params, 1)
    n, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        orc.advance(params, 1)
        n += 1
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    out = {"value": mesh.ncells * n / dt, "unit": METRIC, "cores": cores, "kind": "oracle",
           "sample": f"{n} steps of a 64^3 periodic box (4^3 blocks of 16^3) of the same wave, "
                     f"FP64 oracle, OpenMP over blocks, {dt:.1f} s"}
    # the same oracle on one host thread (the OpenMP runtime's thread count, restored after)
    import ctypes
    try:
        gomp = ctypes.CDLL("libgomp.so.1")
    except OSError:
        gomp = None
    if gomp is not None:
        nmax = gomp.omp_get_max_threads()
        gomp.omp_set_num_threads(1)
        try:
            n1, t1 = 0, time.perf_counter()
            while time.perf_counter() - t1 < seconds / 2:
                orc.advance(params, 1)
                n1 += 1
            d1 = time.perf_counter() - t1
        finally:
            gomp.omp_set_num_threads(nmax)
        out["single_thread"] = {"value": mesh.ncells * n1 / d1, "unit": METRIC, "cores": 1,
                                "sample": f"{n1} steps of the same box on one thread, {d1:.1f} s"}
    return out


def run_reference(args):
    """Reference arm: the FP64 CPU oracle, timed on this host, bounded sample per step."""
    rank = int(os.environ.get("RANK", "0"))
    if not prints_line(rank):
        return                                        # the other ranks exit without work
    from workloads.problems import config_alfven3d
    import workloads as w
    from oracle import Oracle
    params = dict(config_alfven3d()["params"])
    mesh = w.uniform_mesh(3, 16, (2, 2, 2))          # 32^3 sample per step (8 blocks)
    U = w.evaluate_on_mesh(mesh, w.alfven_wave, ndim=3)
    orc = Oracle(mesh, U)
    for _ in range(args.warmup):
        orc.advance(params, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        orc.advance(params, 1)
    el = time.perf_counter() - t0
    val = mesh.ncells * args.steps / el
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {"metric": METRIC, "value": val, "unit": METRIC, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "sample": "32^3 periodic box (8 blocks of 16^3) per step"},
            "cpu_baseline": {"value": val, "unit": METRIC, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} steps of a 32^3 periodic box of the same wave"},
            "e2e": {"value": val, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_workload(args):
    """Secondary configurations: cell-updates/s of the batched FP32 + FP64-fix form (with
    regrid every few steps on the AMR ones), the plain FP64 form on the same input, and the
    FP32 form's per-variable L1 and Linf error against the FP64 form."""
    import torch
    import workloads as w
    from workloads.problems import CONFIGS, initial_state
    from paper_1204_5849_gb300 import MAP_FP32_FIX64, MAP_FP64, Pool
    cfg = CONFIGS[args.workload](small=args.small)
    mesh0 = cfg["mesh"]
    U0 = initial_state(cfg)
    params = dict(cfg["params"], fp64_fix_tau=1e-2)
    every = cfg.get("regrid_every", 0)
    refine = cfg.get("refine")
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    sptr = stream.cuda_stream
    cap = 4 * mesh0.nleaves + 4096
    out = {"workload": cfg["name"], "leaves": mesh0.nleaves, "cells": mesh0.ncells}
    settle = (refine["max_level"] + 2) if (every and refine) else 0
    for prec, key in ((MAP_FP32_FIX64, "fp32_batched"), (MAP_FP64, "fp64_plain")):
        pool = Pool(mesh0, prec, max_blocks=cap, stream=sptr)
        pool.write_leaves(U0)
        # AMR: let the refinement criterion settle the initial mesh (adapt + one step, a few
        # times) before timing
        for _ in range(settle):
            pool.adapt(params, refine)
            pool.fill_ghosts(); pool.cfl_dt(params); pool.step(params)
        out.setdefault("leaves_settled", {})[key] = pool.nleaves
        nsteps = args.steps if prec == MAP_FP32_FIX64 else max(2, min(args.steps, 8))
        for _ in range(args.warmup):
            if prec == MAP_FP32_FIX64:
                pool.advance(params, 1)
            else:
                pool.fill_ghosts(); pool.cfl_dt(params); pool.step(params)
        torch.cuda.synchronize()
        cell_updates = 0
        adapt_ms = 0.0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        for s in range(nsteps):
            if every and refine and s > 0 and s % every == 0:
                a0 = time.perf_counter()
                pool.adapt(params, refine)
                adapt_ms += 1e3 * (time.perf_counter() - a0)
            if prec == MAP_FP32_FIX64:
                pool.advance(params, 1)
            else:
                pool.fill_ghosts(); pool.cfl_dt(params); pool.step(params)
            cell_updates += pool.nleaves * mesh0.cells_per_block
        e1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        ms = e0.elapsed_time(e1)
        out[key] = {"value": cell_updates / (ms * 1e-3), "unit": METRIC, "ms_per_step": ms / nsteps,
                    "steps": nsteps, "wall_s": wall, "leaves_end": pool.nleaves,
                    "adapt_ms_total": adapt_ms, "check": pool.check()}
        if params.get("conduction", "off") != "off":
            # the conduction share: the same steps without conduction, and the substep count
            _, nsub = pool.last_conduction()
            p_off = dict(params, conduction="off")
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            for s in range(nsteps):
                if prec == MAP_FP32_FIX64:
                    pool.advance(p_off, 1)
                else:
                    pool.fill_ghosts(); pool.cfl_dt(p_off); pool.step(p_off)
            f1.record(stream)
            torch.cuda.synchronize()
            ms_off = f0.elapsed_time(f1)
            n = int(nsub.max())
            per_sub = (ms - ms_off) / nsteps / max(n, 1)
            cells = pool.nleaves * mesh0.cells_per_block
            bpc = 9 * (4 if prec == MAP_FP32_FIX64 else 8)     # read 8 variables + write e
            out[key]["conduction"] = {"substeps_per_step": n, "ms_per_step_without": ms_off / nsteps,
                                      "ms_per_substep": per_sub,
                                      "substep_cells_per_s": cells / (per_sub * 1e-3),
                                      "algorithmic_gbs": bpc * cells / (per_sub * 1e-3) / 1e9,
                                      "bytes_per_cell": bpc}
        pool.close()
    if every and refine:
        # the initial mesh held fixed (no regrid): at t = 0 the refinement criterion keeps
        # only the steep regions refined, so the settled mesh above is much smaller
        pool = Pool(mesh0, MAP_FP32_FIX64, max_blocks=cap, stream=sptr)
        pool.write_leaves(U0)
        for _ in range(args.warmup):
            pool.advance(params, 1)
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        pool.advance(params, args.steps)
        g1.record(stream)
        torch.cuda.synchronize()
        ms = g0.elapsed_time(g1)
        out["fp32_batched_fixed_mesh"] = {"value": mesh0.ncells * args.steps / (ms * 1e-3), "unit": METRIC,
                                          "ms_per_step": ms / args.steps, "leaves": mesh0.nleaves,
                                          "check": pool.check()}
        pool.close()
    # accuracy of the FP32 form against the plain FP64 form on the same input and mesh (no
    # regrid), per variable: L1 of the difference over the mean |FP64| and Linf over max |FP64|
    # (scales floored at 1e-3 of the largest variable's).  The FP64 form itself matches the
    # FP64 oracle to 1e-12 after one step (the GPU parity tests).
    nacc = 10
    G = {}
    for prec in (MAP_FP32_FIX64, MAP_FP64):
        pool = Pool(mesh0, prec, max_blocks=cap, stream=sptr)
        pool.write_leaves(U0)
        for _ in range(nacc):
            pool.fill_ghosts(); pool.cfl_dt(params); pool.step(params)
        G[prec] = pool.read_leaves()
        pool.close()
    out["error_fp32_vs_fp64"] = dict(steps=nacc, **error_table(G[MAP_FP32_FIX64], G[MAP_FP64]))
    if len(mesh0.problems) > 1:
        # per problem: the largest per-variable L1 of the FP32 form against the FP64 form
        prob = np.array([lf[0] for lf in mesh0.leaves])
        per = []
        for q in range(len(mesh0.problems)):
            sel = prob == q
            t = error_table(G[MAP_FP32_FIX64][sel], G[MAP_FP64][sel])["l1_rel"]
            per.append(max(t.values()))
        cells = [int(mesh0.problems[q].nbase[0] * mesh0.nb) for q in range(len(mesh0.problems))]
        out["error_fp32_vs_fp64_per_problem"] = {
            "steps": nacc, "l1_rel_max_over_variables": per, "edge_cells": cells,
            "max": max(per), "median": float(np.median(per))}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--size", type=int, default=256, help="cells per edge (profiling of smaller cases)")
    ap.add_argument("--quick", action="store_true", help="value and kernel timing only (profiling)")
    ap.add_argument("--prec", type=int, default=32, choices=(32, 64), help="pool precision of --quick runs")
    ap.add_argument("--workload", default="alfven3d",
                    choices=("alfven3d", "ot2d", "rotor_amr", "harris_amr", "ensemble", "conduction"),
                    help="secondary configurations print their own line")
    ap.add_argument("--small", action="store_true", help="small variant of a secondary workload")
    ap.add_argument("--no-tune", action="store_true", help="default launch shape (no autotuner)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload != "alfven3d":
        run_workload(args)
        return

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    from paper_1204_5849_gb300 import MAP_FP32_FIX64, MAP_FP64, Pool
    cfg, mesh, U0, params = build_workload(args.size)
    ncells = mesh.ncells
    # a dedicated non-default stream: the library's kernels and the timing events share it
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    sptr = stream.cuda_stream
    assert sptr != 0

    # -------- FP32 + FP64-fix batched form (the value) --------
    main_prec = MAP_FP64 if (args.quick and args.prec == 64) else MAP_FP32_FIX64
    pool = Pool(mesh, main_prec, max_blocks=mesh.nleaves, stream=sptr)
    pool.write_leaves(U0)
    # launch shape of the step kernel picked by the autotuner (untimed; the state is kept);
    # should a trial fail, the pool keeps its default shape and the line says why
    tune = None
    if not args.no_tune:
        try:
            tune = pool.autotune(params, reps=3)
        except Exception as e:                               # MapError: a trial launch failed
            pool.set_launch(0, 0, 0)
            tune = {"error": str(e)[:200], "grid": 0, "w_pred": 0, "w_face": 0}
    for _ in range(args.warmup):
        pool.advance(params, 1)
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    l0 = pool.kernel_launches()
    # one event before every step and one after the last: the per-step intervals time the
    # graph replay of each step (finalize, a 72-byte memset and the step kernel)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    evs[0].record(stream)
    for i in range(args.steps):
        pool.advance(params, 1)
        evs[i + 1].record(stream)
    barrier()
    ms = evs[0].elapsed_time(evs[-1])
    step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
    launches = pool.kernel_launches() - l0
    ms_max = max_over_ranks(ms, dist)
    value = job_value(world, ncells, args.steps, ms_max)
    assert pool.check() == 0, "device error word set during the benchmark"

    # -------- step kernel alone (map_step, without the fused reductions) ----------------
    pool.fill_ghosts()
    pool.cfl_dt(params)
    nk = min(args.steps, 100)
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(nk)]
    for a, b in kev:
        a.record(stream)
        pool.step(params)
        b.record(stream)
        pool.fill_ghosts()
        pool.cfl_dt(params)
    torch.cuda.synchronize()
    k_ms_alone = statistics.mean(a.elapsed_time(b) for a, b in kev)
    # the dominant kernel's launch duration in the timed region: the mean per-step interval
    # (an upper bound: it also holds the finalize kernel and the memset, about 10 us)
    k_ms = statistics.mean(step_ms)
    hbm, peak_kind = peaks()
    achieved = BYTES_PER_CELL_F32 * ncells / (k_ms * 1e-3) / 1e9
    mhz, mhz_src = sm_max_mhz()
    fp32_peak = SMS * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12            # TFLOP/s
    tflops = FLOPS_PER_CELL * ncells / (k_ms * 1e-3) / 1e12
    traffic = STEP_KERNEL_DRAM_BYTES_512_BLOCKS * mesh.nleaves / 512.0

    if args.quick:
        clocks.stop()
        if prints_line(rank):
            print(json.dumps({"metric": METRIC, "value": value, "ms_per_step": ms_max / args.steps, "launch_shape": tune,
                              "kernel_ms": k_ms, "kernel_ms_alone": k_ms_alone, "achieved_gbs": achieved,
                              "achieved_tflops": tflops, "cells": ncells, "gpu_launches": launches}))
        return

    # -------- the interface fluxes on the same workload (Sec. 3.2-3.3, Sec. 5): the step with
    # HLLC and with HLLD in place of f_m, graph-replayed like the value (untimed by the line's
    # value; the state moves on, and the end-to-end loop below writes its own) --------------
    riemann_ms = {"f_m": ms / args.steps}
    nr = min(args.steps, 20)
    for rs in ("hllc", "hlld"):
        pr = dict(params, riemann=rs)
        for _ in range(2):                          # eager run, then the capture per buffer
            pool.advance(pr, 1)
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        r0.record(stream)
        pool.advance(pr, nr)
        r1.record(stream)
        torch.cuda.synchronize()
        riemann_ms[rs] = r0.elapsed_time(r1) / nr
    assert pool.check() == 0, "device error word set by the interface-flux runs"

    # -------- end to end through the public API: pinned H2D of the inputs, D2H result ----
    # every step copies the host state in (map_write_leaves_async[_f32]: its own copy stream
    # and two staging buffers, so the copy for step k+1 overlaps step k), reads the step's
    # result -- the new state (map_read_leaves_async[_f32]: packed on the pool stream, copied
    # out on a second copy stream into alternating pinned buffers) and dt, c_h, c_p, damping,
    # alpha_g -- back into pinned memory; one synchronisation at the end.  e2e.value uses the
    # FP32 host layout, the FP32 pool's own precision; e2e.fp64_host the FP64 layout, whose
    # blocking calls give e2e.blocking_value_fp64_host.
    pinned = torch.empty(U0.shape, dtype=torch.float64, pin_memory=True)
    pinned.numpy()[...] = U0
    outs = [torch.empty(U0.shape, dtype=torch.float64, pin_memory=True) for _ in range(2)]
    ne = min(args.steps, 100)
    res = torch.zeros((ne, len(mesh.problems), 5), dtype=torch.float64, pin_memory=True)
    for _ in range(2):
        pool.write_leaves_async_ptr(pinned.data_ptr())
        pool.advance(params, 1)
        pool.read_leaves_async_ptr(outs[0].data_ptr())
        pool.speeds_async_ptr(res[0].data_ptr())
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(stream)
    for i in range(ne):
        pool.write_leaves_async_ptr(pinned.data_ptr())
        pool.advance(params, 1)
        pool.read_leaves_async_ptr(outs[i % 2].data_ptr())
        pool.speeds_async_ptr(res[i].data_ptr())
    assert pool.check() == 0                    # synchronises the pool's copy streams
    e1.record(stream)
    barrier()
    e2e_ms = max(e0.elapsed_time(e1), 1e3 * (time.perf_counter() - t0))
    assert np.all(res.numpy()[:, :, 0] > 0), "a step's result was not read back"
    # the last state read back is the state after one step from U0
    last = outs[(ne - 1) % 2].numpy()
    np.testing.assert_array_equal(last, pool.read_leaves())
    # the same with the FP32 host layout both ways (an FP32 pool stores FP32: the device
    # state is bitwise the same as with the FP64 copy, and the FP32 read is exact)
    pinned32 = torch.empty(U0.shape, dtype=torch.float32, pin_memory=True)
    pinned32.numpy()[...] = U0.astype(np.float32)
    outs32 = [torch.empty(U0.shape, dtype=torch.float32, pin_memory=True) for _ in range(2)]
    pool.read_leaves_async_f32_ptr(outs32[0].data_ptr())
    barrier()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    f0.record(stream)
    for i in range(ne):
        pool.write_leaves_async_f32_ptr(pinned32.data_ptr())
        pool.advance(params, 1)
        pool.read_leaves_async_f32_ptr(outs32[i % 2].data_ptr())
        pool.speeds_async_ptr(res[i].data_ptr())
    assert pool.check() == 0
    f1.record(stream)
    barrier()
    e2e32_ms = max(f0.elapsed_time(f1), 1e3 * (time.perf_counter() - t0))
    e2e32 = world * ncells * ne / (e2e32_ms * 1e-3)
    b0 = torch.cuda.Event(enable_timing=True)
    b1 = torch.cuda.Event(enable_timing=True)
    nb_ = min(ne, 20)
    bout = outs[0].numpy()
    for _ in range(2):                          # untimed: first use of the blocking path
        pool.write_leaves_ptr(pinned.data_ptr())
        pool.advance(params, 1)
        pool.read_leaves(out=bout)
        pool.speeds()
    t0 = time.perf_counter()
    b0.record(stream)
    for _ in range(nb_):
        pool.write_leaves_ptr(pinned.data_ptr())
        pool.advance(params, 1)
        pool.read_leaves(out=bout)
        pool.speeds()
    b1.record(stream)
    barrier()
    e2e_blocking = world * ncells * nb_ / (max(b0.elapsed_time(b1), 1e3 * (time.perf_counter() - t0)) * 1e-3)
    clk = clocks.stop()
    h2d = U0.nbytes
    d2h = U0.nbytes + 5 * 8 * len(mesh.problems)
    e2e_val = world * ncells * ne / (e2e_ms * 1e-3)

    # -------- accuracy at the stated error: 200 steps of each form, against the closed-form
    # linear wave at each form's own final time, and FP32 against FP64 ------------------
    nacc = 200

    def run_acc(pl, p):
        pl.write_leaves(U0)
        t = 0.0
        for _ in range(nacc):
            pl.advance(p, 1)
            t += float(pl.speeds()[0][0])
        return pl.read_leaves(), t

    G32, t32 = run_acc(pool, params)
    # the same without the FP64 pressure fallback (it triggers only where e_int < 1e-2 e; on
    # this wave e_int / e = 0.23 everywhere, so both tables agree)
    G32n, _ = run_acc(pool, dict(params, fp64_fix_tau=0.0))
    pool.close()
    del pool

    # -------- plain FP64 form (per-level launches, host-synchronised dt) --------
    p64 = Pool(mesh, MAP_FP64, max_blocks=mesh.nleaves, stream=sptr)
    G64, t64 = run_acc(p64, params)
    p64.write_leaves(U0)
    for _ in range(3):
        p64.fill_ghosts(); p64.cfl_dt(params); p64.step(params)
    n64 = max(3, min(args.steps, 10))
    barrier()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(n64):
        p64.fill_ghosts(); p64.cfl_dt(params); p64.step(params)
    f1.record(stream)
    barrier()
    f64_ms = f0.elapsed_time(f1)
    f64_val = world * ncells * n64 / (f64_ms * 1e-3)
    p64.close()
    # per-variable L1 and Linf of (FP32 - FP64) (error_table); the wave components are 1e-6 of
    # O(1), so they are also given over the wave amplitude
    errs = error_table(G32, G64)
    amp = 1e-6
    wave = {nm: float(np.abs(G32[:, v] - G64[:, v]).mean() / amp) for v, nm in enumerate(NAMES)
            if nm in ("my", "mz", "by", "bz")}
    wave_inf = {nm: float(np.abs(G32[:, v] - G64[:, v]).max() / amp) for v, nm in enumerate(NAMES)
                if nm in ("my", "mz", "by", "bz")}
    closed = {"steps": nacc}
    for key, G, t in (("fp32_batched", G32, t32), ("fp64_plain", G64, t64)):
        import workloads as w
        X = w.evaluate_on_mesh(mesh, w.alfven_wave, ndim=3, t=t)
        closed[key] = {"t": t,
                       "wave_l1_over_amplitude": {nm: float(np.abs(G[:, v] - X[:, v]).mean() / amp)
                                                  for v, nm in enumerate(NAMES) if nm in ("my", "mz", "by", "bz")},
                       "background_l1_rel": {nm: float(np.abs(G[:, v] - X[:, v]).mean() / np.abs(X[:, v]).mean())
                                             for v, nm in enumerate(NAMES) if nm in ("rho", "bx", "e")}}
        del X

    if not prints_line(rank):
        if dist is not None:
            dist.destroy_process_group()
        return
    cpu = None if args.no_cpu else cpu_baseline(params)
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "cells": ncells, "blocks": mesh.nleaves,
                   "block": "16^3 + 2 ghost layers", "form": "fp32+fp64-fix batched, graph-replayed",
                   "l2": "state (1.2 GB) larger than L2; no flush",
                   "launch_shape": tune,
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "roofline": {"bound": "alu", "achieved": tflops, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": tflops / fp32_peak, "traffic": traffic,
                     "kernel": "step_kernel<float,3,16,LF,vanleer>", "kernel_ms": k_ms,
                     "kernel_ms_alone": k_ms_alone, "flops_per_cell": FLOPS_PER_CELL,
                     "peak_source": f"{SMS} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flop/FMA x "
                                    f"{mhz:.0f} MHz ({mhz_src})",
                     "traffic_source": "ncu dram bytes of the 512-block launch x blocks/512",
                     "hbm": {"achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                             "bytes_per_cell": BYTES_PER_CELL_F32, "peak_source": f"{peak_kind} hbm_gbs",
                             "dram_gbs": traffic / (k_ms * 1e-3) / 1e9,
                             "dram_frac": traffic / (k_ms * 1e-3) / 1e9 / hbm}},
        "e2e": {"value": e2e32, "unit": METRIC, "h2d_bytes_per_step": U0.nbytes // 2,
                "d2h_bytes_per_step": U0.nbytes // 2 + 5 * 8 * len(mesh.problems), "steps": ne,
                "host_layout": "fp32: the FP32 pool's own storage precision (an FP64 copy-in gives the "
                               "same device state bit for bit; the FP32 read-back is exact)",
                "copies": "FP32 host state in (pinned, map_write_leaves_async_f32: async copy stream, "
                          "double-buffered staging), the new FP32 state and the step's speeds out "
                          "(pinned, map_read_leaves_async_f32 on a second copy stream, "
                          "map_get_speeds_async); one sync at the end",
                "fp64_host": {"value": e2e_val, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                              "copies": "the same loop with the FP64 host layout both ways "
                                        "(map_write_leaves_async, map_read_leaves_async)"},
                "blocking_value_fp64_host": e2e_blocking},
        "gpu_launches": launches,
        "clocks": clk,
        "fp64_plain": {"value": f64_val, "unit": METRIC, "ms_per_step": f64_ms / n64, "steps": n64},
        "error_fp32_vs_fp64": {"steps": nacc, **errs},
        "error_fp32_without_fix_vs_fp64": {"steps": nacc, **error_table(G32n, G64)},
        "error_fp32_vs_fp64_over_wave_amplitude": {"l1": wave, "linf": wave_inf},
        "error_vs_closed_form": closed,
        "riemann_solvers": {"unit": "ms_per_step", "steps": nr, **riemann_ms,
                            "note": "the same FP32 batched step with the interface flux f_m (the value), "
                                    "HLLC or HLLD"},
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
