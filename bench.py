"""Benchmark of the EBIT phase-change time step on GB300.

Workload (default): the 512^2 planar bubble growing in superheated liquid (rho_l/rho_v = 20,
k_l/k_v = 5, St = 0.2, superheat 1, dt = 1.96e-6), the full step of the method: energy
advection, EBIT marker sweeps and reconnection, sharp-interface energy solve, mass flux,
ghost velocities, momentum predictor and ghost-fluid projection.  Headline precision:
FP32 multigrid-preconditioned CG inside FP64 iterative refinement, every solve to a
1e-8 relative residual; the FP64 path is timed beside it.

metric: cell-steps/s = cells x steps / device time (whole job over all ranks).

One JSON line on rank 0.  `--impl reference` times the CPU oracle (the plain FP64
restatement of the method) on the host cores instead.

Multi-GPU: the single-instance step does not shard (every solver iteration couples the whole
grid), so N ranks run N independent replicas (weak scaling); no collective is on the data
path, only the timing barrier and the max-over-ranks reduction.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# the batched workload replays its instances on 32 worker streams: give each its own hardware
# queue (read when the CUDA context is created, so before torch initialises CUDA)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

import numpy as np

WORKLOADS = {
    "c2_bubble_512": dict(kind="c2", desc="2D planar vapour bubble in superheated liquid, 512x512"),
    "c2_bubble_512_one_fluid": dict(kind="c2of", desc="the 512x512 bubble with the one-fluid variant (one velocity "
                                                     "field, phase-change source in the projection)"),
    "c3_film_1024x2048": dict(kind="c3", desc="2D film boiling over a heated wall, 1024x2048"),
    "c5_film_4096": dict(kind="c5", desc="multi-mode 2D film boiling, 4096x4096"),
    # profiling case: the 4096x4096 film's cell size and physics on half its width (16 modes),
    # small enough for multi-pass ncu captures while its smoother operands exceed L2
    "c5_film_half_2048x4096": dict(kind="c5h", desc="multi-mode 2D film boiling, 2048x4096 half-width strip"),
    "c4_batch_4096": dict(kind="c4", desc="4096 independent Stefan / bubble-growth instances, sides 32..256"),
}
METRIC = "cell-steps/s at 1 GPU, FP32+refine vs FP64, 1e-8 rel residual; %HBM roofline"

# DRAM bytes (read + write) per launch of the finest-grid smoother kernels, from one ncu capture
# of the current kernels (summary and command in the named profiles/ file); an entry is removed
# whenever those kernels change, so that a stale figure is never reported
SMOOTH_L0_TRAFFIC = {
    "c2_bubble_512": {"dram_bytes_per_launch": 5.14e6,
                      "summary": "profiles/smoother_l0_traffic_c2_bubble_512.md"},
}


BATCH_COUNT = None   # --batch-count


def make_problems(name, count=None):
    """The workload's instances (one for every workload but the batched one)."""
    from paper_2402_13677_gb300 import workloads as w
    kind = WORKLOADS[name]["kind"]
    if kind == "c4":
        return w.c4_batch(count if count is not None else (BATCH_COUNT or 4096))
    if kind == "c2":
        return [w.c2_bubble(steps=0)]
    if kind == "c2of":
        return [w.one_fluid(w.c2_bubble(steps=0))]
    if kind == "c3":
        return [w.c3_film(steps=0)]
    if kind == "c5h":
        return [w.c5_film_half(steps=0)]
    return [w.c5_film(steps=0)]


# ------------------------------------------------------------------ clocks sampling
class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def start(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()

    def _run(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.samples.append([s.strip() for s in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def stop(self):
        self._stop.set()
        if self._t:
            self._t.join(timeout=10)
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4)
                          if len(s) > 3 + k and s[3 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


# ------------------------------------------------------------------ reference arm (CPU oracle)
def oracle_rate(name, budget_s=20.0, max_steps=3):
    """Time the oracle (as it stands) on a bounded sample of the workload: whole steps of its
    first instance(s), prepared once each, until the CPU budget is used.  Returns (cell-steps/s,
    cell-steps done, seconds, description of the sample)."""
    from oracle import step as S
    pbs = make_problems(name, count=64) if WORKLOADS[name]["kind"] == "c4" else make_problems(name)
    done, secs, cpu, steps, inst = 0, 0.0, 0.0, 0, 0
    for pb in pbs:
        st = S.prepare(pb)
        inst += 1
        for _ in range(max_steps):
            t0, c0 = time.perf_counter(), time.process_time()
            S.step(st)
            secs += time.perf_counter() - t0
            cpu += time.process_time() - c0
            done += pb.nx * pb.ny
            steps += 1
            if secs > budget_s:
                break
        if secs > budget_s:
            break
    what = (f"{steps} whole oracle steps of {name}" if inst == 1 else
            f"{steps} whole oracle steps over its first {inst} instances")
    return done / secs, done, secs, what, cores_used(cpu, secs)


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    # each timed step is one whole oracle step of the workload; the run stops early (and says
    # so in the sample) once the CPU budget is spent, so it ends within a few minutes
    total_steps, total_s, total_cpu, done = 0, 0.0, 0.0, 0
    from oracle import step as S
    pbs = make_problems(args.workload)
    cells = sum(pb.nx * pb.ny for pb in pbs)
    sts = [S.prepare(pb) for pb in pbs[:1]]
    for k in range(args.steps):
        # one timed step = one whole oracle step of the next instance of the sample
        b = k % len(pbs)
        if b >= len(sts):
            sts.append(S.prepare(pbs[b]))
        t0, c0 = time.perf_counter(), time.process_time()
        S.step(sts[b])
        total_s += time.perf_counter() - t0
        total_cpu += time.process_time() - c0
        done += pbs[b].nx * pbs[b].ny
        total_steps += 1
        if total_s > args.reference_budget:
            break
    value = done / total_s
    cores = cores_used(total_cpu, total_s)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "cell-steps/s", "n_gpus": args.gpus,
            "steps": total_steps, "steps_requested": args.steps, "warmup": 0,
            "ms_per_step": 1e3 * total_s / total_steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "cells": cells, "instances": len(pbs),
                       "instances_sampled": len(sts), "solver": "sparse direct (SuperLU)"},
            "cpu_baseline": {"value": value, "unit": "cell-steps/s", "cores": cores, "kind": "oracle",
                             "implementation": "Python/numpy + scipy SuperLU, single process",
                             "cpu_s_per_wall_s": total_cpu / total_s,
                             "sample": f"{total_steps} of {args.steps} requested whole oracle steps of "
                                       f"{args.workload} from its initial state ({total_s:.1f} s; the run stops "
                                       f"once {args.reference_budget:.0f} s of oracle time is spent)"},
            "e2e": {"value": value, "unit": "cell-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cores_used(cpu_s, wall_s):
    """Cores the oracle kept busy: its process CPU time over the wall time of the same steps
    (numpy and SuperLU run single-threaded here; a threaded BLAS would show as more than 1)."""
    return max(1, int(round(cpu_s / wall_s))) if wall_s > 0 else 1


# ------------------------------------------------------------------ replicas (N > 1)
def replica_max(x, dist, device):
    """Max of a per-rank time over all ranks (the slowest replica sets the job's time)."""
    if not dist:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, cells, steps, secs):
    """Whole-job cell-steps/s: every replica advances its own instance by `steps` steps."""
    return world * cells * steps / secs


# ------------------------------------------------------------------ result summaries
# Bytes per cell that one pass of the step must move (the method's algorithmic minimum, one
# word per value): a preconditioned CG iteration (stencil apply with its dot product, the
# vector updates and a V(2,2) multigrid cycle) moves about 250 B per cell in FP64 and 125 B in
# FP32; the explicit part of the step (advection, operators, projection, diagnostics) about
# 250 B.  Iteration counts are the solver's own (energy, both viscous components, Poisson; the
# mixed path counts its FP32 iterations over all refinement passes).
B_ITER = {"fp64": 250.0, "mixed": 125.0}
B_EXPLICIT = 250.0


def step_roofline(r, cells, steps, prec, peak):
    d = r["diag"]
    iters = d[6] + d[7] + d[8]
    b_cell = iters * B_ITER[prec] + B_EXPLICIT
    achieved = b_cell * cells / (r["secs"] / steps) / 1e9
    return {"bytes_per_cell_step": b_cell, "iterations": [d[6], d[7], d[8]], "achieved": achieved,
            "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "formula": f"(energy + viscous + Poisson iterations) x {B_ITER[prec]:.0f} B + {B_EXPLICIT:.0f} B "
                       f"per cell, iterations of the last timed step"}


def mixed_error(pbs, mixed, fp64, nsteps):
    """The mixed path's error against the FP64 path after the same steps from the same initial
    state: max difference over a field group relative to the group's scale (temperatures: max |T|
    over both phases; velocities: max |u| over both phase fields; pressure: max(|p|, rho_l
    u_max^2), p being defined by its outflow reference)."""
    errs = []
    for b, (fm, fd) in enumerate(zip(mixed["final"], fp64["final"])):
        t_scale = max(float(np.max(np.abs(fd["T_l"]))), float(np.max(np.abs(fd["T_v"]))), 1e-300)
        u_scale = max(float(np.max(np.abs(fd["u_l"]))), float(np.max(np.abs(fd["u_v"]))), 1e-300)
        p_scale = max(float(np.max(np.abs(fd["p"]))), pbs[b].rho_l * u_scale ** 2, 1e-300)
        scale = {"T_l": t_scale, "T_v": t_scale, "u_l": u_scale, "u_v": u_scale, "p": p_scale}
        e = {k: float(np.max(np.abs(fm[k] - fd[k]))) / scale[k] for k in ("T_l", "T_v", "p", "u_l", "u_v")}
        e["vcol"] = int(np.sum(fm["vcol"] != fd["vcol"]))
        e["markers"] = float(max(np.max(np.abs(fm["hx_pos"] - fd["hx_pos"])),
                                 np.max(np.abs(fm["vy_pos"] - fd["vy_pos"]))))
        errs.append(e)
    return {"steps": nsteps, "instances_compared": len(errs),
            **{k: max(e[k] for e in errs) for k in ("T_l", "T_v", "p", "u_l", "u_v")},
            "vertex_colours_differing": sum(e["vcol"] for e in errs),
            "marker_max_abs_diff": max(e["markers"] for e in errs),
            "scales": "T: max|T| both phases; u: max|u| both fields; p: max(|p|, rho_l u_max^2)"}


# ------------------------------------------------------------------ our arm
def run_ours(args):
    import torch
    from paper_2402_13677_gb300 import ebit as E
    import __graft_entry__ as G

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0 or world == 1:
        G.build()
    if dist:
        dist.barrier()
        G.build()
    E.load()

    pbs = make_problems(args.workload)
    cells = sum(pb.nx * pb.ny for pb in pbs)
    stream = torch.cuda.Stream()          # non-default stream: each step is replayed as a CUDA graph
    alloc = E.TorchAllocator()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")   # > 129 MB L2

    def new_ctx(pbs, precision):
        ctx = E.ebit_init([E.config_from_problem(pb, precision, args.rtol, args.max_iter) for pb in pbs],
                          stream.cuda_stream, alloc)
        if args.no_graph:
            E.ebit_set_option(ctx, E.EBIT_OPT_GRAPH, 0)
        for b, pb in enumerate(pbs):
            E.upload_state(ctx, b, pb, pb.vcol, np.where(pb.hx_cut > 0, pb.hx_pos, 0.0),
                           np.where(pb.vy_cut > 0, pb.vy_pos, 0.0),
                           {"T_l": pb.T_l, "T_v": pb.T_v, "u_l": pb.u_l, "u_v": pb.u_v, "ufx_l": pb.ufx_l,
                            "ufx_v": pb.ufx_v, "ufy_l": pb.ufy_l, "ufy_v": pb.ufy_v, "p": pb.p}, pb.t0)
        E.ebit_run_stage(ctx, E.STAGE_PREPARE)
        if not args.no_graph and not args.no_autotune:
            E.ebit_autotune(ctx, 2)   # multigrid schedule per batch / instance (state restored)
        return ctx

    def timed_steps(ctx, k, with_timing=False):
        """k steps, each bracketed by CUDA events on the context's stream; L2 flushed between steps."""
        total = 0.0
        launches0 = E.ebit_launch_count(ctx)
        if with_timing:
            E.ebit_timing_begin(ctx, E.EBIT_KT_SMOOTH_L0)
        for _ in range(k):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            E.ebit_step(ctx, 1, allow_noconv=True)
            e1.record(stream)
            torch.cuda.synchronize()
            total += e0.elapsed_time(e1) / 1e3
        kt = E.ebit_timing_end(ctx) if with_timing else None
        return total, E.ebit_launch_count(ctx) - launches0, kt

    def barrier_max(x):
        return replica_max(x, dist, "cuda")

    def measure(pbs, steps, warmup, prec_list, clocks=None, keep_final=True):
        """Warm-up and timed steps of each precision from the workload's initial state."""
        results = {}
        for name, prec in prec_list:
            ctx = new_ctx(pbs, prec)
            try:
                for _ in range(warmup):
                    E.ebit_step(ctx, 1, allow_noconv=True)
                torch.cuda.synchronize()
                if dist:
                    dist.barrier()
                torch.cuda.synchronize()
                if clocks is not None and name == "mixed":
                    clocks.start()
                secs, launches, kt = timed_steps(ctx, steps, with_timing=(name == "mixed"))
                clk = clocks.stop() if clocks is not None and name == "mixed" else None
                torch.cuda.synchronize()
                if dist:
                    dist.barrier()
                secs = barrier_max(secs)
                d = E.ebit_get_diagnostics(ctx, 0)
                results[name] = dict(secs=secs, launches=launches, kt=kt, diag=d.tolist(), clocks=clk)
                sched = {}
                for b in range(len(pbs)):
                    sm, it, tm, co = E.ebit_get_schedule(ctx, b)
                    key = f"small_max={sm} inner_rtol={it:g} tma={tm} coop={co}"
                    sched[key] = sched.get(key, 0) + 1
                results[name]["schedule"] = sched
                if keep_final and rank == 0:
                    results[name]["final"] = [
                        E.download(ctx, b, pbs[b].nx, pbs[b].ny,
                                   ["T_l", "T_v", "p", "u_l", "u_v", "vcol", "hx_pos", "vy_pos"])
                        for b in range(min(len(pbs), 16))]
            finally:
                E.ebit_destroy(ctx)
        return results

    prec_list = [("mixed", E.EBIT_MIXED), ("fp64", E.EBIT_FP64)]
    if args.profile_only:
        prec_list = prec_list[:1]
    clocks = ClockSampler(local)
    results = measure(pbs, args.steps, args.warmup, prec_list, clocks, keep_final=not args.profile_only)
    clk = results["mixed"]["clocks"]
    if args.profile_only:
        if rank == 0:
            r = results["mixed"]
            print(json.dumps({"profile_only": True, "workload": args.workload, "ms_per_step": 1e3 * r["secs"] / args.steps,
                              "diag": r["diag"], "launches": r["launches"]}), flush=True)
        return 0

    # end to end through the C ABI with HOST buffers: every step uploads its inputs (the whole
    # state, from pinned host memory) with ebit_set_interface / ebit_set_field, steps, and reads
    # the new state and the diagnostics back with ebit_get_field / ebit_get_diagnostics;
    # wall-clock time of the whole sequence
    e2e = None
    if not args.no_e2e and len(pbs) > 64:
        e2e = {"value": None, "skipped": "batched workload: per-instance host buffers for every field of "
                                         f"{len(pbs)} instances are not staged; run a single-instance workload"}
    elif not args.no_e2e:
        ctx = new_ctx(pbs, E.EBIT_MIXED)
        try:
            for _ in range(args.warmup):
                E.ebit_step(ctx, 1, allow_noconv=True)
            ids = {"T_l": E.F_T_L, "T_v": E.F_T_V, "u_l": E.F_U_L, "u_v": E.F_U_V, "ufx_l": E.F_UFX_L,
                   "ufx_v": E.F_UFX_V, "ufy_l": E.F_UFY_L, "ufy_v": E.F_UFY_V, "p": E.F_P, "gc": E.F_GC,
                   "mdot": E.F_MDOT, "vcol": E.F_VCOL, "hx_pos": E.F_HX_POS, "vy_pos": E.F_VY_POS}
            lib = E.load()
            host = [{} for _ in pbs]
            for b in range(len(pbs)):
                for n, f in ids.items():
                    cnt, eb = E.ebit_field_shape(ctx, b, f)
                    host[b][n] = torch.empty(cnt * eb, dtype=torch.uint8, pin_memory=True)
                    lib.ebit_get_field(ctx, b, f, host[b][n].data_ptr(), 0)
            h2d = sum(h.numel() for hb in host for h in hb.values())
            # fields in and out through the batched copies (one synchronisation per call); the
            # id and pointer arrays are built once
            state = [(n, f) for n, f in ids.items() if n not in ("vcol", "hx_pos", "vy_pos")]
            ids_in = (ctypes.c_int * len(state))(*[f for _, f in state])
            ids_out = (ctypes.c_int * len(ids))(*ids.values())
            ptr_in = [(ctypes.c_void_p * len(state))(*[host[b][n].data_ptr() for n, _ in state])
                      for b in range(len(pbs))]
            ptr_out = [(ctypes.c_void_p * len(ids))(*[host[b][n].data_ptr() for n in ids]) for b in range(len(pbs))]
            diag = np.zeros(12)
            total = 0.0
            for _ in range(args.steps):
                flush.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for b in range(len(pbs)):
                    E.check(ctx, lib.ebit_set_interface(ctx, b, host[b]["vcol"].data_ptr(),
                                                        host[b]["hx_pos"].data_ptr(), host[b]["vy_pos"].data_ptr(), 0))
                    E.check(ctx, lib.ebit_set_fields(ctx, b, len(state), ids_in, ptr_in[b], 0))
                E.ebit_run_stage(ctx, E.STAGE_RECONSTRUCT)
                E.ebit_step(ctx, 1, allow_noconv=True)
                for b in range(len(pbs)):
                    E.check(ctx, lib.ebit_get_fields(ctx, b, len(ids), ids_out, ptr_out[b], 0))
                    diag = E.ebit_get_diagnostics(ctx, b)
                total += time.perf_counter() - t0
            total = barrier_max(total)
            e2e = {"value": world * cells * args.steps / total, "unit": "cell-steps/s",
                   "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": h2d + 8 * len(diag) * len(pbs),
                   "timing": "wall clock per step, host buffers in and out through the C ABI"}
        finally:
            E.ebit_destroy(ctx)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    mixed, fp64 = results["mixed"], results["fp64"]
    value = job_rate(world, cells, args.steps, mixed["secs"])
    value64 = job_rate(world, cells, args.steps, fp64["secs"])
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = peaks.get("hbm_gbs", 6800.0)
    peak_source = "MEASURED_PEAKS.json hbm_gbs (measured)" if "hbm_gbs" in peaks else "fallback 6800 GB/s"
    kt_ms, kt_n, kt_bytes = mixed["kt"]
    achieved = (kt_bytes * kt_n) / (kt_ms / 1e3) / 1e9 if kt_ms > 0 else None
    mixed_err = mixed_error(pbs, mixed, fp64, args.warmup + args.steps)
    step_roof = {"mixed": step_roofline(mixed, cells, args.steps, "mixed", peak),
                 "fp64": step_roofline(fp64, cells, args.steps, "fp64", peak)}
    extras = {}
    for wname in [x for x in args.extra.split(",") if x and x != args.workload and world == 1]:
        xp = make_problems(wname)
        xc = sum(pb.nx * pb.ny for pb in xp)
        xs = max(1, args.extra_steps)
        xr = measure(xp, xs, args.extra_warmup, [("mixed", E.EBIT_MIXED), ("fp64", E.EBIT_FP64)])
        xm, xd = xr["mixed"], xr["fp64"]
        km, kn, kb = xm["kt"]
        xa = (kb * kn) / (km / 1e3) / 1e9 if km > 0 else None
        extras[wname] = {
            "desc": WORKLOADS[wname]["desc"], "cells": xc, "steps": xs, "warmup": args.extra_warmup,
            "value": job_rate(1, xc, xs, xm["secs"]), "unit": "cell-steps/s",
            "ms_per_step": 1e3 * xm["secs"] / xs, "timesteps_per_s": xs / xm["secs"],
            "fp64": {"value": job_rate(1, xc, xs, xd["secs"]), "ms_per_step": 1e3 * xd["secs"] / xs,
                     "speedup_mixed_over_fp64": xd["secs"] / xm["secs"]},
            "roofline": {"bound": "hbm", "kernel": "k_pre/k_post<float> on the finest grid", "achieved": xa,
                         "peak": peak, "unit": "GB/s", "frac": (xa / peak) if xa else None,
                         "launches_timed": kn, "avg_launch_us": 1e3 * km / kn if kn else None},
            "step_roofline": {"mixed": step_roofline(xm, xc, xs, "mixed", peak),
                              "fp64": step_roofline(xd, xc, xs, "fp64", peak)},
            "mixed_error_vs_fp64": mixed_error(xp, xm, xd, args.extra_warmup + xs),
            "schedule_mixed": xm["schedule"], "gpu_launches": int(xm["launches"]),
        }
        del xp
    tr = SMOOTH_L0_TRAFFIC.get(args.workload)
    traffic = tr["dram_bytes_per_launch"] if tr else None
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        r, n, secs, what, cores = oracle_rate(args.workload, budget_s=args.cpu_budget)
        cpu = {"value": r, "unit": "cell-steps/s", "cores": cores, "kind": "oracle",
               "implementation": "Python/numpy + scipy SuperLU, single process",
               "sample": f"{what} from the initial state ({n} cell-steps, {secs:.1f} s)"}
    line = {
        "metric": METRIC, "value": value, "unit": "cell-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * mixed["secs"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64-refine", "data": "synthetic",
        "config": {"workload": args.workload, "cells": cells, "instances": len(pbs),
                   "grid": [pbs[0].nx, pbs[0].ny] if len(pbs) == 1 else "sides 32..256", "rtol": args.rtol,
                   "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "fp64": {"value": value64, "unit": "cell-steps/s", "ms_per_step": 1e3 * fp64["secs"] / args.steps,
                 "speedup_mixed_over_fp64": value / value64},
        "mixed_error_vs_fp64": mixed_err,
        "timesteps_per_s": args.steps / mixed["secs"],
        "step_roofline": step_roof,
        "roofline": {"bound": "hbm",
                     "kernel": "k_pre/k_post<float> on the finest grid (tiled red-black GS V-cycle legs)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "launches_timed": kt_n, "bytes_per_launch": kt_bytes,
                     "avg_launch_us": 1e3 * kt_ms / kt_n if kt_n else None, "peak_source": peak_source},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clk,
        "gpu_launches": int(mixed["launches"]),
        "workloads": extras,
        "solver": {"mixed_diag": mixed["diag"], "fp64_diag": fp64["diag"],
                   "schedule_mixed": mixed["schedule"], "schedule_fp64": fp64["schedule"],
                   "autotuned": not args.no_autotune and not args.no_graph},
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2_bubble_512", choices=list(WORKLOADS))
    ap.add_argument("--batch-count", type=int, default=None,
                    help="instances of the batched workload (default 4096; fewer only for quick checks)")
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--max-iter", type=int, default=400)
    ap.add_argument("--cpu-budget", type=float, default=10.0)
    ap.add_argument("--reference-budget", type=float, default=150.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--profile-only", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="launch kernels from the host (profilers)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default multigrid schedule")
    ap.add_argument("--extra", default="c2_bubble_512_one_fluid,c3_film_1024x2048,c5_film_4096,c4_batch_4096",
                    help="further workloads measured in the same run (sub-objects of the line; '' for none)")
    ap.add_argument("--extra-steps", type=int, default=5)
    ap.add_argument("--extra-warmup", type=int, default=3)
    args = ap.parse_args()
    global BATCH_COUNT
    BATCH_COUNT = args.batch_count
    if args.impl == "reference":
        return reference_arm(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
