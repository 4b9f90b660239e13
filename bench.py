"""Benchmark of the ESBI hot path on one GB300 (or N independent replicas).

Workload (default ``crossing_batch``): 96 crossing random seas advanced together,
64 on 256x256 and 32 on 512x512 grids, deep water kp h = 5, 7th-order
successive approximation, low-pass filter on, FP32 FFTs/products with FP64
state and RK4 sums.  A step is one classical RK4 step of every member (four
right-hand sides, each one vertical-velocity diagnostic plus the dynamic
condition).  Metric: grid-point RK4 steps per second (sum over members of
nx*ny, times steps, over the device time of the timed region).

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "grid-point RK4 steps/s"
UNIT = "pt-steps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="crossing_batch",
                    choices=["crossing_batch", "large_variable", "bar_1d", "stokes_2d",
                             "bar_wavemaker_1d", "solitary_1d"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--diagnostic", default="esbi", choices=["esbi", "hos"],
                    help="V by the ESBI successive approximation or the HOS expansion (flat bottom)")
    ap.add_argument("--integrator", default="rk4", choices=["rk4", "lawson", "rk45"],
                    help="classical RK4, the integrating factor with RK4 stages, or with the "
                         "5(4) pair at a fixed step")
    ap.add_argument("--no-fp64-arm", action="store_true", help="skip the FP64 plain-path timing")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--compare-diagnostics", action="store_true",
                    help="instead of the step: time one V evaluation of the first member group by "
                         "the successive scheme and by the implicit form of Appendix A "
                         "(per fixed-point iteration), and print that JSON line")
    ap.add_argument("--members", default=None,
                    help="crossing_batch only: 'S,L' small (256^2) and large (512^2) members "
                         "instead of 64,32 (for profiling runs)")
    ap.add_argument("--shard", default="replicas", choices=["replicas", "split"],
                    help="N > 1: every rank advances its own batch of realisations "
                         "(replicas, weak scaling), or the one batch is split over the ranks "
                         "by cost (split, strong scaling)")
    ap.add_argument("--accuracy", action="store_true",
                    help="instead of timing: run the workload's configured number of steps "
                         "in FP32 and in FP64 on the GPU and print their differences "
                         "(eta, phi~, energy drift) as one JSON line")
    ap.add_argument("--accuracy-steps", type=int, default=None,
                    help="with --accuracy: steps instead of the workload's run length")
    ap.add_argument("--state-fp64", action="store_true",
                    help="FP32 path with the RK4 state and sums in FP64 instead of double-single")
    ap.add_argument("--schedule", type=int, default=0,
                    help="step schedule (sbi_options.schedule): 0 chosen by timing, B > 0 "
                         "units of at most total/B points, -1 serial groups")
    ap.add_argument("--col-staging", type=int, default=0, choices=[-1, 0, 1],
                    help="column-pass inputs (sbi_options.col_staging): 0 chosen by timing, "
                         "1 bulk copies into shared memory, -1 direct loads")
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="CPU time of each oracle baseline sample (1 process and all cores)")
    return ap.parse_args()


def make_workload(name, members=None, rank=0, world=1, shard="replicas"):
    """The workload of one rank.  With replicas (weak scaling) rank r advances
    its own set of realisations of the batched crossing seas (random phases
    seeded from 1000 + 96 r); with split (strong scaling) the one batch of
    seed 1000 is divided over the ranks by cost (largest first into the
    lightest rank) and rank r advances its share.  No data is exchanged."""
    import workloads as W
    if name == "crossing_batch":
        s, l = (64, 32)
        if members:
            s, l = (int(v) for v in members.split(","))
        if shard == "split" and world > 1:
            from paper_2310_19840_gb300 import shard as S
            wl = W.crossing_batch(n_small=s, n_large=l, seed0=1000)
            mine = S.partition([(m.nx, m.ny) for m in wl.members], world)[rank]
            wl.notes["global_members"] = mine
            wl.notes["global_count"] = len(wl.members)
            wl.notes["global_points"] = wl.points
            wl.notes["global_shapes"] = _shape_counts(wl.members)
            wl.members = [wl.members[i] for i in mine]
            return wl
        return W.crossing_batch(n_small=s, n_large=l, seed0=1000 + (s + l) * rank)
    return getattr(W, name)()


def reduce_max(value, world, device=None):
    """Max of a per-rank float over all ranks (the timed region's wall time)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _shape_counts(members):
    shapes = {}
    for m in members:
        key = f"{m.nx}x{m.ny}"
        shapes[key] = shapes.get(key, 0) + 1
    return shapes


INTEGRATOR_NAMES = {"rk4": "classical RK4", "lawson": "lawson (integrating factor, RK4 stages)",
                    "rk45": "integrating factor, Cash-Karp 5(4) pair, fixed step"}


def arm_config(args, wl, world):
    """The config dict of a JSON line; both arms print the same one."""
    cfg = workload_config(wl)
    cfg["integrator"] = INTEGRATOR_NAMES[args.integrator]
    cfg["diagnostic"] = args.diagnostic
    if args.state_fp64:
        cfg["state"] = "FP64 (state_fp64)"
    if world == 1:
        cfg["parallelism"] = "single GPU"
    elif args.shard == "split":
        cfg["parallelism"] = f"batch split over {world} GPUs by cost"
    else:
        cfg["parallelism"] = f"replicas on {world} GPUs"
    return cfg


def workload_config(wl):
    """The workload a line is measured on (for a batch split over ranks: the
    whole batch)."""
    shapes = wl.notes.get("global_shapes") or _shape_counts(wl.members)
    points = wl.notes.get("global_points", wl.points)
    cfg = {"workload": wl.name, "members": shapes, "points": points, "order": wl.order,
           "alias_frac": wl.alpha, "dt": wl.dt,
           "filter": bool(wl.filt_beta1 > 0), "sponge": wl.sponge_w is not None,
           "variable_depth": any(m.delta is not None for m in wl.members),
           "l2": ("inputs larger than L2 (no flush needed)" if points * 150 > 129e6 else
                  "working set fits in L2 (about 150 B per point, not flushed): small-workload timing")}
    if wl.wavemaker:
        cfg["wavemaker"] = {"components": len(wl.wavemaker["amp"]), "x0": wl.wavemaker["x0"]}
    return cfg


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
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
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


# the sources of the row, column and RK kernels whose DRAM traffic the
# committed ncu summary records (host code and the other kernels live in
# sbi_host.cu and sbi_noalloc.cu)
KERNEL_SOURCES = ("bank_model.h", "fft.cuh", "kernels.cuh", "sbi_internal.h", "inst_col_f32.cu",
                  "inst_col_f64.cu", "inst_row_f32.cu", "inst_row_f64.cu")


def source_sha():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2310_19840_gb300", "csrc")
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic_crossing_batch.txt")


def ncu_traffic(family, workload):
    """Per-launch DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of a
    kernel family, scaled to a launch of the full workload, from the committed
    ncu summary; None unless the summary was taken on this workload with the
    current CUDA sources."""
    try:
        lines = open(TRAFFIC_FILE).read().splitlines()
    except OSError:
        return None
    kv = {}
    for ln in lines:
        ln = ln.split("#", 1)[0].split()
        if len(ln) == 2:
            kv[ln[0]] = ln[1]
    if kv.get("source_sha") != source_sha() or kv.get("workload") != workload:
        return None
    try:
        return float(kv[family])
    except (KeyError, ValueError):
        return None


def autotune_summary(report):
    """Block shapes the autotuner chose, counted per pass kind, e.g.
    {"row": {"rpc 16": 5, "rpc 8": 2}, "col": {"cpb 8": 9}, "non_default": 2}."""
    out, changed = {}, 0
    for ln in report.splitlines():
        if ": " not in ln:
            continue
        shape, choice = ln.rsplit(": ", 1)
        knob, vals = choice.split()[:2]
        chosen, deflt = vals.split("/")
        kind = out.setdefault(shape.split()[0], {})
        kind[f"{knob} {chosen}"] = kind.get(f"{knob} {chosen}", 0) + 1
        changed += chosen != deflt
    out["non_default"] = changed
    return out


def schedule_summary(report):
    """The step schedules the library timed (sbi_schedule_report): per
    candidate its role, ms per step (None if not timed), name, mode and
    units, and the name of the one in use."""
    out = {"candidates": []}
    for ln in report.splitlines():
        if " units:" not in ln:
            continue
        role, rest = ln.split(" ", 1)
        ms = None
        if " ms per step: " in rest:
            t, rest = rest.split(" ms per step: ", 1)
            ms = float(t)
        head, units = rest.split(" units:", 1)
        name, _, mode = head.partition(" [")
        out["candidates"].append({"role": role, "ms_per_step": ms, "schedule": name,
                                  "mode": mode.split("]")[0], "units": units.split()})
    picked = [c for c in out["candidates"] if c["role"] in ("chosen", "forced")] or \
        [c for c in out["candidates"] if c["role"] == "default"]
    out["chosen"] = picked[0]["schedule"] if picked else None
    return out


def streamed_split(report):
    """The member-range splits the streamed step timed (the "streamed-" lines
    of sbi_schedule_report): per candidate its units and ms per step, and the
    number of units of the one kept."""
    cands = [c for c in schedule_summary(report)["candidates"] if c["role"].startswith("streamed-")]
    kept = [c for c in cands if c["role"] == "streamed-chosen"]
    return {"candidates": [{"schedule": c["schedule"], "ms_per_step": c["ms_per_step"],
                            "units": len(c["units"])} for c in cands],
            "chosen_units": len(kept[0]["units"]) if kept else None}


def make_context(sbi, wl, precision, stream, **extra):
    grids = [(m.nx, m.ny, m.Lx, m.Ly) for m in wl.members]
    depths = [(m.h0 - m.delta) if m.delta is not None else None for m in wl.members]
    h0 = wl.members[0].h0
    ctx = sbi.Context(grids, wl.gravity, depths, h0=h0, order=wl.order, alias_frac=wl.alpha,
                      precision=precision, filt_beta1=wl.filt_beta1, filt_beta2=wl.filt_beta2,
                      k_ref=wl.k_ref, sponge_w=wl.sponge_w, sponge_nu=wl.sponge_nu,
                      stream=stream, check_finite=0, **extra)
    if wl.wavemaker:
        ctx.set_wavemaker(wl.wavemaker["amp"], wl.wavemaker["omega"], wl.wavemaker["phase"],
                          wl.wavemaker["x0"])
    return ctx


def compare_diagnostics(ctx, wl, torch, args):
    """Wall time of one V evaluation of member 0's group (every call queues
    the whole group's passes and synchronises): the successive scheme of
    Sec. 2.4 against the implicit form of Appendix A, whose cost per
    fixed-point iteration is the slope between 1 and 11 iterations."""
    def t(f, k=10):
        for _ in range(3):
            f()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(k):
            f()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / k * 1e3
    m0 = wl.members[0]
    n_group = sum(1 for m in wl.members if (m.nx, m.ny) == (m0.nx, m0.ny))
    esbi = t(lambda: ctx.vertical_velocity(0))
    one = t(lambda: ctx.vertical_velocity_implicit(0, 1))
    eleven = t(lambda: ctx.vertical_velocity_implicit(0, 11))
    per_it = (eleven - one) / 10.0
    _, inc = ctx.vertical_velocity_implicit(0, 11)
    return {"metric": "V evaluation time of one member group", "unit": "ms",
            "config": {"workload": wl.name, "grid": f"{m0.nx}x{m0.ny}", "order": wl.order,
                       "members_of_that_grid": n_group,
                       "evaluated": "the member group holding member 0"},
            "esbi_successive_ms": esbi, "implicit_1_iteration_ms": one,
            "implicit_ms_per_iteration": per_it, "implicit_setup_ms": one - per_it,
            "implicit_increments_11": [float(v) for v in inc],
            "note": "wall time per call including the copy of one member's V to the host"}


def time_steps(ctx, torch, stream, dt, steps, warmup):
    for _ in range(warmup):
        ctx.step(dt, 1)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        ctx.step(dt, 1)
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / 1000.0


def cpu_oracle_sample(wl, target_s=10.0, integrator="rk4", diagnostic="esbi", parallel=True):
    """The FP64 oracle timed on the host on a bounded sample of the workload:
    whole single-member RK4 steps cycling over the member shapes, about
    target_s seconds of CPU time in one process (one thread) and, with
    `parallel`, as much again in every host core at once (spawned processes,
    one single-threaded oracle each).  The reported value is the all-core
    aggregate when it was measured, the one-thread rate otherwise."""
    jobs = _oracle_jobs(wl)
    pts, steps_done, t_tot = _oracle_steps(jobs, target_s, integrator, diagnostic)
    one = pts / t_tot
    shapes = ",".join(f"{j['member'].nx}x{j['member'].ny}" for j in jobs)
    out = {"value": one, "unit": UNIT, "cores": 1, "threads": 1, "kind": "oracle",
           "sample": f"{steps_done} single-member RK4 steps cycling over member shapes [{shapes}]"
                     f" ({t_tot:.1f} s of CPU time) in one process",
           "one_thread_value": one}
    out.update(host_info())
    if parallel and (os.cpu_count() or 1) > 1:
        par = cpu_oracle_parallel(wl, target_s, integrator, diagnostic)
        out["value"] = par["value"]
        out["cores"] = par["processes"]
        out["threads"] = par["processes"]
        out["all_cores_value"] = par["value"]
        out["sample"] += (f"; then {par['processes']} single-threaded processes at once, "
                          f"{par['steps']} steps ({par['cpu_seconds']:.1f} s of CPU time in all): "
                          "value = sum of their rates")
    return out


def host_info():
    """Host CPU model and logical core count (for the oracle baselines)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    return {"nproc": os.cpu_count(), "cpu_model": model}


def _oracle_jobs(wl):
    """One member of each distinct shape, in workload order, with what a
    worker process needs to step it."""
    seen, jobs = set(), []
    for m in wl.members:
        key = (m.nx, m.ny)
        if key in seen:
            continue
        seen.add(key)
        jobs.append({"member": m, "gravity": wl.gravity, "order": wl.order, "alpha": wl.alpha,
                     "sponge_w": wl.sponge_w, "sponge_nu": wl.sponge_nu,
                     "filt_beta1": wl.filt_beta1, "filt_beta2": wl.filt_beta2, "k_ref": wl.k_ref,
                     "wavemaker": wl.wavemaker, "dt": wl.dt})
    return jobs


def _oracle_steps(jobs, target_s, integrator, diagnostic, start=0):
    """Whole single-member RK4 steps of the oracle, cycling over the jobs from
    `start`, until about target_s seconds: (points, steps, seconds)."""
    from oracle import sbi_oracle as O
    import numpy as np
    t_tot, pts, steps_done, i = 0.0, 0, 0, start
    while t_tot < target_s and steps_done < 64:
        j = jobs[i % len(jobs)]
        m = j["member"]
        wm = j["wavemaker"]
        g = O.Grid(m.nx, m.ny, m.Lx, m.Ly)
        pb = O.Problem(g, j["gravity"], m.h0, delta=m.delta, order=j["order"], alpha=j["alpha"],
                       sponge_w=j["sponge_w"], sponge_nu=j["sponge_nu"], filt_beta1=j["filt_beta1"],
                       filt_beta2=j["filt_beta2"], k_ref=j["k_ref"],
                       wavemaker=None if not wm else O.Wavemaker(
                           np.array(wm["amp"]), np.array(wm["omega"]), np.array(wm["phase"]), wm["x0"]))
        pb.integrator = integrator
        pb.diagnostic = diagnostic
        t0 = time.perf_counter()
        O.step(pb, m.eta, m.phi, j["dt"], 1)
        t_tot += time.perf_counter() - t0
        pts += m.nx * m.ny
        steps_done += 1
        i += 1
    return pts, steps_done, t_tot


def _oracle_worker(payload):
    jobs, target_s, integrator, diagnostic, start = payload
    return _oracle_steps(jobs, target_s, integrator, diagnostic, start)


def cpu_oracle_parallel(wl, target_s, integrator="rk4", diagnostic="esbi", processes=None):
    """The oracle in `processes` spawned single-threaded processes at once (all
    host cores by default), each stepping single members for about target_s
    seconds: the aggregate rate is the sum of the processes' rates."""
    import multiprocessing as mp
    procs = processes or os.cpu_count() or 1
    jobs = _oracle_jobs(wl)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        res = pool.map(_oracle_worker, [(jobs, target_s, integrator, diagnostic, w) for w in range(procs)])
    rate = sum(p / t for p, _, t in res if t > 0)
    steps = sum(s for _, s, _ in res)
    return {"value": rate, "processes": procs, "steps": steps,
            "cpu_seconds": sum(t for _, _, t in res)}


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores, on the same
    workload, metric and config as the GB300 arm.  Each step is a bounded
    sample: every host core steps single members of the workload's shapes
    for about 2 s (spawned single-threaded processes); the value is the mean
    aggregate rate over the timed steps."""
    import multiprocessing as mp
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    wl = make_workload(args.workload, args.members, 0, world, args.shard)
    jobs = _oracle_jobs(wl)
    procs = os.cpu_count() or 1
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    samples, cpu_s, nsteps = [], 0.0, 0
    with mp.get_context("spawn").Pool(procs) as pool:
        for k in range(args.warmup + args.steps):
            res = pool.map(_oracle_worker, [(jobs, 2.0, args.integrator, args.diagnostic, w + k)
                                            for w in range(procs)])
            if k >= args.warmup:
                samples.append(sum(p / t for p, _, t in res if t > 0))
                cpu_s += sum(t for _, _, t in res)
                nsteps += sum(s for _, s, _ in res)
    value = sum(samples) / len(samples)
    shapes = ",".join(f"{j['member'].nx}x{j['member'].ny}" for j in jobs)
    cpu = {"value": value, "unit": UNIT, "cores": procs, "threads": procs, "kind": "oracle",
           "sample": f"each step: {procs} single-threaded processes at once, each stepping single "
                     f"members of shapes [{shapes}] for about 2 s; {nsteps} member steps "
                     f"({cpu_s:.1f} s of CPU time) over the {args.steps} timed steps"}
    cpu.update(host_info())
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": None, "higher_is_better": True,
            "scaling": "strong" if (world > 1 and args.shard == "split") else "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": arm_config(args, wl, world), "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def accuracy_run(args, sbi, torch, stream, wl, integ, diag):
    """The workload's configured run (or --accuracy-steps) in FP64 and in FP32
    on the GPU from the same initial state: per member the relative L2
    difference of eta and phi~ at the end, each path's relative energy drift
    (E_end - E_0) / E_0 and the difference of the two drifts; the JSON record
    gives member 0 and the worst member."""
    import numpy as np
    steps = args.accuracy_steps or wl.steps
    out = {}
    t_run = {}
    for prec in (sbi.SBI_FP64, sbi.SBI_FP32):
        ctx = make_context(sbi, wl, prec, stream.cuda_stream, integrator=integ, diagnostic=diag)
        for i, m in enumerate(wl.members):
            ctx.set_state(i, m.eta, m.phi)
        E0 = [ctx.invariants(i)[1] for i in range(len(wl.members))]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        left = steps
        while left > 0:
            k = min(100, left)
            ctx.step(wl.dt, k)
            left -= k
        torch.cuda.synchronize()
        t_run[prec] = time.perf_counter() - t0
        E1 = [ctx.invariants(i)[1] for i in range(len(wl.members))]
        eta, phi = ctx.get_state_all()
        out[prec] = (ctx.split(eta), ctx.split(phi), E0, E1)
        ctx.close()

    def rel(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    per = []
    for i in range(len(wl.members)):
        e64, p64, E0_64, E1_64 = (out[sbi.SBI_FP64][0][i], out[sbi.SBI_FP64][1][i],
                                  out[sbi.SBI_FP64][2][i], out[sbi.SBI_FP64][3][i])
        e32, p32, E0_32, E1_32 = (out[sbi.SBI_FP32][0][i], out[sbi.SBI_FP32][1][i],
                                  out[sbi.SBI_FP32][2][i], out[sbi.SBI_FP32][3][i])
        d64 = (E1_64 - E0_64) / E0_64
        d32 = (E1_32 - E0_32) / E0_32
        per.append({"member": i, "eta_rel_l2": rel(e32, e64), "phi_rel_l2": rel(p32, p64),
                    "energy_drift_fp64": d64, "energy_drift_fp32": d32,
                    "drift_difference": abs(d32 - d64)})
    worst = {k: max(p[k] for p in per) for k in ("eta_rel_l2", "phi_rel_l2", "drift_difference")}
    return {"accuracy": True, "config": arm_config(args, wl, 1), "steps": steps, "dt": wl.dt,
            "members": len(wl.members), "member0": per[0], "worst": worst,
            "largest_fp64_drift": max(abs(p["energy_drift_fp64"]) for p in per),
            "seconds": {"fp64": t_run[sbi.SBI_FP64], "fp32": t_run[sbi.SBI_FP32]},
            "note": "FP32 path against the FP64 path of the same library over the run; the "
                    "energy drifts include the filter's / sponge's dissipation where those are on"}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if os.environ.get("MASTER_ADDR") is None and int(os.environ.get("WORLD_SIZE", "1")) > 1:
        os.environ["MASTER_ADDR"] = "127.0.0.1"
    import numpy as np
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import __graft_entry__ as ge
    ge.build()
    from paper_2310_19840_gb300 import sbi

    wl = make_workload(args.workload, args.members, rank, world, args.shard)
    prec = sbi.SBI_FP64 if args.precision == "fp64" else sbi.SBI_FP32
    stream = torch.cuda.Stream()
    integ = {"rk4": sbi.SBI_RK4, "lawson": sbi.SBI_LAWSON_RK4, "rk45": sbi.SBI_IF_RK45}[args.integrator]
    diag = sbi.SBI_DIAG_HOS if args.diagnostic == "hos" else sbi.SBI_DIAG_ESBI
    if args.accuracy:
        if rank == 0:
            print(json.dumps(accuracy_run(args, sbi, torch, stream, wl, integ, diag)), flush=True)
        return 0
    knobs = {"schedule": args.schedule, "col_staging": args.col_staging}
    ctx = make_context(sbi, wl, prec, stream.cuda_stream, integrator=integ, diagnostic=diag,
                       state_fp64=int(args.state_fp64), **knobs)
    for i, m in enumerate(wl.members):
        ctx.set_state(i, m.eta, m.phi)
    if args.compare_diagnostics:
        if rank == 0:
            print(json.dumps(compare_diagnostics(ctx, wl, torch, args)))
        return
    def barrier():
        if world > 1:
            torch.distributed.barrier()

    # ---- timed region (device time, max over ranks) ----
    clocks = ClockSampler(torch.cuda.current_device())
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    secs = time_steps(ctx, torch, stream, wl.dt, args.steps, args.warmup)
    clk = clocks.stop()
    secs = reduce_max(secs, world, device="cuda")
    # launches and bytes of a step under the schedule the first step chose
    launches = ctx.step_launches()
    bytes_step = ctx.step_bytes(-1)
    pts = wl.points
    split = world > 1 and args.shard == "split"
    # whole-job rate: every rank's points (a split batch: the batch's points)
    job_points = wl.notes["global_points"] if split else pts * world
    value = job_points * args.steps / secs
    gathered = None
    if split:
        # the invariants of every member of the batch, gathered by one
        # all-reduce (outside the timed region)
        from paper_2310_19840_gb300 import shard as S
        local = {gi: ctx.invariants(li) for li, gi in enumerate(wl.notes["global_members"])}
        table = S.gather_invariants(wl.notes["global_count"], local, world, device="cuda")
        gathered = {"members": int(np.count_nonzero(table[:, 1])), "of": wl.notes["global_count"],
                    "total_mass": float(table[:, 0].sum()), "total_energy": float(table[:, 1].sum())}

    # ---- per-kernel roofline: the same K steps with CUDA-event pairs per pass ----
    ctx.profile_enable(True)
    for _ in range(args.steps):
        ctx.step(wl.dt, 1)
    fams = ctx.profile_read()
    ctx.profile_enable(False)
    fam_bytes = [ctx.step_bytes(i) for i in range(len(fams))]
    # transform-pass model: every 1-D transform pass over a field streams it
    # once in and once out, 2 x (bytes of a real) per point (8 B in FP32)
    per_unit = 2 * (8 if prec == sbi.SBI_FP64 else 4)
    fam_model = [ctx.step_transforms(i) * per_unit for i in range(len(fams))]
    dom = max(range(len(fams)), key=lambda i: fams[i][2])
    name, nlaunch, ms = fams[dom]
    launches_per_step = nlaunch / max(1, args.steps)
    model_per_launch = fam_model[dom] / max(1e-9, launches_per_step)
    fused_per_launch = fam_bytes[dom] / max(1e-9, launches_per_step)
    avg_s = (ms / 1000.0) / max(1, nlaunch)
    achieved = model_per_launch / avg_s / 1e9
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    tr = ncu_traffic(name.split()[0], args.workload) if args.members is None else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": tr,
                "kernel": name, "launches_per_step": launches_per_step,
                "basis": f"transform-pass model: {per_unit} B per point per 1-D transform pass "
                         "over a field (one read, one write)",
                "algorithmic_bytes_per_launch": model_per_launch,
                "fused_bytes_per_launch": fused_per_launch,
                "fused_GBps": fused_per_launch / avg_s / 1e9,
                "fused_frac": fused_per_launch / avg_s / 1e9 / peak,
                "avg_launch_ms": avg_s * 1e3,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback",
                "share_of_step": ms / sum(f[2] for f in fams),
                "families": [{"kernel": f[0], "launches": f[1], "ms": f[2],
                              "model_GBps": (fam_model[i] * args.steps / (f[2] / 1e3) / 1e9)
                              if f[2] > 0 else None,
                              "fused_GBps": (fam_bytes[i] * args.steps / (f[2] / 1e3) / 1e9)
                              if f[2] > 0 else None} for i, f in enumerate(fams)]}
    step_gbps = bytes_step * args.steps / secs / 1e9
    step_model_gbps = ctx.step_transforms(-1) * per_unit * args.steps / secs / 1e9

    # ---- error at this configuration: FP32 path vs FP64 path, member 0 ----
    err = None
    fp64_arm = None
    if not args.no_fp64_arm and prec == sbi.SBI_FP32:
        ctx64 = make_context(sbi, wl, sbi.SBI_FP64, stream.cuda_stream, integrator=integ,
                             diagnostic=diag)
        for i, m in enumerate(wl.members):
            ctx64.set_state(i, m.eta, m.phi)
        ctx_err = make_context(sbi, wl, sbi.SBI_FP32, stream.cuda_stream, integrator=integ,
                               diagnostic=diag)
        ctx_err.set_state(0, wl.members[0].eta, wl.members[0].phi)
        ctx64_0 = ctx64
        V32 = ctx_err.vertical_velocity(0)
        V64 = ctx64_0.vertical_velocity(0)
        err = {"V_rel_l2_fp32_vs_fp64": float(np.linalg.norm(V32 - V64) / np.linalg.norm(V64)),
               "member": 0}
        k64 = max(1, min(3, args.steps))
        s64 = time_steps(ctx64, torch, stream, wl.dt, k64, 1)
        fp64_arm = {"value": pts * k64 / s64, "unit": UNIT, "ms_per_step": s64 / k64 * 1e3,
                    "steps": k64, "dtype": "f64"}
        ctx64.close()
        ctx_err.close()

    # ---- end to end through the C ABI with pinned host buffers ----
    e2e = None
    if not args.no_e2e:
        ctx_e = make_context(sbi, wl, prec, stream.cuda_stream, set_state_dealias=0,
                             integrator=integ, diagnostic=diag, **knobs)
        # every member's eta and phi~, concatenated in member order, in pinned memory
        eta_h = torch.from_numpy(np.concatenate([np.ravel(m.eta) for m in wl.members])).pin_memory()
        phi_h = torch.from_numpy(np.concatenate([np.ravel(m.phi) for m in wl.members])).pin_memory()
        eta_o = torch.empty_like(eta_h).pin_memory()
        phi_o = torch.empty_like(phi_h).pin_memory()

        def e2e_streamed():
            ctx_e.step_streamed(eta_h, phi_h, wl.dt, 1, eta_o, phi_o)

        def e2e_calls():
            ctx_e.set_state_all(eta_h, phi_h)
            ctx_e.step(wl.dt, 1)
            ctx_e.get_state_all(eta_o, phi_o)

        def e2e_time(fn):
            for _ in range(max(1, args.warmup)):
                fn()
            torch.cuda.synchronize()
            ke = max(1, min(args.steps, 10))
            t0 = time.perf_counter()
            for _ in range(ke):
                fn()
            torch.cuda.synchronize()
            return ke, reduce_max(time.perf_counter() - t0, world, device="cuda")
        nbytes = 2 * eta_h.numel() * 8
        ke, te = e2e_time(e2e_streamed)
        kc, tc = e2e_time(e2e_calls)
        e2e = {"value": job_points * ke / te, "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "steps": ke,
               "api": "sbi_step_streamed(pinned host in, dt, 1, pinned host out)",
               "streamed_split": streamed_split(ctx_e.schedule_report()),
               "three_calls": {"value": job_points * kc / tc, "steps": kc,
                               "api": "sbi_set_state_all(pinned host) + sbi_step(dt, 1) + "
                                      "sbi_get_state_all(pinned host)"}}
        ctx_e.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_sample(wl, target_s=args.cpu_seconds, integrator=args.integrator,
                                diagnostic=args.diagnostic)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
            "higher_is_better": True, "scaling": "strong" if split else "weak", "vs_baseline": None,
            "dtype": "f64" if prec == sbi.SBI_FP64 else "f32", "data": "synthetic",
            "config": arm_config(args, wl, world), "clocks": clk,
            "gpu_launches": launches * args.steps,
            "transforms_per_point_step": ctx.step_transforms(-1) / wl.points,
            "autotune": autotune_summary(ctx.autotune_report()),
            "schedule": schedule_summary(ctx.schedule_report()),
            "knobs": knobs,
            "model_step_GBps": step_model_gbps, "fused_step_GBps": step_gbps, "roofline": roofline,
            "cpu_baseline": cpu, "e2e": e2e, "fp64_plain": fp64_arm, "error": err}
    if gathered:
        line["invariants_gathered"] = gathered
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
