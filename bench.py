#!/usr/bin/env python
"""Benchmark: extrapolated GBS macro-steps of 2D acoustics on one GB300.

Workload (one "step" = one macro-step of the whole hot path): periodic 2048^2
grid, 6th-order centred FD, kappa and rho = 1 + 16 seeded Gaussians, Gaussian
pressure pulse (sigma 20 cells), GBS_{8,6} (order 8, 11 sequences, 143
grid-point updates per point per macro-step), FP32 state with FP64 combine,
H = 0.8 x the stability limit.  Metric: grid-point updates per second
(Gpt-updates/s), one update = one point advanced by one FE or LF step of one
sequence.

  python bench.py [--gpus N --steps K --warmup W] [--impl gbs|reference]

Under torchrun each rank advances its own independent problem (replicas: the
single-problem path has no exchange step); value = all ranks' updates / the
slowest rank's time.  --impl reference times the FP64 CPU oracle on the host
cores, on a bounded sample of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to L2 err 1e-6: fused FP32 vs plain FP64 GBS; Gpt-updates/s; % HBM peak"
UNIT = "Gpt-updates/s"
N_GRID = 2048
FD_ORDER = 6
SIGMA = 20.0
N_GAUSS = 16
H_FRACTION = 0.8


PREC_DESC = {0: "FP32 state (increment form) + FP64 combine", 1: "FP64",
             2: "FP64 states in FP32-pair arithmetic + FP64 combine"}


def workload_desc(n=N_GRID, prec=0, arithmetic=None):
    """The headline workload's description; arithmetic overrides the precision's wording."""
    return (f"2D acoustics {n}x{n} periodic, 6th-order FD, GBS_8,6 (11 sequences, 143 updates/pt), "
            f"{arithmetic or PREC_DESC[prec]}, H = {H_FRACTION} x stability limit")


# The time-blocked kernel's sources: DRAM traffic measured by ncu belongs to one build of them.
FUSED_SOURCES = ("paper_1907_11771_gb300/csrc/gbs_fused.cu", "paper_1907_11771_gb300/csrc/gbs_stencil.cuh",
                 "paper_1907_11771_gb300/csrc/gbs_ds.cuh", "paper_1907_11771_gb300/csrc/gbs_internal.h")

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of the time-blocked pass
# kernel on the 2D 2048^2 FP32 workload, from one ncu capture per schedule (hseg, tmax, schedule),
# keyed by the hash of FUSED_SOURCES they were measured on: another build reports no traffic.
PASSES_2D2048_TRAFFIC = {
    ("58541fb99eeb", 256, 4, 0): 5.325961984e9 + 3.071086336e9,
    ("58541fb99eeb", 192, 4, 0): 5.198048256e9 + 3.074904832e9,
    ("58541fb99eeb", 192, 4, 1): 5.235100672e9 + 3.072640768e9,
    ("58541fb99eeb", 384, 4, 0): 5.075866880e9 + 3.076349440e9,
    ("58541fb99eeb", 128, 4, 0): 6.117917440e9 + 3.075159552e9,
}

# Algorithmic minimum bytes per grid point per macro-step (FP32 states): the method must read
# y_in and the two media and write y_out once, (F + 2 + F) x 4 bytes; 2D F = 3, 3D F = 4.
ALG_MIN_BYTES_PER_POINT = {2: 32.0, 3: 40.0}


def strip_comments(src):
    """C/CUDA source without its comments, trailing blanks and empty lines (the code a
    comment-only edit leaves unchanged)."""
    import re
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return "\n".join(line.rstrip() for line in src.splitlines() if line.strip()) + "\n"


def fused_source_hash(read=None):
    """First 12 hex digits of the SHA-256 of the time-blocked kernel's sources, comments
    stripped.  read(rel) -> text overrides reading the working tree."""
    import hashlib
    h = hashlib.sha256()
    for rel in FUSED_SOURCES:
        if read is None:
            with open(os.path.join(ROOT, rel)) as f:
                text = f.read()
        else:
            text = read(rel)
        h.update(strip_comments(text).encode())
    return h.hexdigest()[:12]


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 25 ms during the timed region, and
    in a second nvidia-smi process (so that a field the driver lacks cannot cost the SM record)
    the HBM clock and temperature."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    MEM_FIELDS = "clocks.mem,clocks.max.mem,temperature.memory"

    def __init__(self, index):
        self.index = index
        self.proc = self.mem_proc = None
        self.path = self.mem_path = None

    def _start(self, fields):
        fd, path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        out = open(path, "w")
        try:
            proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={fields}",
                                     "--format=csv,noheader,nounits", "-lms", "25"],
                                    stdout=out, stderr=subprocess.DEVNULL)
        except Exception:
            out.close()
            os.unlink(path)
            raise
        return proc, path, out

    def __enter__(self):
        try:
            self.proc, self.path, self.out = self._start(self.FIELDS)
        except Exception:
            self.proc = None
        try:
            self.mem_proc, self.mem_path, self.mem_out = self._start(self.MEM_FIELDS)
        except Exception:
            self.mem_proc = None
        return self

    def __exit__(self, *a):
        for proc, out in ((self.proc, getattr(self, "out", None)), (self.mem_proc, getattr(self, "mem_out", None))):
            if proc:
                proc.terminate()
                try:
                    proc.wait(timeout=5)
                except Exception:
                    proc.kill()
                out.close()

    def mem_summary(self):
        """Median HBM clock, its maximum and the hottest HBM reading (None where unavailable)."""
        mem, mmax, temp = [], None, []
        if self.mem_proc and self.mem_path and os.path.exists(self.mem_path):
            for line in open(self.mem_path):
                parts = [t.strip() for t in line.split(",")]
                if len(parts) < 3:
                    continue
                try:
                    mem.append(float(parts[0]))
                    mmax = float(parts[1])
                except ValueError:
                    continue
                try:
                    temp.append(float(parts[2]))
                except ValueError:
                    pass
            os.unlink(self.mem_path)
        return {"mem_mhz": statistics.median(mem) if mem else None, "mem_max_mhz": mmax,
                "mem_temp_c_max": max(temp) if temp else None}

    def summary(self):
        if not self.proc or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [t.strip() for t in line.split(",")]
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
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "samples": len(sm), "reasons": sorted(reasons), **self.mem_summary()}


def max_over_ranks(value, ws, device):
    """The slowest rank's value (a time): a MAX all-reduce over the process group when ws > 1."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(ws, units_per_rank, seconds):
    """Units processed by all ranks per second of the slowest rank, in G/s (weak scaling)."""
    return ws * units_per_rank / seconds / 1e9


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------

def oracle_macro_step_timing(side, n_steps=1):
    """Time the FP64 oracle for n_steps macro-steps on a side x side grid of the same recipe."""
    from fractions import Fraction

    from oracle import gbs as OG
    from oracle import mol as OM
    from oracle import weights as OW
    from paper_1907_11771_gb300 import inputs
    from paper_1907_11771_gb300 import schemes as S
    sc = S.GBS_8_6
    steps, c = OW.scheme_weights(sc.order, list(sc.steps_dep), list(sc.steps_free),
                                 [Fraction(t) for t in sc.c_free_text])
    c = OW.to_fp64(c)
    y0, kappa, rho = inputs.acoustic_problem((side, side), 0, N_GAUSS, SIGMA * side / N_GRID)
    b = 1.0 / rho
    f = lambda v: OM.rhs_acoustic(v, kappa, b, [1.0, 1.0], FD_ORDER)
    H = 0.5  # any stable step: the cost does not depend on H
    t0 = time.perf_counter()
    y = y0
    for _ in range(n_steps):
        y = OG.gbs_macro_step(f, y, H, steps, c)
    dt = time.perf_counter() - t0
    return dt, sc.updates_per_point * side * side * n_steps


def pick_oracle_side(budget_s):
    """Largest side (multiple of 64, 128..2048) whose one oracle macro-step fits budget_s.

    Calibrated on one right-hand side of a 512^2 grid; larger grids fall out of
    cache and run slower per point, hence the safety factor."""
    from oracle import mol as OM
    import numpy as np
    side = 512
    y = np.random.default_rng(0).standard_normal((3, side, side))
    k = np.ones((side, side))
    OM.rhs_acoustic(y, k, k, [1.0, 1.0], FD_ORDER)
    t0 = time.perf_counter()
    for _ in range(2):
        OM.rhs_acoustic(y, k, k, [1.0, 1.0], FD_ORDER)
    t_rhs = (time.perf_counter() - t0) / 2
    per_pt = t_rhs / (side * side) * 1.15 * 1.8     # GBS updates on top; out-of-cache slowdown
    pts = budget_s / (143 * per_pt)
    s = int((pts ** 0.5) // 64 * 64)
    return max(128, min(N_GRID, s))


def host_cores():
    """CPUs this process may run on (its affinity set), else the host's count."""
    try:
        return len(os.sched_getaffinity(0)) or 1
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def _oracle_worker(side):
    return oracle_macro_step_timing(side)


def cpu_baseline(budget_s=15.0):
    """The FP64 oracle on the host: one process (one core), and one process per core running
    the same macro-step concurrently (the oracle is single-threaded numpy; its processes are
    started with spawn, after the GPU work)."""
    import multiprocessing as mp
    side = pick_oracle_side(budget_s)
    dt, upd = oracle_macro_step_timing(side)
    single = {"value": upd / dt / 1e9, "cores": 1, "seconds": dt}
    cores = host_cores()
    side_all = pick_oracle_side(budget_s / 2)     # memory bandwidth is shared by the processes
    try:
        t0 = time.perf_counter()
        with mp.get_context("spawn").Pool(cores) as pool:
            res = pool.map(_oracle_worker, [side_all] * cores)
        wall = time.perf_counter() - t0
        all_cores = {"value": sum(u for _, u in res) / wall / 1e9, "cores": cores, "seconds": wall,
                     "side": side_all}
    except Exception as e:  # no process pool on this host: report the single-core figure only
        all_cores = {"value": None, "cores": cores, "error": str(e)[:200]}
    best = all_cores if all_cores.get("value") else single
    return {"value": best["value"], "unit": UNIT, "cores": best["cores"], "kind": "oracle",
            "sample": (f"1 macro-step of GBS_8,6 on a {side_all}x{side_all} grid of the same recipe in each of "
                       f"{cores} concurrent processes (numpy FP64, one core each; wall time incl. process start)"
                       if best is all_cores else
                       f"1 macro-step of GBS_8,6 on a {side}x{side} grid of the same recipe (numpy FP64)"),
            "single_core": {"value": single["value"], "unit": UNIT, "cores": 1,
                            "sample": f"1 macro-step on {side}x{side} ({upd} updates, {dt:.1f} s)"},
            "all_cores": all_cores}


def run_reference(args):
    """The oracle on the host cores: every step runs one macro-step of the same sample in each of
    host_cores() concurrent processes (the oracle is single-threaded numpy; the processes are
    started once, with spawn), or in this process alone where no process pool can start."""
    import multiprocessing as mp
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    budget = 100.0 / max(1, args.steps + args.warmup)
    cores = host_cores()
    pool = None
    if cores > 1:
        try:
            pool = mp.get_context("spawn").Pool(cores)
        except Exception:
            pool = None
    used = cores if pool else 1
    side = pick_oracle_side(budget / 2 if pool else budget)   # memory bandwidth is shared

    def one_step():
        if pool is None:
            return oracle_macro_step_timing(side)
        t0 = time.perf_counter()
        res = pool.map(_oracle_worker, [side] * cores)
        return time.perf_counter() - t0, sum(u for _, u in res)

    try:
        for _ in range(args.warmup):
            one_step()
        total_t, total_u = 0.0, 0
        for _ in range(args.steps):
            dt, upd = one_step()
            total_t += dt
            total_u += upd
    finally:
        if pool is not None:
            pool.close()
            pool.join()
    v = total_u / total_t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_desc(side, arithmetic="FP64 CPU oracle"),
                       "grid": [side, side]},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": used, "kind": "oracle",
                             "sample": f"each step: 1 macro-step of GBS_8,6 on a {side}x{side} grid of the "
                                       f"same recipe in each of {used} concurrent process(es), numpy FP64, one "
                                       f"core each (the full {N_GRID}^2 grid does not fit the time budget)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def make_workload(args, rank):
    """Solver, initial state, step size, updates per macro-step and config dict of a workload."""
    import numpy as np
    import torch

    from paper_1907_11771_gb300 import binding as B
    from paper_1907_11771_gb300 import inputs
    from paper_1907_11771_gb300 import schemes as S
    from paper_1907_11771_gb300.solver import GBSSolver

    F32 = B.GBS_F32_STATE_F64_COMBINE
    prec = B.GBS_F64 if args.f64 else B.GBS_F32X2 if args.f32x2 else F32
    dt = np.float32 if prec == F32 else np.float64
    tdt = torch.float32 if prec == F32 else torch.float64
    wl = args.workload
    if wl == "2d":
        n = args.grid
        y0, kappa, rho = inputs.acoustic_problem((n, n), rank, N_GAUSS, SIGMA * n / N_GRID, dtype=dt)
        shapes, sch = [(n, n)], S.GBS_8_6
        order = FD_ORDER
        desc = workload_desc(n, prec)
        if prec == F32 and args.combine == "pairs":
            desc = desc.replace("FP64 combine", "compensated FP32-pair combine")
        slots = None
    elif wl == "3d":
        n = args.grid if args.grid != N_GRID else 512
        y0, kappa, rho = inputs.acoustic_problem((n, n, n), rank, 64, 4.0, n_pulses=3, centred=False, dtype=dt)
        shapes, sch, order = [(n, n, n)], S.GBS_8_6, 4
        desc = f"3D acoustics {n}^3 periodic, 4th-order FD, GBS_8,6, H = {H_FRACTION} x stability limit"
        slots = None
    elif wl == "batch":
        sides = inputs.batch_sides(256, rank)
        probs = [inputs.acoustic_problem((s, s), 1000 + i, N_GAUSS, SIGMA * s / N_GRID, dtype=dt)
                 for i, s in enumerate(sides)]
        y0 = np.concatenate([p[0].ravel() for p in probs])
        kappa = np.concatenate([p[1].ravel() for p in probs])
        rho = np.concatenate([p[2].ravel() for p in probs])
        shapes, sch, order = [(s, s) for s in sides], S.GBS_8_6, FD_ORDER
        slots = [i % 2 for i in range(len(sides))]
        desc = ("256 independent 2D acoustics problems, sides from {128..1024}, 6th-order FD, "
                "optimised order-8 (GBS_8,6) and order-6 (GBS_6,6) schemes alternating, one launch per macro-step")
    else:
        raise ValueError(wl)
    tk = torch.tensor(kappa.ravel(), dtype=tdt, device="cuda")
    tr = torch.tensor(rho.ravel(), dtype=tdt, device="cuda")
    sol = GBSSolver(B.GBS_ACOUSTIC, [tuple(reversed(s)) for s in shapes], [(1.0,) * len(shapes[0])] * len(shapes),
                    fd_order=order, precision=prec, kappa=tk, rho=tr)
    sol._keep = (tk, tr)
    sol.set_scheme(sch, slot=0)
    upd = sum(int(np.prod(s)) for s in shapes) * sch.updates_per_point
    if slots is not None:
        sol.set_scheme(S.GBS_6_6, slot=1)
        sol.assign_slots(slots)
        upd = sum(int(np.prod(s)) * (S.GBS_8_6 if sl == 0 else S.GBS_6_6).updates_per_point
                  for s, sl in zip(shapes, slots))
    Hs = [H_FRACTION * h for h in sol.stability_limit()]
    y = torch.tensor(np.asarray(y0).ravel(), dtype=tdt, device="cuda")
    cfg = {"workload": desc, "shapes": shapes if len(shapes) < 4 else f"{len(shapes)} problems",
           "scheme": sch.name, "updates_per_step_per_gpu": upd,
           "updates_per_point": upd / sum(int(np.prod(s)) for s in shapes), "shape_zyx": list(shapes[0])}
    return sol, y, (Hs if len(Hs) > 1 else Hs[0]), upd, cfg


def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1907_11771_gb300 import binding as B
    from paper_1907_11771_gb300 import build as Bld
    from paper_1907_11771_gb300 import inputs
    from paper_1907_11771_gb300 import schemes as S
    from paper_1907_11771_gb300.solver import GBSSolver

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    Bld.build()

    sol, y, H, upd_per_step, cfg = make_workload(args, rank)
    kernel = {"auto": B.GBS_KERNEL_AUTO, "plain": B.GBS_KERNEL_PLAIN, "fused": B.GBS_KERNEL_FUSED}[args.kernel]
    sol.set_option("kernel", kernel)
    tuned = None
    if args.hseg:
        sol.set_option("hseg", args.hseg)
    if args.tmax:
        sol.set_option("tmax", args.tmax)
    if args.schedule >= 0:
        sol.set_option("schedule", args.schedule)
    if args.zseg:
        sol.set_option("zseg", args.zseg)
    if args.seqfuse != -1:
        sol.set_option("seqfuse", args.seqfuse)
    if args.seqgroup != -1:
        sol.set_option("seqgroup", args.seqgroup)
    if args.tma != -1:
        sol.set_option("tma", args.tma)
    if args.combine == "pairs":
        sol.set_option("combine", 1)
    if not (args.hseg or args.tmax or args.zseg or args.schedule >= 0 or args.no_autotune):
        from paper_1907_11771_gb300 import autotune as AT
        r = AT.autotune(sol, y, H, cache=os.path.join(tempfile.gettempdir(), "gbs_gb300_tune.json"))
        if r is not None:
            tuned = {"options": r["options"], "from_cache": r["cached"], "macro_step_s": r["seconds"],
                     "candidates": len(r.get("table", []))}
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > 129 MB L2

    def barrier():
        if ws > 1:
            dist.barrier()

    for _ in range(args.warmup):
        sol.step(y, y, H, 1)
    torch.cuda.synchronize()
    barrier()
    l0 = sol.kernel_launches
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    # the clock sampler runs over the timed region and the kernel-timing pass after it (the same
    # macro-steps again), so that short timed regions still get several samples under load
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        barrier()
        for i in range(args.steps):
            flush.fill_(float(i))
            evs[i][0].record(stream)
            sol.step(y, y, H, 1)
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        barrier()
        launches = sol.kernel_launches - l0

        # dominant-kernel roofline: CUDA events recorded by the library around each launch
        sol.set_option("time_kernels", 1)
        sol.kernel_time()
        for i in range(args.steps):
            flush.fill_(float(i))
            sol.step(y, y, H, 1)
        nl, kms, kbytes = sol.kernel_time()
        sol.set_option("time_kernels", 0)
    ms = sum(a.elapsed_time(b) for a, b in evs)
    ms_max = max_over_ranks(ms, ws, "cuda")
    value = whole_job_rate(ws, upd_per_step * args.steps, ms_max / 1e3)

    # the opt-in variant of the time-blocked FP32 path: the combine in compensated FP32 pairs
    variant = None
    if sol_kernel_is_fused(sol, B) and not (args.f64 or args.f32x2) and args.combine == "f64":
        sol.set_option("combine", 1)
        for _ in range(args.warmup):
            sol.step(y, y, H, 1)
        torch.cuda.synchronize()
        barrier()
        vev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for i in range(args.steps):
            flush.fill_(float(i))
            vev[i][0].record(stream)
            sol.step(y, y, H, 1)
            vev[i][1].record(stream)
        torch.cuda.synchronize()
        vms = max_over_ranks(sum(a.elapsed_time(b) for a, b in vev), ws, "cuda")
        sol.set_option("combine", 0)
        variant = {"combine_dtype": "f32 pairs (compensated, about 2^-48 of sum_k |c_k d*_k|)",
                   "value": whole_job_rate(ws, upd_per_step * args.steps, vms / 1e3), "unit": UNIT,
                   "ms_per_step": vms / args.steps}
    peak, peak_kind = peaks()
    fused = sol_kernel_is_fused(sol, B)
    launch_s = kms / nl / 1e3 if nl else None
    # one launch of the time-blocked kernel is a whole macro-step; the one-level kernel runs one
    # leap-frog level of one sequence, nl / steps launches per macro-step
    pts = upd_per_step / cfg["updates_per_point"]
    per_launch_share = args.steps / nl if nl else 0.0
    esz = 8 if (args.f64 or args.f32x2) else 4
    alg_min = ALG_MIN_BYTES_PER_POINT[len(cfg["shape_zyx"])] * esz / 4 * pts * per_launch_share
    sched_bytes = kbytes / nl if nl else None
    achieved = alg_min / launch_s / 1e9 if nl else None
    traffic, traffic_key = None, None
    if args.workload == "2d" and args.grid == N_GRID and not (args.f64 or args.f32x2) and fused:
        traffic_key = (fused_source_hash(),) + tuple(int(sol.get_option(k)) for k in ("hseg", "tmax", "schedule"))
        traffic = PASSES_2D2048_TRAFFIC.get(traffic_key)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak if achieved else None, "traffic": traffic,
            "peak_kind": f"{peak_kind} HBM copy bandwidth",
            "kernel": ("3D time-blocked pass (k_tb3)" if len(cfg["shape_zyx"]) == 3 else "fused pass (k_passes)")
                      if fused else ("sequence-fused tiled leap-frog step (k_lf_tiled_seqs)" if sol.get_option("seqfuse")
                                     else "tiled leap-frog step (k_lf_tiled)"),
            "avg_launch_ms": launch_s * 1e3 if nl else None,
            "achieved_basis": "algorithmic minimum: y_in, kappa, rho read and y_out written once per macro-step "
                              f"({ALG_MIN_BYTES_PER_POINT[len(cfg['shape_zyx'])] * esz / 4:.0f} B per grid point)",
            "algorithmic_min_bytes_per_launch": alg_min,
            "schedule_bytes_per_launch": sched_bytes,
            "frac_sched": sched_bytes / launch_s / 1e9 / peak if nl else None,
            "frac_dram": traffic / launch_s / 1e9 / peak if (traffic and nl) else None,
            "traffic_key": list(traffic_key) if traffic_key else None}

    # end to end through the C ABI with host buffers: every step copies its input state from
    # pinned host memory, runs one macro-step and copies its result back (gbs_step_host_stream:
    # the copies of neighbouring steps overlap the macro-steps)
    e2e = None
    if not isinstance(H, list):
        hbuf = torch.empty(y.numel(), dtype=y.dtype, pin_memory=True)
        hbuf.copy_(y.cpu())
        hout = torch.empty(y.numel(), dtype=y.dtype, pin_memory=True)   # empty_like would not pin
        sol.step_host_stream([hbuf] * 2, [hout] * 2, H, 1)
        barrier()
        t0 = time.perf_counter()
        sol.step_host_stream([hbuf] * args.steps, [hout] * args.steps, H, 1)
        e2e_s = max_over_ranks(time.perf_counter() - t0, ws, "cuda")
        nbytes = y.numel() * y.element_size()
        e2e = {"value": whole_job_rate(ws, upd_per_step * args.steps, e2e_s), "unit": UNIT,
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
               "api": "gbs_step_host_stream (host copies of neighbouring steps overlap the macro-steps)"}

    sol.sync()
    line = None
    if rank == 0:
        fused = sol_kernel_is_fused(sol, B)
        if tuned is not None:
            cfg["autotuned_schedule"] = tuned
        cfg.update({"combine_dtype": ("f32 pairs (double-single, ~48-bit)" if fused and args.combine == "pairs"
                                      else "f64"),
                    "kernel": roof["kernel"], "l2": "flushed (256 MB write) before every timed step",
                    "sequence_fused": {"in_use": int(sol.get_option("seqfuse")),
                                       "group": int(sol.get_option("seqgroup"))},
                    "parallelism": f"replicas x{ws}"})
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if args.f64 else "f32x2" if args.f32x2 else "f32",
                "data": "synthetic", "config": cfg,
                "clocks": clk.summary(), "gpu_launches": launches, "roofline": roof, "e2e": e2e}
        if variant is not None:
            line["variant_pair_combine"] = variant
        if ws == 1 and not args.no_tts and args.workload == "2d" and not (args.f64 or args.f32x2):
            sol.close()
            # the headline scheme, and the classical {2,4,6,8} whose small weights keep the FP32
            # rounding floor below 1e-6 at its stability-limited step
            line["time_to_1e6"] = time_to_solution(args, 1, compact=True,
                                                   schemes={"GBS_8,6": 1, "SQ8{2,4,6,8}": 1})
        if ws == 1 and not args.no_cpu_baseline and args.workload == "2d" and not (args.f64 or args.f32x2):
            line["cpu_baseline"] = cpu_baseline()
        print(json.dumps(line), flush=True)
    sol.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


def run_adjoint(args):
    """Misfit-gradient throughput: one step = J and dJ/dkappa over M macro-steps (forward sweep with
    a checkpoint every C, then the backward sweep recomputing each segment and running the
    adjoint macro-steps; with --adj-snapshots S a binomial schedule of S stored states instead),
    2D acoustics n x n (default 1024^2), 4th-order FD, rho = 1, 16-Gaussian kappa, Gaussian
    pressure source sigma = 8, 64 receivers on the row 3n/4, GBS_8,6 in FP32 (--f64: FP64 states;
    --f32x2: FP64 states in FP32 pairs, forward and adjoint in pair arithmetic).  Counted work: M
    forward plus M adjoint macro-steps of P x 143 updates; the checkpoint recomputation is
    overhead.  Observed data: a forward run of the same solver with a perturbed
    kappa (kappa + 0.05 x one more seeded Gaussian)."""
    import numpy as np
    import torch

    from paper_1907_11771_gb300 import binding as B
    from paper_1907_11771_gb300 import build as Bld
    from paper_1907_11771_gb300 import inputs
    from paper_1907_11771_gb300 import schemes as S
    from paper_1907_11771_gb300.autograd import gbs_misfit_and_grad
    from paper_1907_11771_gb300.solver import GBSSolver

    torch.cuda.set_device(0)
    Bld.build()
    n = args.grid if args.grid != N_GRID else 1024
    M, C = args.adj_macro, args.adj_checkpoint
    SN = args.adj_snapshots or None
    ckpt_desc = f"binomial checkpointing with {SN} stored states" if SN else f"checkpoint every {C}"
    prec = B.GBS_F64 if args.f64 else B.GBS_F32X2 if args.f32x2 else B.GBS_F32_STATE_F64_COMBINE
    dt = np.float32 if prec == B.GBS_F32_STATE_F64_COMBINE else np.float64
    tdt = torch.float32 if dt == np.float32 else torch.float64
    esz = 4 if dt == np.float32 else 8
    prec_name = {B.GBS_F64: "FP64", B.GBS_F32X2: "FP64 states in FP32 pairs"}.get(prec, "FP32")
    y0, kappa, rho = inputs.acoustic_problem((n, n), 0, N_GAUSS, 8.0, const_rho=True, dtype=dt)
    bump = inputs.smooth_media((n, n), 1, 7, 1.0) - 1.0        # one more seeded Gaussian
    tk = torch.tensor(kappa.ravel(), device="cuda")
    tr = torch.tensor(rho.ravel(), device="cuda")
    sol = GBSSolver(B.GBS_ACOUSTIC, [(n, n)], [(1.0, 1.0)], fd_order=4, precision=prec,
                    kappa=tk, rho=tr, enable_adjoint=True)
    sol.set_scheme(S.GBS_8_6)
    H = H_FRACTION * sol.stability_limit()[0]
    rcv = torch.tensor(inputs.line_receivers(n, 64), device="cuda")
    y = torch.tensor(y0.ravel(), device="cuda")
    # observed data from the perturbed medium
    k_true = torch.tensor((kappa + 0.05 * np.asarray(bump, dtype=dt)).ravel(), device="cuda")
    sol.set_media(k_true, tr)
    data = torch.empty(M, rcv.numel(), dtype=tdt, device="cuda")
    yy = y.clone()
    for m in range(M):
        sol.step(yy, yy, H, 1)
        data[m] = yy[rcv]
    sol.set_media(tk, tr)
    P = n * n
    upd = 2 * M * P * S.GBS_8_6.updates_per_point
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        gbs_misfit_and_grad(sol, y, H, M, rcv, data, C, SN)
    torch.cuda.synchronize()
    l0 = sol.kernel_launches
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(0) as clk:
        for i in range(args.steps):
            flush.fill_(float(i))
            evs[i][0].record()
            J, g = gbs_misfit_and_grad(sol, y, H, M, rcv, data, C, SN)
            evs[i][1].record()
        torch.cuda.synchronize()
    launches = sol.kernel_launches - l0
    ms = sum(a.elapsed_time(b) for a, b in evs)
    value = upd * args.steps / (ms / 1e3) / 1e9
    # roofline of the adjoint's reverse leap-frog kernel: library events around its launches
    lam = torch.zeros_like(y)
    grad = torch.zeros(P, dtype=torch.float64, device="cuda")
    sol.set_option("time_kernels", 1)
    sol.kernel_time()
    for i in range(3):
        flush.fill_(float(i))
        sol.adjoint_step(y, lam, lam, grad, H)
    nl, kms, kbytes = sol.kernel_time()
    sol.set_option("time_kernels", 0)
    peak, peak_kind = peaks()
    achieved = (kbytes / nl) / (kms / nl / 1e3) / 1e9 if nl else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak if achieved else None, "traffic": None,
            "peak_kind": f"{peak_kind} HBM copy bandwidth", "kernel": "adjoint reverse leap-frog step (k_adj_rev)",
            "algorithmic_bytes_per_launch": kbytes / nl if nl else None, "avg_launch_ms": kms / nl if nl else None}
    # end to end: inputs from pinned host memory, gradient back to the host, every step
    hy = y.cpu().pin_memory()
    hk = tk.cpu().pin_memory()
    hd = data.cpu().pin_memory()
    hg = torch.empty(P, dtype=torch.float64).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(args.steps):
        y.copy_(hy, non_blocking=True)
        tk.copy_(hk, non_blocking=True)
        data.copy_(hd, non_blocking=True)
        J, g = gbs_misfit_and_grad(sol, y, H, M, rcv, data, C, SN)
        hg.copy_(g, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    e2e_s = e0.elapsed_time(e1) / 1e3
    e2e = {"value": upd * args.steps / e2e_s / 1e9, "unit": UNIT,
           "h2d_bytes_per_step": (hy.numel() + hk.numel() + hd.numel()) * esz, "d2h_bytes_per_step": hg.numel() * 8}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {4: "f32"}.get(esz, "f32x2" if args.f32x2 else "f64"), "data": "synthetic",
            "config": {"workload": (f"misfit gradient: 2D acoustics {n}x{n}, 4th-order FD, rho = 1, 64 receivers, "
                                    f"GBS_8,6 {prec_name}, {M} macro-steps, {ckpt_desc}; one step = forward + "
                                    f"checkpointed backward; updates counted: {M} forward + {M} adjoint macro-steps"),
                       "shapes": [[n, n]], "scheme": "GBS_8,6", "updates_per_step_per_gpu": upd,
                       "macro_steps": M, "checkpoint_every": None if SN else C, "snapshots": SN, "misfit_J": J,
                       "l2": "flushed (256 MB write) before every timed step", "parallelism": "replicas x1"},
            "clocks": clk.summary(), "gpu_launches": launches, "roofline": roof, "e2e": e2e}
    print(json.dumps(line), flush=True)
    sol.close()
    return 0


def run_oneway(args):
    """Sec. 4's test problem on the GPU: the one-way wave u_t + u_x = 0 with spectral derivatives.
    Throughput: a batch of 256 problems of n = 1024, GBS_8,6 at 0.99 x the stability limit.  The
    FFTs run in FP64, so the kernel is bound by GB300's FP64 rate: its roofline counts
    algorithmic FP64 flops (per right-hand side two radix-2 FFTs of length n/2, the real signal
    packed as a half-length complex one, 10 flops per butterfly, plus the bins' pairing and the
    scaling) against the nominal FP64 rate
    (1.25 TFLOP/s: 152 SMs x 2 FP64 FMA per clock x 2 flops x 2.07 GHz).  The config also
    carries Sec. 4's convergence study: the error after one trip around the interval at
    lambda = dt/dx = 0.99 ISB / pi for GBS_8,6 and GBS_12,8, n = 16 .. 1024."""
    import numpy as np
    import torch

    from paper_1907_11771_gb300 import binding as B
    from paper_1907_11771_gb300 import build as Bld
    from paper_1907_11771_gb300 import schemes as S
    from paper_1907_11771_gb300.solver import GBSSolver

    torch.cuda.set_device(0)
    Bld.build()
    study = {}
    for sch in (S.GBS_8_6, S.GBS_12_8):
        rows = []
        for n in (16, 32, 64, 128, 256, 512, 1024):
            sol = GBSSolver(B.GBS_ONEWAY_SPECTRAL, [(n,)], [(1.0 / n,)], fd_order=0, precision=B.GBS_F64)
            sol.set_scheme(sch)
            isb = sol.weights()[2]
            M = int(np.ceil(1.0 / (0.99 / np.pi * isb / n)))
            u0 = 0.5 * (1 - np.cos(2 * np.pi * np.arange(n) / n))
            y = torch.tensor(u0, dtype=torch.float64, device="cuda")
            sol.step(y, y, 1.0 / M, M)
            sol.sync()
            rows.append({"n": n, "macro_steps": M, "max_error": float(np.max(np.abs(y.cpu().numpy() - u0)))})
            sol.close()
        study[sch.name] = rows
    nb, n = 256, 1024
    sol = GBSSolver(B.GBS_ONEWAY_SPECTRAL, [(n,)] * nb, [(1.0 / n,)] * nb, fd_order=0, precision=B.GBS_F64)
    sol.set_scheme(S.GBS_8_6)
    H = 0.99 * sol.stability_limit()[0]
    rng = np.random.default_rng(0)
    y = torch.tensor(rng.standard_normal(nb * n), dtype=torch.float64, device="cuda")
    upd = nb * n * S.GBS_8_6.updates_per_point
    for _ in range(args.warmup):
        sol.step(y, y, H, 1)
    torch.cuda.synchronize()
    l0 = sol.kernel_launches
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(0) as clk:
        for i in range(args.steps):
            evs[i][0].record()
            sol.step(y, y, H, 1)
            evs[i][1].record()
        torch.cuda.synchronize()
    launches = sol.kernel_launches - l0
    ms = sum(a.elapsed_time(b) for a, b in evs)
    value = upd * args.steps / (ms / 1e3) / 1e9
    m, logm = n // 2, int(np.log2(n)) - 1
    # per right-hand side: two FFTs of length n/2 (the real signal as a half-length complex one;
    # 10 flops per butterfly), the pairing of bins k, m - k with the -i k multiply (46 flops per
    # pair) and the scaling of the n samples
    rhs_flops = 2 * (m // 2) * logm * 10 + (m // 2) * 46 + 2 * n
    evals = 1 + sum(S.GBS_8_6.steps)                     # shared f0 plus one per leap-frog step
    flops = nb * evals * rhs_flops * args.steps
    peak_tf = 152 * 2 * 2 * 2.07e9 / 1e12
    achieved = flops / (ms / 1e3) / 1e12
    hy = y.cpu().pin_memory()
    ho = torch.empty_like(hy).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(args.steps):
        y.copy_(hy, non_blocking=True)
        sol.step(y, y, H, 1)
        ho.copy_(y, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    e2e = {"value": upd * args.steps / (e0.elapsed_time(e1) / 1e3) / 1e9, "unit": UNIT,
           "h2d_bytes_per_step": hy.numel() * 8, "d2h_bytes_per_step": ho.numel() * 8}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": (f"Sec. 4 one-way wave u_t + u_x = 0, spectral derivatives, {nb} problems of "
                                    f"n = {n}, GBS_8,6 FP64, H = 0.99 x stability limit"),
                       "shapes": f"{nb} x [{n}]", "scheme": "GBS_8,6", "updates_per_step_per_gpu": upd,
                       "section4_convergence": study, "parallelism": "replicas x1"},
            "clocks": clk.summary(), "gpu_launches": launches,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tf, "unit": "TFLOP/s",
                         "frac": achieved / peak_tf, "traffic": None,
                         "peak_kind": "FP64 from unit counts and clock (152 SMs x 2 FMA/clk x 2 flops x 2.07 GHz)",
                         "kernel": "spectral macro-step (k_spectral_macro)"},
            "e2e": e2e}
    print(json.dumps(line), flush=True)
    sol.close()
    return 0


def run_time_to_solution(args):
    print(json.dumps(time_to_solution(args, args.tts_levels)), flush=True)
    return 0


def time_to_solution(args, levels, compact=False, schemes=None):
    """Time to a relative L2 error of 1e-6 at t = T (2D acoustics, same recipe on an n x n grid;
    T = tts_macro macro-steps of GBS_8,6 at H0 = 0.8 x its stability limit): for each scheme
    raced, the FP32-state paths (time-blocked and plain), the plain FP64 path, and FP64 states in
    FP32-pair arithmetic on the plain and the time-blocked kernels, each swept over
    H = H_s / 2^j, j < levels (H_s the fewest macro-steps of the scheme at 0.8 x its own
    stability limit that reach T), against an FP64 GBS_12,8 reference run at a quarter of its own
    0.8 x limit and checked against one at an eighth.  schemes: {name: levels} (default the
    one scheme --tts-scheme with `levels`).  compact: per path only the fastest time that reaches
    1e-6 and the smallest error reached."""
    import numpy as np
    import torch

    from paper_1907_11771_gb300 import binding as B
    from paper_1907_11771_gb300 import build as Bld
    from paper_1907_11771_gb300 import inputs
    from paper_1907_11771_gb300 import schemes as S
    from paper_1907_11771_gb300.solver import GBSSolver

    Bld.build()
    n, M_T = args.tts_grid, args.tts_macro
    y0, kappa, rho = inputs.acoustic_problem((n, n), 0, N_GAUSS, SIGMA * n / N_GRID)
    if schemes is None:
        schemes = {args.tts_scheme: levels}

    def solver(prec, scheme, kernel):
        dt = np.float32 if prec == B.GBS_F32_STATE_F64_COMBINE else np.float64
        tk = torch.tensor(kappa.astype(dt).ravel(), device="cuda")
        tr = torch.tensor(rho.astype(dt).ravel(), device="cuda")
        s = GBSSolver(B.GBS_ACOUSTIC, [(n, n)], [(1.0, 1.0)], fd_order=FD_ORDER, precision=prec, kappa=tk, rho=tr)
        s.set_scheme(scheme)
        s.set_option("kernel", kernel)
        s._keep = (tk, tr)
        return s

    def run(sol, H, M, dt):
        y = torch.tensor(y0.ravel(), dtype=dt, device="cuda")
        out = torch.empty_like(y)
        sol.step(y, out, H, 1)           # warm-up (graph capture)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        sol.step(y, out, H, M)
        e1.record()
        torch.cuda.synchronize()
        return out.double(), e0.elapsed_time(e1) / 1e3

    f64 = solver(B.GBS_F64, S.GBS_8_6, B.GBS_KERNEL_PLAIN)
    T = M_T * H_FRACTION * f64.stability_limit()[0]
    ref_sol = solver(B.GBS_F64, S.GBS_12_8, B.GBS_KERNEL_PLAIN)
    Mref = int(np.ceil(T / (H_FRACTION * ref_sol.stability_limit()[0]))) * 4
    ref, _ = run(ref_sol, T / Mref, Mref, torch.float64)
    ref2, _ = run(ref_sol, T / (2 * Mref), 2 * Mref, torch.float64)
    ref_sol.close()
    rel = lambda a: (f64.norms(a, ref)[0] / f64.norms(ref)[0]) ** 0.5
    ref_err = rel(ref2)
    paths = [("fused FP32 state + FP64 combine", B.GBS_F32_STATE_F64_COMBINE, B.GBS_KERNEL_FUSED, torch.float32),
             ("plain FP32 state + FP64 combine", B.GBS_F32_STATE_F64_COMBINE, B.GBS_KERNEL_PLAIN, torch.float32),
             ("plain FP64", B.GBS_F64, B.GBS_KERNEL_PLAIN, torch.float64),
             ("plain FP32 pairs (FP64 states)", B.GBS_F32X2, B.GBS_KERNEL_PLAIN, torch.float64),
             ("fused FP32 pairs (FP64 states)", B.GBS_F32X2, B.GBS_KERNEL_FUSED, torch.float64)]
    races = {}
    for sname, lev in schemes.items():
        scheme = S.ALL[sname]
        sch = solver(B.GBS_F64, scheme, B.GBS_KERNEL_PLAIN)
        M0 = int(np.ceil(T / (H_FRACTION * sch.stability_limit()[0] * (1.0 + 1e-12))))
        sch.close()
        rows, tuned = {}, {}
        for name, prec, kernel, dt in paths:
            sol = solver(prec, scheme, kernel)
            if kernel == B.GBS_KERNEL_FUSED and not args.no_autotune:
                from paper_1907_11771_gb300 import autotune as AT
                yt = torch.tensor(y0.ravel(), dtype=dt, device="cuda")
                r = AT.autotune(sol, yt, T / M0, cache=os.path.join(tempfile.gettempdir(), "gbs_gb300_tune.json"))
                if r is not None:
                    tuned[name] = r["options"]
            rows[name] = []
            for j in range(lev):
                M = M0 * 2 ** j
                out, secs = run(sol, T / M, M, dt)
                rows[name].append({"H_over_H0": 2.0 ** -j, "macro_steps": M, "seconds": secs, "rel_l2": rel(out),
                                   "gpt_updates_per_s": scheme.updates_per_point * n * n * M / secs / 1e9})
            sol.close()
        best = {k: min((r["seconds"] for r in v if r["rel_l2"] <= 1e-6), default=None) for k, v in rows.items()}
        race = {"H0": T / M0, "macro_steps_at_H0": M0, "time_to_1e-6_s": best, "autotuned_schedule": tuned}
        if compact:
            race["smallest_rel_l2"] = {k: min(r["rel_l2"] for r in v) for k, v in rows.items()}
            race["H_over_H0_swept"] = [2.0 ** -j for j in range(lev)]
        else:
            race["paths"] = rows
        races[sname] = race
    f64.close()
    fastest = {}
    for sname, race in races.items():
        for k, v in race["time_to_1e-6_s"].items():
            if v is not None and (k not in fastest or v < fastest[k]["seconds"]):
                fastest[k] = {"seconds": v, "scheme": sname}
    out = {"study": "time to relative L2 error 1e-6", "grid": [n, n], "t_final": T,
           "reference": f"GBS_12,8 FP64, {Mref} macro-steps", "reference_self_check_rel_l2": ref_err,
           "fastest_to_1e-6": fastest, "schemes": races}
    return out


def sol_kernel_is_fused(sol, B):
    try:
        return sol.uses_fused()
    except Exception:
        return False


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gbs", "reference"], default="gbs")
    ap.add_argument("--kernel", choices=["auto", "plain", "fused"], default="auto")
    ap.add_argument("--grid", type=int, default=N_GRID)
    ap.add_argument("--workload", choices=["2d", "3d", "batch", "adjoint", "oneway"], default="2d",
                    help="2d (default, the headline workload), 3d (512^3), batch (256 problems), "
                         "adjoint (misfit gradient, 1024^2) or oneway (Sec. 4 spectral test problem)")
    ap.add_argument("--adj-macro", type=int, default=100, help="macro-steps of one misfit gradient (adjoint workload)")
    ap.add_argument("--adj-checkpoint", type=int, default=50, help="checkpoint interval (adjoint workload)")
    ap.add_argument("--adj-snapshots", type=int, default=0,
                    help="binomial checkpointing with this many stored states instead (adjoint workload)")
    ap.add_argument("--f64", action="store_true", help="FP64 state (plain kernels)")
    ap.add_argument("--f32x2", action="store_true", help="FP64 states computed in FP32 pairs (plain kernels)")
    ap.add_argument("--hseg", type=int, default=0, help="row-segment height of the time-blocked tiles (0: default)")
    ap.add_argument("--zseg", type=int, default=0, help="z-planes per block of the 3D time-blocked passes (0: default)")
    ap.add_argument("--seqfuse", type=int, choices=[-1, 0, 1], default=-1,
                    help="one-level kernels: all sequences of a level per launch (1), one (0), by dimension (-1)")
    ap.add_argument("--seqgroup", type=int, default=-1, help="most sequences per fused one-level launch (-1: default)")
    ap.add_argument("--tmax", type=int, default=0, help="most leap-frog levels per time-blocked pass (0: default)")
    ap.add_argument("--schedule", type=int, default=-1, help="work-queue order of the time-blocked kernel (-1: default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--combine", choices=["f64", "pairs"], default="f64",
                    help="combine of the time-blocked FP32 path: FP64 (default) or compensated FP32 pairs")
    ap.add_argument("--tma", type=int, default=-1, choices=[-1, 0, 1],
                    help="tensor-copy staging of the plain step kernel: -1 default (3D), 1 always, 0 never")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default time-blocked schedule instead of autotuning it first")
    ap.add_argument("--time-to-solution", action="store_true",
                    help="run the time-to-1e-6 study (fused FP32 vs plain FP64) instead of the throughput bench")
    ap.add_argument("--no-tts", action="store_true",
                    help="leave the time-to-1e-6 race (1024^2, two step sizes) out of the default line")
    ap.add_argument("--tts-grid", type=int, default=1024)
    ap.add_argument("--tts-macro", type=int, default=100)
    ap.add_argument("--tts-levels", type=int, default=3)
    ap.add_argument("--tts-scheme", default="GBS_8,6", help="scheme raced in the time-to-solution study (schemes.ALL)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gbs":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.time_to_solution:
        return run_time_to_solution(args)
    if args.workload == "adjoint":
        return run_adjoint(args)
    if args.workload == "oneway":
        return run_oneway(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
