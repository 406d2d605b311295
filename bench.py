"""Benchmark: Newton multigrid steady solve of the 2D partial-dry channel.

Workload: 1024 x 1024 cells on [0,4] x [0,1], 16 seeded Gaussian bumps with
dry tops, inflow discharge hu ~ U[0.5, 1.5] at x = 0, outflow depth 0.6 at
x = 4, reflective walls, LLF flux with the wet/dry speed increase; mixed
precision (FP32 multigrid inner solve, FP64 residual / Jacobian / update /
norms), W-cycles (gamma = 2, N_L = 7 with an exact solve on the 8 x 8
coarsest level, N_mg = 3), eps_p = 2, tol 1e-10.

One step = one complete swnmg_solve (Algorithm 1 including its Step 1) from
the same initial state, with inputs resident in HBM.  value = cells x
multigrid cycles / second over the timed steps; ms_per_step = time to
sum ||R_i||_1 < 1e-10.  The FP64 path is timed on the same problem and
reported beside it.  e2e repeats the mixed solve through host buffers
(pinned H2D of the initial state, D2H of the steady state inside the timed
region).  Multi-GPU: independent replicas (the lexicographic sweeps do not
shard), weak scaling.

--impl reference times the CPU FP64 oracle (the reference restatement of the
method) on a bounded sample of the same workload: one Newton step
(BLU-SGS sweep, Jacobian, N_mg cycles, update) from the initial state.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell*cycles/s to residual 1e-10 at 1024^2 (mixed FP32-MG / FP64), time to 1e-10"
UNIT = "cell*cycles/s"
NX = NY = 1024
LEVELS = 7


def workload(precision, nx=NX, ny=NY):
    from paper_1608_06721_gb300 import workloads as W
    return W.channel_bench(nx, ny, precision, n_levels=LEVELS)


def config_dict(p, flush):
    prm = p.params
    return {"workload": "2D partial-dry channel %dx%d (LLF, W-cycle N_L=%d exact coarsest, N_mg=%d, eps_p=%g, seed 301)"
            % (p.nx, p.ny, prm.n_levels, prm.n_mg, prm.eps_p),
            "cells": p.n,
            "precision": ("mixed FP32 multigrid and FP32 Step 1 BLU-SGS / FP64 residual+update"
                          if prm.precision == 2 else "mixed FP32 multigrid / FP64 residual+update"),
            "l2": flush, "tol": prm.tol}


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) >= 9:
                for k, nm in enumerate(names):
                    if r[5 + k].lower().startswith("active"):
                        reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- peaks

def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            hbm = d.get("hbm_gbs") or d.get("hbm_GBps")
            if hbm:
                return float(hbm), "measured (MEASURED_PEAKS.json hbm_gbs)"
        except (ValueError, OSError):
            pass
    return 6800.0, "fallback 6.8 TB/s (MEASURED_PEAKS.json absent)"


# FP64 unit peak of GB300: 152 SMs x 2 FP64 lanes/clk x 2.07 GHz = 0.63e12
# FP64 instructions/s (1.26 TFLOP/s counting an FMA as two); the flux
# kernels are compiled without FMA contraction, so one counted add, mul,
# div or sqrt is compared against one instruction slot.
FP64_OPS_PEAK = 152 * 2 * 2.07e9


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per cell of one
# launch, from ncu captures of one BLU-SGS and one SGS half-sweep of the
# 512 x 512 channel; a launch's traffic grows with the cells it processes, so
# it is scaled to the timed launches by their cell counts.  Both kernels
# changed after those captures (the Roe flux, the Froude-number boundary and
# the time-step term entered the BLU-SGS cell update; the SGS cell update
# became one explicit-FMA function), so `traffic` is null until the next
# capture, and the captured figure is kept as `traffic_previous_build`.
TRAFFIC_PER_CELL = {"blusgs": 36.2, "blusgs_coarse": 36.2, "sgs_fine": 217.9, "sgs_coarse": 217.9}
TRAFFIC_CURRENT = False


def algorithmic(cls, p, fp32):
    """(bound, algorithmic units per cell) of a kernel class: bytes for the
    block-SGS smoother, FP64 operations for the flux kernels.  One edge
    evaluation (reconstruction, two reciprocals, two square roots, the flux
    and the sources) is about 53 FP64 operations; a cell owns about 2.5 edge
    evaluations in the residual (130), 7 per edge in the FD Jacobian (1035),
    and a BLU-SGS cell update makes 16 plus a 3x3 elimination (1020).
    Multiplied by the cells the timed launches processed, as reported by the
    library."""
    nc = p.ncomp
    w = 4 if fp32 else 8
    if cls in ("sgs_fine", "sgs_coarse"):
        return "hbm", (5 * nc * nc - nc * nc + 9 + 3 + 2 * nc) * w + 1   # blocks, LU, b, x in/out, piv
    if cls in ("blusgs", "blusgs_coarse"):
        return "alu", 1020.0
    if cls == "jacobian":
        return "alu", 1035.0
    if cls == "residual":
        return "alu", 130.0
    return None, None


# ---------------------------------------------------------------- ranks

def rank_env():
    """(world, rank, local rank) from the torchrun environment (1, 0, 0 alone)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x, world, device):
    """Largest x over the ranks of the default process group (x alone when world == 1)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, world, device):
    """Sum of x over the ranks (x alone when world == 1)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def shard(items, rank, world):
    """The independent problems a rank solves: every world-th one from rank."""
    return list(items)[rank::world]


# ---------------------------------------------------------------- GPU arm

def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1608_06721_gb300 import swnmg, workloads as W

    world, rank, local = rank_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            dist.barrier()

    p = workload(W.PREC_MIXED_STEP1 if args.step1_fp32 else W.PREC_MIXED, args.nx, args.nx)
    stream = torch.cuda.current_stream()
    S = swnmg.Solver(p, stream=stream)
    U0 = torch.as_tensor(p.U0, dtype=torch.float64, device=dev).contiguous()
    U = torch.empty_like(U0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 256 MB > L2

    def one_solve():
        U.copy_(U0)
        info = S.solve(U)
        if info["status"] != 0:
            raise RuntimeError("solve did not converge: %s" % info)
        return info

    for _ in range(args.warmup):
        one_solve()
    torch.cuda.synchronize()
    S.set_timing(True)
    n0 = swnmg.lib().swnmg_launch_count()
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    total_ms, cycles, infos = 0.0, 0, []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = one_solve()
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        cycles += info["n_vcycles"]
        infos.append(info)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    launches = swnmg.lib().swnmg_launch_count() - n0
    timing = S.get_timing()
    S.set_timing(False)
    total_ms = max_over_ranks(total_ms, world, dev)
    value = world * p.n * cycles / (total_ms * 1e-3)
    ms_per_step = total_ms / args.steps

    # roofline of the dominant kernel class (live CUDA events on the solver's stream)
    dom = max((k for k in timing if timing[k][1] > 0), key=lambda k: timing[k][0])
    bound, per_cell = algorithmic(dom, p, True)
    roof = None
    if bound is not None:
        avg_ms = timing[dom][0] / timing[dom][1]
        units = per_cell * timing[dom][2] / timing[dom][1]    # per launch
        cells_per_launch = timing[dom][2] / timing[dom][1]
        captured = TRAFFIC_PER_CELL[dom] * cells_per_launch if dom in TRAFFIC_PER_CELL else None
        traffic = captured if TRAFFIC_CURRENT else None
        if bound == "hbm":
            pk, src = peaks()
            ach = units / (avg_ms * 1e-3) / 1e9
            roof = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": pk, "unit": "GB/s",
                    "frac": ach / pk, "traffic": traffic, "traffic_previous_build": captured,
                    "peak_source": src, "units_per_launch": units, "avg_launch_ms": avg_ms}
        else:
            ach = units / (avg_ms * 1e-3) / 1e12
            pk = FP64_OPS_PEAK / 1e12
            roof = {"bound": "alu", "kernel": dom, "achieved": ach, "peak": pk,
                    "unit": "TFLOP/s (FP64 ops, no FMA)", "frac": ach / pk, "traffic": traffic,
                    "traffic_previous_build": captured,
                    "peak_source": "derived: 152 SMs x 2 FP64 lanes/clk x 2.07 GHz",
                    "units_per_launch": units, "avg_launch_ms": avg_ms}
    total_dev = sum(v[0] for v in timing.values())
    shares = {k: {"ms": round(v[0], 3), "launches": v[1], "cells": v[2],
                  "share": round(v[0] / total_dev, 4) if total_dev else 0}
              for k, v in timing.items() if v[1] > 0}

    # FP64 path on the same problem
    fp64 = None
    if args.fp64_steps > 0 and rank == 0:
        p64 = workload(W.PREC_FP64, args.nx, args.nx)
        S64 = swnmg.Solver(p64, stream=stream)
        U64 = torch.empty_like(U0)
        U64.copy_(U0)
        S64.solve(U64)   # warm-up
        t64, c64, n64 = 0.0, 0, 0
        for _ in range(args.fp64_steps):
            U64.copy_(U0)
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            i64 = S64.solve(U64)
            e1.record(stream)
            e1.synchronize()
            t64 += e0.elapsed_time(e1)
            c64 += i64["n_vcycles"]
            n64 = i64["n_newton"]
        diff = float((U64 - U).abs().max() / U64.abs().max())
        fp64 = {"ms_per_step": t64 / args.fp64_steps, "cell_cycles_per_s": p.n * c64 / (t64 * 1e-3),
                "n_newton": n64, "status": i64["status"], "max_rel_diff_mixed_vs_fp64": diff}
        S64.close()

    # end to end through the public API with host buffers
    hU0 = torch.empty(U0.shape, dtype=torch.float64, pin_memory=True)
    hU0.copy_(U0.cpu())
    hU = torch.empty_like(hU0).pin_memory()
    e2e_ms, e2e_cycles = 0.0, 0
    for _ in range(max(1, args.e2e_steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        U.copy_(hU0, non_blocking=True)
        info = S.solve(U)
        hU.copy_(U, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms += (time.perf_counter() - t0) * 1e3
        e2e_cycles += info["n_vcycles"]
    e2e_ms = max_over_ranks(e2e_ms, world, dev)
    e2e = {"value": world * p.n * e2e_cycles / (e2e_ms * 1e-3), "unit": UNIT,
           "h2d_bytes_per_step": int(hU0.numel() * 8), "d2h_bytes_per_step": int(hU.numel() * 8),
           "ms_per_step": e2e_ms / max(1, args.e2e_steps)}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32 (FP32 multigrid, FP64 residual/update)",
           "data": "synthetic (seeded Gaussian-bump topography)", "config": config_dict(p, "256 MB flush between steps; working set > L2"),
           "newton_steps": infos[-1]["n_newton"], "cycles_per_solve": infos[-1]["n_vcycles"],
           "step1_blusgs_sweeps": infos[-1]["blusgs_sweeps"], "final_res": infos[-1]["final_res"],
           "fp64": fp64, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
           "roofline": roof, "kernels": shares}
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_sample(args.nx, args.cpu_sample_steps)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------- batched workload

def run_batch(args):
    """--workload batch: 64 independent channel problems of mixed sizes
    (128^2 .. 1024^2, seed 401, mixed precision) solved by one batched
    swnmg_batch_solve per step, autotuned, N_mg cycles replayed from a CUDA
    graph.  value = converged problems per second; beside it cell*cycles/s
    over all problems and, with --sequential, the same problems solved one by
    one through the single-problem API.  Under torchrun the problems are
    dealt to the ranks (every N-th from the rank's index), each rank solving
    its share as one batch on its GPU: no data-path collective, and value =
    all ranks' converged problems / the slowest rank's time."""
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1608_06721_gb300 import swnmg, workloads as W

    world, rank, local = rank_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    all_probs = W.batch_channels(seed=401, count=args.batch_count)
    probs = shard(all_probs, rank, world)
    stream = torch.cuda.current_stream()
    bt = swnmg.BatchSolver(probs, stream=stream)
    U0 = bt.states()
    t0 = time.perf_counter()
    chunks, blocks = bt.tune([u.clone() for u in U0])
    tune_s = time.perf_counter() - t0
    bt.set_graph(True)
    Us = [torch.empty_like(u) for u in U0]

    def one():
        for u, v in zip(Us, U0):
            u.copy_(v)
        return bt.solve(Us)

    for _ in range(args.warmup):
        one()
    torch.cuda.synchronize()
    n0 = swnmg.lib().swnmg_launch_count()
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    total_ms, infos = 0.0, None
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos = one()
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    launches = swnmg.lib().swnmg_launch_count() - n0
    ms = max_over_ranks(total_ms / args.steps, world, dev)
    ok = sum_over_ranks(sum(i["status"] == 0 for i in infos), world, dev)
    cells = sum(p.n for p in all_probs)
    cc = sum_over_ranks(sum(i["n_vcycles"] * p.n for i, p in zip(infos, probs)), world, dev)
    status_names = {0: "ok", 3: "not_converged", 4: "nonfinite", 5: "diverged"}
    by = {}
    for i, p in zip(infos, probs):
        k = status_names.get(i["status"], str(i["status"]))
        by.setdefault(k, []).append(p.nx)
    out = {"metric": "batched steady solves/s (64 seeded channels 128^2..1024^2, mixed precision)",
           "value": ok / (ms * 1e-3), "unit": "converged solves/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "strong",
           "vs_baseline": None, "dtype": "f64+f32 (FP32 multigrid, FP64 residual/update)",
           "data": "synthetic (seeded Gaussian-bump topography)",
           "config": {"workload": "%d channel problems, sizes %s, seed 401, W-cycle, eps_p=2, exact 8x8 coarsest"
                                  % (len(all_probs), sorted(set(p.nx for p in all_probs))),
                      "cells": cells, "parallelism": "problems dealt to %d rank(s)" % world,
                      "l2": "working set %.1f GB > L2" % (cells * 3 * 8 * 12 / 1e9)},
           "cell_cycles_per_s": cc / (ms * 1e-3), "converged": int(ok), "problems": len(all_probs),
           "status_by_size_rank0": {k: sorted(v) for k, v in by.items()},
           "max_newton_steps_rank0": max(i["n_newton"] for i in infos),
           "tuning_rank0": {"sgs_chunk": chunks, "blusgs_blocks": blocks, "seconds": tune_s},
           "gpu_launches": int(launches), "clocks": clk}
    if args.sequential and world == 1:
        tot, cyc, okn = 0.0, 0, 0
        for p in probs:
            S = swnmg.Solver(p, stream=stream)
            U = torch.as_tensor(np.ascontiguousarray(p.U0), dtype=torch.float64, device="cuda").contiguous()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = S.solve(U)
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
            cyc += info["n_vcycles"] * p.n
            okn += info["status"] == 0
            S.close()
        out["sequential_single"] = {"ms": tot, "converged_solves_per_s": okn / (tot * 1e-3),
                                    "cell_cycles_per_s": cyc / (tot * 1e-3), "speedup_batched": tot / ms}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------- CPU oracle

def cpu_sample(nx, nsteps=1):
    """The CPU oracle on a bounded sample of the same workload: nsteps Newton
    steps (BLU-SGS sweep, Jacobian, N_mg cycles, update) from the initial
    state, one host thread."""
    from oracle.oracle import Oracle
    from paper_1608_06721_gb300 import workloads as W
    p = workload(W.PREC_FP64, nx, nx)
    o = Oracle(p, init_mode=W.INIT_NONE, max_newton=nsteps, tol=0.0)
    t0 = time.perf_counter()
    U, info = o.solve()
    dt = time.perf_counter() - t0
    return {"value": p.n * info["n_vcycles"] / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d Newton step(s) of the %dx%d workload from its initial state (Step 2 only), "
                      "FP64 oracle, %.1f s" % (nsteps, nx, nx, dt), "seconds": dt}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    for _ in range(args.warmup):
        cpu_sample(args.nx, 1)
    vals, secs = [], 0.0
    for _ in range(args.steps):
        r = cpu_sample(args.nx, 1)
        vals.append(r["value"])
        secs += r["seconds"]
    value = sum(vals) / len(vals)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded Gaussian-bump topography)",
           "config": {"workload": "2D partial-dry channel %dx%d, one Newton step per step" % (args.nx, args.nx)},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": "one Newton step (Step 2) of the %dx%d workload per step" % (args.nx, args.nx)},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------- profiling cases

def _event_ms(fn):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    fn()
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1)


def run_profile_case(args):
    """Small fixed launch sequences for ncu and CUDA-event timing of single
    kernels (no JSON line).

    sweeps: on the n x n channel (mixed precision, the benchmark's levels
      for n): residual, Jacobian, one symmetric BLU-SGS sweep twice, a level-0
      SGS forward and backward half-sweep twice; every kernel of interest
      launches at least twice, so `-s 1 -c 1` on one kernel name captures a
      warm launch.
    cycle: Jacobian then one multigrid cycle of the benchmark configuration,
      for a launch list of every level's kernels."""
    import torch
    from paper_1608_06721_gb300 import swnmg, workloads as W
    n = args.nx
    p = W.channel_bench(n, n, W.PREC_MIXED)
    S = swnmg.Solver(p)
    U = torch.as_tensor(p.U0, dtype=torch.float64, device="cuda").contiguous()
    if args.profile_case == "sweeps":
        for k in range(2):
            ms = _event_ms(lambda: S.residual(U))
        print("residual %dx%d: %.3f ms" % (n, n, ms))
        for k in range(2):
            ms = _event_ms(lambda: S.jacobian(U))
        print("jacobian (with hierarchy and LU) %dx%d: %.3f ms" % (n, n, ms))
        V = U.clone()
        for k in range(2):
            ms = _event_ms(lambda: S.blusgs(V, 0, 1))
        print("blusgs symmetric sweep %dx%d: %.3f ms" % (n, n, ms))
        S.jacobian(U)
        R, _, _ = S.residual(U)
        x = torch.zeros_like(U)
        for fw in (True, False):
            for k in range(2):
                ms = _event_ms(lambda: S.sgs_sweep(0, -R, x, fw))
            print("sgs half-sweep %s %dx%d: %.3f ms" % ("forward" if fw else "backward", n, n, ms))
    elif args.profile_case == "cycle":
        S.jacobian(U)
        R, _, _ = S.residual(U)
        x = torch.zeros_like(U)
        n0 = swnmg.lib().swnmg_launch_count()
        ms = _event_ms(lambda: S.vcycle(-R, x, 1))
        print("one cycle (gamma=%d, N_L=%d) %dx%d: %.3f ms, %d launches"
              % (p.params.gamma, p.params.n_levels, n, n, ms, swnmg.lib().swnmg_launch_count() - n0))
    else:
        raise SystemExit("unknown profile case " + args.profile_case)
    S.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nx", type=int, default=NX)
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--cpu-sample-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--levels", type=int, default=LEVELS)
    ap.add_argument("--workload", default="channel1024", choices=["channel1024", "batch"])
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--sequential", action="store_true")
    ap.add_argument("--step1-fp32", action="store_true",
                    help="Step 1's coarse-level BLU-SGS in FP32 (precision MIXED_STEP1)")
    ap.add_argument("--profile-case", choices=["sweeps", "cycle"], default=None,
                    help="run a small fixed launch sequence for ncu instead of the benchmark")
    args = ap.parse_args()
    globals()["LEVELS"] = args.levels
    if args.profile_case:
        run_profile_case(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
