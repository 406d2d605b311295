"""Benchmark: Newton multigrid steady solve of the 2D partial-dry channel.

Workload: 1024 x 1024 cells on [0,4] x [0,1], 16 seeded Gaussian bumps with
dry tops, inflow discharge hu ~ U[0.5, 1.5] at x = 0, outflow depth 0.6 at
x = 4, reflective walls, LLF flux with the wet/dry speed increase; mixed
precision (FP32 multigrid inner solve, FP64 residual / Jacobian / update /
norms), W-cycles (gamma = 2, N_L = 7 with an exact solve on the 8 x 8
coarsest level, N_mg = 3), eps_p = 2, tol 1e-10.

One step = one complete swnmg_solve (Algorithm 1 including its Step 1) from
the same initial state, with inputs resident in HBM.  value = cells x
multigrid cycles / second over the timed steps (no per-launch
instrumentation inside them); ms_per_step = time to sum ||R_i||_1 < 1e-10.
One instrumented solve after the timed steps gives each kernel class's
device time (CUDA events around its launches) for the roofline entries.
The FP64 path is timed on the same problem and reported beside it.  e2e
repeats the mixed solve through host buffers (pinned H2D of the initial
state, D2H of the steady state inside the timed region), three samples.
The variants (FP32 Step 1, two-colour smoother) and the like-for-like line
(the oracle's and the GPU's full solve of the 256^2 channel) are reported
beside the headline.  Multi-GPU: independent replicas (the lexicographic
sweeps do not shard), weak scaling.

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


# Algorithmic work and measured DRAM traffic per cell of one launch of each
# kernel class, from ncu captures on the 512 x 512 channel (profiles/); a
# launch's work grows with the cells it processes, so both are scaled to the
# timed launches by their cell counts.
# FP64_PER_CELL: FP64 lane instructions (dadd + dmul + dfma, predicated on)
# of an implementation that evaluates every edge once and shares each
# reciprocal (the two-pass residual and Jacobian, the BLU-SGS cell update of
# 16 lanes), including the instruction sequences of the correctly rounded
# divisions and square roots: the method's work as the GPU executes it,
# compared against the measured FP64 lane instruction rate (swnmg_fp64_rate).
# The fused tile kernels evaluate a tile's border edges twice (+8 %) and the
# two-warp BLU-SGS kernel forms the cell's half of a new-side edge term in one
# warp and the combination in the other; that extra work is not counted.
# The SGS classes are HBM-bound kernels whose algorithmic bytes per cell come
# from the operator layout (below).
# TRAFFIC_PER_CELL: dram__bytes_read.sum + dram__bytes_write.sum of the
# current kernels (k_res_tile, k_jac_tile, k_blusgs_ws, k_sgs_ws); at
# 512 x 512 their outputs stay in the 126 MB L2, so the writes are not seen.
# The BLU-SGS figure includes the tagged words the strips hand on (48 bytes
# per column of a two-row strip, written and read back).
FP64_PER_CELL = {"residual": 181.1, "jacobian": 1380.5, "blusgs": 1485.8, "blusgs_coarse": 1485.8}
TRAFFIC_PER_CELL = {"residual": 32.3, "jacobian": 76.3, "blusgs": 62.1, "blusgs_coarse": 62.1,
                    "sgs_fine": 218.5, "sgs_coarse": 218.5}
# the kernels of these classes are unchanged since the captures above
TRAFFIC_CURRENT = {"residual", "jacobian", "blusgs", "blusgs_coarse", "sgs_fine", "sgs_coarse"}


def algorithmic(cls, p, fp32):
    """(bound, algorithmic units per cell) of a kernel class: bytes of the
    operator blocks, LU factors, pivot code, b, and x read and written for
    the block-SGS smoother; counted FP64 lane instructions for the flux
    kernels."""
    nc = p.ncomp
    w = 4 if fp32 else 8
    if cls in ("sgs_fine", "sgs_coarse"):
        return "hbm", (5 * nc * nc - nc * nc + 9 + 3 + 2 * nc) * w + 1   # blocks, LU, b, x in/out, piv
    if cls in FP64_PER_CELL:
        return "alu", FP64_PER_CELL[cls]
    return None, None


def roofline_entry(cls, timing, p, fp32, fp64_peak, hbm_peak, hbm_src):
    """achieved / peak of one kernel class from its CUDA-event totals."""
    ms, launches, cells = timing[cls]
    if launches <= 0:
        return None
    bound, per_cell = algorithmic(cls, p, fp32)
    if bound is None:
        return None
    avg_ms = ms / launches
    cells_per_launch = cells / launches
    units = per_cell * cells_per_launch
    captured = TRAFFIC_PER_CELL[cls] * cells_per_launch if cls in TRAFFIC_PER_CELL else None
    traffic = captured if cls in TRAFFIC_CURRENT else None
    if bound == "hbm":
        ach = units / (avg_ms * 1e-3) / 1e9
        return {"bound": "hbm", "kernel": cls, "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                "frac": ach / hbm_peak, "traffic": traffic, "peak_source": hbm_src + ", of measured",
                "units_per_launch": units, "avg_launch_ms": avg_ms}
    ach = units / (avg_ms * 1e-3) / 1e12
    pk = fp64_peak / 1e12
    return {"bound": "alu", "kernel": cls, "achieved": ach, "peak": pk,
            "unit": "T FP64 lane instructions/s", "frac": ach / pk, "traffic": traffic,
            "peak_source": "measured by swnmg_fp64_rate (chains of adds on every SM)",
            "units_per_launch": units, "avg_launch_ms": avg_ms}


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

    def one_solve(solver, out):
        out.copy_(U0)
        info = solver.solve(out)
        if info["status"] != 0:
            raise RuntimeError("solve did not converge: %s" % info)
        return info

    def timed(solver, out, k):
        """k solves from U0 (each after an L2 flush), device ms from CUDA
        events on the solver's stream."""
        t, infos = 0.0, []
        for _ in range(k):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            infos.append(one_solve(solver, out))
            e1.record(stream)
            e1.synchronize()
            t += e0.elapsed_time(e1)
        return t, infos

    for _ in range(args.warmup):
        one_solve(S, U)
    torch.cuda.synchronize()
    # timed region: no per-launch instrumentation
    n0 = swnmg.lib().swnmg_launch_count()
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    total_ms, infos = timed(S, U, args.steps)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    launches = swnmg.lib().swnmg_launch_count() - n0
    cycles = sum(i["n_vcycles"] for i in infos)
    total_ms = max_over_ranks(total_ms, world, dev)
    value = world * p.n * cycles / (total_ms * 1e-3)
    ms_per_step = total_ms / args.steps

    # per-kernel-class device time from one instrumented solve of the same
    # workload after the timed steps (CUDA events around every launch)
    hbm_peak, hbm_src = peaks()
    fp64_peak = swnmg.fp64_rate(1)
    S.set_timing(True)
    one_solve(S, U)
    timing = S.get_timing()
    S.set_timing(False)
    dom = max((k for k in timing if timing[k][1] > 0), key=lambda k: timing[k][0])
    roof = roofline_entry(dom, timing, p, True, fp64_peak, hbm_peak, hbm_src)
    kernel_roofs = {k: roofline_entry(k, timing, p, True, fp64_peak, hbm_peak, hbm_src)
                    for k in ("residual", "jacobian", "sgs_fine", "sgs_coarse", "blusgs", "blusgs_coarse")}
    total_dev = sum(v[0] for v in timing.values())
    shares = {k: {"ms": round(v[0], 3), "launches": v[1], "cells": v[2],
                  "share": round(v[0] / total_dev, 4) if total_dev else 0}
              for k, v in timing.items() if v[1] > 0}

    # FP64 path on the same problem
    fp64 = None
    if args.fp64_steps > 0 and rank == 0:
        S64 = swnmg.Solver(workload(W.PREC_FP64, args.nx, args.nx), stream=stream)
        U64 = torch.empty_like(U0)
        one_solve(S64, U64)   # warm-up
        t64, i64 = timed(S64, U64, args.fp64_steps)
        c64 = sum(i["n_vcycles"] for i in i64)
        diff = float((U64 - U).abs().max() / U64.abs().max())
        fp64 = {"ms_per_step": t64 / args.fp64_steps, "cell_cycles_per_s": p.n * c64 / (t64 * 1e-3),
                "n_newton": i64[-1]["n_newton"], "status": i64[-1]["status"], "max_rel_diff_mixed_vs_fp64": diff}
        S64.close()

    # end to end through the public API with host buffers
    hU0 = torch.empty(U0.shape, dtype=torch.float64, pin_memory=True)
    hU0.copy_(U0.cpu())
    hU = torch.empty_like(hU0).pin_memory()
    e2e_ms, e2e_cycles, e2e_samples = 0.0, 0, []
    for _ in range(max(1, args.e2e_steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        U.copy_(hU0, non_blocking=True)
        info = S.solve(U)
        hU.copy_(U, non_blocking=True)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) * 1e3
        e2e_samples.append(round(dt, 2))
        e2e_ms += dt
        e2e_cycles += info["n_vcycles"]
    e2e_ms = max_over_ranks(e2e_ms, world, dev)
    e2e = {"value": world * p.n * e2e_cycles / (e2e_ms * 1e-3), "unit": UNIT,
           "h2d_bytes_per_step": int(hU0.numel() * 8), "d2h_bytes_per_step": int(hU.numel() * 8),
           "ms_per_step": e2e_ms / max(1, args.e2e_steps), "samples_ms": e2e_samples}

    variants = run_variants(args, p, U0, U, stream, timed, one_solve, fp64_peak, hbm_peak, hbm_src) \
        if rank == 0 and args.variants else None

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32 (FP32 multigrid, FP64 residual/update)",
           "data": "synthetic (seeded Gaussian-bump topography)",
           "config": config_dict(p, "256 MB flush between steps; working set > L2"),
           "newton_steps": infos[-1]["n_newton"], "cycles_per_solve": infos[-1]["n_vcycles"],
           "step1_blusgs_sweeps": infos[-1]["blusgs_sweeps"], "final_res": infos[-1]["final_res"],
           "fp64": fp64, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
           "roofline": roof, "kernel_rooflines": kernel_roofs, "fp64_peak_lane_inst_per_s": fp64_peak,
           "kernels": shares, "kernel_timing": "one instrumented solve after the timed steps",
           "variants": variants}
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_sample(args.nx, args.cpu_sample_steps)
        if args.like_for_like:
            out["like_for_like"] = like_for_like(args, stream)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_variants(args, p, U0, U, stream, timed, one_solve, fp64_peak, hbm_peak, hbm_src):
    """Separately reported variants on the same problem, one solve each
    after a warm-up: Step 1's coarse-level BLU-SGS in FP32, and the
    two-colour block SGS smoother (its level-0 half-sweep roofline from one
    instrumented solve)."""
    import torch
    from paper_1608_06721_gb300 import swnmg, workloads as W
    out = {}
    Uv = torch.empty_like(U0)
    S1 = swnmg.Solver(workload(W.PREC_MIXED_STEP1, args.nx, args.nx), stream=stream)
    one_solve(S1, Uv)
    t, inf = timed(S1, Uv, 1)
    out["step1_fp32"] = {"ms_per_step": t, "cell_cycles_per_s": p.n * inf[0]["n_vcycles"] / (t * 1e-3),
                         "n_newton": inf[0]["n_newton"], "step1_blusgs_sweeps": inf[0]["blusgs_sweeps"],
                         "max_rel_diff_vs_mixed": float((Uv - U).abs().max() / U.abs().max()),
                         "precision": "Step 1 coarse-level BLU-SGS in FP32 (FD step 2^-12), else as mixed"}
    S1.close()
    pc = workload(W.PREC_MIXED, args.nx, args.nx).with_params(smoother=W.SMOOTH_COLOUR)
    S2 = swnmg.Solver(pc, stream=stream)
    one_solve(S2, Uv)
    t, inf = timed(S2, Uv, 1)
    S2.set_timing(True)
    one_solve(S2, Uv)
    tm = S2.get_timing()
    S2.set_timing(False)
    out["colour_smoother"] = {
        "ms_per_step": t, "cell_cycles_per_s": p.n * inf[0]["n_vcycles"] / (t * 1e-3),
        "n_newton": inf[0]["n_newton"], "cycles_per_solve": inf[0]["n_vcycles"],
        "max_rel_diff_vs_mixed": float((Uv - U).abs().max() / U.abs().max()),
        "sgs_fine_roofline": roofline_entry("sgs_fine", tm, pc, True, fp64_peak, hbm_peak, hbm_src),
        "sgs_coarse_ms": round(tm["sgs_coarse"][0], 3), "sgs_fine_ms": round(tm["sgs_fine"][0], 3),
        "smoother": "two colours (ix + iy) mod 2; not the paper's lexicographic order"}
    out["colour_smoother"]["sgs_fine_roofline"]["traffic"] = None   # not captured by ncu
    S2.close()
    return out


def like_for_like(args, stream):
    """The same solve on both sides: the CPU oracle's time to sum ||R_i||_1 <
    1e-10 on the 256^2 channel (benchmark parameters, one core) beside the
    GPU's, FP64 and mixed."""
    import numpy as np
    import torch
    from oracle.oracle import Oracle
    from paper_1608_06721_gb300 import swnmg, workloads as W
    n = 256
    p = W.channel_bench(n, n, W.PREC_FP64)
    t0 = time.perf_counter()
    Uo, io = Oracle(p).solve()
    cpu_s = time.perf_counter() - t0
    out = {"workload": "2D partial-dry channel 256x256 (W-cycle, N_L = 5, exact coarsest, seed 301)",
           "cpu_oracle_s": cpu_s, "cpu_cores": 1, "cpu_newton": io["n_newton"]}
    for prec, key in ((W.PREC_FP64, "gpu_fp64_s"), (W.PREC_MIXED, "gpu_mixed_s")):
        S = swnmg.Solver(p.with_params(precision=prec), stream=stream)
        U0 = torch.as_tensor(p.U0, dtype=torch.float64, device="cuda").contiguous()
        U = U0.clone()
        S.solve(U)   # warm-up
        U.copy_(U0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = S.solve(U)
        e1.record(stream)
        e1.synchronize()
        out[key] = e0.elapsed_time(e1) * 1e-3
        out[key.replace("_s", "_newton")] = info["n_newton"]
        out[key.replace("_s", "_max_rel_diff_vs_oracle")] = float(np.abs(U.cpu().numpy() - Uo).max() / np.abs(Uo).max())
        S.close()
    out["speedup_fp64"] = cpu_s / out["gpu_fp64_s"]
    out["speedup_mixed"] = cpu_s / out["gpu_mixed_s"]
    return out


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
    if args.eps_p_rule:   # the paper's rule: 1 % of each problem's initial residual
        all_probs = [p.with_params(eps_p=-0.01) for p in all_probs]
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
           "config": {"workload": "%d channel problems, sizes %s, seed 401, W-cycle, eps_p=%s, exact 8x8 coarsest"
                                  % (len(all_probs), sorted(set(p.nx for p in all_probs)),
                                     "1 % of the initial residual" if args.eps_p_rule else "2"),
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
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-variants", dest="variants", action="store_false",
                    help="skip the FP32 Step 1 and two-colour smoother variant lines")
    ap.add_argument("--no-like-for-like", dest="like_for_like", action="store_false",
                    help="skip the oracle-vs-GPU full solve on the 256^2 channel")
    ap.add_argument("--cpu-sample-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--levels", type=int, default=LEVELS)
    ap.add_argument("--workload", default="channel1024", choices=["channel1024", "batch"])
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--sequential", action="store_true")
    ap.add_argument("--eps-p-rule", action="store_true",
                    help="batch: Step 1's eps_p by the paper's rule (1 %% of each problem's initial residual)")
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
