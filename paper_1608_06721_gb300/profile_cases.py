"""Small fixed cases for profiling single kernels of the library (ncu, CUDA
events).  Usage:

    python -m paper_1608_06721_gb300.profile_cases sweeps N

builds the NxN partial-dry channel (W-cycle, eps_p = 2, N_L = 6, mixed
precision), then runs: one symmetric BLU-SGS sweep (warm-up), one timed
symmetric BLU-SGS sweep, a Jacobian, one SGS half-sweep (warm-up) and one
timed SGS half-sweep, printing the two CUDA-event timings.
"""
import sys

import torch

from . import swnmg, workloads as W


def sweeps(n: int):
    p = W.channel_2d(nx=n, ny=n, precision=W.PREC_MIXED).with_params(gamma=2, eps_p=2.0, n_levels=6)
    S = swnmg.Solver(p)
    U = torch.as_tensor(p.U0, dtype=torch.float64, device="cuda").contiguous()
    S.blusgs(U, 0, 1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    S.blusgs(U, 0, 1)
    e1.record()
    e1.synchronize()
    print("blusgs symmetric sweep %dx%d: %.3f ms" % (n, n, e0.elapsed_time(e1)))
    R = torch.zeros_like(U)
    x = torch.zeros_like(U)
    S.jacobian(U)
    S.sgs_sweep(0, R, x, True)
    e0.record()
    S.sgs_sweep(0, R, x, True)
    e1.record()
    e1.synchronize()
    print("sgs half-sweep %dx%d: %.3f ms" % (n, n, e0.elapsed_time(e1)))


if __name__ == "__main__":
    what = sys.argv[1] if len(sys.argv) > 1 else "sweeps"
    n = int(sys.argv[2]) if len(sys.argv) > 2 else 256
    if what == "sweeps":
        sweeps(n)
    else:
        raise SystemExit("unknown case " + what)
