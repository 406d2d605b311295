"""Python binding of libswnmg (include/swnmg.h): argument marshalling only.

Every step of the method runs in the CUDA library; PyTorch only provides the
device tensors and the stream.  There is no CPU fallback: if the library or a
CUDA device is missing, the constructor raises.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os

import numpy as np
import torch

from . import workloads as W
from .build import build

HIST = 512

OK, ERR_ARG, ERR_CUDA, ERR_NOT_CONVERGED, ERR_NONFINITE, ERR_DIVERGED, ERR_TIMEOUT, ERR_OOM = range(8)
STATUS = {0: "ok", 1: "arg", 2: "cuda", 3: "not_converged", 4: "nonfinite", 5: "diverged",
          6: "timeout", 7: "oom"}


class _BC(C.Structure):
    _fields_ = [("kind", C.c_int32), ("h", C.c_double), ("q", C.c_double), ("ut", C.c_double)]


class Problem(C.Structure):
    _fields_ = [("dim", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32),
                ("x0", C.c_double), ("x1", C.c_double), ("y0", C.c_double), ("y1", C.c_double),
                ("g", C.c_double), ("bc", _BC * 4)]


class Params(C.Structure):
    _fields_ = [("flux", C.c_int32), ("llf_wetdry", C.c_int32),
                ("alpha", C.c_double), ("fd_eps", C.c_double), ("tau", C.c_double),
                ("h_eps", C.c_double), ("eps_r", C.c_double), ("eps_p", C.c_double),
                ("tol", C.c_double),
                ("n_levels", C.c_int32), ("n_mg", C.c_int32), ("nu1", C.c_int32), ("nu2", C.c_int32),
                ("gamma", C.c_int32), ("coarse_sweeps", C.c_int32), ("max_newton", C.c_int32),
                ("max_blusgs", C.c_int32), ("init_mode", C.c_int32), ("precision", C.c_int32),
                ("eps_f", C.c_double), ("smoother", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("status", C.c_int32), ("n_newton", C.c_int32), ("n_vcycles", C.c_int32),
                ("blusgs_sweeps", C.c_int32 * 16), ("init_res", C.c_double),
                ("final_res", C.c_double), ("res_hist", C.c_double * HIST),
                ("ms_step1", C.c_double), ("ms_newton", C.c_double)]


_lib = None


def lib():
    """Loads (building first if needed) the in-tree CUDA library."""
    global _lib
    if _lib is None:
        path = build()
        if not os.path.exists(path):
            raise RuntimeError("libswnmg.so is missing: run __graft_entry__.build()")
        L = C.CDLL(path)
        vp, dp = C.c_void_p, C.POINTER(C.c_double)
        L.swnmg_default_params.argtypes = [C.c_int32, C.POINTER(Params)]
        L.swnmg_create.argtypes = [C.POINTER(Problem), C.POINTER(Params), vp, vp, C.POINTER(vp)]
        L.swnmg_destroy.argtypes = [vp]
        L.swnmg_last_error.argtypes = [vp]
        L.swnmg_last_error.restype = C.c_char_p
        L.swnmg_set_params.argtypes = [vp, C.POINTER(Params)]
        L.swnmg_set_mesh.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.swnmg_residual.argtypes = [vp, vp, vp, vp, dp]
        L.swnmg_jacobian.argtypes = [vp, vp]
        L.swnmg_get_blocks.argtypes = [vp, C.c_int32, vp]
        L.swnmg_vcycle.argtypes = [vp, vp, vp, C.c_int32]
        L.swnmg_sgs_sweep.argtypes = [vp, C.c_int32, vp, vp, C.c_int32]
        L.swnmg_blusgs.argtypes = [vp, vp, C.c_int32, C.c_int32]
        L.swnmg_solve.argtypes = [vp, vp, C.POINTER(Stats)]
        L.swnmg_set_timing.argtypes = [vp, C.c_int32]
        L.swnmg_get_timing.argtypes = [vp, dp, C.POINTER(C.c_int64), dp]
        L.swnmg_residual_noalloc.argtypes = [C.POINTER(Problem), C.POINTER(Params), vp, vp, vp, vp, vp, vp]
        L.swnmg_residual_noalloc.restype = C.c_int
        L.swnmg_adjoint.argtypes = [vp, vp, vp, vp, vp, dp, C.c_int32, C.c_double, C.POINTER(C.c_int32)]
        L.swnmg_time_step.argtypes = [vp, vp, C.c_double, C.c_double, C.POINTER(Stats)]
        L.swnmg_level_cells.argtypes = [vp, C.c_int32]
        L.swnmg_batch_create.argtypes = [C.POINTER(Problem), C.POINTER(C.c_int32), C.c_int32, C.POINTER(Params),
                                         C.POINTER(vp), vp, C.POINTER(vp)]
        L.swnmg_batch_destroy.argtypes = [vp]
        L.swnmg_batch_last_error.argtypes = [vp]
        L.swnmg_batch_last_error.restype = C.c_char_p
        L.swnmg_batch_solve.argtypes = [vp, C.POINTER(vp), C.POINTER(Stats)]
        L.swnmg_batch_set_graph.argtypes = [vp, C.c_int32]
        L.swnmg_batch_tune.argtypes = [vp, C.POINTER(vp), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
        L.swnmg_batch_set_tuning.argtypes = [vp, C.POINTER(C.c_int32), C.c_int32]
        L.swnmg_level_cells.restype = C.c_int64
        L.swnmg_set_wait_limit.argtypes = [C.c_int32]
        L.swnmg_fp64_rate.argtypes = [C.c_int32, C.POINTER(C.c_double)]
        L.swnmg_fp64_rate.restype = C.c_int
        L.swnmg_set_wait_limit.restype = C.c_int32
        for f in ("swnmg_default_params", "swnmg_create", "swnmg_destroy", "swnmg_set_params",
                  "swnmg_residual", "swnmg_jacobian", "swnmg_get_blocks", "swnmg_vcycle",
                  "swnmg_sgs_sweep", "swnmg_blusgs", "swnmg_solve", "swnmg_set_timing",
                  "swnmg_get_timing", "swnmg_adjoint", "swnmg_time_step", "swnmg_batch_create",
                  "swnmg_batch_destroy",
                  "swnmg_batch_solve", "swnmg_batch_set_graph", "swnmg_batch_tune", "swnmg_batch_set_tuning"):
            getattr(L, f).restype = C.c_int
        _lib = L
    return _lib


KERNEL_CLASSES = ["residual", "jacobian", "galerkin_lu", "sgs_fine", "sgs_coarse", "transfer",
                  "blusgs", "update", "coarse_exact", "blusgs_coarse"]


class SwnmgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("swnmg status %d (%s): %s" % (status, STATUS.get(status, "?"), msg))
        self.status = status


def make_problem(p: W.Problem, allow_mesh: bool = False) -> Problem:
    """The C struct of a problem.  A curvilinear problem's vertices go to the
    library separately (swnmg_set_mesh, single problems only): without
    allow_mesh such a problem is refused."""
    if getattr(p, "mesh_x", None) is not None and not allow_mesh:
        raise NotImplementedError("batches solve on uniform Cartesian meshes only; "
                                  "problem %r has a curvilinear mesh" % p.name)
    s = Problem()
    s.dim, s.nx, s.ny = p.dim, p.nx, (p.ny if p.dim == 2 else 1)
    s.x0, s.x1, s.y0, s.y1, s.g = p.x0, p.x1, p.y0, p.y1, p.g
    for k in range(4):
        b = p.bc[k]
        s.bc[k].kind, s.bc[k].h, s.bc[k].q, s.bc[k].ut = b.kind, b.h, b.q, b.ut
    return s


def make_params(prm: W.Params) -> Params:
    s = Params()
    for f, _ in Params._fields_:
        setattr(s, f, getattr(prm, f))
    return s


def _ptr(t: torch.Tensor):
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return C.c_void_p(t.data_ptr())


class Solver:
    """One problem on the current CUDA device; tensors are float64 SoA."""

    def __init__(self, prob: W.Problem, params: W.Params | None = None, stream=None, z=None):
        if not torch.cuda.is_available():
            raise RuntimeError("swnmg needs a CUDA device (no CPU fallback)")
        self.L = lib()
        self.prob = prob
        self.params = params or prob.params
        self.nc = prob.ncomp
        self.stream = stream or torch.cuda.current_stream()
        self.z = z if z is not None else torch.as_tensor(np.ascontiguousarray(prob.z), dtype=torch.float64,
                                                         device="cuda")
        self._pp = make_problem(prob, allow_mesh=True)
        self._pr = make_params(self.params)
        h = C.c_void_p()
        rc = self.L.swnmg_create(C.byref(self._pp), C.byref(self._pr), _ptr(self.z),
                                 C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if rc != OK:
            raise SwnmgError(rc, self.L.swnmg_last_error(None).decode())
        self.h = h
        if getattr(prob, "mesh_x", None) is not None:   # structured curvilinear mesh
            mx = np.ascontiguousarray(prob.mesh_x, dtype=np.float64)
            my = np.ascontiguousarray(prob.mesh_y, dtype=np.float64)
            if mx.shape != (prob.ny + 1, prob.nx + 1) or my.shape != mx.shape:
                self.close()
                raise ValueError("mesh vertices must be (ny + 1, nx + 1) arrays")
            P = C.POINTER(C.c_double)
            self._check(self.L.swnmg_set_mesh(self.h, mx.ctypes.data_as(P), my.ctypes.data_as(P)))

    def _check(self, rc):
        if rc != OK:
            raise SwnmgError(rc, self.L.swnmg_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.L.swnmg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, **kw):
        self.params = self.params.replace(**kw)
        self._pr = make_params(self.params)
        self._check(self.L.swnmg_set_params(self.h, C.byref(self._pr)))

    def level_cells(self, level):
        return int(self.L.swnmg_level_cells(self.h, level))

    def tensor(self, a=None, level=0):
        n = self.level_cells(level)
        if a is None:
            return torch.zeros((self.nc, n), dtype=torch.float64, device="cuda")
        return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda").reshape(self.nc, n).contiguous()

    def residual(self, U, with_sum=True):
        n = self.level_cells(0)
        R = torch.empty((self.nc, n), dtype=torch.float64, device="cuda")
        rn = torch.empty(n, dtype=torch.float64, device="cuda")
        s = C.c_double(0.0)
        self._check(self.L.swnmg_residual(self.h, _ptr(U), _ptr(R), _ptr(rn),
                                          C.byref(s) if with_sum else None))
        return R, rn, s.value

    def jacobian(self, U):
        self._check(self.L.swnmg_jacobian(self.h, _ptr(U)))

    def get_blocks(self, level=0):
        n = self.level_cells(level)
        out = np.zeros((n, 5, self.nc, self.nc))
        self._check(self.L.swnmg_get_blocks(self.h, level, out.ctypes.data_as(C.c_void_p)))
        return out

    def vcycle(self, rhs, dU, ncycles=1):
        self._check(self.L.swnmg_vcycle(self.h, _ptr(rhs), _ptr(dU), ncycles))
        return dU

    def sgs_sweep(self, level, rhs, x, forward=True):
        self._check(self.L.swnmg_sgs_sweep(self.h, level, _ptr(rhs), _ptr(x), 1 if forward else 0))
        return x

    def blusgs(self, U, level=0, nsweeps=1):
        self._check(self.L.swnmg_blusgs(self.h, _ptr(U), level, nsweeps))
        return U

    def set_timing(self, enable=True):
        self._check(self.L.swnmg_set_timing(self.h, 1 if enable else 0))

    def get_timing(self):
        """{class: (device ms, launches, cells processed)} since set_timing(True)."""
        k = len(KERNEL_CLASSES)
        ms = (C.c_double * k)()
        nl = (C.c_int64 * k)()
        cells = (C.c_double * k)()
        self._check(self.L.swnmg_get_timing(self.h, ms, nl, cells))
        return {name: (ms[i], nl[i], cells[i]) for i, name in enumerate(KERNEL_CLASSES)}

    def solve(self, U, check=False):
        """Algorithm 1 in place on U; returns a dict of the solver counters."""
        st = Stats()
        rc = self.L.swnmg_solve(self.h, _ptr(U), C.byref(st))
        if check:
            self._check(rc)
        elif rc not in (OK, ERR_NOT_CONVERGED, ERR_NONFINITE, ERR_DIVERGED):
            self._check(rc)
        return {"status": st.status, "n_newton": st.n_newton, "n_vcycles": st.n_vcycles,
                "blusgs_sweeps": list(st.blusgs_sweeps)[:self.params.n_levels + 1],
                "init_res": st.init_res, "final_res": st.final_res,
                "res_hist": list(st.res_hist)[:min(st.n_newton, HIST)],
                "ms_step1": st.ms_step1, "ms_newton": st.ms_newton}

    def time_step(self, U, dt, beta=0.0, check=False):
        """Remark 2.6: U (U^n) becomes U^{n+1} in place; returns the counters."""
        st = Stats()
        rc = self.L.swnmg_time_step(self.h, _ptr(U), float(dt), float(beta), C.byref(st))
        if check:
            self._check(rc)
        elif rc not in (OK, ERR_NOT_CONVERGED, ERR_NONFINITE, ERR_DIVERGED):
            self._check(rc)
        return _stats_dict(st, self.params.n_levels)

    def adjoint(self, U, g, max_cycles=100, rtol=1e-12, check=True):
        """swnmg_adjoint: lambda with J(U)^T lambda = g by multigrid cycles on the
        transposed hierarchy, gz = -lambda^T dR/dz (n) and gq = -lambda^T
        dR/dq (4 sides), the loss gradient's parts through U*.
        Returns (lam, gz, gq, cycles)."""
        n = self.level_cells(0)
        lam = torch.empty((self.nc, n), dtype=torch.float64, device="cuda")
        gz = torch.empty(n, dtype=torch.float64, device="cuda")
        gq = (C.c_double * 4)()
        cyc = C.c_int32(0)
        rc = self.L.swnmg_adjoint(self.h, _ptr(U), _ptr(g), _ptr(lam), _ptr(gz), gq, max_cycles,
                                  rtol, C.byref(cyc))
        if check or rc != ERR_NOT_CONVERGED:
            self._check(rc)
        return lam, gz, np.array(list(gq)), cyc.value


def _stats_dict(st, n_levels):
    return {"status": st.status, "n_newton": st.n_newton, "n_vcycles": st.n_vcycles,
            "blusgs_sweeps": list(st.blusgs_sweeps)[:n_levels + 1],
            "init_res": st.init_res, "final_res": st.final_res,
            "res_hist": list(st.res_hist)[:min(st.n_newton, HIST)],
            "ms_step1": st.ms_step1, "ms_newton": st.ms_newton}


class BatchSolver:
    """Many independent 2D problems solved together (swnmg_batch_*).  Each
    problem keeps its own grid, bed, boundary data and number of levels
    (prob.params.n_levels); the other parameters are shared (``params``,
    default the first problem's)."""

    SGS_LEVELS = 13

    def __init__(self, probs, params: W.Params | None = None, stream=None):
        if not torch.cuda.is_available():
            raise RuntimeError("swnmg needs a CUDA device (no CPU fallback)")
        self.L = lib()
        self.probs = list(probs)
        self.B = len(self.probs)
        self.params = params or self.probs[0].params
        self.stream = stream or torch.cuda.current_stream()
        self.z = [torch.as_tensor(np.ascontiguousarray(p.z), dtype=torch.float64, device="cuda")
                  for p in self.probs]
        arr = (Problem * self.B)(*[make_problem(p) for p in self.probs])
        nl = (C.c_int32 * self.B)(*[p.params.n_levels for p in self.probs])
        zp = (C.c_void_p * self.B)(*[t.data_ptr() for t in self.z])
        self._pr = make_params(self.params)
        h = C.c_void_p()
        rc = self.L.swnmg_batch_create(arr, nl, self.B, C.byref(self._pr), zp, C.c_void_p(self.stream.cuda_stream),
                                       C.byref(h))
        if rc != OK:
            raise SwnmgError(rc, self.L.swnmg_batch_last_error(None).decode())
        self.h = h

    def _check(self, rc):
        if rc != OK:
            raise SwnmgError(rc, self.L.swnmg_batch_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.L.swnmg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def states(self):
        """Initial states of the problems as float64 CUDA tensors (3, n)."""
        return [torch.as_tensor(np.ascontiguousarray(p.U0), dtype=torch.float64, device="cuda").contiguous()
                for p in self.probs]

    def _ptrs(self, Us):
        if len(Us) != self.B:
            raise ValueError("expected %d states" % self.B)
        return (C.c_void_p * self.B)(*[_ptr(u).value for u in Us])

    def solve(self, Us, check=False):
        """Algorithm 1 on every problem in place; returns one counters dict each."""
        st = (Stats * self.B)()
        rc = self.L.swnmg_batch_solve(self.h, self._ptrs(Us), st)
        if check:
            self._check(rc)
        elif rc not in (OK, ERR_NOT_CONVERGED, ERR_NONFINITE, ERR_DIVERGED):
            self._check(rc)
        return [_stats_dict(st[p], self.probs[p].params.n_levels) for p in range(self.B)]

    def set_graph(self, enable=True):
        self._check(self.L.swnmg_batch_set_graph(self.h, 1 if enable else 0))

    def tune(self, Us):
        """Autotuner; returns (SGS chunk per level, BLU-SGS grid blocks per level)."""
        ch = (C.c_int32 * self.SGS_LEVELS)()
        nb = (C.c_int32 * self.SGS_LEVELS)()
        self._check(self.L.swnmg_batch_tune(self.h, self._ptrs(Us), ch, nb))
        return list(ch), list(nb)

    def set_tuning(self, chunks=None, blusgs_blocks=0):
        ch = (C.c_int32 * self.SGS_LEVELS)(*chunks) if chunks is not None else None
        self._check(self.L.swnmg_batch_set_tuning(self.h, ch, blusgs_blocks))


def with_discharge(prob: W.Problem, q) -> W.Problem:
    """prob with the prescribed discharge of side s replaced by q[s]."""
    bc = [dataclasses.replace(b, q=float(q[k])) for k, b in enumerate(prob.bc)]
    return dataclasses.replace(prob, bc=bc)


class SteadySWE(torch.autograd.Function):
    """U* = NMGM(z, q): Algorithm 1 run to its tolerance, with the discrete
    adjoint (swnmg_adjoint) as the backward pass:
        grad_z = -lambda^T dR/dz,  grad_q = -lambda^T dR/dq,  J^T lambda = grad_U.
    z: (n,) float64 CUDA bed; q: (4,) float64 discharge per side (only
    inflow-discharge sides carry a gradient); U0: initial state (ncomp, n)
    for the solve.  The loss's own dependence on z (e.g. through h + z) is
    added by autograd outside this function."""

    @staticmethod
    def forward(ctx, z, q, prob, params, U0, adj_cycles, adj_rtol):
        qh = q.detach().cpu().numpy()
        solver = Solver(with_discharge(prob, qh), params, z=z.detach().contiguous())
        U = U0.detach().clone().contiguous()
        solver.solve(U, check=True)
        ctx.solver = solver
        ctx.adj = (adj_cycles, adj_rtol)
        ctx.q_meta = (q.device, q.dtype)
        ctx.save_for_backward(U)
        return U

    @staticmethod
    def backward(ctx, gU):
        (U,) = ctx.saved_tensors
        _, gz, gq, _ = ctx.solver.adjoint(U, gU.contiguous(), ctx.adj[0], ctx.adj[1])
        gq = torch.as_tensor(gq, dtype=ctx.q_meta[1], device=ctx.q_meta[0])
        return gz, gq, None, None, None, None, None


def steady_state(z, q, prob: W.Problem, params: W.Params | None = None, U0=None, adj_cycles=400,
                 adj_rtol=1e-10):
    """Differentiable steady state: SteadySWE.apply with defaults."""
    params = params or prob.params
    if U0 is None:
        U0 = torch.as_tensor(np.ascontiguousarray(prob.U0), dtype=torch.float64, device="cuda")
    return SteadySWE.apply(z, q, prob, params, U0, adj_cycles, adj_rtol)


def residual_noalloc(prob: W.Problem, z, U, R, rnorm=None, l1=None, params: W.Params | None = None,
                     stream=None):
    """swnmg_residual_noalloc: the residual without a context and without any
    device allocation by the library (scratch is a fixed device array), for
    callers that must not allocate.  z, U, R (and rnorm, l1 when given) are
    the caller's float64 CUDA tensors; the work is enqueued on `stream`."""
    L = lib()
    pp, pr = make_problem(prob), make_params(params or prob.params)
    st = stream or torch.cuda.current_stream()
    rc = L.swnmg_residual_noalloc(C.byref(pp), C.byref(pr), _ptr(z), _ptr(U), _ptr(R),
                                  _ptr(rnorm) if rnorm is not None else None,
                                  _ptr(l1) if l1 is not None else None, C.c_void_p(st.cuda_stream))
    if rc != OK:
        raise SwnmgError(rc, L.swnmg_last_error(None).decode())


def set_wait_limit(polls: int) -> int:
    """swnmg_set_wait_limit: polls of every device-side wait before a sweep
    gives up with ERR_TIMEOUT (<= 0: the default); returns the old limit."""
    return int(lib().swnmg_set_wait_limit(int(polls)))


def fp64_rate(op: int = 1) -> float:
    """swnmg_fp64_rate: measured FP64 lane operations per second of the
    current device (op 0: FMA chains, op 1: additions)."""
    v = C.c_double(0.0)
    rc = lib().swnmg_fp64_rate(int(op), C.byref(v))
    if rc != OK:
        raise SwnmgError(rc, lib().swnmg_last_error(None).decode())
    return v.value


def default_params(dim: int) -> dict:
    p = Params()
    rc = lib().swnmg_default_params(dim, C.byref(p))
    if rc != OK:
        raise SwnmgError(rc, lib().swnmg_last_error(None).decode())
    return {f: getattr(p, f) for f, _ in Params._fields_}
