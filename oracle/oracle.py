"""ctypes front end of the CPU FP64 oracle (swnmg_oracle.c).

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline may import this module.  It builds the oracle with gcc
(-O2 -ffp-contract=off) into oracle/_build/ on first use.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "swnmg_oracle.c")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle.so")

HIST = 512


class _BC(C.Structure):
    _fields_ = [("kind", C.c_int), ("h", C.c_double), ("q", C.c_double), ("ut", C.c_double)]


class Cfg(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int),
                ("x0", C.c_double), ("x1", C.c_double), ("y0", C.c_double), ("y1", C.c_double),
                ("g", C.c_double), ("bc", _BC * 4),
                ("flux", C.c_int), ("llf_wetdry", C.c_int),
                ("alpha", C.c_double), ("fd_eps", C.c_double), ("tau", C.c_double),
                ("h_eps", C.c_double), ("eps_r", C.c_double), ("eps_p", C.c_double),
                ("tol", C.c_double),
                ("n_levels", C.c_int), ("n_mg", C.c_int), ("nu1", C.c_int), ("nu2", C.c_int),
                ("gamma", C.c_int), ("coarse_sweeps", C.c_int), ("max_newton", C.c_int),
                ("max_blusgs", C.c_int), ("init_mode", C.c_int), ("eps_f", C.c_double),
                ("t_ka", C.c_double), ("t_omb", C.c_double), ("t_src", C.c_void_p),
                ("mesh_x", C.c_void_p), ("mesh_y", C.c_void_p), ("t_kai", C.c_void_p),
                ("smoother", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("status", C.c_int), ("n_newton", C.c_int), ("n_vcycles", C.c_int),
                ("blusgs_sweeps", C.c_int * 16), ("init_res", C.c_double),
                ("final_res", C.c_double), ("res_hist", C.c_double * HIST)]


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, FP64, no FMA contraction)."""
    os.makedirs(BUILD, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.POINTER(C.c_double)
        cfgp = C.POINTER(Cfg)
        _lib.orc_residual.argtypes = [cfgp, C.c_int, P, P, P, P]
        _lib.orc_residual_sum.argtypes = [cfgp, C.c_int, P, P]
        _lib.orc_residual_sum.restype = C.c_double
        _lib.orc_jacobian.argtypes = [cfgp, C.c_int, P, P, P, P, P]
        _lib.orc_edge_flux.argtypes = [cfgp] + [C.c_double] * 8 + [P]
        _lib.orc_ghost.argtypes = [cfgp, C.c_int, C.c_double, C.c_double, C.c_double, P]
        _lib.orc_galerkin.argtypes = [cfgp, C.c_int, P, P]
        _lib.orc_restrict.argtypes = [cfgp, C.c_int, P, P, P, P]
        _lib.orc_prolong.argtypes = [cfgp, C.c_int, P, P]
        _lib.orc_sgs.argtypes = [cfgp, C.c_int, P, P, P, C.c_int]
        _lib.orc_coarse_solve.argtypes = [cfgp, C.c_int, P, P, P]
        _lib.orc_vcycle.argtypes = [cfgp, P, P, P, C.c_int]
        _lib.orc_hierarchy.argtypes = [cfgp, P, P]
        _lib.orc_blusgs.argtypes = [cfgp, C.c_int, P, P, C.c_int]
        _lib.orc_average.argtypes = [cfgp, C.c_int, C.c_int, P, P]
        _lib.orc_solve.argtypes = [cfgp, P, P, C.POINTER(Stats)]
        _lib.orc_level_cells.argtypes = [cfgp, C.c_int]
        _lib.orc_cell_areas.argtypes = [cfgp, C.c_int, P]
        _lib.orc_transpose_blocks.argtypes = [cfgp, C.c_int, P, P]
        _lib.orc_adjoint.argtypes = [cfgp, P, P, P, P, P, P, C.c_int]
        _lib.orc_time_step.argtypes = [cfgp, P, P, C.c_double, C.c_double, C.POINTER(Stats)]
    return _lib


def _p(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_cfg(prob, **over) -> Cfg:
    """Oracle configuration from a workloads.Problem (+ parameter overrides).
    A curvilinear problem's vertex arrays are referenced, not copied: the
    configuration keeps them alive as ``_mesh``."""
    prm = prob.params.replace(**over) if over else prob.params
    c = Cfg()
    if getattr(prob, "mesh_x", None) is not None:
        mx = np.ascontiguousarray(prob.mesh_x, dtype=np.float64)
        my = np.ascontiguousarray(prob.mesh_y, dtype=np.float64)
        assert mx.shape == my.shape == (prob.ny + 1, prob.nx + 1)
        c._mesh = (mx, my)
        c.mesh_x, c.mesh_y = mx.ctypes.data, my.ctypes.data
    c.dim, c.nx, c.ny = prob.dim, prob.nx, (prob.ny if prob.dim == 2 else 1)
    c.x0, c.x1, c.y0, c.y1, c.g = prob.x0, prob.x1, prob.y0, prob.y1, prob.g
    for s in range(4):
        b = prob.bc[s]
        c.bc[s].kind, c.bc[s].h, c.bc[s].q, c.bc[s].ut = b.kind, b.h, b.q, b.ut
    for f in ("flux", "llf_wetdry", "alpha", "fd_eps", "tau", "h_eps", "eps_r", "eps_p", "tol",
              "n_levels", "n_mg", "nu1", "nu2", "gamma", "coarse_sweeps", "max_newton",
              "max_blusgs", "init_mode", "eps_f", "smoother"):
        setattr(c, f, getattr(prm, f))
    return c


class Oracle:
    """Per-problem convenience wrapper; arrays are float64 numpy."""

    def __init__(self, prob, **over):
        self.prob = prob
        self.cfg = make_cfg(prob, **over)
        self.nc = prob.ncomp
        self.L = lib()

    def reconfigure(self, **over):
        return Oracle(self.prob, **over)

    def ncells(self, level=0):
        return self.L.orc_level_cells(C.byref(self.cfg), level)

    def areas(self, level=0):
        """|K_i| of the cells of a curvilinear mesh's level."""
        out = np.zeros(self.ncells(level))
        assert self.L.orc_cell_areas(C.byref(self.cfg), level, _p(out)) == 0
        return out

    def z_levels(self):
        zs = [np.ascontiguousarray(self.prob.z, dtype=np.float64)]
        for l in range(self.cfg.n_levels):
            zc = np.zeros(self.ncells(l + 1))
            self.L.orc_average(C.byref(self.cfg), l, 1, _p(zs[-1]), _p(zc))
            zs.append(zc)
        return zs

    def average(self, level, v):
        v = np.ascontiguousarray(v, dtype=np.float64)
        k = v.shape[0] if v.ndim == 2 else 1
        out = np.zeros((k, self.ncells(level + 1))) if v.ndim == 2 else np.zeros(self.ncells(level + 1))
        self.L.orc_average(C.byref(self.cfg), level, k, _p(v), _p(out))
        return out

    def residual(self, U, level=0, z=None):
        z = self.prob.z if z is None else z
        z = np.ascontiguousarray(z, dtype=np.float64)
        U = np.ascontiguousarray(U, dtype=np.float64)
        n = self.ncells(level)
        R = np.zeros((self.nc, n))
        rn = np.zeros(n)
        self.L.orc_residual(C.byref(self.cfg), level, _p(z), _p(U), _p(R), _p(rn))
        return R, rn

    def residual_sum(self, U, level=0, z=None):
        z = self.prob.z if z is None else z
        return self.L.orc_residual_sum(C.byref(self.cfg), level,
                                       _p(np.ascontiguousarray(z, dtype=np.float64)),
                                       _p(np.ascontiguousarray(U, dtype=np.float64)))

    def jacobian(self, U, level=0, z=None):
        """(R, rn, blocks[n,5,nc,nc]) with blocks D (incl. alpha*rn), W, E, S, N."""
        z = self.prob.z if z is None else z
        z = np.ascontiguousarray(z, dtype=np.float64)
        U = np.ascontiguousarray(U, dtype=np.float64)
        n = self.ncells(level)
        R = np.zeros((self.nc, n))
        rn = np.zeros(n)
        blk = np.zeros((n, 5, self.nc, self.nc))
        self.L.orc_jacobian(C.byref(self.cfg), level, _p(z), _p(U), _p(R), _p(rn), _p(blk))
        return R, rn, blk

    def edge_flux(self, hL, uL, vL, zL, hR, uR, vR, zR):
        out = np.zeros(5)
        self.L.orc_edge_flux(C.byref(self.cfg), hL, uL, vL, zL, hR, uR, vR, zR, _p(out))
        return out

    def ghost(self, side, hI, uI, vI=0.0):
        out = np.zeros(3)
        self.L.orc_ghost(C.byref(self.cfg), side, hI, uI, vI, _p(out))
        return out

    def galerkin(self, level, blk):
        blk = np.ascontiguousarray(blk, dtype=np.float64)
        out = np.zeros((self.ncells(level + 1), 5, self.nc, self.nc))
        self.L.orc_galerkin(C.byref(self.cfg), level, _p(blk), _p(out))
        return out

    def restrict(self, level, blk, b, x):
        out = np.zeros((self.nc, self.ncells(level + 1)))
        self.L.orc_restrict(C.byref(self.cfg), level, _p(np.ascontiguousarray(blk)),
                            _p(np.ascontiguousarray(b)), _p(np.ascontiguousarray(x)), _p(out))
        return out

    def prolong(self, level, xc, xf):
        xf = np.array(xf, dtype=np.float64, copy=True)
        self.L.orc_prolong(C.byref(self.cfg), level, _p(np.ascontiguousarray(xc)), _p(xf))
        return xf

    def sgs(self, level, blk, b, x, forward=True):
        x = np.array(x, dtype=np.float64, copy=True)
        self.L.orc_sgs(C.byref(self.cfg), level, _p(np.ascontiguousarray(blk)),
                       _p(np.ascontiguousarray(b)), _p(x), 1 if forward else 0)
        return x

    def coarse_solve(self, level, blk, b, x):
        x = np.array(x, dtype=np.float64, copy=True)
        self.L.orc_coarse_solve(C.byref(self.cfg), level, _p(np.ascontiguousarray(blk)),
                                _p(np.ascontiguousarray(b)), _p(x))
        return x

    def vcycle(self, blk0, b, x, ncycles=1):
        x = np.array(x, dtype=np.float64, copy=True)
        self.L.orc_vcycle(C.byref(self.cfg), _p(np.ascontiguousarray(blk0)),
                          _p(np.ascontiguousarray(b)), _p(x), ncycles)
        return x

    def hierarchy(self, blk0):
        sizes = [self.ncells(l) for l in range(self.cfg.n_levels + 1)]
        out = np.zeros(sum(sizes) * 5 * self.nc * self.nc)
        self.L.orc_hierarchy(C.byref(self.cfg), _p(np.ascontiguousarray(blk0)), _p(out))
        res, off = [], 0
        for n in sizes:
            m = n * 5 * self.nc * self.nc
            res.append(out[off:off + m].reshape(n, 5, self.nc, self.nc))
            off += m
        return res

    def blusgs(self, U, nsweeps=1, level=0, z=None):
        z = self.prob.z if z is None else z
        U = np.array(U, dtype=np.float64, copy=True)
        self.L.orc_blusgs(C.byref(self.cfg), level, _p(np.ascontiguousarray(z, dtype=np.float64)),
                          _p(U), nsweeps)
        return U

    def transpose_blocks(self, blk, level=0):
        out = np.zeros_like(np.ascontiguousarray(blk, dtype=np.float64))
        self.L.orc_transpose_blocks(C.byref(self.cfg), level, _p(np.ascontiguousarray(blk)), _p(out))
        return out

    def adjoint(self, U, g, ncycles=0, z=None):
        """(lambda, lambda^T dR/dz, lambda^T dR/dq[4]) at U for g = (dL/dU)^T."""
        z = self.prob.z if z is None else z
        U = np.ascontiguousarray(U, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        lam = np.zeros_like(U)
        dRz = np.zeros(U.shape[1])
        dRq = np.zeros(4)
        self.L.orc_adjoint(C.byref(self.cfg), _p(np.ascontiguousarray(z, dtype=np.float64)), _p(U), _p(g),
                           _p(lam), _p(dRz), _p(dRq), ncycles)
        return lam, dRz, dRq

    def time_step(self, U, dt, beta=0.0):
        """Remark 2.6: U^{n+1} from U^n = U (returns a new array and the counters)."""
        U = np.array(U, dtype=np.float64, copy=True)
        st = Stats()
        self.L.orc_time_step(C.byref(self.cfg), _p(np.ascontiguousarray(self.prob.z, dtype=np.float64)), _p(U),
                             float(dt), float(beta), C.byref(st))
        info = {"status": st.status, "n_newton": st.n_newton, "final_res": st.final_res,
                "res_hist": list(st.res_hist)[:min(st.n_newton, HIST)]}
        return U, info

    def solve(self, U0=None):
        U = np.array(self.prob.U0 if U0 is None else U0, dtype=np.float64, copy=True)
        st = Stats()
        self.L.orc_solve(C.byref(self.cfg), _p(np.ascontiguousarray(self.prob.z, dtype=np.float64)),
                         _p(U), C.byref(st))
        info = {"status": st.status, "n_newton": st.n_newton, "n_vcycles": st.n_vcycles,
                "blusgs_sweeps": list(st.blusgs_sweeps)[:self.cfg.n_levels + 1],
                "init_res": st.init_res, "final_res": st.final_res,
                "res_hist": list(st.res_hist)[:min(st.n_newton, HIST)]}
        return U, info
