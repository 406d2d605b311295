"""Pins of the oracle's implicit / semi-implicit time step (Remark 2.6):
|K_i| (U^{n+1} - U^n)/dt + beta R(U^n) + (1 - beta) R(U^{n+1}) = 0, solved by
Steps 2-3 of Algorithm 1.  Checked against what the discretisation fixes:
the lake at rest stays at rest, a closed basin keeps its mass, an infinite
step is the steady solve, a small backward-Euler step differs from the
forward-Euler step by O(dt^2), and over a fixed time backward Euler
(beta = 0) converges at first order and Crank-Nicolson (beta = 1/2) at
second order."""

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_1608_06721_gb300 import workloads as W


def _ex31(n=64):
    # tol 1e-10: the time-step residual carries |K|/dt U (|K|/dt up to 1e4
    # here), whose rounding floor is near 1e-11
    return W.smooth_subcritical_1d(n)


def test_lake_at_rest_stays_at_rest():
    p = W.lake_at_rest_2d(n=32, flux=W.FLUX_LLF).with_params(n_levels=2)
    o = Oracle(p)
    U1, info = o.time_step(p.U0, dt=0.05, beta=0.0)
    assert info["status"] == 0
    assert np.abs(U1 - p.U0).max() <= 1e-12


@pytest.mark.parametrize("flux,amp", [(W.FLUX_LLF, 0.02), (W.FLUX_HLLC, 0.002)])
def test_closed_basin_keeps_its_mass(flux, amp):
    """A disturbed lake with dry islands and walls all round: the fluxes'
    mass parts telescope and the sources have none, so sum h is kept by
    every step (to the solve's tolerance).  (With HLL-type fluxes a rough
    0.02 disturbance of the shore cells makes Newton's iteration fail: the
    wet/dry wave speeds are not smooth; LLF takes it.)"""
    p = W.lake_at_rest_2d(n=32, flux=flux).with_params(n_levels=2)
    rng = np.random.default_rng(3)
    U = p.U0.copy()
    U[0] = U[0] + amp * (U[0] > 0) * rng.random(U.shape[1])
    o = Oracle(p)
    m0 = U[0].sum()
    for beta in (0.0, 0.5):
        V = U.copy()
        for _ in range(3):
            V, info = o.time_step(V, dt=0.01, beta=beta)
            assert info["status"] == 0
        assert abs(V[0].sum() - m0) <= 1e-11 * m0


def test_infinite_step_is_the_steady_solve():
    p = _ex31()
    Us, _ = Oracle(p, init_mode=W.INIT_NONE).solve(p.U0)
    U1, info = Oracle(p).time_step(p.U0, dt=1e14, beta=0.0)
    assert info["status"] == 0
    assert np.abs(U1 - Us).max() <= 1e-9 * np.abs(Us).max()


def test_small_backward_euler_step_matches_forward_euler_to_second_order():
    p = _ex31()
    o = Oracle(p)
    dx = (p.x1 - p.x0) / p.nx
    R0, _ = o.residual(p.U0)
    diffs = []
    for dt in (2e-3, 1e-3):
        Ub, info = o.time_step(p.U0, dt=dt, beta=0.0)
        assert info["status"] == 0
        Uf = p.U0 - (dt / dx) * R0
        diffs.append(np.abs(Ub - Uf).max())
    assert 3.5 < diffs[0] / diffs[1] < 4.5, diffs


@pytest.mark.parametrize("beta,order", [(0.0, 1), (0.5, 2)])
def test_time_accuracy_order(beta, order):
    """Error at t = 0.04 against a reference of 256 Crank-Nicolson steps."""
    p = _ex31()
    o = Oracle(p)
    T = 0.04

    def run(nsteps, b):
        U = p.U0.copy()
        for _ in range(nsteps):
            U, info = o.time_step(U, dt=T / nsteps, beta=b)
            assert info["status"] == 0
        return U

    ref = run(256, 0.5)
    e1 = np.abs(run(8, beta) - ref).max()
    e2 = np.abs(run(16, beta) - ref).max()
    rate = np.log2(e1 / e2)
    assert abs(rate - order) < 0.3, (e1, e2, rate)
