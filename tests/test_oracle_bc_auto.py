"""Pins of the open boundary that picks its condition by the local Froude
number (Remark 2.3): in each of the four regimes -- subcritical or
supercritical, inflow or outflow -- its ghost state is that of the
corresponding fixed boundary kind (themselves pinned in test_oracle_flux.py);
a dry interior cell counts as supercritical outflow; and a subcritical
problem solved with it on both open ends is the problem with the explicit
kinds, bit for bit."""
import copy

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_1608_06721_gb300 import workloads as W

G = 9.81


def _with_bc(p, side, kind):
    q = copy.deepcopy(p)
    q.bc[side] = W.BC(kind, h=0.8, q=1.7, ut=0.25)
    return q


def _base():
    return W.channel_2d(nx=8, ny=8, n_levels=1, redraw=False)


# (side, interior h, u along +axis, tangential v, expected fixed kind)
CASES = [
    (0, 1.0, 0.5, 0.1, W.BC_INFLOW_DISCHARGE),   # west side: outward u_n = -u < 0, inflow
    (0, 1.0, -0.5, 0.1, W.BC_OUTFLOW_DEPTH),
    (0, 0.2, 3.0, 0.0, W.BC_SUPER_INFLOW),
    (0, 0.2, -3.0, 0.0, W.BC_SUPER_OUTFLOW),
    (1, 1.0, 0.5, -0.2, W.BC_OUTFLOW_DEPTH),
    (1, 1.0, -0.5, -0.2, W.BC_INFLOW_DISCHARGE),
    (1, 0.2, 3.0, 0.0, W.BC_SUPER_OUTFLOW),
    (1, 0.2, -3.0, 0.0, W.BC_SUPER_INFLOW),
]


def _expected_kind(side, h, u, v):
    sigma = 1.0 if side & 1 else -1.0
    sup = u * u + v * v >= G * h
    inflow = sigma * u < 0.0
    if sup:
        return W.BC_SUPER_INFLOW if inflow else W.BC_SUPER_OUTFLOW
    return W.BC_INFLOW_DISCHARGE if inflow else W.BC_OUTFLOW_DEPTH


@pytest.mark.parametrize("side,h,u,v,_k", CASES)
def test_auto_ghost_is_the_regimes_fixed_ghost(side, h, u, v, _k):
    kind = _expected_kind(side, h, u, v)
    auto = Oracle(_with_bc(_base(), side, W.BC_AUTO_FROUDE)).ghost(side, h, u, v)
    fixed = Oracle(_with_bc(_base(), side, kind)).ghost(side, h, u, v)
    assert np.array_equal(auto, fixed), (kind, auto, fixed)


def test_all_four_regimes_are_reached():
    kinds = {_expected_kind(s, h, u, v) for s, h, u, v, _ in CASES}
    assert kinds == {W.BC_INFLOW_DISCHARGE, W.BC_OUTFLOW_DEPTH, W.BC_SUPER_INFLOW, W.BC_SUPER_OUTFLOW}


def test_dry_interior_is_supercritical_outflow():
    o = Oracle(_with_bc(_base(), 1, W.BC_AUTO_FROUDE))
    assert np.array_equal(o.ghost(1, 0.0, 0.0, 0.0), np.zeros(3))


def test_subcritical_problem_matches_explicit_kinds():
    """Example 3.1 (subcritical at both ends): at the explicit problem's steady
    state the automatic boundary picks the same conditions (the residuals
    agree bit for bit), and a solve from the initial state -- where u = 0 on
    the inflow side picks the outflow condition at first -- reaches the same
    steady state in the same number of Newton steps."""
    p = W.smooth_subcritical_1d(64)
    q = copy.deepcopy(p)
    q.bc[0] = W.BC(W.BC_AUTO_FROUDE, h=p.bc[1].h, q=p.bc[0].q)
    q.bc[1] = W.BC(W.BC_AUTO_FROUDE, h=p.bc[1].h, q=p.bc[0].q)
    Up, ip = Oracle(p).solve()
    assert ip["status"] == 0
    Rp, _ = Oracle(p).residual(Up)
    Rq, _ = Oracle(q).residual(Up)
    assert np.array_equal(Rp, Rq)
    Uq, iq = Oracle(q).solve()
    assert iq["status"] == 0 and iq["n_newton"] == ip["n_newton"]
    assert np.abs(Uq - Up).max() <= 1e-11 * np.abs(Up).max()
