"""Pins of the oracle's Newton multigrid iteration (Algorithm 1) against what
the paper and the mathematics fix: the lake at rest survives a Newton step,
1D steady states converge at first order to the Bernoulli closed form and to
Example 3.1's cubic, Example 3.3 lands on h = max(0.1 - z, 0), explicit time
marching reaches the same root, and the paper's printed Newton counts and
spectral radii (Tables 3.1, 3.2, 3.4; tests/golden/paper_tables.txt)."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_1608_06721_gb300 import workloads as W
from tests import dense
from tests.golden import tables

G = 9.81
PAPER = tables.load()
NS = [int(v) for v in PAPER["N"]]


@pytest.mark.parametrize("flux", [W.FLUX_LLF, W.FLUX_HLLC])
def test_lake_at_rest_survives_newton_step(flux):
    """Section 3 / eq. GNeqsSTEEADY2: one forced Newton step (tol = 0, warm
    start) keeps h + z = 0.5 and u = v = 0 to 1e-13; dry cells stay dry."""
    p = W.lake_at_rest_2d(n=64, flux=flux)
    U, info = Oracle(p, tol=0.0, max_newton=1, init_mode=W.INIT_NONE).solve()
    assert info["n_newton"] == 1
    wet = p.U0[0] > 0
    assert np.abs(U[0][wet] + p.z[wet] - 0.5).max() <= 1e-13
    assert np.abs(U[1:]).max() <= 1e-13
    assert np.all(U[:, ~wet] == 0.0)


def _bernoulli_depth(q, E, z):
    h = np.full_like(z, 3.0)
    for _ in range(100):
        f = q * q / (2 * h * h) + G * (h + z) - E
        h = h - f / (-q * q / h ** 3 + G)
    return h


def test_bernoulli_first_order():
    """Subcritical flow over a bump: hu = q and u^2/2 + g(h+z) = E (E from the
    outflow depth) hold to O(dx): the L1 depth error halves with dx."""
    errs = []
    for n in (200, 400, 800):
        p = W.subcritical_bump_1d(n=n)
        U, info = Oracle(p).solve()
        assert info["status"] == 0
        q = p.meta["q"]
        he = _bernoulli_depth(q, q * q / 8.0 + 2.0 * G, p.z)
        errs.append(np.abs(U[0] - he).mean())
    assert errs[0] < 2e-3
    for a, b in zip(errs, errs[1:]):
        assert 1.8 < a / b < 2.2


def test_example31_cubic_first_order():
    """Example 3.1: u^3 + (2gz - 2g - 1)u + 2g = 0, hu = 1; first-order error."""
    errs = []
    for n in (128, 256, 512):
        p = W.smooth_subcritical_1d(n)
        U, info = Oracle(p).solve()
        assert info["status"] == 0
        ue = np.ones(n)
        for _ in range(100):
            ue = ue - (ue ** 3 + (2 * G * p.z - 2 * G - 1) * ue + 2 * G) / (3 * ue ** 2 + (2 * G * p.z - 2 * G - 1))
        errs.append(np.abs(U[1] / U[0] - ue).mean())
    assert errs[0] < 1e-2
    for a, b in zip(errs, errs[1:]):
        assert 1.8 < a / b < 2.2


@pytest.mark.parametrize("n", [64, 128, 256, 512])
def test_example33_wet_dry_steady_state(n):
    """Example 3.3: the solve reaches h = max(0.1 - z, 0), u = 0."""
    p = W.wetdry_lake_1d(n)
    U, info = Oracle(p).solve()
    assert info["status"] == 0
    assert np.abs(U[0] - np.maximum(0.1 - p.z, 0.0)).max() <= 1e-8
    assert np.abs(U[1]).max() <= 1e-8


def _explicit_march(o, U, dt_over_area, steps, h_eps=1e-6):
    for _ in range(steps):
        R, _ = o.residual(U)
        U = U - dt_over_area * R
        U[:, U[0] < h_eps] = 0.0
    return U


def test_explicit_time_marching_reaches_same_root_1d():
    """The Newton root is the steady state of |K| dU/dt + R(U) = 0 (Example
    3.7 compares NMGM with explicit LLF marching the same way)."""
    p = W.subcritical_bump_1d(n=32, n_levels=2)
    o = Oracle(p)
    Un, info = o.solve()
    dx = 25.0 / 32
    U = _explicit_march(o, p.U0.copy(), 0.4 * dx / 12.0 / dx, 30000)
    assert o.residual_sum(U) < 1e-9
    assert np.abs(U - Un).max() <= 1e-8


def test_explicit_time_marching_reaches_same_root_2d_wetdry():
    p = W.hill_wetdry_2d(16, 8, n_levels=2)
    o = Oracle(p)
    Un, info = o.solve()
    assert info["status"] == 0
    dx, dy = 25.0 / 16, 10.0 / 8
    U = _explicit_march(o, p.U0.copy(), 0.3 * min(dx, dy) / 3.0 / (dx * dy), 40000)
    assert o.residual_sum(U) < 1e-9
    assert np.abs(U - Un).max() <= 1e-7


def _count(prob, **kw):
    U, info = Oracle(prob, **kw).solve()
    return info["n_newton"] if info["status"] == 0 else -1


def test_paper_newton_counts_table31_hll():
    """Table 3.1, HLL, V-cycle N_L = 3: N_step within one of the paper's (the
    paper does not state its stopping tolerance; ours is 1e-10)."""
    for n, ref in zip(NS[:4], PAPER["t31_hll_V_NL3_Nstep"]):
        assert abs(_count(W.smooth_subcritical_1d(n)) - ref) <= 1
    for n, ref in zip(NS[:2], PAPER["t31_llf_V_NL3_Nstep"]):
        assert abs(_count(W.smooth_subcritical_1d(n, flux=W.FLUX_LLF)) - ref) <= 1


def test_paper_newton_counts_table32_and_34():
    for n, ref in zip(NS[:4], PAPER["t32_hll_V_NL3_Nstep"]):
        assert abs(_count(W.transcritical_1d(n, 1)) - ref) <= 1
    for n, ref in zip(NS[:3], PAPER["t34_llf_V_NL3_Nstep"]):
        assert abs(_count(W.wetdry_lake_1d(n)) - ref) <= 1


def _steady_rho(p):
    o = Oracle(p)
    U, info = o.solve()
    assert info["status"] == 0
    R, rn, blk = o.jacobian(U)
    return dense.sgs_iteration_radius(dense.assemble(blk, p.nx, 1), p.ncomp)


@pytest.mark.parametrize("k,n", [(0, 64), (1, 128)])
def test_paper_spectral_radius_table31(k, n):
    """Table 3.1: spectral radius of the block SGS iteration matrix at the
    steady state (dense eigenvalues) -- pins the Jacobian, the boundary ghosts
    and the lexicographic sweep order together."""
    assert abs(_steady_rho(W.smooth_subcritical_1d(n)) - PAPER["t31_hll_rho"][k]) <= 2e-3
    assert abs(_steady_rho(W.smooth_subcritical_1d(n, flux=W.FLUX_LLF)) - PAPER["t31_llf_rho"][k]) <= 5e-5


def test_paper_spectral_radius_table32():
    assert abs(_steady_rho(W.transcritical_1d(64, 1)) - PAPER["t32_hll_rho"][0]) <= 5e-3


@pytest.mark.parametrize("flux,key", [(W.FLUX_HLL, "hll"), (W.FLUX_LLF, "llf"), (W.FLUX_ROE, "roe")])
def test_paper_table33_shock(flux, key):
    """Table 3.3 (Example 3.2 (II), transcritical flow with a hydraulic jump):
    V-cycle (N_L = 3) Newton steps within one at N = 64, 128 and the block
    SGS spectral radius at the steady state (N = 64 within 1e-4: measured
    0.39174 / 0.92514 / 0.25370; N = 128 within 1e-3)."""
    for k, n in enumerate((64, 128)):
        p = W.transcritical_1d(n, 2, flux=flux)
        if flux == W.FLUX_LLF:
            p = p.with_params(llf_wetdry=0)
        o = Oracle(p)
        U, info = o.solve()
        assert info["status"] == 0
        assert abs(info["n_newton"] - PAPER["t33_%s_V_NL3_Nstep" % key][k]) <= 1
        R, rn, blk = o.jacobian(U)
        rho = dense.sgs_iteration_radius(dense.assemble(blk, p.nx, 1), p.ncomp)
        assert abs(rho - PAPER["t33_%s_rho" % key][k]) <= (1e-4 if n == 64 else 1e-3), rho

