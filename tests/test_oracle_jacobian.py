"""Pins of the oracle's residual assembly and finite-difference Jacobian
(eq. Res, eq. NumerDiff with the boundary rule, eq. NewtonREG): the lake at
rest (well-balancing), conservation, and the assembled block matrix against
a central-difference Jacobian of the whole residual map."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_1608_06721_gb300 import workloads as W
from tests import dense


@pytest.mark.parametrize("flux", [W.FLUX_LLF, W.FLUX_HLLC, W.FLUX_HLL])
def test_lake_at_rest_2d_dry_islands(flux):
    """h + z = const, u = 0 with dry bump tops is an exact discrete steady
    state (eq. GNeqsSTEEADY2; the 2D lake-at-rest workload): sum ||R_i||_1 <= 1e-13."""
    p = W.lake_at_rest_2d(n=256, flux=flux)
    assert (p.U0[0] == 0).mean() > 0.01
    R, rn = Oracle(p).residual(p.U0)
    assert rn.sum() <= 1e-13


def test_lake_at_rest_1d_emerged_bump():
    """Example 3.3's steady state h = max(0.1 - z, 0), u = 0 with depth 0.1
    prescribed at both ends is an exact discrete steady state."""
    p = W.wetdry_lake_1d(256)
    U = np.stack([np.maximum(0.1 - p.z, 0.0), np.zeros(p.n)])
    assert Oracle(p).residual_sum(U) <= 1e-14


def test_mass_conservation_closed_basin():
    """With walls on every side the mass components of R telescope to zero."""
    p = W.lake_at_rest_2d(n=32)
    U = W.random_state(p, 7, wet_frac=0.5)
    R, _ = Oracle(p).residual(U)
    assert abs(R[0].sum()) <= 1e-13 * np.abs(R[0]).sum()


def _central_jacobian(o, U, nc, step=1e-6):
    n = U.shape[1]
    J = np.zeros((n * nc, n * nc))
    for j in range(n):
        for k in range(nc):
            Up, Um = U.copy(), U.copy()
            Up[k, j] += step
            Um[k, j] -= step
            Rp, _ = o.residual(Up)
            Rm, _ = o.residual(Um)
            J[:, j * nc + k] = dense.vec((Rp - Rm) / (2 * step))
    return J


@pytest.mark.parametrize("case", ["1d_bump", "2d_channel", "2d_walls"])
def test_fd_jacobian_matches_central_difference(case):
    """The assembled blocks (diagonal with alpha||R_i||_1 removed) equal the
    Jacobian of the full residual map, boundary ghosts included."""
    if case == "1d_bump":
        p = W.subcritical_bump_1d(n=16, n_levels=1)
        ny = 1
    else:
        p = W.channel_2d(nx=8, ny=6, redraw=False, n_levels=1)
        ny = 6
        if case == "2d_walls":
            p.bc = [W.BC(W.BC_WALL_REFLECT) for _ in range(4)]
            p = p.with_params(flux=W.FLUX_HLLC, llf_wetdry=0)
    rng = np.random.default_rng(5)
    nc = p.ncomp
    U = np.empty((nc, p.n))
    U[0] = 1.0 + 0.1 * rng.random(p.n)             # wet, away from the max(0, .) kinks
    for k in range(1, nc):
        U[k] = 0.2 * U[0] * rng.standard_normal(p.n)
    o = Oracle(p)
    R, rn, blk = o.jacobian(U)
    A = dense.assemble(blk, p.nx, ny)
    for i in range(p.n):
        for s in range(nc):
            A[i * nc + s, i * nc + s] -= p.params.alpha * rn[i]
    J = _central_jacobian(o, U, nc)
    err = np.abs(A - J).max() / np.abs(J).max()
    assert err < 2e-6, err
    # the regularisation term is exactly alpha * ||R_i||_1 on the diagonal
    R0, rn0, blk0 = Oracle(p, alpha=0.0).jacobian(U)
    d = blk[:, 0] - blk0[:, 0]
    for i in range(p.n):
        np.testing.assert_allclose(np.diag(d[i]), p.params.alpha * rn[i], rtol=1e-9, atol=1e-15)
    np.testing.assert_array_equal(blk[:, 1:], blk0[:, 1:])
    np.testing.assert_array_equal(R, R0)
