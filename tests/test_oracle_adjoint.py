"""Pins of the oracle's discrete adjoint (the gradient form of the method;
the paper has no adjoint): the transposed block operator, lambda against a
dense solve of J^T lambda = g, the vector-Jacobian products lambda^T dR/dz and
lambda^T dR/dq against central differences of the residual map, and the
gradient of a gauge loss against central differences with re-solved steady
states (implicit function theorem)."""
import numpy as np

from oracle.oracle import Oracle
from paper_1608_06721_gb300 import workloads as W
from tests import dense


def kink_free_cells(p, U, gap=1e-4, hmin=0.05):
    """Wet cells whose bed differs from every neighbour's by more than gap
    (max(z_i, z_j) of the reconstruction is smooth there)."""
    z = p.z.reshape(p.ny, p.nx)
    ok = np.ones_like(z, dtype=bool)
    for dz in (np.abs(np.diff(z, axis=1)), np.abs(np.diff(z, axis=0))):
        bad = dz <= gap
        if dz.shape[1] == p.nx - 1:
            ok[:, :-1] &= ~bad
            ok[:, 1:] &= ~bad
        else:
            ok[:-1, :] &= ~bad
            ok[1:, :] &= ~bad
    return np.flatnonzero(ok.ravel() & (U[0] > hmin))


def _small(nx=16, ny=8, nl=2):
    p = W.channel_2d(nx=nx, ny=ny, n_levels=nl, redraw=False).with_params(gamma=2, coarse_sweeps=0)
    o = Oracle(p)
    U, info = o.solve()
    assert info["status"] == 0
    return p, o, U


def test_transposed_blocks_are_AT():
    p, o, U = _small()
    R, rn, blk = o.jacobian(U)
    A = dense.assemble(blk, p.nx, p.ny)
    AT = dense.assemble(o.transpose_blocks(blk), p.nx, p.ny)
    np.testing.assert_array_equal(AT, A.T)


def test_lambda_solves_transposed_system():
    p, o, U = _small()
    g = np.random.default_rng(1).standard_normal(U.shape)
    lam, _, _ = o.adjoint(U, g, ncycles=0)
    R, rn, blk = o.jacobian(U)
    A = dense.assemble(blk, p.nx, p.ny)
    np.testing.assert_allclose(dense.vec(lam), np.linalg.solve(A.T, dense.vec(g)), rtol=1e-10, atol=1e-12)
    lam_mg, _, _ = o.adjoint(U, g, ncycles=40)
    assert np.abs(lam_mg - lam).max() <= 1e-10 * np.abs(lam).max()


def test_vjp_against_central_differences_of_the_residual():
    p, o, U = _small()
    rng = np.random.default_rng(2)
    lam = rng.standard_normal(U.shape)
    A = dense.assemble(o.jacobian(U)[2], p.nx, p.ny)
    g = dense.unvec(A.T @ dense.vec(lam), p.ncomp)
    lam2, dRz, dRq = o.adjoint(U, g, ncycles=0)   # lambda = J^{-T} g with g = J^T lam
    np.testing.assert_allclose(lam2, lam, rtol=1e-8, atol=1e-10)
    d = 1e-6
    cells = kink_free_cells(p, U)
    assert len(cells) >= 12
    for j in rng.choice(cells, 12, replace=False):
        zp, zm = p.z.copy(), p.z.copy()
        zp[j] += d
        zm[j] -= d
        fd = np.sum(lam * (o.residual(U, z=zp)[0] - o.residual(U, z=zm)[0])) / (2 * d)
        assert abs(dRz[j] - fd) <= 1e-6 * max(abs(fd), np.abs(dRz).max() * 1e-3), (j, dRz[j], fd)
    import copy
    pq, pm = copy.deepcopy(p), copy.deepcopy(p)
    pq.bc[0].q += d
    pm.bc[0].q -= d
    fd = np.sum(lam * (Oracle(pq).residual(U)[0] - Oracle(pm).residual(U)[0])) / (2 * d)
    assert abs(dRq[0] - fd) <= 1e-6 * abs(fd)
    assert dRq[1] == dRq[2] == dRq[3] == 0.0


def _loss(U, z, gauges, eta):
    return float(np.sum((U[0][gauges] + z[gauges] - eta) ** 2))


def test_gauge_loss_gradient_matches_resolved_central_differences():
    """dL/dz = dL/dz|direct - lambda^T dR/dz and dL/dq = -lambda^T dR/dq,
    J^T lambda = dL/dU, against L(U_s(z +- d e_j)) re-solved to 1e-13."""
    p, o, U = _small(32, 16, 2)
    rng = np.random.default_rng(3)
    gauges = np.sort(rng.choice(np.flatnonzero(U[0] > 0.05), 10, replace=False))
    eta = U[0][gauges] + p.z[gauges] + 0.01 * rng.standard_normal(10)
    g = np.zeros_like(U)
    g[0][gauges] = 2 * (U[0][gauges] + p.z[gauges] - eta)
    lam, dRz, dRq = o.adjoint(U, g, ncycles=0)
    dLdz = -dRz
    dLdz[gauges] += 2 * (U[0][gauges] + p.z[gauges] - eta)
    d = 1e-5
    warm = Oracle(p, init_mode=W.INIT_NONE, tol=1e-13, max_newton=50)
    for j in rng.choice(kink_free_cells(p, U), 6, replace=False):
        Ls = []
        for sgn in (1, -1):
            pz = p.with_params()
            pz.z = p.z.copy()
            pz.z[j] += sgn * d
            Uj, info = Oracle(pz, init_mode=W.INIT_NONE, tol=1e-13, max_newton=50).solve(U)
            assert info["status"] == 0
            Ls.append(_loss(Uj, pz.z, gauges, eta))
        fd = (Ls[0] - Ls[1]) / (2 * d)
        assert abs(dLdz[j] - fd) <= 1e-6 * max(abs(fd), np.abs(dLdz).max()), (j, dLdz[j], fd)
    import copy
    Ls = []
    for sgn in (1, -1):
        pq = copy.deepcopy(p)
        pq.bc[0].q += sgn * d
        Uq, info = Oracle(pq, init_mode=W.INIT_NONE, tol=1e-13, max_newton=50).solve(U)
        Ls.append(_loss(Uq, p.z, gauges, eta))
    fd = (Ls[0] - Ls[1]) / (2 * d)
    assert abs(-dRq[0] - fd) <= 1e-6 * abs(fd), (-dRq[0], fd)
