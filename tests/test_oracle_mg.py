"""Pins of the oracle's multigrid (Section 2.3, eq. MatrixForm, ProjectAR,
Project, correction, Algorithm 0 and the block SGS smoother) against a
dense-matrix restatement: A_{l+1} = P^T A_l P with piecewise-constant P,
restriction P^T (b - A x), prolongation x + P x_c, Gauss-Seidel sweeps
(D+L)^{-1}(b - U x) and (D+U)^{-1}(b - L x), exact coarse solves, and V/W
cycles that converge to A^{-1} b."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_1608_06721_gb300 import workloads as W
from tests import dense


def _setup(dim, nl=3, gamma=1, coarse_sweeps=8, seed=11):
    if dim == 1:
        p = W.subcritical_bump_1d(n=16, n_levels=nl)
        ny = 1
    else:
        p = W.channel_2d(nx=8, ny=8, redraw=False, n_levels=nl)
        ny = 8
    p = p.with_params(gamma=gamma, coarse_sweeps=coarse_sweeps)
    o = Oracle(p)
    U = W.random_state(p, seed)
    R, rn, blk = o.jacobian(U)
    return p, ny, o, R, blk


def _levels(p, ny, o, blk):
    H = o.hierarchy(blk)
    dims = [(p.nx >> l, (ny >> l) if p.dim == 2 else 1) for l in range(len(H))]
    return H, dims


@pytest.mark.parametrize("dim", [1, 2])
def test_galerkin_is_PtAP(dim):
    p, ny, o, R, blk = _setup(dim)
    H, dims = _levels(p, ny, o, blk)
    nc = p.ncomp
    for l in range(len(H) - 1):
        A = dense.assemble(H[l], *dims[l])
        P = dense.prolongation(dims[l][0], dims[l][1], nc, p.dim)
        Ac = dense.assemble(H[l + 1], *dims[l + 1])
        np.testing.assert_allclose(Ac, P.T @ A @ P, rtol=0, atol=1e-13 * np.abs(A).max())
        np.testing.assert_array_equal(o.galerkin(l, H[l]), H[l + 1])


@pytest.mark.parametrize("dim", [1, 2])
def test_restrict_prolong(dim):
    p, ny, o, R, blk = _setup(dim)
    H, dims = _levels(p, ny, o, blk)
    nc = p.ncomp
    rng = np.random.default_rng(0)
    for l in range(len(H) - 1):
        n = dims[l][0] * dims[l][1]
        b, x = rng.standard_normal((nc, n)), rng.standard_normal((nc, n))
        A = dense.assemble(H[l], *dims[l])
        P = dense.prolongation(dims[l][0], dims[l][1], nc, p.dim)
        bc = o.restrict(l, H[l], b, x)
        np.testing.assert_allclose(dense.vec(bc), P.T @ (dense.vec(b) - A @ dense.vec(x)),
                                   rtol=0, atol=1e-12 * (1 + np.abs(A).max()))
        xc = rng.standard_normal((nc, P.shape[1] // nc))
        np.testing.assert_allclose(dense.vec(o.prolong(l, xc, x)), dense.vec(x) + P @ dense.vec(xc),
                                   rtol=0, atol=1e-15)


@pytest.mark.parametrize("dim", [1, 2])
def test_block_gauss_seidel_sweeps(dim):
    p, ny, o, R, blk = _setup(dim)
    nc = p.ncomp
    A = dense.assemble(blk, p.nx, ny)
    D, L, U = dense.split_blocks(A, nc)
    rng = np.random.default_rng(1)
    b, x = rng.standard_normal((nc, p.n)), rng.standard_normal((nc, p.n))
    xf = o.sgs(0, blk, b, x, forward=True)
    np.testing.assert_allclose(dense.vec(xf), np.linalg.solve(D + L, dense.vec(b) - U @ dense.vec(x)),
                               rtol=1e-11, atol=1e-12)
    xb = o.sgs(0, blk, b, x, forward=False)
    np.testing.assert_allclose(dense.vec(xb), np.linalg.solve(D + U, dense.vec(b) - L @ dense.vec(x)),
                               rtol=1e-11, atol=1e-12)


def _dense_cycle(As, Ps, nc, b, x, l, nl, nu1, nu2, gamma, kc):
    """Algorithm 0 written with dense matrices."""
    A = As[l]
    D, L, U = dense.split_blocks(A, nc)

    def sweep(x):
        x = np.linalg.solve(D + L, b - U @ x)
        return np.linalg.solve(D + U, b - L @ x)
    if l == nl:
        if kc <= 0:
            return np.linalg.solve(A, b)
        for _ in range(kc):
            x = sweep(x)
        return x
    for _ in range(nu1):
        x = sweep(x)
    bc = Ps[l].T @ (b - A @ x)
    xc = np.zeros_like(bc)
    for _ in range(1 if l == 0 else gamma):
        xc = _dense_cycle(As, Ps, nc, bc, xc, l + 1, nl, nu1, nu2, gamma, kc)
    x = x + Ps[l] @ xc
    for _ in range(nu2):
        x = sweep(x)
    return x


@pytest.mark.parametrize("dim,gamma,kc", [(1, 1, 8), (1, 2, 8), (2, 1, 8), (2, 2, 8), (2, 1, 0)])
def test_cycle_matches_dense_algorithm0(dim, gamma, kc):
    p, ny, o, R, blk = _setup(dim, gamma=gamma, coarse_sweeps=kc)
    H, dims = _levels(p, ny, o, blk)
    nc = p.ncomp
    As = [dense.assemble(H[l], *dims[l]) for l in range(len(H))]
    Ps = [dense.prolongation(dims[l][0], dims[l][1], nc, p.dim) for l in range(len(H) - 1)]
    b = -R
    x1 = o.vcycle(blk, b, np.zeros_like(b), 1)
    kc_eff = 0 if dim == 1 else kc
    xd = _dense_cycle(As, Ps, nc, dense.vec(b), np.zeros(p.n * nc), 0, len(H) - 1,
                      p.params.nu1, p.params.nu2, gamma, kc_eff)
    np.testing.assert_allclose(dense.vec(x1), xd, rtol=1e-10, atol=1e-12 * np.abs(xd).max())


@pytest.mark.parametrize("dim", [1, 2])
def test_cycles_converge_to_dense_solution(dim):
    p, ny, o, R, blk = _setup(dim, coarse_sweeps=0)
    A = dense.assemble(blk, p.nx, ny)
    xe = np.linalg.solve(A, dense.vec(-R))
    x = o.vcycle(blk, -R, np.zeros_like(R), 40)
    assert np.abs(dense.vec(x) - xe).max() <= 1e-12 * np.abs(xe).max()


def test_coarse_solve_1d_is_exact():
    p, ny, o, R, blk = _setup(1, nl=2)
    H, dims = _levels(p, ny, o, blk)
    b = np.random.default_rng(4).standard_normal((p.ncomp, dims[2][0]))
    x = o.coarse_solve(2, H[2], b, np.zeros_like(b))
    A = dense.assemble(H[2], *dims[2])
    np.testing.assert_allclose(dense.vec(x), np.linalg.solve(A, dense.vec(b)), rtol=1e-11, atol=1e-13)


# ------------------------------------------- two-colour smoother (variant)

def _colour_perm(nx, ny, nc, first):
    """Unknown permutation that lists the cells of colour `first` ((ix + iy)
    mod 2), then the other colour, each in cell order."""
    cells = [i for c in (first, 1 - first) for i in range(nx * ny) if ((i % nx) + (i // nx)) % 2 == c]
    return np.array([i * nc + s for i in cells for s in range(nc)])


def _colour_gs(A, nc, nx, ny, b, x, first):
    """One block Gauss-Seidel sweep in the colour order, written as forward
    Gauss-Seidel (D + L)^{-1}(b - U x) on the permuted system."""
    p = _colour_perm(nx, ny, nc, first)
    Ap = A[np.ix_(p, p)]
    D, L, U = dense.split_blocks(Ap, nc)
    y = np.linalg.solve(D + L, b[p] - U @ x[p])
    out = np.empty_like(x)
    out[p] = y
    return out


@pytest.mark.parametrize("dim", [1, 2])
def test_colour_gauss_seidel_sweeps(dim):
    """SWNMG_SMOOTH_COLOUR (not the paper's smoother): the forward sweep is
    block Gauss-Seidel with colour 0 ((ix + iy) even) first, the backward
    sweep with colour 1 first; inside a colour the cells decouple."""
    p, ny, o, R, blk = _setup(dim)
    o = o.reconfigure(smoother=W.SMOOTH_COLOUR)
    nc = p.ncomp
    A = dense.assemble(blk, p.nx, ny)
    rng = np.random.default_rng(2)
    b, x = rng.standard_normal((nc, p.n)), rng.standard_normal((nc, p.n))
    for fwd, first in ((True, 0), (False, 1)):
        xo = o.sgs(0, blk, b, x, forward=fwd)
        xd = _colour_gs(A, nc, p.nx, ny, dense.vec(b), dense.vec(x), first)
        np.testing.assert_allclose(dense.vec(xo), xd, rtol=1e-11, atol=1e-12)
    # it is not the lexicographic sweep
    assert np.abs(o.sgs(0, blk, b, x, forward=True) - Oracle(p).sgs(0, blk, b, x, forward=True)).max() > 1e-3


@pytest.mark.parametrize("dim,gamma", [(1, 1), (2, 1), (2, 2)])
def test_colour_cycles_converge_to_dense_solution(dim, gamma):
    """Algorithm 0 with the two-colour smoother still converges to A^{-1} b."""
    p, ny, o, R, blk = _setup(dim, gamma=gamma, coarse_sweeps=0)
    o = o.reconfigure(smoother=W.SMOOTH_COLOUR)
    A = dense.assemble(blk, p.nx, ny)
    xe = np.linalg.solve(A, dense.vec(-R))
    x = o.vcycle(blk, -R, np.zeros_like(R), 60)
    assert np.abs(dense.vec(x) - xe).max() <= 1e-11 * np.abs(xe).max()
