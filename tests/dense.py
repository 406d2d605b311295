"""Dense-matrix restatements used to pin the oracle (test helpers only).

Everything here is plain numpy linear algebra on the assembled global matrix:
the block operator A = [D, W, E, S, N] becomes one dense matrix with unknowns
ordered cell-major (i*nc + s), the aggregation prolongation becomes a 0/1
matrix P, and Algorithm 0 is written with those matrices.
"""
import numpy as np


def nbr(nx, ny, i, side):
    ix, iy = i % nx, i // nx
    if side == 0:
        return i - 1 if ix > 0 else -1
    if side == 1:
        return i + 1 if ix < nx - 1 else -1
    if side == 2:
        return i - nx if iy > 0 else -1
    return i + nx if iy < ny - 1 else -1


def assemble(blk, nx, ny):
    n, _, nc, _ = blk.shape
    A = np.zeros((n * nc, n * nc))
    for i in range(n):
        A[i * nc:(i + 1) * nc, i * nc:(i + 1) * nc] = blk[i, 0]
        for side in range(4):
            j = nbr(nx, ny, i, side)
            if j >= 0:
                A[i * nc:(i + 1) * nc, j * nc:(j + 1) * nc] = blk[i, 1 + side]
    return A


def vec(v):
    """SoA (nc, n) -> cell-major flat vector"""
    return np.ascontiguousarray(v.T).ravel()


def unvec(x, nc):
    return np.ascontiguousarray(x.reshape(-1, nc).T)


def prolongation(nx, ny, nc, dim):
    """P maps coarse unknowns to fine ones by piecewise-constant injection."""
    if dim == 1:
        ncx = nx // 2
        P = np.zeros((nx * nc, ncx * nc))
        for i in range(nx):
            I = i // 2
            for s in range(nc):
                P[i * nc + s, I * nc + s] = 1.0
        return P
    ncx, ncy = nx // 2, ny // 2
    P = np.zeros((nx * ny * nc, ncx * ncy * nc))
    for iy in range(ny):
        for ix in range(nx):
            i = ix + nx * iy
            I = ix // 2 + ncx * (iy // 2)
            for s in range(nc):
                P[i * nc + s, I * nc + s] = 1.0
    return P


def split_blocks(A, nc):
    """block diagonal, strictly lower and strictly upper parts (cell order)"""
    D = np.zeros_like(A)
    m = A.shape[0] // nc
    for i in range(m):
        D[i * nc:(i + 1) * nc, i * nc:(i + 1) * nc] = A[i * nc:(i + 1) * nc, i * nc:(i + 1) * nc]
    return D, np.tril(A - D), np.triu(A - D)


def sgs_iteration_radius(A, nc):
    """spectral radius of the symmetric block Gauss-Seidel iteration matrix"""
    D, L, U = split_blocks(A, nc)
    M = np.eye(A.shape[0]) - np.linalg.solve(D + U, D) @ np.linalg.solve(D + L, A)
    return float(np.abs(np.linalg.eigvals(M)).max())
