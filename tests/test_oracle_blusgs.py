"""Pins of the oracle's BLU-SGS iteration (Algorithm 1, Steps 1 and 2.1) and
of its Step 1 cascade, against restatements that do not go through the
oracle's cell update, and against the paper's BLU-SGS step counts
(Table 3.1).

The restatements take only the oracle's residual map R(U) (pinned on its own
by the flux, well-balance and closed-form tests) and rebuild the rest from
the paper's text with numpy: the diagonal block dR_i/dU_i by differencing the
whole residual map, the regularised block solve
(alpha ||R_i||_1 I + dR_i/dU_i)^{-1} R_i, the dry rule of Remark 2.5, the
lexicographic forward then backward cell order, the averages to the coarse
levels, the thresholds eps_p 2^{-l} and the injection to the finer level."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_1608_06721_gb300 import workloads as W
from tests.golden import tables

PAPER = tables.load()


# ---------------------------------------------------------------- restatement

def _diag_block(o, U, i, level=0, z=None):
    """dR_i/dU_i by the paper's forward difference (eq. NumerDiff, eps =
    1e-8) of the whole residual map, one column per component of U_i.  The
    forward form is the paper's definition, and it matters: the map has
    kinks (h = 0, u = 0 in the LLF speeds) where a central difference gives
    another value."""
    nc = U.shape[0]
    d = o.cfg.fd_eps
    R0, _ = o.residual(U, level, z)
    D = np.zeros((nc, nc))
    for k in range(nc):
        Up = U.copy()
        Up[k, i] += d
        D[:, k] = (o.residual(Up, level, z)[0][:, i] - R0[:, i]) / d
    return R0[:, i], D


def _cell_update(o, U, i, level=0, z=None):
    """One BLU-SGS cell update, restated from Algorithm 1 and Remark 2.5."""
    alpha, h_eps = o.cfg.alpha, o.cfg.h_eps
    Ri, D = _diag_block(o, U, i, level, z)
    rn = np.abs(Ri).sum()
    if rn == 0.0:
        return
    dU = np.linalg.solve(D + alpha * rn * np.eye(len(Ri)), Ri)
    if U[0, i] < h_eps:          # dry when its update starts: depth only
        dU[1:] = 0.0
    U[:, i] -= dU
    if U[0, i] < h_eps:          # Remark 2.5: reset to a dry cell
        U[:, i] = 0.0


def _sweep(o, U, level=0, z=None):
    U = U.copy()
    n = U.shape[1]
    for i in range(n):
        _cell_update(o, U, i, level, z)
    for i in reversed(range(n)):
        _cell_update(o, U, i, level, z)
    return U


def _state_1d_smooth(n=16):
    p = W.smooth_subcritical_1d(n, n_levels=1)
    rng = np.random.default_rng(7)
    U = np.stack([1.0 - p.z + 0.05 * rng.standard_normal(n), 1.0 + 0.2 * rng.standard_normal(n)])
    return p, U


def _state_1d_wetdry(n=24):
    """Example 3.3 near its steady state, with dry cells on the emerged bump,
    a wet cell next to them and a dry cell that the sweep wets."""
    p = W.wetdry_lake_1d(n, n_levels=1)
    rng = np.random.default_rng(8)
    h = np.maximum(0.1 - p.z, 0.0)
    wet = h > 0
    h[wet] += 0.01 * rng.standard_normal(wet.sum())
    h = np.maximum(h, 0.0)
    U = np.stack([h, np.where(h > 0, 0.02 * rng.standard_normal(n), 0.0)])
    dry = np.nonzero(~wet)[0]
    assert len(dry) >= 3
    # a shallow wet cell on the bump's flank; no momentum is exactly zero in a
    # wet cell (|u| in the LLF speed has its kink there)
    U[:, dry[0]] = (0.3, 0.003)
    return p, U


def _state_2d_wetdry():
    """Example 3.7's hill on a 6 x 4 grid (LLF, inflow, outflow, walls): one
    hill cell is dry, the other holds a film of depth 2e-6 that runs off and
    dries out, the rest is wet with random depths and momenta."""
    p = W.hill_wetdry_2d(6, 4, n_levels=1)
    rng = np.random.default_rng(9)
    h = p.U0[0].copy()
    wet = h > 0
    assert (~wet).sum() >= 2
    h[wet] = h[wet] * (1.0 + 0.3 * rng.uniform(-1, 1, wet.sum()))
    U = np.stack([h, 0.05 * rng.standard_normal(h.size) * wet, 0.05 * rng.standard_normal(h.size) * wet])
    i_thin = np.nonzero(~wet)[0][0]
    U[:, i_thin] = (2e-6, 1e-7, -1e-7)
    return p, U


CASES = {"1d_smooth_hll": _state_1d_smooth, "1d_wetdry_llf": _state_1d_wetdry,
         "2d_hill_wetdry_llf": _state_2d_wetdry}


@pytest.mark.parametrize("case", list(CASES))
def test_blusgs_sweep_matches_restatement(case):
    """One symmetric BLU-SGS sweep (forward then backward, Algorithm 1 Step
    2.1) equals the restated cell updates to 1e-6 of max|U|.  What differs
    is rounding: the oracle differences each edge term and sums, this test
    differences the summed residual."""
    p, U = CASES[case]()
    o = Oracle(p)
    got = o.blusgs(U, 1)
    want = _sweep(o, U)
    scale = np.abs(want).max()
    assert np.abs(got - want).max() <= 1e-6 * scale, np.abs(got - want).max() / scale
    # the sweep does something: the state moves by far more than the bar
    assert np.abs(got - U).max() > 1e-3 * scale


def test_blusgs_sweep_exercises_dry_rules():
    """The wet/dry cases reach both branches of Remark 2.5's rule: a cell
    that is dry when its update starts becomes wet with zero momentum, and a
    barely wet cell is reset to zero."""
    p, U = _state_2d_wetdry()
    o = Oracle(p)
    got = o.blusgs(U, 1)
    i_thin = np.nonzero(p.U0[0] == 0)[0][0]
    assert U[0, i_thin] > o.cfg.h_eps and np.all(got[:, i_thin] == 0.0)
    p1, U1 = _state_1d_wetdry()
    got1 = Oracle(p1).blusgs(U1, 1)
    wetted = (U1[0] == 0.0) & (got1[0] > 0.0)
    assert wetted.any()
    # cells wetted in the forward half are updated again in the backward half
    # with their momentum free, so only their first update keeps it at zero:
    # check that rule on a forward-only restatement of the first such cell
    o1 = Oracle(p1)
    i = int(np.nonzero(wetted)[0][0])
    V = U1.copy()
    for k in range(i + 1):
        _cell_update(o1, V, k)
    assert V[0, i] > 0.0 and V[1, i] == 0.0


# ----------------------------------------------------------- Step 1 cascade

def _children_mean(p, v, nx, ny):
    """Average of the 2 (1D) or 2 x 2 (2D) children of every coarse cell,
    summed in the child order (0,0), (1,0), (0,1), (1,1) and scaled by 1/2 or
    1/4, so that it rounds like any left-to-right sum of the children."""
    if p.dim == 1:
        a = v.reshape(v.shape[:-1] + (nx // 2, 2))
        return (a[..., 0] + a[..., 1]) * 0.5
    a = v.reshape(v.shape[:-1] + (ny // 2, 2, nx // 2, 2))
    s = ((a[..., 0, :, 0] + a[..., 0, :, 1]) + a[..., 1, :, 0]) + a[..., 1, :, 1]
    return (s * 0.25).reshape(v.shape[:-1] + ((nx // 2) * (ny // 2),))


def _inject(p, v, nx, ny):
    """U_{j,l-1} = U_{I,l} for the children j of I (piecewise constant)."""
    if p.dim == 1:
        return np.repeat(v, 2, axis=-1)
    a = v.reshape(v.shape[:-1] + (ny, nx))
    a = np.repeat(np.repeat(a, 2, axis=-1), 2, axis=-2)
    return a.reshape(v.shape[:-1] + (4 * nx * ny,))


def _step1(o, p):
    """Algorithm 1, Step 1: averages to the coarsest level, BLU-SGS on level l
    until sum_i ||R_{i,l}||_1 < eps_p 2^{-l}, injection to level l - 1, for
    l = N_L ... 1.  Returns the level-0 initial guess and the sweep counts."""
    NL, eps_p, cap = o.cfg.n_levels, o.cfg.eps_p, o.cfg.max_blusgs
    if eps_p < 0:   # the paper's rule: a fraction of the initial data's residual
        eps_p = -eps_p * o.residual_sum(p.U0)
    sizes = [(p.nx >> l, (p.ny >> l) if p.dim == 2 else 1) for l in range(NL + 1)]
    zs, Us = [np.asarray(p.z, dtype=float)], [np.asarray(p.U0, dtype=float)]
    for l in range(NL):
        zs.append(_children_mean(p, zs[-1], *sizes[l]))
        Us.append(_children_mean(p, Us[-1], *sizes[l]))
    U = Us[NL]
    sweeps = [0] * (NL + 1)
    for l in range(NL, 0, -1):
        while o.residual_sum(U, l, zs[l]) >= eps_p / 2 ** l and sweeps[l] < cap:
            U = o.blusgs(U, 1, level=l, z=zs[l])
            sweeps[l] += 1
        U = _inject(p, U, *sizes[l])
    return U, sweeps


def _coarse_problem(p, l, z_l):
    """The same problem posed on level l's mesh (nx / 2^l cells)."""
    import dataclasses
    q = dataclasses.replace(p, nx=p.nx >> l, ny=(p.ny >> l) if p.dim == 2 else p.ny)
    q.z = z_l
    return q


@pytest.mark.parametrize("make", [lambda: W.smooth_subcritical_1d(64),
                                  lambda: W.wetdry_lake_1d(64),
                                  lambda: W.hill_wetdry_2d(32, 16, n_levels=2),
                                  lambda: W.channel_2d(nx=32, ny=16, n_levels=2),
                                  lambda: W.channel_2d(nx=32, ny=16, n_levels=2).with_params(eps_p=-0.01),
                                  lambda: W.smooth_subcritical_1d(64).with_params(eps_p=-0.01)],
                         ids=["ex31", "ex33", "ex37_2d", "channel_2d", "channel_2d_rule", "ex31_rule"])
def test_step1_cascade_matches_restatement(make):
    """The oracle's Step 1 (orc_solve with no Newton step) equals the
    restated cascade: the same BLU-SGS sweep count on every level and the
    same level-0 initial guess to 1e-14.  A coarse level's residual equals
    the residual of the same problem posed on the coarse mesh (|e| = 2^l dx)."""
    p = make()
    o = Oracle(p)
    U_orc, info = Oracle(p, max_newton=0).solve()
    U_re, sweeps = _step1(o, p)
    assert info["blusgs_sweeps"][1:] == sweeps[1:], (info["blusgs_sweeps"], sweeps)
    assert sum(sweeps) > 0
    scale = np.abs(U_re).max()
    assert np.abs(U_orc - U_re).max() <= 1e-14 * scale
    # coarse-level geometry: level l of p is level 0 of the coarse problem
    l = o.cfg.n_levels
    z_l = o.z_levels()[l]
    U_l = np.asarray(p.U0, dtype=float)
    for m in range(l):
        U_l = o.average(m, U_l)
    Rc, _ = Oracle(_coarse_problem(p, l, z_l)).residual(U_l)
    Rl, _ = o.residual(U_l, l, z_l)
    assert np.abs(Rc - Rl).max() <= 1e-13 * max(1.0, np.abs(Rl).max())


# ------------------------------------------------- Table 3.1 BLU-SGS counts

def _blusgs_counts(p, tols, cap):
    """BLU-SGS sweeps on the finest mesh from Step 1's initial guess until
    sum_i ||R_i||_1 < tol, for each tol (the paper's stop tolerance is not
    printed)."""
    U, _ = Oracle(p, max_newton=0).solve()
    o = Oracle(p)
    out, k = {}, 0
    r = o.residual_sum(U)
    for tol in sorted(tols, reverse=True):
        while r >= tol and k < cap and np.isfinite(r):
            U = o.blusgs(U, 1)
            k += 1
            r = o.residual_sum(U)
        out[tol] = k if r < tol else -1
    return out


@pytest.mark.parametrize("flux,key,ns", [(W.FLUX_HLL, "hll", (64, 128, 256)),
                                         (W.FLUX_ROE, "roe", (64, 128, 256)),
                                         (W.FLUX_LLF, "llf", (64, 128))])
def test_paper_blusgs_counts_table31(flux, key, ns):
    """Table 3.1, block LU-SGS rows: started from Step 1's initial guess
    (N_L = 3, eps_p = 0.2), the sweeps needed to bring sum_i ||R_i||_1 below
    1e-10 and below 1e-12 bracket the printed N_step within one sweep
    (HLL 33/39/40, Roe 35/38/39, LLF 576/1370).  The bracket stands for the
    paper's unstated tolerance; the LLF rows are linear convergence at the
    block-SGS rate near 1, so they also pin the sweep order and the
    regularisation's decay."""
    for k, n in enumerate(ns):
        p = W.smooth_subcritical_1d(n, flux=flux)
        if flux == W.FLUX_LLF:
            p = p.with_params(llf_wetdry=0)
        c = _blusgs_counts(p, (1e-10, 1e-12), 4000)
        ref = PAPER["t31_%s_BLUSGS_Nstep" % key][k]
        assert c[1e-10] - 1 <= ref <= c[1e-12] + 1, (n, c, ref)


def test_table34_blusgs_known_discrepancy():
    """Table 3.4's BLU-SGS row (Example 3.3, LLF, wet/dry) is NOT reproduced:
    from Step 1's initial guess the oracle needs 30/46/99 sweeps to 1e-10
    (36/56/119 to 1e-12) at N = 64/128/256 against the printed 42/69/129,
    10-35 % fewer.  This test records the measured counts so that a change
    shows up; it is not a pin of the paper's numbers."""
    got = []
    for n in (64, 128, 256):
        c = _blusgs_counts(W.wetdry_lake_1d(n), (1e-10, 1e-12), 4000)
        got.append((c[1e-10], c[1e-12]))
    assert got == [(30, 36), (46, 56), (99, 119)], got
    for (lo, hi), ref in zip(got, PAPER["t34_llf_BLUSGS_Nstep"][:3]):
        assert hi < ref
