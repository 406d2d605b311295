"""GPU parity on structured curvilinear meshes (swnmg_set_mesh; eq. totalFlux
with each edge's |e_ij| and n_ij, Examples 3.4 and 3.5) against the CPU
oracle on the same inputs.

Bar, as on the uniform mesh: residual, finite-difference Jacobian blocks with
the Galerkin hierarchy, and BLU-SGS sweeps bit for bit (the geometry is
computed on the device without FMA contraction, in the oracle's order); full
solves and time steps with the same Newton and Step 1 counts and states
within 1e-10 relative.  The uniform mesh given as vertices reproduces the
uniform path bit for bit.  A degenerate mesh, the adjoint and batches are
refused."""
import numpy as np
import pytest
import torch

from oracle.oracle import Oracle
from paper_1608_06721_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def swnmg():
    from paper_1608_06721_gb300 import swnmg as S
    S.lib()
    return S


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _first_diff(a, b):
    d = np.flatnonzero(a.ravel() != b.ravel())
    if d.size == 0:
        return "identical"
    k = d[0]
    return "first difference at flat index %d: gpu %r oracle %r (%d differ)" % (k, a.ravel()[k], b.ravel()[k],
                                                                                d.size)


def _warped(nx, ny, amp=0.25):
    """[0,3]x[0,2] with every vertex displaced by amp cell widths along sine
    modes (curved boundaries too)."""
    xs = 3.0 * np.arange(nx + 1) / nx
    ys = 2.0 * np.arange(ny + 1) / ny
    X, Y = np.meshgrid(xs, ys)
    Xw = X + amp * (3.0 / nx) * np.sin(np.pi * Y) * np.sin(2 * np.pi * X / 3.0)
    Yw = Y + amp * (2.0 / ny) * np.sin(2 * np.pi * X / 3.0 + 0.5) * np.cos(0.5 * np.pi * Y)
    return Xw, Yw


def _warped_basin(nx=48, ny=32, flux=W.FLUX_LLF):
    """Closed basin on the warped mesh: two bumps, dry islands, walls."""
    n = nx * ny
    p = W.Problem("warped_basin", 2, nx, ny, 0.0, 3.0, 0.0, 2.0, np.zeros(n), np.zeros((3, n)),
                  [W.BC(W.BC_WALL_REFLECT) for _ in range(4)],
                  W.Params(flux=flux, n_levels=2, n_mg=3, llf_wetdry=1 if flux == W.FLUX_LLF else 0))
    p = W.with_mesh(p, *_warped(nx, ny))
    Xc, Yc = p.centres()
    p.z = W.gaussian_bumps(Xc, Yc, [0.7, 0.35], [0.25, 0.3], [1.0, 2.1], [0.8, 1.3])
    h = np.maximum(0.5 - p.z, 0.0)
    p.U0 = np.stack([h, np.zeros_like(h), np.zeros_like(h)])
    return p


def _inflow_noise(p, seed, rel=0.1):
    U = p.U0.copy()
    U = U * (1.0 + rel * np.random.default_rng(seed).standard_normal(U.shape))
    U[2] = U[2] + rel * np.abs(U[1]).max() * np.random.default_rng(seed + 1).standard_normal(U.shape[1])
    return U


def _cases():
    out = []
    p = W.constricted_channel("I", 72, 40)
    out.append(("channel_I_72x40", p, lambda p: _inflow_noise(p, 1)))
    p = W.constricted_channel("II", 72, 40, flux=W.FLUX_ROE)
    out.append(("channel_II_72x40_roe", p, lambda p: _inflow_noise(p, 2)))
    p = W.hubbard_channel(1.2)
    out.append(("hubbard_F1.2_96x32", p, lambda p: _inflow_noise(p, 3, 0.3)))
    p = _warped_basin()
    out.append(("warped_basin_48x32_llf", p, lambda p: W.random_state(p, 4, wet_frac=0.5)))
    p = _warped_basin(flux=W.FLUX_HLLC)
    out.append(("warped_basin_48x32_hllc", p, lambda p: W.random_state(p, 5, wet_frac=0.5)))
    return out


CASES = _cases()
IDS = [c[0] for c in CASES]


@pytest.mark.parametrize("name,prob,gen", CASES, ids=IDS)
def test_residual_bitwise(swnmg, name, prob, gen):
    U = gen(prob)
    S = swnmg.Solver(prob)
    R, rn, tot = S.residual(_dev(U))
    Ro, rno = Oracle(prob).residual(U)
    assert np.array_equal(R.cpu().numpy(), Ro), _first_diff(R.cpu().numpy(), Ro)
    assert np.array_equal(rn.cpu().numpy(), rno)


@pytest.mark.parametrize("name,prob,gen", CASES, ids=IDS)
def test_jacobian_and_hierarchy_bitwise(swnmg, name, prob, gen):
    U = gen(prob)
    S = swnmg.Solver(prob)
    S.jacobian(_dev(U))
    o = Oracle(prob)
    R, rn, blk = o.jacobian(U)
    for l, Ho in enumerate(o.hierarchy(blk)):
        Hg = S.get_blocks(l)
        assert np.array_equal(Hg, Ho), "level %d: %s" % (l, _first_diff(Hg, Ho))


@pytest.mark.parametrize("name,prob,gen", CASES, ids=IDS)
def test_blusgs_bitwise_fine_and_coarse(swnmg, name, prob, gen):
    """Level 0, and the coarsest level with its area-averaged bed and state."""
    U = gen(prob)
    S = swnmg.Solver(prob)
    o = Oracle(prob)
    Ug = _dev(U)
    S.blusgs(Ug, 0, 2)
    Uo = o.blusgs(U, 2)
    assert np.array_equal(Ug.cpu().numpy(), Uo), _first_diff(Ug.cpu().numpy(), Uo)
    NL = prob.params.n_levels
    Uc = U
    for l in range(NL):
        Uc = o.average(l, Uc)
    Ucg = _dev(Uc)
    S.blusgs(Ucg, NL, 2)
    Uco = o.blusgs(Uc, 2, level=NL, z=o.z_levels()[NL])
    assert np.array_equal(Ucg.cpu().numpy(), Uco), _first_diff(Ucg.cpu().numpy(), Uco)


def test_uniform_mesh_as_vertices_is_the_uniform_path(swnmg):
    p = W.channel_2d(nx=64, ny=32, n_levels=2, redraw=False)
    q = W.with_mesh(p, *W.cartesian_vertices(p))
    U = W.random_state(p, 6, wet_frac=0.5)
    Sp, Sq = swnmg.Solver(p), swnmg.Solver(q)
    Rp, _, _ = Sp.residual(_dev(U))
    Rq, _, _ = Sq.residual(_dev(U))
    assert np.array_equal(Rp.cpu().numpy(), Rq.cpu().numpy())
    Sp.jacobian(_dev(U))
    Sq.jacobian(_dev(U))
    assert np.array_equal(Sp.get_blocks(0), Sq.get_blocks(0))
    Up, Uq = _dev(p.U0), _dev(p.U0)
    ip, iq = Sp.solve(Up), Sq.solve(Uq)
    assert ip["status"] == iq["status"] == 0 and ip["n_newton"] == iq["n_newton"]
    assert torch.equal(Up, Uq)


SOLVES = [
    ("channel_I_72x40", W.constricted_channel("I", 72, 40)),
    ("channel_II_72x40", W.constricted_channel("II", 72, 40)),
    ("hubbard_F0.5", W.hubbard_channel(0.5)),
    ("hubbard_F1.2", W.hubbard_channel(1.2)),
    ("hubbard_F2", W.hubbard_channel(2.0)),
]


@pytest.mark.parametrize("name,prob", SOLVES, ids=[s[0] for s in SOLVES])
def test_solve_fp64(swnmg, name, prob):
    Uo, io = Oracle(prob).solve()
    S = swnmg.Solver(prob)
    Ug = _dev(prob.U0)
    ig = S.solve(Ug)
    assert io["status"] == 0 and ig["status"] == 0, (io, ig)
    assert ig["n_newton"] == io["n_newton"]
    assert ig["blusgs_sweeps"] == io["blusgs_sweeps"]
    assert np.abs(Ug.cpu().numpy() - Uo).max() <= 1e-10 * np.abs(Uo).max()


def test_solve_mixed_channel_I(swnmg):
    """Mixed precision (FP32 multigrid): the FP64 oracle's steady state to 1e-9."""
    prob = W.constricted_channel("I", 72, 40).with_params(precision=W.PREC_MIXED)
    Uo, io = Oracle(prob).solve()
    S = swnmg.Solver(prob)
    Ug = _dev(prob.U0)
    ig = S.solve(Ug)
    assert ig["status"] == 0
    assert np.abs(Ug.cpu().numpy() - Uo).max() <= 1e-9 * np.abs(Uo).max()


@pytest.mark.parametrize("beta", [0.0, 0.5], ids=["backward_euler", "crank_nicolson"])
def test_time_steps_match_oracle(swnmg, beta):
    """A disturbed closed basin on the warped mesh: |K_i|/dt per cell."""
    p = _warped_basin()
    U0 = p.U0.copy()
    U0[0] = U0[0] + 0.02 * (U0[0] > 0) * np.random.default_rng(7).random(p.n)
    o = Oracle(p)
    S = swnmg.Solver(p)
    Uo, Ug = U0.copy(), _dev(U0)
    for k in range(2):
        Uo, io = o.time_step(Uo, dt=0.01, beta=beta)
        ig = S.time_step(Ug, dt=0.01, beta=beta)
        assert io["status"] == 0 and ig["status"] == 0, (k, io, ig)
        assert ig["n_newton"] == io["n_newton"]
        assert np.abs(Ug.cpu().numpy() - Uo).max() <= 1e-10 * np.abs(Uo).max()


def test_degenerate_mesh_is_refused(swnmg):
    p = W.constricted_channel("I", 72, 40)
    X, Y = p.mesh_x.copy(), p.mesh_y.copy()
    X[5, 7] = X[5, 8]          # two vertices on top of each other: a zero-length edge
    Y[5, 7] = Y[5, 8]
    with pytest.raises(swnmg.SwnmgError) as e:
        swnmg.Solver(W.with_mesh(p, X, Y))
    assert e.value.status == swnmg.ERR_ARG


def test_adjoint_and_batches_are_refused(swnmg):
    p = W.constricted_channel("I", 72, 40)
    S = swnmg.Solver(p)
    U = _dev(p.U0)
    with pytest.raises(swnmg.SwnmgError) as e:
        S.adjoint(U, torch.zeros_like(U))
    assert e.value.status == swnmg.ERR_ARG
    with pytest.raises(NotImplementedError):
        swnmg.BatchSolver([p])
