"""GPU implicit / semi-implicit time steps (swnmg_time_step, Remark 2.6)
against the oracle's on the same inputs: the same Newton steps per time
step and the state within 1e-10 relative (FP64; the step's residual and
Jacobian are the oracle's operation by operation, the multigrid agrees to
1e-12 per cycle).  After a time step the context's residual is the steady
one again."""
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
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda").contiguous()


def _lake():
    p = W.lake_at_rest_2d(n=32, flux=W.FLUX_LLF).with_params(n_levels=2)
    U = p.U0.copy()
    U[0] = U[0] + 0.02 * (U[0] > 0) * np.random.default_rng(3).random(U.shape[1])
    return p, U


CASES = [
    ("ex31_64", lambda: (W.smooth_subcritical_1d(64), W.smooth_subcritical_1d(64).U0), 0.01, 3),
    ("lake32_llf", _lake, 0.01, 2),
    ("channel_32", lambda: (W.channel_2d(nx=32, ny=32, n_levels=2, redraw=False).with_params(
        gamma=2, coarse_sweeps=0), None), 0.002, 2),
]


@pytest.mark.parametrize("beta", [0.0, 0.5], ids=["backward_euler", "crank_nicolson"])
@pytest.mark.parametrize("name,make,dt,steps", CASES, ids=[c[0] for c in CASES])
def test_time_steps_match_oracle(swnmg, name, make, dt, steps, beta):
    p, U0 = make()
    U0 = p.U0 if U0 is None else U0
    o = Oracle(p)
    S = swnmg.Solver(p)
    Uo = U0.copy()
    Ug = _dev(U0)
    for k in range(steps):
        Uo, io = o.time_step(Uo, dt=dt, beta=beta)
        ig = S.time_step(Ug, dt=dt, beta=beta)
        assert io["status"] == 0 and ig["status"] == 0, (k, io, ig)
        assert ig["n_newton"] == io["n_newton"], (k, ig["n_newton"], io["n_newton"])
        Ugh = Ug.cpu().numpy()
        assert np.abs(Ugh - Uo).max() <= 1e-10 * np.abs(Uo).max(), np.abs(Ugh - Uo).max()
    # the context is steady again
    R, rn, _ = S.residual(Ug)
    Ro, _ = o.residual(Ug.cpu().numpy())
    assert np.array_equal(R.cpu().numpy(), Ro)


def test_time_step_rejects_bad_arguments(swnmg):
    p = W.smooth_subcritical_1d(64)
    S = swnmg.Solver(p)
    U = _dev(p.U0)
    for dt, beta in ((0.0, 0.0), (-1.0, 0.0), (0.01, 1.0), (0.01, -0.1)):
        with pytest.raises(swnmg.SwnmgError) as e:
            S.time_step(U, dt=dt, beta=beta, check=True)
        assert e.value.status == swnmg.ERR_ARG
