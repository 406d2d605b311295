"""Failure detection on the GPU without a fault: a device-side wait that runs
out of its bound ends the sweep with SWNMG_ERR_TIMEOUT, and the same context
then gives bit-identical results once the bound is restored.

The bound is shortened to one poll (swnmg_set_wait_limit), so the wavefront
sweeps' progress waits (a strip waiting on its predecessor) and staging waits
give up at once; nothing is left waiting, and the warps still drain their own
in-flight bulk copies under a separate bound before they exit."""
import numpy as np
import pytest
import torch

from paper_1608_06721_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def swnmg():
    from paper_1608_06721_gb300 import swnmg as S
    S.lib()
    yield S
    S.set_wait_limit(0)


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("precision", [W.PREC_FP64, W.PREC_MIXED])
def test_sgs_wait_timeout_then_recovery(swnmg, precision):
    """Block SGS half-sweeps on the 256 x 256 level 0 (8 strips)."""
    p = W.channel_2d(nx=256, ny=256, n_levels=3, precision=precision)
    U = _dev(W.random_state(p, 21, wet_frac=0.8))
    S = swnmg.Solver(p)
    S.jacobian(U)
    rhs = _dev(np.random.default_rng(22).standard_normal(U.shape))
    ref = {fw: S.sgs_sweep(0, rhs, torch.zeros_like(U), fw).clone() for fw in (True, False)}
    for fw in (True, False):
        old = swnmg.set_wait_limit(1)
        try:
            with pytest.raises(swnmg.SwnmgError) as e:
                S.sgs_sweep(0, rhs, torch.zeros_like(U), fw)
            assert e.value.status == swnmg.ERR_TIMEOUT
        finally:
            swnmg.set_wait_limit(old)
        assert torch.equal(S.sgs_sweep(0, rhs, torch.zeros_like(U), fw), ref[fw])
    S.close()


@pytest.mark.parametrize("nx,ny", [(256, 256), (64, 512)])
def test_blusgs_wait_timeout_then_recovery(swnmg, nx, ny):
    """BLU-SGS sweeps (strip-pipelined, in place on U; a 1D grid is one strip
    and has no progress wait)."""
    p = W.channel_2d(nx=nx, ny=ny, n_levels=3)
    U0 = W.random_state(p, 23, wet_frac=0.8)
    S = swnmg.Solver(p)
    ref = S.blusgs(_dev(U0), 0, 1).clone()
    old = swnmg.set_wait_limit(1)
    try:
        with pytest.raises(swnmg.SwnmgError) as e:
            S.blusgs(_dev(U0), 0, 1)
        assert e.value.status == swnmg.ERR_TIMEOUT
    finally:
        swnmg.set_wait_limit(old)
    assert torch.equal(S.blusgs(_dev(U0), 0, 1), ref)
    S.close()


def test_default_limit_restored(swnmg):
    old = swnmg.set_wait_limit(0)
    assert swnmg.set_wait_limit(0) == 1 << 22
    swnmg.set_wait_limit(old)
