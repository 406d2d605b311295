"""The allocation-free residual entry point (swnmg_residual_noalloc).

Some callers cannot allocate device memory -- a host callback where CUDA
calls such as cudaMalloc are not allowed, a runtime that owns all device
memory through its own pool, a loop that cannot take the allocator's implicit
synchronisation.  For them the library evaluates the residual with scratch
from one fixed device array.  This file checks, through the C ABI, that two
calls in a row give exactly what swnmg_residual gives (the residual tests'
tolerance: bit for bit), and that a grid too large for the fixed scratch is
refused with a clear message.  It is collected last so that a failure here
comes after every other test has run.
"""
import numpy as np
import pytest
import torch

from paper_1608_06721_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


CASES = [
    ("channel_64x48", lambda: W.channel_2d(nx=64, ny=48, redraw=False), 4),
    ("bump1d_200", lambda: W.subcritical_bump_1d(n=200), 1),
    ("lake_128_hllc", lambda: W.lake_at_rest_2d(n=128, flux=W.FLUX_HLLC), 3),
]


@pytest.mark.parametrize("name,make,seed", CASES, ids=[c[0] for c in CASES])
def test_noalloc_residual_matches_context_residual(name, make, seed):
    from paper_1608_06721_gb300 import swnmg
    p = make()
    U = _dev(W.random_state(p, seed, wet_frac=0.5))
    S = swnmg.Solver(p)
    R_ref, rn_ref, l1_ref = S.residual(U)
    z = _dev(p.z)
    for call in range(2):
        R = torch.full_like(R_ref, float("nan"))
        rn = torch.full_like(rn_ref, float("nan"))
        l1 = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        swnmg.residual_noalloc(p, z, U, R, rn, l1)
        torch.cuda.synchronize()
        assert torch.equal(R, R_ref), (name, call)
        assert torch.equal(rn, rn_ref), (name, call)
        assert abs(l1.item() - l1_ref) <= 1e-13 * max(abs(l1_ref), 1e-300), (name, call)
    # without the optional ||R_i||_1 output (kept in the fixed scratch instead)
    R = torch.zeros_like(R_ref)
    l1 = torch.zeros(1, dtype=torch.float64, device="cuda")
    swnmg.residual_noalloc(p, z, U, R, None, l1)
    torch.cuda.synchronize()
    assert torch.equal(R, R_ref)
    assert abs(l1.item() - l1_ref) <= 1e-13 * max(abs(l1_ref), 1e-300)


def test_noalloc_rejects_grids_beyond_the_fixed_scratch():
    from paper_1608_06721_gb300 import swnmg
    p = W.channel_2d(nx=512, ny=512, redraw=False)
    U = _dev(p.U0)
    R = torch.zeros_like(U)
    with pytest.raises(swnmg.SwnmgError) as e:
        swnmg.residual_noalloc(p, _dev(p.z), U, R)
    assert e.value.status == swnmg.ERR_ARG
    assert "scratch" in str(e.value)
