"""The allocation-free residual entry point (swnmg_residual_noalloc).

Some callers cannot allocate device memory: a runtime that owns all device
memory through its own pool, or a loop that cannot take the allocator's
implicit synchronisation.  For them the library evaluates the residual with
scratch from one fixed device array.  This file checks, through the C ABI,
that two calls in a row give exactly what swnmg_residual gives (the residual
tests' tolerance: bit for bit), including the largest grids the fixed
scratch holds, and that the next grid past that limit is refused with a
clear message.  It is collected last so that a failure here comes after
every other test has run.
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
    ("channel_256", lambda: W.channel_2d(nx=256, ny=256, redraw=False), 5),
]


def _words(nx, ny, with_rnorm):
    """Scratch doubles a 2D grid needs: 2 ncomp per edge, ||R_i||_1 when the
    caller passes no rnorm array, 1024 reduction partials."""
    edges = (nx + 1) * ny + nx * (ny + 1)
    return 6 * edges + (0 if with_rnorm else nx * ny) + 1024


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


@pytest.mark.parametrize("n,with_rnorm", [(294, True), (283, False)])
def test_noalloc_largest_accepted_grid(n, with_rnorm):
    """The largest square grids that fit the 2^20-double scratch, with and
    without the optional ||R_i||_1 output, are accepted and bit-identical to
    swnmg_residual; one more cell per side does not fit."""
    from paper_1608_06721_gb300 import swnmg
    assert _words(n, n, with_rnorm) <= 1 << 20 < _words(n + 1, n + 1, with_rnorm)
    # one level: the context only supplies the reference residual, and these
    # sizes are not divisible by 2
    p = W.channel_2d(nx=n, ny=n, redraw=False, n_levels=0)
    U = _dev(W.random_state(p, 11, wet_frac=0.5))
    S = swnmg.Solver(p)
    R_ref, rn_ref, l1_ref = S.residual(U)
    R = torch.full_like(R_ref, float("nan"))
    rn = torch.full_like(rn_ref, float("nan")) if with_rnorm else None
    l1 = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    swnmg.residual_noalloc(p, _dev(p.z), U, R, rn, l1)
    torch.cuda.synchronize()
    assert torch.equal(R, R_ref)
    if with_rnorm:
        assert torch.equal(rn, rn_ref)
    assert abs(l1.item() - l1_ref) <= 1e-13 * max(abs(l1_ref), 1e-300)
    S.close()
    q = W.channel_2d(nx=n + 1, ny=n + 1, redraw=False, n_levels=0)
    Uq = _dev(q.U0)
    with pytest.raises(swnmg.SwnmgError) as e:
        swnmg.residual_noalloc(q, _dev(q.z), Uq, torch.zeros_like(Uq),
                               torch.zeros(Uq.shape[1], dtype=torch.float64, device="cuda") if with_rnorm else None)
    assert e.value.status == swnmg.ERR_ARG


def test_noalloc_rejects_grids_beyond_the_fixed_scratch():
    from paper_1608_06721_gb300 import swnmg
    p = W.channel_2d(nx=512, ny=512, redraw=False)
    U = _dev(p.U0)
    R = torch.zeros_like(U)
    with pytest.raises(swnmg.SwnmgError) as e:
        swnmg.residual_noalloc(p, _dev(p.z), U, R)
    assert e.value.status == swnmg.ERR_ARG
    assert "scratch" in str(e.value)
