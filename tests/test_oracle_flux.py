"""Pins of the oracle's numerical fluxes, reconstruction and ghost states
against properties the paper and the mathematics fix (Section 2.1, Remarks
2.2-2.3): consistency, upwinding, mirror antisymmetry, flow direction, the
wet/dry speed increase, hydrostatic reconstruction and the Riemann-invariant
boundary conditions."""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_1608_06721_gb300 import workloads as W

G = 9.81
FLUXES = [W.FLUX_HLL, W.FLUX_HLLC, W.FLUX_LLF]


def _orc(flux, llf_wetdry=0):
    p = W.lake_at_rest_2d(n=8, flux=flux)
    return Oracle(p, flux=flux, llf_wetdry=llf_wetdry)


def phys(h, u, v):
    return np.array([h * u, h * u * u + 0.5 * G * h * h, h * u * v])


@pytest.mark.parametrize("flux", FLUXES)
def test_consistency(flux):
    """F_hat(U, U) = F_n(U) (Section 2.1, consistency of the numerical flux)."""
    o = _orc(flux)
    rng = np.random.default_rng(1)
    for _ in range(200):
        h = rng.uniform(0.01, 3.0)
        u, v = rng.uniform(-3, 3, 2)
        out = o.edge_flux(h, u, v, 0.0, h, u, v, 0.0)
        np.testing.assert_allclose(out[:3], phys(h, u, v), rtol=1e-13, atol=1e-15)
        assert out[3] == out[4]
        np.testing.assert_allclose(out[3], 0.5 * G * h * h, rtol=1e-15)


@pytest.mark.parametrize("flux", FLUXES)
def test_still_water_flows_downhill(flux):
    """Two resting states of different depth: mass flows from the deep side."""
    o = _orc(flux)
    for hl, hr in [(1.0, 0.5), (0.3, 0.0), (0.0, 0.7), (2.0, 1.9)]:
        f = o.edge_flux(hl, 0.0, 0.0, 0.0, hr, 0.0, 0.0, 0.0)
        assert math.copysign(1.0, f[0]) == math.copysign(1.0, hl - hr) and f[0] != 0.0


@pytest.mark.parametrize("flux", FLUXES)
def test_mirror_antisymmetry(flux):
    """Reflecting the Riemann problem x -> -x (swap sides, negate normal
    velocity) negates the mass and tangential fluxes and keeps the normal
    momentum flux."""
    o = _orc(flux)
    rng = np.random.default_rng(2)
    for _ in range(200):
        hl, hr = rng.uniform(0.05, 2.0, 2)
        ul, ur, vl, vr = rng.uniform(-2.5, 2.5, 4)
        f = o.edge_flux(hl, ul, vl, 0.0, hr, ur, vr, 0.0)
        m = o.edge_flux(hr, -ur, vr, 0.0, hl, -ul, vl, 0.0)
        scale = np.abs(f[:3]).max() + 1.0
        assert abs(m[0] + f[0]) <= 1e-13 * scale
        assert abs(m[1] - f[1]) <= 1e-13 * scale
        if flux != W.FLUX_HLLC:
            assert abs(m[2] + f[2]) <= 1e-13 * scale


@pytest.mark.parametrize("flux", [W.FLUX_HLL, W.FLUX_HLLC])
def test_supersonic_upwinding(flux):
    """HLL/HLLC: s_L >= 0 gives F(U-), s_R <= 0 gives F(U+), bit for bit."""
    o = _orc(flux)
    f = o.edge_flux(1.0, 8.0, 0.3, 0.0, 0.8, 7.5, -0.2, 0.0)
    assert np.array_equal(f[:3], phys(1.0, 8.0, 0.3)) or np.allclose(f[:3], phys(1.0, 8.0, 0.3), rtol=1e-15)
    f = o.edge_flux(1.0, -8.0, 0.3, 0.0, 0.8, -7.5, -0.2, 0.0)
    np.testing.assert_allclose(f[:3], phys(0.8, -7.5, -0.2), rtol=1e-15)


def test_hllc_contact():
    """HLLC: equal tangential velocities reproduce HLL; otherwise the
    tangential flux is u_tau of the upwind side of the contact times f1."""
    hll, hllc = _orc(W.FLUX_HLL), _orc(W.FLUX_HLLC)
    a = hll.edge_flux(1.0, 0.4, 0.7, 0.0, 0.6, 0.2, 0.7, 0.0)
    b = hllc.edge_flux(1.0, 0.4, 0.7, 0.0, 0.6, 0.2, 0.7, 0.0)
    np.testing.assert_allclose(b, a, rtol=1e-13)
    b = hllc.edge_flux(1.0, 0.5, 0.9, 0.0, 1.0, 0.5, -0.4, 0.0)   # contact moves right
    assert b[0] > 0 and b[2] == 0.9 * b[0]
    b = hllc.edge_flux(1.0, -0.5, 0.9, 0.0, 1.0, -0.5, -0.4, 0.0)  # contact moves left
    assert b[0] < 0 and b[2] == -0.4 * b[0]


@pytest.mark.parametrize("flux", FLUXES)
def test_dry_dry_edge(flux):
    o = _orc(flux)
    assert np.all(o.edge_flux(0.0, 1.0, 0.0, 0.3, 0.0, -1.0, 0.0, 0.1) == 0.0)


def test_llf_wetdry_speed_increase():
    """eq. LLFflux: the wet/dry variant adds eps_r sqrt(g max h) to s_max,
    i.e. -1/2 eps_r sqrt(g max h) (U+ - U-) to the flux."""
    a, b = _orc(W.FLUX_LLF, 0), _orc(W.FLUX_LLF, 1)
    hl, hr, ul, ur = 0.9, 0.4, 0.3, -0.1
    fa = a.edge_flux(hl, ul, 0.0, 0.0, hr, ur, 0.0, 0.0)
    fb = b.edge_flux(hl, ul, 0.0, 0.0, hr, ur, 0.0, 0.0)
    d = 0.03 * math.sqrt(G * max(hl, hr))
    np.testing.assert_allclose(fb[0] - fa[0], -0.5 * d * (hr - hl), rtol=1e-12)
    np.testing.assert_allclose(fb[1] - fa[1], -0.5 * d * (hr * ur - hl * ul), rtol=1e-12)


@pytest.mark.parametrize("flux", FLUXES)
def test_hydrostatic_reconstruction(flux):
    """Lake at rest across a bed step: h_{e,-} = h_{e,+} = eta - max(z), the
    mass flux vanishes and the momentum flux equals both pressure terms."""
    o = _orc(flux)
    eta, zl, zr = 1.0, 0.25, 0.5
    out = o.edge_flux(eta - zl, 0.0, 0.0, zl, eta - zr, 0.0, 0.0, zr)
    he = eta - max(zl, zr)
    assert out[0] == 0.0
    np.testing.assert_allclose(out[3], 0.5 * G * he * he, rtol=1e-15)
    np.testing.assert_allclose(out[4], 0.5 * G * he * he, rtol=1e-15)
    np.testing.assert_allclose(out[1], out[3], rtol=1e-14)
    out = o.edge_flux(0.1, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.5)   # water below a dry step
    assert out[3] == 0.0 and out[4] == 0.0 and out[0] == 0.0


def test_ghost_states():
    """Remark 2.3: subcritical inflow keeps R = u_n + 2 sqrt(g h) and the
    prescribed discharge; subcritical outflow keeps R with the prescribed
    depth; the reflective wall mirrors the normal velocity."""
    p = W.channel_2d(nx=8, ny=8, redraw=False)
    p.bc[0] = W.BC(W.BC_INFLOW_DISCHARGE, q=0.9)
    p.bc[1] = W.BC(W.BC_OUTFLOW_DEPTH, h=0.6)
    p.bc[3] = W.BC(W.BC_INFLOW_DISCHARGE, q=-0.4, ut=0.1)   # inflow through the north side
    o = Oracle(p)
    rng = np.random.default_rng(3)
    for _ in range(100):
        h = rng.uniform(0.2, 1.5)
        u, v = rng.uniform(-0.5, 0.5, 2)
        for side, sigma, q in [(0, -1.0, 0.9), (3, 1.0, -0.4)]:
            hg, ug, vg = o.ghost(side, h, u, v)
            lhs = sigma * ug + 2 * math.sqrt(G * hg)
            rhs = sigma * u + 2 * math.sqrt(G * h)
            assert abs(lhs - rhs) <= 1e-12 * abs(rhs)
            assert abs(hg * ug - q) <= 1e-12 * abs(q)
        hg, ug, vg = o.ghost(1, h, u, v)
        assert hg == 0.6 and vg == v
        assert abs((ug + 2 * math.sqrt(G * 0.6)) - (u + 2 * math.sqrt(G * h))) <= 1e-13 * 10
        hg, ug, vg = o.ghost(2, h, u, v)
        assert (hg, ug, vg) == (h, -u, v)


@pytest.mark.parametrize("flux", FLUXES)
def test_wall_mass_flux_is_zero(flux):
    o = _orc(flux)
    for h, u, v in [(0.7, 0.3, -0.2), (1.2, -0.9, 0.4), (0.05, 0.01, 0.0)]:
        hg, ug, vg = o.ghost(1, h, u, v)
        assert o.edge_flux(h, u, v, 0.0, hg, ug, vg, 0.0)[0] == 0.0
