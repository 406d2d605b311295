"""The float restatement of the flux (Remark 2.2), the hydrostatic
reconstruction and the ghosts (Remark 2.3) used by the FP32 Step 1 sweep
(csrc/flux32.cuh), built for the host with nvcc and compared with the FP64
oracle on random states: every flux and every boundary kind to FP32
accuracy, allowing the rare state where float rounding flips a wave-speed
branch."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_1608_06721_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_1608_06721_gb300", "csrc", "flux32.cuh")

WRAP = r'''
#include "%s"
using namespace swnmg;
extern "C" void f32_edge(int flux, int llf_wetdry, double g, double eps_r, double eps_f, const double* in8,
                         double* out5) {
  DevLevel L{};
  L.g = g; L.half_g = 0.5 * g; L.flux = flux; L.llf_wetdry = llf_wetdry; L.eps_r = eps_r; L.eps_f = eps_f;
  const f32::P32 a{(float)in8[0], (float)in8[1], (float)in8[2]}, b{(float)in8[4], (float)in8[5], (float)in8[6]};
  float o[5];
  f32::edge_eval32(L, a, (float)in8[3], b, (float)in8[7], o);
  for (int k = 0; k < 5; ++k) out5[k] = o[k];
}
extern "C" void f32_ghost(int kind, double bh, double bq, double but, double g, int side, const double* in3,
                          double* out3) {
  DevLevel L{};
  L.g = g; L.half_g = 0.5 * g;
  L.bc[side].kind = kind; L.bc[side].h = bh; L.bc[side].q = bq; L.bc[side].ut = but;
  const f32::P32 I{(float)in3[0], (float)in3[1], (float)in3[2]};
  const f32::P32 o = f32::ghost32(L, side, I);
  out3[0] = o.h; out3[1] = o.u; out3[2] = o.v;
}
'''


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("flux32")
    src, so = d / "wrap.cu", d / "libf32.so"
    src.write_text(WRAP % HDR)
    subprocess.check_call([nvcc, "-O2", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
                           "-shared", "-gencode", "arch=compute_103a,code=sm_103a", "-o", str(so), str(src)])
    L = C.CDLL(str(so))
    P = C.POINTER(C.c_double)
    L.f32_edge.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, P, P]
    L.f32_ghost.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int, P, P]
    return L


def _p(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _close(a, b, scale):
    return np.abs(a - b).max() <= 2e-5 * scale


@pytest.mark.parametrize("flux", [W.FLUX_HLL, W.FLUX_HLLC, W.FLUX_LLF, W.FLUX_ROE])
def test_edge_flux_matches_the_oracle(lib, flux):
    p = W.channel_2d(nx=8, ny=8, n_levels=1, redraw=False).with_params(flux=flux, llf_wetdry=1)
    o = Oracle(p)
    rng = np.random.default_rng(40 + flux)
    bad = 0
    N = 2000
    for _ in range(N):
        hL, hR = rng.uniform(0.0, 2.0, 2) * (rng.random(2) > 0.1)
        uL, vL, uR, vR = rng.uniform(-3.0, 3.0, 4)
        zL, zR = rng.uniform(0.0, 0.5, 2)
        ref = o.edge_flux(hL, uL, vL, zL, hR, uR, vR, zR)
        x = np.array([hL, uL, vL, zL, hR, uR, vR, zR])
        out = np.zeros(5)
        lib.f32_edge(flux, 1, p.g, p.params.eps_r, p.params.eps_f, _p(x), _p(out))
        scale = 1.0 + np.abs(ref).max() + 5.0 * max(hL, hR)
        bad += not _close(out, ref, scale)
    assert bad <= N // 100, bad


@pytest.mark.parametrize("kind", list(range(7)))
def test_ghosts_match_the_oracle(lib, kind):
    base = W.channel_2d(nx=8, ny=8, n_levels=1, redraw=False)
    rng = np.random.default_rng(70 + kind)
    bad = 0
    N = 400
    for side in range(4):
        p = base.with_params()
        p.bc = list(base.bc)
        p.bc[side] = W.BC(kind, h=0.8, q=1.7 if side % 2 == 0 else -1.7, ut=0.25)
        o = Oracle(p)
        for _ in range(N // 4):
            h = rng.uniform(0.05, 2.0)
            u, v = rng.uniform(-4.0, 4.0, 2)
            ref = o.ghost(side, h, u, v)
            out = np.zeros(3)
            lib.f32_ghost(kind, 0.8, p.bc[side].q, 0.25, p.g, side, _p(np.array([h, u, v])), _p(out))
            bad += not _close(out, ref, 1.0 + np.abs(ref).max())
    assert bad <= N // 100, bad
