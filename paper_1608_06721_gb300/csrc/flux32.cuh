// flux32.cuh -- the flux of Remark 2.2, the hydrostatic reconstruction and
// the ghosts of Remark 2.3 in float, for the FP32 Step 1 sweep (blusgs32.cu).
// Host and device: the host build serves a test against the FP64 oracle.
#pragma once

#include <math.h>

#include "common.cuh"

namespace swnmg {
namespace f32 {

struct P32 { float h, u, v; };

constexpr float FD32 = 1.0f / 4096.0f;

__host__ __device__ inline float fmin2(float a, float b) { return (a < b) ? a : b; }
__host__ __device__ inline float fmax2(float a, float b) { return (a > b) ? a : b; }

__host__ __device__ inline P32 prim32(float h, float qa, float qb, float h_eps) {
  P32 p;
  p.h = h;
  if (h >= h_eps) {
    const float r = 1.0f / h;
    p.u = qa * r;
    p.v = qb * r;
  } else {
    p.u = 0.0f;
    p.v = 0.0f;
  }
  return p;
}

__host__ __device__ inline float harten32(float x, float ef) {
  const float a = fabsf(x);
  return (a < 2.0f * ef) ? (x * x) / (4.0f * ef) + ef : a;
}

// numerical flux between reconstructed states, Remark 2.2 (as in flux.cu)
__host__ __device__ inline void num_flux32(const DevLevel& L, float hl, float ul, float vl, float hr, float ur, float vr,
                           float F[3]) {
  if (hl == 0.0f && hr == 0.0f) {
    F[0] = 0.0f; F[1] = 0.0f; F[2] = 0.0f;
    return;
  }
  const float g = (float)L.g, hg = (float)L.half_g;
  const float cl = sqrtf(g * hl), cr = sqrtf(g * hr);
  const float ql = hl * ul, qr = hr * ur;
  const float FL0 = ql, FL1 = ql * ul + hg * (hl * hl), FL2 = ql * vl;
  const float FR0 = qr, FR1 = qr * ur + hg * (hr * hr), FR2 = qr * vr;
  const float dU0 = hr - hl, dU1 = qr - ql, dU2 = hr * vr - hl * vl;
  if (L.flux == FX_ROE) {
    const float ef = (float)L.eps_f;
    const float sl = sqrtf(hl), sr = sqrtf(hr);
    const float rs = 1.0f / (sl + sr);
    const float uh = (sl * ul + sr * ur) * rs, vh = (sl * vl + sr * vr) * rs;
    const float ch = sqrtf(g * ((hl + hr) * 0.5f));
    const float l1 = uh - ch, l3 = uh + ch, r2c = 1.0f / (2.0f * ch);
    const float a1 = (l3 * dU0 - dU1) * r2c, a3 = (dU1 - l1 * dU0) * r2c, a2 = dU2 - vh * dU0;
    const float w1 = harten32(l1, ef) * a1, w2 = harten32(uh, ef) * a2, w3 = harten32(l3, ef) * a3;
    F[0] = ((FL0 + FR0) - (w1 + w3)) * 0.5f;
    F[1] = ((FL1 + FR1) - (w1 * l1 + w3 * l3)) * 0.5f;
    F[2] = ((FL2 + FR2) - ((w1 * vh + w2) + w3 * vh)) * 0.5f;
    return;
  }
  if (L.flux == FX_LLF) {
    float smax = fmax2(fabsf(ul) + cl, fabsf(ur) + cr);
    if (L.llf_wetdry) smax = smax + (float)L.eps_r * fmax2(cl, cr);
    F[0] = ((FL0 + FR0) - smax * dU0) * 0.5f;
    F[1] = ((FL1 + FR1) - smax * dU1) * 0.5f;
    F[2] = ((FL2 + FR2) - smax * dU2) * 0.5f;
    return;
  }
  const float us = ((ul + ur) * 0.5f + cl) - cr;
  const float t = (cl + cr) + (ul - ur) * 0.5f;
  const float cs = fabsf(t) * 0.5f;
  const float sL = (hl == 0.0f) ? ur - 2.0f * cr : fmin2(ul - cl, us - cs);
  const float sR = (hr == 0.0f) ? ul + 2.0f * cl : fmax2(ur + cr, us + cs);
  if (sL >= 0.0f) { F[0] = FL0; F[1] = FL1; F[2] = FL2; return; }
  if (sR <= 0.0f) { F[0] = FR0; F[1] = FR1; F[2] = FR2; return; }
  const float rden = 1.0f / (sR - sL), p = sL * sR;
  F[0] = ((sR * FL0 - sL * FR0) + p * dU0) * rden;
  F[1] = ((sR * FL1 - sL * FR1) + p * dU1) * rden;
  F[2] = ((sR * FL2 - sL * FR2) + p * dU2) * rden;
  if (L.flux == FX_HLLC) {
    const float a = hr * (ur - sR), b = hl * (ul - sL);
    const float sM = (sL * a - sR * b) / (a - b);
    F[2] = (sM >= 0.0f) ? vl * F[0] : vr * F[0];
  }
}

__host__ __device__ inline void edge_eval32(const DevLevel& L, P32 a, float za, P32 b, float zb, float out[5]) {
  const float zs = fmax2(za, zb);
  const float tl = (a.h + za) - zs, tr = (b.h + zb) - zs;
  const float hl = (tl > 0.0f) ? tl : 0.0f, hr = (tr > 0.0f) ? tr : 0.0f;
  num_flux32(L, hl, a.u, a.v, hr, b.u, b.v, out);
  const float hg = (float)L.half_g;
  out[3] = hg * (hl * hl);
  out[4] = hg * (hr * hr);
}

__host__ __device__ inline float inflow_celerity32(float g, float RI, float qn) {
  const float gq = g * qn;
  float c = (RI > 0.0f) ? RI : 1.0f;
  for (int k = 0; k < 200; ++k) {
    if (((2.0f * c - RI) * c) * c + gq > 0.0f) break;
    c = 2.0f * c;
  }
  for (int it = 0; it < 60; ++it) {
    const float f = ((2.0f * c - RI) * c) * c + gq;
    const float fp = (6.0f * c - 2.0f * RI) * c;
    if (!(fp > 0.0f)) break;
    const float cn = c - f / fp;
    if (!(cn < c)) break;
    c = cn;
  }
  return c;
}

// Remark 2.3 ghost from the interior state in the edge frame (as in flux.cu)
__host__ __device__ inline P32 ghost32(const DevLevel& L, int side, P32 I) {
  const DevBC& bc = L.bc[side];
  const float sigma = (side & 1) ? 1.0f : -1.0f, g = (float)L.g;
  const float bh = (float)bc.h, bq = (float)bc.q, but = (float)bc.ut;
  P32 o;
  int kind = bc.kind;
  if (kind == BC_AUTO) {
    const bool super = (I.u * I.u + I.v * I.v) >= g * I.h;
    const bool in = (sigma * I.u) < 0.0f;
    kind = super ? (in ? BC_SUPER_IN : BC_SUPER_OUT) : (in ? BC_INFLOW : BC_OUTFLOW);
  }
  switch (kind) {
    case BC_SLIP: o.h = I.h; o.u = 0.0f; o.v = I.v; break;
    case BC_INFLOW: {
      const float qn = sigma * bq;
      const float c = inflow_celerity32(g, sigma * I.u + 2.0f * sqrtf(g * I.h), qn);
      const float h = (c * c) / g;
      o.h = h; o.u = sigma * ((h > 0.0f) ? qn / h : 0.0f); o.v = but;
      break;
    }
    case BC_OUTFLOW: {
      const float un = (sigma * I.u + 2.0f * sqrtf(g * I.h)) - 2.0f * sqrtf(g * bh);
      o.h = bh; o.u = sigma * un; o.v = I.v;
      break;
    }
    case BC_SUPER_IN: o.h = bh; o.u = (bh > 0.0f) ? bq / bh : 0.0f; o.v = but; break;
    case BC_SUPER_OUT: o = I; break;
    default: o.h = I.h; o.u = -I.u; o.v = I.v; break;
  }
  return o;
}

}  // namespace f32
}  // namespace swnmg
