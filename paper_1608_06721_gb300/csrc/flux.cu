// flux.cu -- residual, finite-difference Jacobian, BLU-SGS and Newton update
// kernels (Sections 2.1, 2.2 and 2.4 of Wu & Tang, arXiv:1608.06721).
//
// Built with -fmad=false: every product and sum rounds separately, in the
// fixed evaluation order documented next to each formula, so that R and the
// finite-difference Jacobian (whose 1/eps = 1e8 amplifies any rounding
// difference) are reproducible bit for bit.  Divisions and square roots use
// CUDA's correctly rounded double operators.
#include "common.cuh"

namespace swnmg {

namespace {

struct Prim { double h, u, v; };   // edge frame: u along +axis, v tangential

__device__ __forceinline__ double dmin(double a, double b) { return (a < b) ? a : b; }
__device__ __forceinline__ double dmax(double a, double b) { return (a > b) ? a : b; }

// Comparisons of doubles on the integer pipe, with the results of the FP64
// comparisons they replace (NaN operands and signed zeros included).  A GB300
// SM issues one FP64 instruction per warp every 64 cycles, so on the cell
// update's dependent chain every FP64 comparison costs as much as a multiply.
// The bit patterns of doubles with a clear sign bit order like their values;
// patterns above infinity's are NaNs.
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
constexpr long long kInfBits = 0x7ff0000000000000LL;
// x > 0.0
__device__ __forceinline__ bool gt_zero(double x) {
  const long long u = dbits(x);
  return u > 0 && u <= kInfBits;
}
// x >= c for a positive c (not NaN)
__device__ __forceinline__ bool ge_pos(double x, double c) {
  const long long u = dbits(x);
  return u >= dbits(c) && u <= kInfBits;
}
// x < c for a positive c (not NaN)
__device__ __forceinline__ bool lt_pos(double x, double c) {
  const long long u = dbits(x);
  return u < dbits(c) && (u & 0x7fffffffffffffffLL) <= kInfBits;
}
// x == 0.0 (either zero)
__device__ __forceinline__ bool is_zero(double x) { return (dbits(x) << 1) == 0; }
// (a > b) ? a : b for a and b that are NaN or at least +0 (never -0)
__device__ __forceinline__ double dmax_nonneg(double a, double b) {
  const long long ua = dbits(a), ub = dbits(b);
  return (ua > ub && ua <= kInfBits && ub <= kInfBits && ub >= 0) ? a : b;
}

// cell velocities from the conserved state: 1/h once, zero below h_eps
// (a cell with h < h_eps is treated as dry, Remark 2.5)
__device__ __forceinline__ Prim to_prim(double h, double qa, double qb, double h_eps) {
  Prim p;
  p.h = h;
  if (ge_pos(h, h_eps)) {
    double r = 1.0 / h;
    p.u = qa * r;
    p.v = qb * r;
  } else {
    p.u = 0.0;
    p.v = 0.0;
  }
  return p;
}

// Harten's entropy fix (Remark 2.2): |x|, or x^2/(4 eps_f) + eps_f below 2 eps_f
__device__ __forceinline__ double harten_q(double x, double ef) {
  const double a = fabs(x);
  return (a < 2.0 * ef) ? (x * x) / (4.0 * ef) + ef : a;
}

// Numerical flux of Remark 2.2 between reconstructed states (hl, ul, vl) and
// (hr, ur, vr): HLL (eq. HLLflux) with the wet/dry wave speeds, HLLC's contact
// choice for the tangential flux, LLF (eq. LLFflux) with the optional wet/dry
// speed increase, or Roe with Harten's entropy fix (eq. ROEflux: mean depth,
// sqrt(h)-weighted velocities, waves u - c, u, u + c).  Both depths zero:
// zero flux.  FX is the flux (compile time); num_flux below picks it at run
// time, so every kernel evaluates the same operations.
template <int FX>
__device__ __forceinline__ void num_flux_t(const DevLevel& L, double hl, double ul, double vl, double hr,
                                           double ur, double vr, double F[3]) {
  if (is_zero(hl) && is_zero(hr)) {
    F[0] = 0.0; F[1] = 0.0; F[2] = 0.0;
    return;
  }
  const double g = L.g, hg = L.half_g;
  const double cl = sqrt(g * hl), cr = sqrt(g * hr);
  const double ql = hl * ul, qr = hr * ur;                 // h u_n of each side
  const double FL0 = ql, FL1 = ql * ul + hg * (hl * hl), FL2 = ql * vl;
  const double FR0 = qr, FR1 = qr * ur + hg * (hr * hr), FR2 = qr * vr;
  const double dU0 = hr - hl, dU1 = qr - ql, dU2 = hr * vr - hl * vl;   // U+ - U-
  if constexpr (FX == FX_ROE) {
    const double ef = L.eps_f;
    const double sl = sqrt(hl), sr = sqrt(hr);
    const double rs = 1.0 / (sl + sr);
    const double uh = (sl * ul + sr * ur) * rs;
    const double vh = (sl * vl + sr * vr) * rs;
    const double ch = sqrt(g * ((hl + hr) * 0.5));
    const double l1 = uh - ch, l3 = uh + ch;
    const double r2c = 1.0 / (2.0 * ch);
    const double a1 = (l3 * dU0 - dU1) * r2c;   // wave strengths
    const double a3 = (dU1 - l1 * dU0) * r2c;
    const double a2 = dU2 - vh * dU0;
    const double w1 = harten_q(l1, ef) * a1, w2 = harten_q(uh, ef) * a2, w3 = harten_q(l3, ef) * a3;
    const double D0 = w1 + w3;
    const double D1 = w1 * l1 + w3 * l3;
    const double D2 = (w1 * vh + w2) + w3 * vh;
    F[0] = ((FL0 + FR0) - D0) * 0.5;
    F[1] = ((FL1 + FR1) - D1) * 0.5;
    F[2] = ((FL2 + FR2) - D2) * 0.5;
    return;
  } else if constexpr (FX == FX_LLF) {
    double smax = dmax_nonneg(fabs(ul) + cl, fabs(ur) + cr);
    // sqrt(g max(h-, h+)) equals max(sqrt(g h-), sqrt(g h+)) bit for bit:
    // scaling by g > 0 and the correctly rounded sqrt are both monotone
    if (L.llf_wetdry) smax = smax + L.eps_r * dmax_nonneg(cl, cr);
    F[0] = ((FL0 + FR0) - smax * dU0) * 0.5;
    F[1] = ((FL1 + FR1) - smax * dU1) * 0.5;
    F[2] = ((FL2 + FR2) - smax * dU2) * 0.5;
    return;
  } else {
    // u_* and sqrt(g h_*) = |t|/2 (h_* = t^2 / (4g))
    const double us = ((ul + ur) * 0.5 + cl) - cr;
    const double t = (cl + cr) + (ul - ur) * 0.5;
    const double cs = fabs(t) * 0.5;
    const double sL = is_zero(hl) ? ur - 2.0 * cr : dmin(ul - cl, us - cs);
    const double sR = is_zero(hr) ? ul + 2.0 * cl : dmax(ur + cr, us + cs);
    if (sL >= 0.0) { F[0] = FL0; F[1] = FL1; F[2] = FL2; return; }
    if (sR <= 0.0) { F[0] = FR0; F[1] = FR1; F[2] = FR2; return; }
    const double rden = 1.0 / (sR - sL), p = sL * sR;
    F[0] = ((sR * FL0 - sL * FR0) + p * dU0) * rden;
    F[1] = ((sR * FL1 - sL * FR1) + p * dU1) * rden;
    F[2] = ((sR * FL2 - sL * FR2) + p * dU2) * rden;
    if constexpr (FX == FX_HLLC) {
      const double a = hr * (ur - sR), b = hl * (ul - sL);
      const double sM = (sL * a - sR * b) / (a - b);
      F[2] = (sM >= 0.0) ? vl * F[0] : vr * F[0];
    }
  }
}

__device__ void num_flux(const DevLevel& L, double hl, double ul, double vl, double hr, double ur,
                         double vr, double F[3]) {
  if (L.flux == FX_ROE) num_flux_t<FX_ROE>(L, hl, ul, vl, hr, ur, vr, F);
  else if (L.flux == FX_LLF) num_flux_t<FX_LLF>(L, hl, ul, vl, hr, ur, vr, F);
  else if (L.flux == FX_HLLC) num_flux_t<FX_HLLC>(L, hl, ul, vl, hr, ur, vr, F);
  else num_flux_t<FX_HLL>(L, hl, ul, vl, hr, ur, vr, F);
}

// eq. totalFlux with the hydrostatic reconstruction; a is the lower-index
// side.  out: F (3), g/2 h_{e,-}^2, g/2 h_{e,+}^2.
__device__ __forceinline__ void edge_eval(const DevLevel& L, Prim a, double za, Prim b, double zb,
                                          double out[5]) {
  const double zs = dmax(za, zb);
  const double tl = (a.h + za) - zs, tr = (b.h + zb) - zs;
  const double hl = gt_zero(tl) ? tl : 0.0, hr = gt_zero(tr) ? tr : 0.0;
  num_flux(L, hl, a.u, a.v, hr, b.u, b.v, out);
  out[3] = L.half_g * (hl * hl);
  out[4] = L.half_g * (hr * hr);
}

// edge_eval with the flux fixed at compile time
template <int FX>
__device__ __forceinline__ void edge_eval_t(const DevLevel& L, Prim a, double za, Prim b, double zb,
                                            double out[5]) {
  const double zs = dmax(za, zb);
  const double tl = (a.h + za) - zs, tr = (b.h + zb) - zs;
  const double hl = gt_zero(tl) ? tl : 0.0, hr = gt_zero(tr) ? tr : 0.0;
  num_flux_t<FX>(L, hl, a.u, a.v, hr, b.u, b.v, out);
  out[3] = L.half_g * (hl * hl);
  out[4] = L.half_g * (hr * hr);
}

// Subcritical inflow: celerity c of the ghost from f(c) = 2c^3 - R c^2 + g qn
// = 0.  Start right of the largest root (c = R, or 1, doubled until f > 0),
// then Newton steps while the iterate keeps decreasing (at most 60).
__device__ double inflow_celerity(double g, double RI, double qn) {
  const double gq = g * qn;
  double c = (RI > 0.0) ? RI : 1.0;
  for (int k = 0; k < 200; ++k) {
    const double f = ((2.0 * c - RI) * c) * c + gq;
    if (f > 0.0) break;
    c = 2.0 * c;
  }
  for (int it = 0; it < 60; ++it) {
    const double f = ((2.0 * c - RI) * c) * c + gq;
    const double fp = (6.0 * c - 2.0 * RI) * c;
    if (!(fp > 0.0)) break;
    const double cn = c - f / fp;
    if (!(cn < c)) break;
    c = cn;
  }
  return c;
}

// Ghost state of Remark 2.3 for boundary side s (0 W, 1 E, 2 S, 3 N) from the
// interior primitive state; sigma*u is the outward normal velocity.
__device__ Prim ghost_state(const DevLevel& L, int side, Prim I) {
  const DevBC& bc = L.bc[side];
  const double sigma = (side & 1) ? 1.0 : -1.0;
  const double g = L.g;
  Prim o;
  int kind = bc.kind;
  if (kind == BC_AUTO) {
    // Remark 2.3's choice by the interior's local Froude number (|u|^2 >= g h:
    // supercritical, a dry cell included) and the sign of the outward u_n
    const bool super = (I.u * I.u + I.v * I.v) >= g * I.h;
    const bool in = (sigma * I.u) < 0.0;
    kind = super ? (in ? BC_SUPER_IN : BC_SUPER_OUT) : (in ? BC_INFLOW : BC_OUTFLOW);
  }
  switch (kind) {
    case BC_SLIP: o.h = I.h; o.u = 0.0; o.v = I.v; break;
    case BC_INFLOW: {
      const double qn = sigma * bc.q;
      const double RI = sigma * I.u + 2.0 * sqrt(g * I.h);
      const double c = inflow_celerity(g, RI, qn);
      const double h = (c * c) / g;
      const double un = (h > 0.0) ? qn / h : 0.0;
      o.h = h; o.u = sigma * un; o.v = bc.ut;
      break;
    }
    case BC_OUTFLOW: {
      const double un = (sigma * I.u + 2.0 * sqrt(g * I.h)) - 2.0 * sqrt(g * bc.h);
      o.h = bc.h; o.u = sigma * un; o.v = I.v;
      break;
    }
    case BC_SUPER_IN: o.h = bc.h; o.u = (bc.h > 0.0) ? bc.q / bc.h : 0.0; o.v = bc.ut; break;
    case BC_SUPER_OUT: o = I; break;
    default: o.h = I.h; o.u = -I.u; o.v = I.v; break;   // reflective wall
  }
  return o;
}

// conserved global state (h, hu, hv) -> primitive in the frame of `axis`
template <int NC>
__device__ __forceinline__ Prim prim_axis(const DevLevel& L, const double* c, int axis) {
  if (NC == 2) return to_prim(c[0], c[1], 0.0, L.h_eps);
  return axis == 0 ? to_prim(c[0], c[1], c[2], L.h_eps) : to_prim(c[0], c[2], c[1], L.h_eps);
}

// G received by the left and right cell of an edge, in global components:
// left  (F0, F1 - sL, F2), right -(F0, F1 - sR, F2); y-edges swap the two
// momentum components back to (hu, hv).
template <int NC>
__device__ __forceinline__ void edge_G(const double o[5], int axis, double GL[NC], double GR[NC]) {
  const double gl1 = o[1] - o[3], gr1 = -(o[1] - o[4]);
  GL[0] = o[0];
  GR[0] = -o[0];
  if (NC == 2) { GL[1] = gl1; GR[1] = gr1; return; }
  if (axis == 0) {
    GL[1] = gl1; GL[2] = o[2];
    GR[1] = gr1; GR[2] = -o[2];
  } else {
    GL[1 % NC] = o[2]; GL[2 % NC] = gl1;
    GR[1 % NC] = -o[2]; GR[2 % NC] = gr1;
  }
}

// ---- structured curvilinear meshes (Examples 3.4, 3.5) ----------------------
// The edge frame is (n, tau): n from L.geo, tau = n turned by +90 degrees on
// x-edges and by -90 degrees on y-edges, so that on a uniform mesh it is the
// frame above (tau-velocity v on x-edges, u on y-edges; a boundary's q is
// along n, its u_tau along tau).  States go to the frame as u_n = u n^x +
// v n^y, u_tau = u tau^x + v tau^y; the flux comes back as F_1 n + F_2 tau,
// and the source term g/2 h_{e,-}^2 (n^x, n^y) is subtracted there.
struct Frame { double nx, ny, tx, ty; };

__device__ __forceinline__ long long level_edges(const DevLevel& L) {
  return (long long)(L.nx + 1) * L.ny + (L.dim == 2 ? (long long)L.nx * (L.ny + 1) : 0);
}

__device__ __forceinline__ Frame edge_frame(const DevLevel& L, long long e, int axis) {
  const long long ne = level_edges(L);
  Frame f;
  f.nx = L.geo[ne + e];
  f.ny = L.geo[2 * ne + e];
  if (axis == 0) { f.tx = -f.ny; f.ty = f.nx; }
  else { f.tx = f.ny; f.ty = -f.nx; }
  return f;
}

// global primitive (h, u, v) -> (h, u_n, u_tau)
__device__ __forceinline__ Prim to_frame(Prim g, const Frame& f) {
  Prim p;
  p.h = g.h;
  p.u = g.u * f.nx + g.v * f.ny;
  p.v = g.u * f.tx + g.v * f.ty;
  return p;
}

// G of the left and right cell in global components on a curvilinear mesh
__device__ __forceinline__ void edge_G_frame(const double o[5], const Frame& f, double GL[3], double GR[3]) {
  const double fx = o[1] * f.nx + o[2] * f.tx, fy = o[1] * f.ny + o[2] * f.ty;
  GL[0] = o[0];
  GL[1] = fx - o[3] * f.nx;
  GL[2] = fy - o[3] * f.ny;
  GR[0] = -o[0];
  GR[1] = -(fx - o[4] * f.nx);
  GR[2] = -(fy - o[4] * f.ny);
}

// a cell's primitive state in the edge's frame (fr: curvilinear, else the axis frame)
template <int NC>
__device__ __forceinline__ Prim prim_edge(const DevLevel& L, const double* c, int axis, const Frame* fr) {
  if constexpr (NC == 3) {
    if (fr) return to_frame(to_prim(c[0], c[1], c[2], L.h_eps), *fr);
  }
  return prim_axis<NC>(L, c, axis);
}

// One edge with conserved states cL / cR (NULL = boundary, ghost computed
// from the other side); returns G of both cells.  fr: the edge's frame on a
// curvilinear mesh, NULL on the uniform one.
template <int NC>
__device__ __forceinline__ void eval_edge_states(const DevLevel& L, int axis, const double* cL,
                                                 double zL, const double* cR, double zR,
                                                 double GL[NC], double GR[NC], const Frame* fr = nullptr) {
  Prim a, b;
  double za = zL, zb = zR;
  if (cL && cR) {
    a = prim_edge<NC>(L, cL, axis, fr);
    b = prim_edge<NC>(L, cR, axis, fr);
  } else if (cR) {
    b = prim_edge<NC>(L, cR, axis, fr);
    a = ghost_state(L, 2 * axis, b);
    za = zR;
  } else {
    a = prim_edge<NC>(L, cL, axis, fr);
    b = ghost_state(L, 2 * axis + 1, a);
    zb = zL;
  }
  double o[5];
  edge_eval(L, a, za, b, zb, o);
  if constexpr (NC == 3) {
    if (fr) {
      edge_G_frame(o, *fr, GL, GR);
      return;
    }
  }
  edge_G<NC>(o, axis, GL, GR);
}

// eval_edge_states with the cells' states held by reference and their
// presence as flags (no pointer to a local array, which would force it into
// local memory): the same operations
template <int NC>
__device__ __forceinline__ void eval_edge_flags(const DevLevel& L, int axis, bool hasL, const double (&cL)[NC],
                                                double zL, bool hasR, const double (&cR)[NC], double zR,
                                                double GL[NC], double GR[NC], const Frame* fr) {
  Prim a, b;
  double za = zL, zb = zR;
  if (hasL && hasR) {
    a = prim_edge<NC>(L, cL, axis, fr);
    b = prim_edge<NC>(L, cR, axis, fr);
  } else if (hasR) {
    b = prim_edge<NC>(L, cR, axis, fr);
    a = ghost_state(L, 2 * axis, b);
    za = zR;
  } else {
    a = prim_edge<NC>(L, cL, axis, fr);
    b = ghost_state(L, 2 * axis + 1, a);
    zb = zL;
  }
  double o[5];
  edge_eval(L, a, za, b, zb, o);
  if constexpr (NC == 3) {
    if (fr) {
      edge_G_frame(o, *fr, GL, GR);
      return;
    }
  }
  edge_G<NC>(o, axis, GL, GR);
}

// edge e -> (axis, left cell, right cell, |e|); -1 marks a boundary side
__device__ __forceinline__ void edge_cells(const DevLevel& L, int e, int n_xe, int& axis, int& iL,
                                           int& iR, double& len) {
  if (e < n_xe) {
    const int ie = e % (L.nx + 1), iy = e / (L.nx + 1);
    axis = 0;
    iL = ie > 0 ? (ie - 1) + L.nx * iy : -1;
    iR = ie < L.nx ? ie + L.nx * iy : -1;
    len = L.geo ? L.geo[e] : L.ex;
  } else {
    const int f = e - n_xe, ix = f % L.nx, je = f / L.nx;
    axis = 1;
    iL = je > 0 ? ix + L.nx * (je - 1) : -1;
    iR = je < L.ny ? ix + L.nx * je : -1;
    len = L.geo ? L.geo[e] : L.ey;
  }
}

// the frame of edge e on a curvilinear mesh (fr filled, returned), else NULL
template <int NC>
__device__ __forceinline__ const Frame* frame_of(const DevLevel& L, int e, int axis, Frame& fr) {
  if constexpr (NC == 3) {
    if (L.geo) {
      fr = edge_frame(L, e, axis);
      return &fr;
    }
  }
  return nullptr;
}

template <int NC>
__device__ __forceinline__ void load_c(const double* U, int n, int i, double c[NC]) {
  for (int s = 0; s < NC; ++s) c[s] = U[s * n + i];
}

template <typename T>
__device__ __forceinline__ void st(void* p, long long idx, double v) {
  static_cast<T*>(p)[idx] = static_cast<T>(v);
}

// ---- residual: per-edge G, then per-cell sums --------------------------------

template <int NC>
__device__ __forceinline__ void res_edge(const DevLevel& L, const double* __restrict__ z,
                                         const double* __restrict__ U, double* __restrict__ eb, int n_xe,
                                         int n_e, int e, long long es, int el) {
  int axis, iL, iR;
  double len;
  edge_cells(L, e, n_xe, axis, iL, iR, len);
  double cL[NC], cR[NC], GL[NC], GR[NC];
  if (iL >= 0) load_c<NC>(U, L.n, iL, cL);
  if (iR >= 0) load_c<NC>(U, L.n, iR, cR);
  Frame fr;
  const Frame* pf = frame_of<NC>(L, e, axis, fr);
  eval_edge_states<NC>(L, axis, iL >= 0 ? cL : nullptr, iL >= 0 ? z[iL] : 0.0,
                       iR >= 0 ? cR : nullptr, iR >= 0 ? z[iR] : 0.0, GL, GR, pf);
  for (int s = 0; s < NC; ++s) {
    eb[s * es + el] = GL[s];
    eb[(NC + s) * es + el] = GR[s];
  }
}

template <int NC>
__global__ void k_res_edges(DevLevel L, const double* __restrict__ z, const double* __restrict__ U,
                            double* __restrict__ eb, int n_xe, int n_e) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n_e) res_edge<NC>(L, z, U, eb, n_xe, n_e, e, n_e, e);
}

// cell edges: W (x-edge, cell on the right), E (x-edge, left), S, N
__device__ __forceinline__ void cell_edges(const DevLevel& L, int i, int n_xe, int& eW, int& eE,
                                           int& eS, int& eN) {
  const int ix = i % L.nx, iy = i / L.nx;
  eW = ix + (L.nx + 1) * iy;
  eE = eW + 1;
  eS = n_xe + ix + L.nx * iy;
  eN = eS + L.nx;
}

// R_i = sum over W, E, S, N of |e| G (eq. Res), ||R_i||_1
// (a non-finite cell state makes ||R_i||_1 NaN, so that the sums report it:
// the reconstruction's max(0, .) would otherwise hide a NaN depth)
// Remark 2.6: an off-diagonal Jacobian entry of a time step is (1 - beta) x
__device__ __forceinline__ double time_scale(const DevLevel& L, double v) {
  return L.t_ka > 0.0 ? L.t_omb * v : v;
}

// |K_i|/dt of a time step: one value on the uniform mesh, per cell on a curvilinear one
__device__ __forceinline__ double tka(const DevLevel& L, long long i) { return L.t_kai ? L.t_kai[i] : L.t_ka; }

// |e| of a cell's W/E (x) or S/N (y) edge e
__device__ __forceinline__ double elen(const DevLevel& L, int e, int axis) {
  return L.geo ? L.geo[e] : (axis == 0 ? L.ex : L.ey);
}

// Remark 2.6: the time-step residual of cell i from its flux sum r
template <int NC>
__device__ __forceinline__ void time_residual(const DevLevel& L, const double* __restrict__ U, int i,
                                              double r[NC]) {
  const long long n = L.n;
  for (int s = 0; s < NC; ++s) r[s] = (L.t_omb * r[s] + tka(L, i) * U[s * n + i]) - L.t_src[s * n + i];
}

// eb holds the edge pieces at eb[f * es + b], b in the edge numbering of
// (bW, bE, bS, bN): the global one for the edge buffer, a tile's own for the
// fused kernels
template <int NC>
__device__ __forceinline__ void res_cell(const DevLevel& L, const double* __restrict__ eb,
                                         const double* __restrict__ U, double* __restrict__ R,
                                         double* __restrict__ rn, int n_xe, int n_e, int i, long long es,
                                         int bW, int bE, int bS, int bN) {
  int eW, eE, eS, eN;
  cell_edges(L, i, n_xe, eW, eE, eS, eN);
  const double lW = elen(L, eW, 0), lE = elen(L, eE, 0);
  const double lS = L.dim == 2 ? elen(L, eS, 1) : 0.0, lN = L.dim == 2 ? elen(L, eN, 1) : 0.0;
  double r[NC];
  for (int s = 0; s < NC; ++s) {
    double a = 0.0;
    a = a + lW * eb[(NC + s) * es + bW];
    a = a + lE * eb[s * es + bE];
    if (L.dim == 2) {
      a = a + lS * eb[(NC + s) * es + bS];
      a = a + lN * eb[s * es + bN];
    }
    r[s] = a;
  }
  if (L.t_ka > 0.0) time_residual<NC>(L, U, i, r);
  for (int s = 0; s < NC; ++s) R[s * (long long)L.n + i] = r[s];
  double m = fabs(r[0]) + fabs(r[1]);
  if (NC == 3) m = m + fabs(r[NC - 1]);
  bool fin = true;
  for (int s = 0; s < NC; ++s) fin = fin && isfinite(U[(long long)s * L.n + i]);
  if (rn) rn[i] = fin ? m : __longlong_as_double(0x7ff8000000000000LL);
}

template <int NC>
__global__ void k_res_cells(DevLevel L, const double* __restrict__ eb, const double* __restrict__ U,
                            double* __restrict__ R, double* __restrict__ rn, int n_xe, int n_e) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < L.n) {
    int eW, eE, eS, eN;
    cell_edges(L, i, n_xe, eW, eE, eS, eN);
    res_cell<NC>(L, eb, U, R, rn, n_xe, n_e, i, n_e, eW, eE, eS, eN);
  }
}

// ---- finite-difference Jacobian ---------------------------------------------
// Edge buffer fields (each n_e long): GL[NC], GR[NC], dLL[NC*NC], dRR[NC*NC],
// where dLL = |e| (G_L(U_L + eps e_k) - G_L(U)) / eps is the left cell's
// diagonal contribution (ghost recomputed on boundary edges); the
// off-diagonal blocks go straight to the level's block arrays.

template <int NC, typename T>
__device__ __forceinline__ void jac_edge(const DevLevel& L, const double* __restrict__ z,
                                         const double* __restrict__ U, double* __restrict__ eb,
                                         void* __restrict__ blk, int n_xe, int n_e, int e, long long es,
                                         int el) {
  int axis, iL, iR;
  double len;
  edge_cells(L, e, n_xe, axis, iL, iR, len);
  const long long P = skew_slots(L.nx, L.ny);
  const long long sL = iL >= 0 ? skew_pos(iL % L.nx, iL / L.nx, L.nx) : 0;
  const long long sR = iR >= 0 ? skew_pos(iR % L.nx, iR / L.nx, L.nx) : 0;
  double cL[NC], cR[NC], GLb[NC], GRb[NC], GL[NC], GR[NC];
  const bool hL = iL >= 0, hR = iR >= 0;
  for (int s = 0; s < NC; ++s) {
    cL[s] = hL ? U[s * (long long)L.n + iL] : 0.0;
    cR[s] = hR ? U[s * (long long)L.n + iR] : 0.0;
  }
  const double zL = hL ? z[iL] : 0.0, zR = hR ? z[iR] : 0.0;
  Frame fr;
  const Frame* pf = frame_of<NC>(L, e, axis, fr);
  eval_edge_flags<NC>(L, axis, hL, cL, zL, hR, cR, zR, GLb, GRb, pf);
  for (int s = 0; s < NC; ++s) {
    eb[s * es + el] = GLb[s];
    eb[(NC + s) * es + el] = GRb[s];
  }
  const int f_dLL = 2 * NC, f_dRR = 2 * NC + NC * NC;
  const int bR = axis == 0 ? 1 : 3;   // block of the right cell pointing left (W / S)
  const int bL = axis == 0 ? 2 : 4;   // block of the left cell pointing right (E / N)
  // perturb the left cell
  for (int k = 0; k < NC; ++k) {
    if (iL >= 0) {
      double c[NC];
      for (int s = 0; s < NC; ++s) c[s] = (s == k) ? cL[s] + L.eps : cL[s];
      eval_edge_flags<NC>(L, axis, true, c, zL, hR, cR, zR, GL, GR, pf);
      for (int s = 0; s < NC; ++s) {
        eb[(f_dLL + s * NC + k) * es + el] = len * ((GL[s] - GLb[s]) * L.reps);
        if (iR >= 0) st<T>(blk, ((long long)(bR * NC * NC + s * NC + k)) * P + sR,
                           time_scale(L, len * ((GR[s] - GRb[s]) * L.reps)));
      }
    } else {
      for (int s = 0; s < NC; ++s) {
        eb[(f_dLL + s * NC + k) * es + el] = 0.0;
        st<T>(blk, ((long long)(bR * NC * NC + s * NC + k)) * P + sR, 0.0);
      }
    }
  }
  // perturb the right cell
  for (int k = 0; k < NC; ++k) {
    if (iR >= 0) {
      double c[NC];
      for (int s = 0; s < NC; ++s) c[s] = (s == k) ? cR[s] + L.eps : cR[s];
      eval_edge_flags<NC>(L, axis, hL, cL, zL, true, c, zR, GL, GR, pf);
      for (int s = 0; s < NC; ++s) {
        eb[(f_dRR + s * NC + k) * es + el] = len * ((GR[s] - GRb[s]) * L.reps);
        if (iL >= 0) st<T>(blk, ((long long)(bL * NC * NC + s * NC + k)) * P + sL,
                           time_scale(L, len * ((GL[s] - GLb[s]) * L.reps)));
      }
    } else {
      for (int s = 0; s < NC; ++s) {
        eb[(f_dRR + s * NC + k) * es + el] = 0.0;
        st<T>(blk, ((long long)(bL * NC * NC + s * NC + k)) * P + sL, 0.0);
      }
    }
  }
}

template <int NC, typename T>
__global__ void k_jac_edges(DevLevel L, const double* __restrict__ z, const double* __restrict__ U,
                            double* __restrict__ eb, void* __restrict__ blk, int n_xe, int n_e) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n_e) jac_edge<NC, T>(L, z, U, eb, blk, n_xe, n_e, e, n_e, e);
}

// Diagonal block D_i = sum_{W,E,S,N} dG + alpha ||R_i||_1 I (eq. NewtonREG),
// residual and its norm.  1D cells have only W and E.
template <int NC, typename T>
__device__ __forceinline__ void jac_cell(const DevLevel& L, const double* __restrict__ eb,
                                         const double* __restrict__ U, double* __restrict__ R,
                                         double* __restrict__ rn, void* __restrict__ blk, int n_xe, int n_e,
                                         int i, long long es, int bW, int bE, int bS, int bN) {
  int eW, eE, eS, eN;
  cell_edges(L, i, n_xe, eW, eE, eS, eN);
  const long long n = L.n, P = skew_slots(L.nx, L.ny);
  const long long si = skew_pos(i % L.nx, i / L.nx, L.nx);
  const double lW = elen(L, eW, 0), lE = elen(L, eE, 0);
  const double lS = L.dim == 2 ? elen(L, eS, 1) : 0.0, lN = L.dim == 2 ? elen(L, eN, 1) : 0.0;
  double r[NC];
  for (int s = 0; s < NC; ++s) {
    double a = 0.0;
    a = a + lW * eb[(NC + s) * es + bW];
    a = a + lE * eb[s * es + bE];
    if (L.dim == 2) {
      a = a + lS * eb[(NC + s) * es + bS];
      a = a + lN * eb[s * es + bN];
    }
    r[s] = a;
  }
  const bool tm = L.t_ka > 0.0;   // time step: scaled blocks, |K|/dt on the diagonal
  if (tm) time_residual<NC>(L, U, i, r);
  for (int s = 0; s < NC; ++s) R[s * n + i] = r[s];
  double m = fabs(r[0]) + fabs(r[1]);
  if (NC == 3) m = m + fabs(r[NC - 1]);
  if (rn) rn[i] = m;
  const int f_dLL = 2 * NC, f_dRR = 2 * NC + NC * NC;
  const double am = L.alpha * m;
  for (int s = 0; s < NC; ++s)
    for (int k = 0; k < NC; ++k) {
      const int f = s * NC + k;
      double d = 0.0;
      d = d + eb[(f_dRR + f) * es + bW];
      d = d + eb[(f_dLL + f) * es + bE];
      if (L.dim == 2) {
        d = d + eb[(f_dRR + f) * es + bS];
        d = d + eb[(f_dLL + f) * es + bN];
      }
      if (tm) {
        d = L.t_omb * d;
        if (s == k) d = d + tka(L, i);
      }
      if (s == k) d = d + am;
      st<T>(blk, (long long)f * P + si, d);
    }
}

template <int NC, typename T>
__global__ void k_jac_cells(DevLevel L, const double* __restrict__ eb, const double* __restrict__ U,
                            double* __restrict__ R, double* __restrict__ rn, void* __restrict__ blk, int n_xe,
                            int n_e) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < L.n) {
    int eW, eE, eS, eN;
    cell_edges(L, i, n_xe, eW, eE, eS, eN);
    jac_cell<NC, T>(L, eb, U, R, rn, blk, n_xe, n_e, i, n_e, eW, eE, eS, eN);
  }
}

// ---- fused residual and Jacobian: one CTA per tile of TX x TY cells (2D) ---
// The tile's edges (its cells' own and the ones on its border, which the
// neighbouring tile evaluates as well) are evaluated into shared memory by
// res_edge / jac_edge, then every cell sums its sides from there by
// res_cell / jac_cell: the same operations in the same order as the two-pass
// kernels above, without the per-edge pieces going through HBM.  Tile edge
// numbering: the x-edges, TX + 1 per tile row, then the y-edges, TX per
// edge row.  A CTA has NT >= TX * TY threads, so that the tile's edges take
// two rounds (552 edges on 288 threads for 32 x 8 cells) instead of two and
// a small third.  The Jacobian's off-diagonal blocks go straight to the level's
// block arrays; a border edge's blocks are written by both tiles with the
// same bits.
template <int TX, int TY>
__device__ __forceinline__ bool tile_edge(const DevLevel& L, int n_xe, int x0, int y0, int le, int& e) {
  constexpr int NXE = (TX + 1) * TY;
  if (le < NXE) {
    const int gx = x0 + le % (TX + 1), gy = y0 + le / (TX + 1);
    if (gx > L.nx || gy >= L.ny) return false;
    e = gx + (L.nx + 1) * gy;
    return true;
  }
  const int l2 = le - NXE;
  const int gx = x0 + l2 % TX, gy = y0 + l2 / TX;
  if (gx >= L.nx || gy > L.ny) return false;
  e = n_xe + gx + L.nx * gy;
  return true;
}

template <int TX, int TY>
constexpr int tile_edges() { return (TX + 1) * TY + TX * (TY + 1); }

template <int NC, int TX, int TY, int NT>
__global__ void __launch_bounds__(NT) k_res_tile(DevLevel L, const double* __restrict__ z,
                                                      const double* __restrict__ U, double* __restrict__ R,
                                                      double* __restrict__ rn, int n_xe, int n_e) {
  constexpr int NXE = (TX + 1) * TY, NE = tile_edges<TX, TY>();
  __shared__ double eb[2 * NC * NE];
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  for (int le = threadIdx.x; le < NE; le += NT) {
    int e;
    if (tile_edge<TX, TY>(L, n_xe, x0, y0, le, e)) res_edge<NC>(L, z, U, eb, n_xe, n_e, e, NE, le);
  }
  __syncthreads();
  const int lx = threadIdx.x % TX, ly = threadIdx.x / TX;
  const int gx = x0 + lx, gy = y0 + ly;
  if (ly < TY && gx < L.nx && gy < L.ny) {
    const int bW = lx + (TX + 1) * ly, bS = NXE + lx + TX * ly;
    res_cell<NC>(L, eb, U, R, rn, n_xe, n_e, gx + L.nx * gy, NE, bW, bW + 1, bS, bS + TX);
  }
}

template <int NC, typename T, int TX, int TY, int NT>
__global__ void __launch_bounds__(NT) k_jac_tile(DevLevel L, const double* __restrict__ z,
                                                      const double* __restrict__ U, double* __restrict__ R,
                                                      double* __restrict__ rn, void* __restrict__ blk, int n_xe,
                                                      int n_e) {
  constexpr int NXE = (TX + 1) * TY, NE = tile_edges<TX, TY>();
  extern __shared__ double ebj[];   // (2 NC + 2 NC^2) fields x NE edges
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  for (int le = threadIdx.x; le < NE; le += NT) {
    int e;
    if (tile_edge<TX, TY>(L, n_xe, x0, y0, le, e)) jac_edge<NC, T>(L, z, U, ebj, blk, n_xe, n_e, e, NE, le);
  }
  __syncthreads();
  const int lx = threadIdx.x % TX, ly = threadIdx.x / TX;
  const int gx = x0 + lx, gy = y0 + ly;
  if (ly < TY && gx < L.nx && gy < L.ny) {
    const int bW = lx + (TX + 1) * ly, bS = NXE + lx + TX * ly;
    jac_cell<NC, T>(L, ebj, U, R, rn, blk, n_xe, n_e, gx + L.nx * gy, NE, bW, bW + 1, bS, bS + TX);
  }
}

// ---- block solve with the same elimination as the reference definition -----
// Gaussian elimination with partial pivoting (largest |entry|, lowest row on
// ties); a pivot <= 1e-14 max|D| marks its unknown singular (correction 0).
// Every index is a compile-time constant (row swaps and the permutation are
// selections), so the block stays in registers; the arithmetic is the
// elimination's, operation by operation.
template <int NC>
__device__ __forceinline__ void small_solve(double m[NC * NC], const double b[NC], double x[NC]) {
  // max |entry|, NaN entries counting as 0 (as in a running "if (a > amax)
  // amax = a" from 0).  The bit patterns of non-negative doubles order like
  // their values, so the maximum is taken on the integer pipe: |x| is x's
  // pattern without the sign bit, and a NaN (pattern above infinity's) is
  // replaced by 0.  The result is the same double, without a chain of FP64
  // comparisons on the cell update's critical path.
  unsigned long long amax_bits = 0ull;
#pragma unroll
  for (int e = 0; e < NC * NC; ++e) {
    unsigned long long u = (unsigned long long)__double_as_longlong(m[e]) & 0x7fffffffffffffffull;
    u = (u > 0x7ff0000000000000ull) ? 0ull : u;
    amax_bits = (u > amax_bits) ? u : amax_bits;
  }
  const double amax = __longlong_as_double((long long)amax_bits);
  const double tiny = 1e-14 * amax;
  int perm[NC];
  bool sing[NC];
#pragma unroll
  for (int r = 0; r < NC; ++r) { perm[r] = r; sing[r] = false; }
#pragma unroll
  for (int col = 0; col < NC; ++col) {
    // the pivot row: "if (|a| > best)" over the rows below, compared on the
    // magnitudes' bit patterns (a NaN on either side compares false, as in
    // FP64); kb ends as the pattern of the chosen entry's magnitude
    int p = col;
    unsigned long long kb = (unsigned long long)__double_as_longlong(m[col * NC + col]) & 0x7fffffffffffffffull;
#pragma unroll
    for (int r = col + 1; r < NC; ++r) {
      const unsigned long long ka =
          (unsigned long long)__double_as_longlong(m[r * NC + col]) & 0x7fffffffffffffffull;
      if (ka <= 0x7ff0000000000000ull && kb <= 0x7ff0000000000000ull && ka > kb) { kb = ka; p = r; }
    }
#pragma unroll
    for (int r = col + 1; r < NC; ++r)
      if (r == p) {
#pragma unroll
        for (int k = 0; k < NC; ++k) {
          const double t = m[col * NC + k];
          m[col * NC + k] = m[r * NC + k];
          m[r * NC + k] = t;
        }
        const int t = perm[col]; perm[col] = perm[r]; perm[r] = t;
      }
    if (!(kb > (unsigned long long)dbits(tiny) && kb <= (unsigned long long)kInfBits)) {   // !(best > tiny), tiny >= +0
      sing[col] = true;
#pragma unroll
      for (int r = col + 1; r < NC; ++r) m[r * NC + col] = 0.0;
    } else {
#pragma unroll
      for (int r = col + 1; r < NC; ++r) {
        const double l = m[r * NC + col] / m[col * NC + col];
        m[r * NC + col] = l;
#pragma unroll
        for (int k = col + 1; k < NC; ++k) m[r * NC + k] = m[r * NC + k] - l * m[col * NC + k];
      }
    }
  }
  double y[NC];
#pragma unroll
  for (int r = 0; r < NC; ++r) {
    double v = b[0];
#pragma unroll
    for (int k = 1; k < NC; ++k)
      if (perm[r] == k) v = b[k];
    y[r] = v;
  }
#pragma unroll
  for (int r = 0; r < NC; ++r)
#pragma unroll
    for (int k = 0; k < r; ++k) y[r] = y[r] - m[r * NC + k] * y[k];
#pragma unroll
  for (int r = NC - 1; r >= 0; --r) {
    double s = y[r];
#pragma unroll
    for (int k = r + 1; k < NC; ++k) s = s - m[r * NC + k] * x[k];
    x[r] = sing[r] ? 0.0 : s / m[r * NC + r];
  }
}

// ---- BLU-SGS: one anti-diagonal of the lexicographic sweep ------------------
// Cells with ix + iy = d depend only on diagonal d-1 (new values) and d+1
// (old values), so updating one diagonal at a time in increasing (forward)
// or decreasing (backward) order reproduces the lexicographic sweep exactly
// (the whole sweep runs in one cooperative launch, k_blusgs_sweep below).
// Each cell has a group of lanes, one per (side, perturbation p): p = 0
// evaluates the side's G at U_i, p = k+1 at U_i + eps e_k.  All lanes run the
// same edge evaluation (the cell is put on the edge's left or right by
// selection, not by branching); the p = 0 lane of a side shares 1/h_i and the
// neighbour's velocities with its perturbation lanes (the same values they
// would compute).  The group's first lane sums the sides in W, E, S, N order
// and updates U_i -= (alpha||R_i||_1 I + dR_i/dU_i)^{-1} R_i.
template <bool L2>
__device__ __forceinline__ double ldU(const double* p) { return L2 ? __ldcg(p) : *p; }

// The cell's primitive state along `axis` in perturbation p (p = k + 1 adds
// eps to component k); rinv = 1/h of the unperturbed cell (0 when dry).
// 1/h is recomputed only when the depth is the perturbed component.
template <int NC>
__device__ __forceinline__ Prim pert_prim(const DevLevel& L, const double c[NC], int p, double rinv, int axis,
                                          const Frame* fr = nullptr) {
  if constexpr (NC == 3) {
    if (fr) {   // curvilinear: global velocities, then the edge frame
      Prim gl;
      gl.h = c[0];
      if (ge_pos(c[0], L.h_eps)) {
        const double r = (p == 1) ? 1.0 / c[0] : rinv;
        gl.u = c[1] * r;
        gl.v = c[2] * r;
      } else {
        gl.u = 0.0;
        gl.v = 0.0;
      }
      return to_frame(gl, *fr);
    }
  }
  Prim me;
  me.h = c[0];
  const double qa = (NC == 2) ? c[1] : (axis == 0 ? c[1] : c[NC - 1]);
  const double qb = (NC == 2) ? 0.0 : (axis == 0 ? c[NC - 1] : c[1]);
  if (ge_pos(c[0], L.h_eps)) {
    const double r = (p == 1) ? 1.0 / c[0] : rinv;
    me.u = qa * r;
    me.v = qb * r;
  } else {
    me.u = 0.0;
    me.v = 0.0;
  }
  return me;
}

// edge of side sd (0 W, 1 E, 2 S, 3 N) of cell (ix, iy), in edge_cells' numbering
__device__ __forceinline__ int side_edge(const DevLevel& L, int ix, int iy, int sd) {
  const int n_xe = (L.nx + 1) * L.ny;
  switch (sd) {
    case 0: return ix + (L.nx + 1) * iy;
    case 1: return ix + 1 + (L.nx + 1) * iy;
    case 2: return n_xe + ix + L.nx * iy;
    default: return n_xe + ix + L.nx * (iy + 1);
  }
}

// Ghost states of every boundary cell of a level for the base state and each
// perturbation, before a BLU-SGS half-sweep: a cell's state does not change
// until its own update, so its ghosts are the ones the sweep would compute
// (the inflow ghost's cubic solve then leaves the per-diagonal critical
// path).  gbuf[((side * glen + k) * NP + p) * 3 + {h, u, v}], k the position
// along the side, glen = max(nx, ny).
template <int NC, int NS>
__device__ __forceinline__ void ghost_prologue(const DevLevel& L, const double* U, double* gbuf, int tid,
                                               int nthreads) {
  constexpr int NP = NC + 1;
  const long long n = L.n;
  const int glen = L.nx > L.ny ? L.nx : L.ny;
  const int total = NS * glen * NP;
  for (int t = tid; t < total; t += nthreads) {
    const int p = t % NP, k = (t / NP) % glen, sd = t / (NP * glen);
    if (k >= (sd < 2 ? L.ny : L.nx)) continue;
    const int ix = sd == 0 ? 0 : (sd == 1 ? L.nx - 1 : k);
    const int iy = sd < 2 ? k : (sd == 2 ? 0 : L.ny - 1);
    const int i = ix + L.nx * iy;
    double c[NC];
    for (int s = 0; s < NC; ++s) c[s] = __ldcg(&U[s * n + i]);
    const double rinv = ge_pos(c[0], L.h_eps) ? 1.0 / c[0] : 0.0;
    if (p > 0) c[p - 1] = c[p - 1] + L.eps;
    Frame fr;
    const Frame* pf = frame_of<NC>(L, side_edge(L, ix, iy, sd), sd >> 1, fr);
    const Prim gh = ghost_state(L, sd, pert_prim<NC>(L, c, p, rinv, sd >> 1, pf));
    gbuf[(long long)t * 3 + 0] = gh.h;
    gbuf[(long long)t * 3 + 1] = gh.u;
    gbuf[(long long)t * 3 + 2] = gh.v;
  }
}

// One cell group of a BLU-SGS diagonal.  With L2 = true the state is read
// through L2 only (the persistent sweep, where other SMs update it during the
// launch).  All 32 lanes of the warp must call it together.
template <int NC, int NS, int GRP, bool L2>
__device__ __forceinline__ void blusgs_group(const DevLevel& L, const double* __restrict__ z,
                                             double* U, const double* gbuf, int d, int ix0, int ncell,
                                             int cell, int g) {
  constexpr int NP = NC + 1;                 // perturbations incl. the base
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int side = g / NP, p = g % NP;
  const int gbase = lane - g;                // first lane of the cell's group
  const bool cell_ok = cell < ncell;
  const bool act = cell_ok && side < NS;
  const int ix = ix0 + (cell_ok ? cell : 0), iy = d - ix;
  const int i = ix + L.nx * iy;
  const long long n = L.n;
  const int sd = side < NS ? side : 0;
  const int axis = sd >> 1, upper = sd & 1;
  int j = -1;
  if (act) {
    if (sd == 0 && ix > 0) j = i - 1;
    if (sd == 1 && ix < L.nx - 1) j = i + 1;
    if (sd == 2 && iy > 0) j = i - L.nx;
    if (sd == 3 && iy < L.ny - 1) j = i + L.nx;
  }
  double ci[NC];
  for (int s = 0; s < NC; ++s) ci[s] = act ? ldU<L2>(&U[s * n + i]) : 0.0;
  const double zi = act ? z[i] : 0.0, zj = (j >= 0) ? z[j] : zi;
  const int eidx = L.dim == 2 ? side_edge(L, ix, iy, sd) : 0;   // a valid edge on every lane
  Frame fr;
  const Frame* pf = frame_of<NC>(L, eidx, axis, fr);
  // base lane: 1/h_i and the neighbour's primitive state
  double rinv = 0.0;
  Prim nb{0.0, 0.0, 0.0};
  if (act && p == 0) {
    if (ge_pos(ci[0], L.h_eps)) rinv = 1.0 / ci[0];
    if (j >= 0) {
      double cj[NC];
      for (int s = 0; s < NC; ++s) cj[s] = ldU<L2>(&U[s * n + j]);
      nb = prim_edge<NC>(L, cj, axis, pf);
    }
  }
  const int src0 = gbase + sd * NP;          // the side's p = 0 lane
  rinv = __shfl_sync(full, rinv, src0);
  nb.h = __shfl_sync(full, nb.h, src0);
  nb.u = __shfl_sync(full, nb.u, src0);
  nb.v = __shfl_sync(full, nb.v, src0);
  double G[NC];
  for (int s = 0; s < NC; ++s) G[s] = 0.0;
  if (act) {
    double c[NC];
    for (int s = 0; s < NC; ++s) c[s] = ci[s];
    if (p > 0) c[p - 1] = c[p - 1] + L.eps;
    const Prim me = pert_prim<NC>(L, c, p, rinv, axis, pf);
    Prim other = nb;
    if (j < 0) {
      if (gbuf) {   // precomputed by ghost_prologue
        const int glen = L.nx > L.ny ? L.nx : L.ny;
        const long long t = ((long long)(sd * glen + (sd < 2 ? iy : ix)) * NP + p) * 3;
        other.h = __ldcg(&gbuf[t]);
        other.u = __ldcg(&gbuf[t + 1]);
        other.v = __ldcg(&gbuf[t + 2]);
      } else {
        other = ghost_state(L, sd, me);
      }
    }
    const double zo = (j >= 0) ? zj : zi;
    const Prim a = upper ? me : other, b = upper ? other : me;
    const double za = upper ? zi : zo, zb = upper ? zo : zi;
    double o[5], GL[NC], GR[NC];
    edge_eval(L, a, za, b, zb, o);
    bool done = false;
    if constexpr (NC == 3) {
      if (pf) {
        edge_G_frame(o, *pf, GL, GR);
        done = true;
      }
    }
    if (!done) edge_G<NC>(o, axis, GL, GR);
    for (int s = 0; s < NC; ++s) G[s] = upper ? GL[s] : GR[s];
  }
  // p = 0 lanes hold |e| G; p = k+1 lanes column k of |e| dG/dU_i
  const double len = L.dim == 2 ? elen(L, eidx, axis) : L.ex;
  double v[NC];
  for (int s = 0; s < NC; ++s) {
    const double gb = __shfl_sync(full, G[s], src0);
    v[s] = (p == 0) ? len * G[s] : len * ((G[s] - gb) * L.reps);
  }
  // Sum over the sides, lane-parallel: lane g < NC*NP of the group owns
  // entry (s, pp) = (g / NP, g % NP) and adds the sides' values in the order
  // W, E, S, N (the same additions, in the same order, as one lane summing
  // every entry), then the group's first lane collects the NC*NP sums.
  const int es = g / NP < NC ? g / NP : 0, ep = g % NP;
  double acc = 0.0;
  for (int q = 0; q < NS; ++q) {
    double w = 0.0;
#pragma unroll
    for (int s = 0; s < NC; ++s) {
      const double t = __shfl_sync(full, v[s], gbase + q * NP + ep);
      if (s == es) w = t;
    }
    acc = acc + w;
  }
  double Rs[NC], D[NC * NC];
#pragma unroll
  for (int s = 0; s < NC; ++s)
#pragma unroll
    for (int pp = 0; pp < NP; ++pp) {
      const double t = __shfl_sync(full, acc, gbase + s * NP + pp);
      if (pp == 0) Rs[s] = t;
      else D[s * NC + (pp - 1)] = t;
    }
  if (!cell_ok || g != 0) return;
  if (gt_zero(L.t_ka)) {   // time step (Remark 2.6): the step's residual and diagonal block
    const double ka = tka(L, i);
    for (int s = 0; s < NC; ++s) Rs[s] = (L.t_omb * Rs[s] + ka * ci[s]) - L.t_src[s * n + i];
    for (int e = 0; e < NC * NC; ++e) D[e] = L.t_omb * D[e];
    for (int s = 0; s < NC; ++s) D[s * NC + s] = D[s * NC + s] + ka;
  }
  double m = fabs(Rs[0]) + fabs(Rs[1]);
  if (NC == 3) m = m + fabs(Rs[NC - 1]);
  const double am = L.alpha * m;
  for (int s = 0; s < NC; ++s) D[s * NC + s] = D[s * NC + s] + am;
  double x[NC];
  small_solve<NC>(D, Rs, x);
  if (lt_pos(ci[0], L.h_eps))   // dry at the start: momentum stays zero (Remark 2.5)
    for (int s = 1; s < NC; ++s) x[s] = 0.0;
  double un[NC];
  for (int s = 0; s < NC; ++s) un[s] = ci[s] - x[s];
  if (lt_pos(un[0], L.h_eps))
    for (int s = 0; s < NC; ++s) un[s] = 0.0;
  for (int s = 0; s < NC; ++s) U[s * n + i] = un[s];
}

// ---- BLU-SGS: whole half-sweep in one cooperative launch -------------------
// Every block walks the anti-diagonals in sweep order; after a diagonal the
// blocks meet at a grid barrier (arrival counter, release/acquire), so the
// next diagonal sees the new values.  The barrier wait is bounded: on expiry
// the kernel sets the sticky error word and the abort flag, and every block
// leaves at its next barrier.  sync: [0] arrivals, [1] abort.
__device__ __forceinline__ int ld_acq(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Bounded grid barrier number q + 1 (all blocks co-resident): false when the
// wait ran out or another block gave up (the sticky error is then set).
__device__ __forceinline__ bool grid_barrier(int* sync, int q, int* sticky_err, int spin_limit) {
  __shared__ int s_go;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(&sync[0], 1);
    const int target = (q + 1) * gridDim.x;
    int ok = 0;
    for (int it = 0; it < spin_limit; ++it) {
      if (ld_acq(&sync[0]) >= target) { ok = 1; break; }
      if (ld_acq(&sync[1])) break;
      __nanosleep(20);
    }
    if (!ok) {
      if (!ld_acq(&sync[1])) atomicOr(sticky_err, 1);
      atomicExch(&sync[1], 1);
    }
    s_go = ok;
  }
  __syncthreads();
  return s_go != 0;
}

// gbuf: ghost scratch (ghost_prologue), 4 * max(nx, ny) * (NC + 1) * 3 doubles
template <int NC, int NS, int GRP>
__global__ void __launch_bounds__(128) k_blusgs_sweep(DevLevel L, const double* __restrict__ z,
                                                      double* U, double* gbuf, int forward, int* sync,
                                                      int* sticky_err, int spin_limit) {
  const int ndiag = L.nx + L.ny - 1;
  const int wpb = blockDim.x >> 5, warp = threadIdx.x >> 5;
  // warp-major numbering: consecutive cell pairs go to different SMs first,
  // so a short diagonal puts one warp per SM (GB300 issues about two FP64
  // operations per clock per SM; four warps of one SM would queue on it)
  const int gw = warp * gridDim.x + blockIdx.x, nw = gridDim.x * wpb;
  const int cpw = 32 / GRP;                     // cells per warp and round
  ghost_prologue<NC, NS>(L, U, gbuf, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
  if (!grid_barrier(sync, 0, sticky_err, spin_limit)) return;
  for (int q = 0; q < ndiag; ++q) {
    const int d = forward ? q : ndiag - 1 - q;
    const int ix0 = d - (L.ny - 1) > 0 ? d - (L.ny - 1) : 0;
    const int ix1 = d < L.nx - 1 ? d : L.nx - 1;
    const int ncell = ix1 - ix0 + 1;
    for (int c0 = gw * cpw; c0 < ncell; c0 += nw * cpw)   // warp-uniform loop
      blusgs_group<NC, NS, GRP, true>(L, z, U, gbuf, d, ix0, ncell, c0 + (threadIdx.x & 31) / GRP,
                                      (threadIdx.x & 31) % GRP);
    if (!grid_barrier(sync, q + 1, sticky_err, spin_limit)) return;
  }
}

// ---- BLU-SGS: strip-pipelined half-sweep ------------------------------------
// The same cell updates as k_blusgs_sweep, ordered by point-to-point waits
// instead of a grid barrier per anti-diagonal.  Strip q holds R = 32 / GRP
// consecutive rows, counted from the sweep's first row (the bottom row
// forward, the top row backward), and columns are counted from the sweep's
// first column.  At step t the strip's warp updates row r at column t - r,
// so the cells of a step lie on one anti-diagonal.  A cell's neighbours
// before it in the sweep order are then new values: inside the strip they
// were updated at step t - 1 by this warp, and the first row's neighbour is
// in the last row of strip q - 1, which this strip waits for (bounded) until
// that row has passed column t.  Its neighbours after it in the sweep order
// are still old values: they are updated later by this warp, or by strip
// q + 1, which waits for this strip's last row.  The lane that wrote the
// last row's cell publishes the progress with a release store after it (in
// a forward step that cell is cell 0, in a backward step the last cell).
// Strips are claimed in order through an atomic ticket, so a strip only
// waits for one that a running warp owns.  The ghosts come from
// k_ghost_prologue, launched before.
// sync: [0] ticket, [1] abort, [2 + q] columns completed by strip q's last row.
__device__ __forceinline__ void st_rel(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <int NC, int NS>
__global__ void __launch_bounds__(128) k_ghost_prologue(DevLevel L, const double* __restrict__ U,
                                                        double* gbuf) {
  ghost_prologue<NC, NS>(L, U, gbuf, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

template <int NC, int NS, int GRP>
__global__ void __launch_bounds__(32) k_blusgs_strip(DevLevel L, const double* __restrict__ z, double* U,
                                                     const double* gbuf, int forward, int* sync,
                                                     int* sticky_err, int spin_limit) {
  constexpr int R = 32 / GRP;
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int nstrips = (L.ny + R - 1) / R;
  int* prog = sync + 2;
  for (;;) {
    int q = 0;
    if (lane == 0) q = atomicAdd(&sync[0], 1);
    q = __shfl_sync(full, q, 0);
    if (q >= nstrips) return;
    const int rows = (L.ny - q * R < R) ? L.ny - q * R : R;
    const int nsteps = L.nx + rows - 1;
    int known = 0;
    for (int t = 0; t < nsteps; ++t) {
      if (q > 0 && t < L.nx && known < t + 1) {   // the previous strip's last row at column t
        int pg = 0, it = 0;
        do {
          if (lane == 0) {
            pg = ld_acq(&prog[q - 1]);
            if (pg < t + 1 && ld_acq(&sync[1])) pg = -1;
          }
          pg = __shfl_sync(full, pg, 0);
          if (pg >= t + 1 || pg < 0) break;
          __nanosleep(32);
        } while (++it < spin_limit);
        if (pg < t + 1) {
          if (lane == 0) {
            if (pg >= 0) atomicOr(sticky_err, 1);
            atomicExch(&sync[1], 1);
          }
          return;
        }
        known = pg;
      }
      __syncwarp();   // lane 0's acquire before the other lanes' loads of that row
      const int c_lo = t - rows + 1 > 0 ? t - rows + 1 : 0;
      const int c_hi = t < L.nx - 1 ? t : L.nx - 1;
      const int ncell = c_hi - c_lo + 1;
      int d, ix0;
      if (forward) {   // ix = c, iy = qR + (t - c)
        d = q * R + t;
        ix0 = c_lo;
      } else {         // ix = nx-1-c, iy = ny-1-qR-(t - c)
        d = (L.nx - 1) + (L.ny - 1) - (q * R + t);
        ix0 = L.nx - 1 - c_hi;
      }
      blusgs_group<NC, NS, GRP, true>(L, z, U, gbuf, d, ix0, ncell, lane / GRP, lane % GRP);
      __syncwarp();
      const int done = t - rows + 2;                  // columns completed by the last row
      if (q + 1 < nstrips && done >= 1 && done <= L.nx) {
        const int rel = forward ? 0 : (ncell - 1) * GRP;
        if (lane == rel) st_rel(&prog[q], done);
      }
    }
  }
}

// ---- BLU-SGS, strip-pipelined, 2D uniform mesh, flux fixed at compile time --
// The schedule of k_blusgs_strip (one warp per strip of R = 2 rows, 16 lanes
// per cell: side sd in W, E, S, N order times perturbation p = 0..3; strips
// claimed by ticket; bounded waits on the previous strip's published
// progress) and the same operations in the same order, so the sweeps are
// bit-identical.  What changes is how the operands reach the lanes:
//   * the two neighbours that are new in this sweep (the previous column and
//     the previous row) come in registers: the previous column is the group's
//     own last result, the previous row the result of the group below it in
//     the warp, by shuffle; only the strip's first row loads its previous-row
//     neighbour from global memory, after the progress wait;
//   * the cell's own state and the two neighbours that are still old (the
//     next column and row), the beds and the boundary ghosts do not change
//     before the cell's update, so they are loaded one step ahead, at the
//     start of the previous step (double-buffered), where the load latency
//     hides behind that step's flux and elimination;
//   * every lane computes its reciprocals itself (the same values a shared
//     lane would broadcast), the side sums go through shared memory, and the
//     perturbed component is chosen by selection, not by indexing.
template <int FX>
__global__ void __launch_bounds__(32) k_blusgs_lean(DevLevel L, const double* __restrict__ z, double* U,
                                                    const double* __restrict__ gbuf, int forward, int* sync,
                                                    int* sticky_err, int spin_limit) {
  constexpr int NC = 3, NP = 4, GRP = 16, R = 2;
  __shared__ double sv[R][GRP][NC];
  __shared__ double ss[R][GRP];
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int grp = lane / GRP, g = lane % GRP;
  const int sd = g / NP, p = g % NP;
  const int axis = sd >> 1, upper = sd & 1;
  // the side's role in this sweep: 0 previous column, 1 next column,
  // 2 previous row (new values), 3 next row (old values)
  const int role = forward ? sd : (sd ^ 1);
  const long long n = L.n;
  const int nstrips = (L.ny + R - 1) / R;
  const int glen = L.nx > L.ny ? L.nx : L.ny;
  const double len = axis == 0 ? L.ex : L.ey;
  const int src0 = lane - p;                 // the side's p = 0 lane
  int* prog = sync + 2;
  for (;;) {
    int q = 0;
    if (lane == 0) q = atomicAdd(&sync[0], 1);
    q = __shfl_sync(full, q, 0);
    if (q >= nstrips) return;
    const int rows = (L.ny - q * R < R) ? L.ny - q * R : R;
    const int nsteps = L.nx + rows - 1;
    const int rr = q * R + grp;              // this group's row, counted in sweep order
    const bool row_ok = grp < rows;
    const int iy = forward ? rr : L.ny - 1 - rr;
    const bool has_py = rr > 0, has_ny = rr < L.ny - 1;
    // operands of the group's cell (ci ...) and of its next one (n*), the
    // latter loaded during the current step
    double ci[NC], cj[NC], zi = 0.0, zj = 0.0;
    Prim gh{0.0, 0.0, 0.0};
    double nci[NC], ncj[NC], nzi = 0.0, nzj = 0.0;
    Prim ngh{0.0, 0.0, 0.0};
    for (int k = 0; k < NC; ++k) { ci[k] = cj[k] = nci[k] = ncj[k] = 0.0; }
    auto fetch = [&](int c) {
      const int ix = forward ? c : L.nx - 1 - c;
      const int i = ix + L.nx * iy;
      for (int k = 0; k < NC; ++k) nci[k] = __ldcg(&U[k * n + i]);
      nzi = z[i];
      const bool has = role == 0 ? c > 0 : role == 1 ? c < L.nx - 1 : role == 2 ? has_py : has_ny;
      int j = i;
      if (sd == 0) j = i - 1;
      else if (sd == 1) j = i + 1;
      else if (sd == 2) j = i - L.nx;
      else j = i + L.nx;
      if (has) {
        nzj = z[j];
        if (role == 1 || role == 3)
          for (int k = 0; k < NC; ++k) ncj[k] = __ldcg(&U[k * n + j]);
      } else {                               // precomputed by ghost_prologue
        const long long t3 = ((long long)(sd * glen + (sd < 2 ? iy : ix)) * NP + p) * 3;
        ngh.h = __ldcg(&gbuf[t3]);
        ngh.u = __ldcg(&gbuf[t3 + 1]);
        ngh.v = __ldcg(&gbuf[t3 + 2]);
      }
    };
    auto advance = [&]() {   // the next cell's operands become the current ones
      for (int k = 0; k < NC; ++k) { ci[k] = nci[k]; cj[k] = ncj[k]; }
      zi = nzi;
      zj = nzj;
      gh = ngh;
    };
    if (row_ok && grp == 0) {
      fetch(0);
      advance();
    }
    double prevx[NC] = {0.0, 0.0, 0.0};      // the group's last result (new)
    int known = 0;
    for (int t = 0; t < nsteps; ++t) {
      if (q > 0 && t < L.nx && known < t + 1) {   // the previous strip's last row at column t
        int pg = 0, it = 0;
        do {
          if (lane == 0) {
            pg = ld_acq(&prog[q - 1]);
            if (pg < t + 1 && ld_acq(&sync[1])) pg = -1;
          }
          pg = __shfl_sync(full, pg, 0);
          if (pg >= t + 1 || pg < 0) break;
          __nanosleep(32);
        } while (++it < spin_limit);
        if (pg < t + 1) {
          if (lane == 0) {
            if (pg >= 0) atomicOr(sticky_err, 1);
            atomicExch(&sync[1], 1);
          }
          return;
        }
        known = pg;
      }
      __syncwarp();   // lane 0's acquire before the other lanes' loads of that row
      const int c = t - grp;
      const bool act = row_ok && c >= 0 && c < L.nx;
      const int ix = forward ? c : L.nx - 1 - c;
      const int i = ix + L.nx * iy;
      // operands of the next cell (its own state is still old: nobody else
      // writes it before this group's next step)
      const bool next_ok = row_ok && c + 1 >= 0 && c + 1 < L.nx;
      if (next_ok) fetch(c + 1);
      // the previous row's new values: the group below, or the previous strip
      double py[NC];
      for (int k = 0; k < NC; ++k) py[k] = __shfl_up_sync(full, prevx[k], GRP);
      double G[NC] = {0.0, 0.0, 0.0};
      if (act) {
        const bool has = role == 0 ? c > 0 : role == 1 ? c < L.nx - 1 : role == 2 ? has_py : has_ny;
        double cn[NC];
        for (int k = 0; k < NC; ++k) cn[k] = role == 0 ? prevx[k] : cj[k];
        if (role == 2 && has) {
          if (grp > 0) {
            for (int k = 0; k < NC; ++k) cn[k] = py[k];
          } else {
            const int j = forward ? i - L.nx : i + L.nx;
            for (int k = 0; k < NC; ++k) cn[k] = __ldcg(&U[k * n + j]);
          }
        }
        // this lane's perturbation of the cell (component p - 1 by eps)
        double cp[NC];
        for (int k = 0; k < NC; ++k) cp[k] = (k == p - 1) ? ci[k] + L.eps : ci[k];
        Prim me;
        me.h = cp[0];
        const double qa = axis == 0 ? cp[1] : cp[2], qb = axis == 0 ? cp[2] : cp[1];
        if (ge_pos(cp[0], L.h_eps)) {
          const double r = 1.0 / cp[0];
          me.u = qa * r;
          me.v = qb * r;
        } else {
          me.u = 0.0;
          me.v = 0.0;
        }
        const Prim other = has ? to_prim(cn[0], axis == 0 ? cn[1] : cn[2], axis == 0 ? cn[2] : cn[1], L.h_eps) : gh;
        const double zo = has ? zj : zi;
        const Prim a = upper ? me : other, b = upper ? other : me;
        const double za = upper ? zi : zo, zb = upper ? zo : zi;
        double o[5], GL[NC], GR[NC];
        edge_eval_t<FX>(L, a, za, b, zb, o);
        edge_G<NC>(o, axis, GL, GR);
        for (int k = 0; k < NC; ++k) G[k] = upper ? GL[k] : GR[k];
      }
      // p = 0 lanes hold |e| G, p = k+1 lanes column k of |e| dG/dU_i
      for (int k = 0; k < NC; ++k) {
        const double gb = __shfl_sync(full, G[k], src0);
        sv[grp][g][k] = len * ((p == 0) ? G[k] : (G[k] - gb) * L.reps);   // |e| G, or |e| (G - G_0) / eps
      }
      __syncwarp();
      if (g < NC * NP) {   // entry (component g / NP, perturbation g % NP): sides in W, E, S, N order
        const int es = g / NP, ep = g % NP;
        double acc = 0.0;
        for (int qs = 0; qs < 4; ++qs) acc = acc + sv[grp][qs * NP + ep][es];
        ss[grp][g] = acc;
      }
      __syncwarp();
      double un[NC] = {0.0, 0.0, 0.0};
      if (act && g == 0) {
        double Rs[NC], D[NC * NC];
        for (int k = 0; k < NC; ++k) {
          Rs[k] = ss[grp][k * NP];
          for (int pp = 1; pp < NP; ++pp) D[k * NC + (pp - 1)] = ss[grp][k * NP + pp];
        }
        if (gt_zero(L.t_ka)) {   // time step (Remark 2.6): the step's residual and diagonal block
          const double ka = tka(L, i);
          for (int k = 0; k < NC; ++k) Rs[k] = (L.t_omb * Rs[k] + ka * ci[k]) - L.t_src[k * n + i];
          for (int e = 0; e < NC * NC; ++e) D[e] = L.t_omb * D[e];
          for (int k = 0; k < NC; ++k) D[k * NC + k] = D[k * NC + k] + ka;
        }
        double m = fabs(Rs[0]) + fabs(Rs[1]);
        m = m + fabs(Rs[2]);
        const double am = L.alpha * m;
        for (int k = 0; k < NC; ++k) D[k * NC + k] = D[k * NC + k] + am;
        double x[NC];
        small_solve<NC>(D, Rs, x);
        if (lt_pos(ci[0], L.h_eps))   // dry at the start: momentum stays zero (Remark 2.5)
          for (int k = 1; k < NC; ++k) x[k] = 0.0;
        for (int k = 0; k < NC; ++k) un[k] = ci[k] - x[k];
        if (lt_pos(un[0], L.h_eps))
          for (int k = 0; k < NC; ++k) un[k] = 0.0;
        for (int k = 0; k < NC; ++k) U[k * n + i] = un[k];
      }
      for (int k = 0; k < NC; ++k) {
        const double v = __shfl_sync(full, un[k], grp * GRP);
        if (act) prevx[k] = v;
      }
      if (next_ok) advance();
      const int done = t - rows + 2;                  // columns completed by the last row
      if (q + 1 < nstrips && done >= 1 && done <= L.nx && lane == (rows - 1) * GRP)
        st_rel(&prog[q], done);   // orders this lane's store of the last row's cell
    }
  }
}

// ---- BLU-SGS with the edge flux split between two warps (LLF, 2D uniform) ---
// The LLF flux of eq. LLFflux between hydrostatically reconstructed states
// splits into what each side contributes on its own (reconstructed depth,
// celerity, momentum, the flux of that side, the wave-speed bound, the source
// term) and their combination.  Half and llf_combine are those two parts of
// edge_eval_t<FX_LLF> with its operations in its order, so together they give
// its bits.
struct Half {
  double h, c, q, f1, f2, hv, s, src;   // h*, sqrt(g h*), h* u, q u + g/2 h*^2, q v, h* v, |u| + c, g/2 h*^2
};

// one side of the edge: state p on bed zp, zs = max of the two beds
__device__ __forceinline__ Half llf_half(const DevLevel& L, const Prim& p, double zp, double zs) {
  Half o;
  const double t = (p.h + zp) - zs;
  o.h = gt_zero(t) ? t : 0.0;
  o.c = sqrt(L.g * o.h);
  o.q = o.h * p.u;
  o.src = L.half_g * (o.h * o.h);
  o.f1 = o.q * p.u + o.src;
  o.f2 = o.q * p.v;
  o.hv = o.h * p.v;
  o.s = fabs(p.u) + o.c;
  return o;
}

// the flux from the two sides (l: the lower-index cell's side) and the cell's
// G on the side `upper` (as edge_G)
template <int NC>
__device__ __forceinline__ void llf_combine(const DevLevel& L, const Half& l, const Half& r, int axis, bool upper,
                                            double G[NC]) {
  double o[5];
  if (is_zero(l.h) && is_zero(r.h)) {
    o[0] = 0.0; o[1] = 0.0; o[2] = 0.0;
  } else {
    const double dU0 = r.h - l.h, dU1 = r.q - l.q, dU2 = r.hv - l.hv;
    double smax = dmax_nonneg(l.s, r.s);
    if (L.llf_wetdry) smax = smax + L.eps_r * dmax_nonneg(l.c, r.c);
    o[0] = ((l.q + r.q) - smax * dU0) * 0.5;
    o[1] = ((l.f1 + r.f1) - smax * dU1) * 0.5;
    o[2] = ((l.f2 + r.f2) - smax * dU2) * 0.5;
  }
  o[3] = l.src;
  o[4] = r.src;
  double GL[NC], GR[NC];
  edge_G<NC>(o, axis, GL, GR);
#pragma unroll
  for (int k = 0; k < NC; ++k) G[k] = upper ? GL[k] : GR[k];
}

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void bl_mbar_init(uint64_t* b) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool bl_mbar_try_wait(uint64_t* b, unsigned parity) {
  unsigned ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
               : "=r"(ok)
               : "r"(smem_u32(b)), "r"(parity)
               : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bl_mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ int bl_ld_vol(const int* p) {
  int v;
  asm volatile("ld.volatile.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_tagged_g(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_tagged_g(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void bl_sts_vol(int* p, int v) {
  asm volatile("st.volatile.shared.s32 [%0], %1;" ::"r"(smem_u32(p)), "r"(v) : "memory");
}
__device__ __forceinline__ int bl_lds_vol(const int* p) {
  int v;
  asm volatile("ld.volatile.shared.s32 %0, [%1];" : "=r"(v) : "r"(smem_u32(p)) : "memory");
  return v;
}

// BLU-SGS half-sweep (Algorithm 1, Steps 1 and 2.1) on a 2D uniform mesh with
// the LLF flux: the cell order, the operations and so the bits of
// k_blusgs_lean, with the step's work divided between two warps.  One CTA per
// strip of two rows in flight, 16 lanes per cell (side sd in W, E, S, N order
// times perturbation p):
//   warp 1 (helper), up to two steps ahead, loads the next cells' old
//     operands and forms every edge term that does not involve a value new in
//     this sweep: the whole G of the sides whose neighbour is old or a
//     boundary ghost, and the cell's own half of the other sides; then it
//     waits for the previous strip's new last-row value the first row needs
//     and passes it on;
//   warp 0 (critical) finishes the sides with a new neighbour (the own last
//     result, the row below, or the passed-on value: its half of the flux and
//     the combination), sums the sides, solves the 3x3 system and updates the
//     cell.  On a GB300 a warp issues one FP64 instruction per 64 cycles, so
//     the critical warp's FP64 instruction count sets the step time.
// Hand-offs inside the CTA go through two buffers and mbarriers (bounded
// waits); between strips the last row's new values travel as tagged 64-bit
// words (32 bits of a value and the launch's epoch), as in the SGS kernel.
// sync: [0] ticket, [1] abort.  edge: (strip q, column c, word w) at
// (q * nx + c) * 6 + 2 k + h (component k, half h).
__global__ void __launch_bounds__(64, 1) k_blusgs_ws(DevLevel L, const double* __restrict__ z, double* U,
                                                     const double* __restrict__ gbuf, int forward, int* sync,
                                                     unsigned long long* edge, unsigned epoch, int* sticky_err,
                                                     int spin_limit) {
  constexpr int NC = 3, NP = 4, GRP = 16, R = 2, NF = 16;
  // per buffer, field, lane: kinds 0 (the critical warp supplies the new
  // neighbour) and 2 (field 10-12: the previous strip's value): fields 0-7
  // the cell's half, 8 max bed, 9 neighbour bed; kind 3: fields 0-2 G.
  // Fields 13-15: the cell's old state.
  __shared__ double rec[2][NF][32];
  __shared__ int kind[2][32];
  __shared__ double sv[R][GRP][NC];
  __shared__ double ss[R][GRP];
  __shared__ __align__(8) uint64_t bar[4];   // full[0..1] helper -> critical, empty[2..3] back
  __shared__ int ctl[2];                      // [0] strip, [1] fail
  const unsigned full = 0xffffffffu;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane / GRP, g = lane % GRP;
  const int sd = g / NP, p = g % NP;
  const int axis = sd >> 1, upper = sd & 1;
  const int role = forward ? sd : (sd ^ 1);   // 0 previous column, 1 next column, 2 previous row, 3 next row
  const bool newside = (role & 1) == 0;       // neighbour updated earlier in this sweep
  const long long n = L.n;
  const int nstrips = (L.ny + R - 1) / R;
  const int glen = L.nx > L.ny ? L.nx : L.ny;
  const double len = axis == 0 ? L.ex : L.ey;
  const int src0 = lane - p;                  // the side's p = 0 lane
  if (threadIdx.x == 0) {
    for (int k = 0; k < 4; ++k) bl_mbar_init(&bar[k]);
    ctl[1] = 0;
  }
  __syncthreads();
  unsigned pf = 0u, pe = 0u, used = 0u;   // per buffer (bit b): full parity, empty parity, written once
  for (;;) {
    if (threadIdx.x == 0) ctl[0] = atomicAdd(&sync[0], 1);
    __syncthreads();
    const int q = ctl[0];
    if (q >= nstrips) return;
    const int rows = (L.ny - q * R < R) ? L.ny - q * R : R;
    const int nsteps = L.nx + rows - 1;
    const int rr = q * R + grp;
    const bool row_ok = grp < rows;
    const int iy = forward ? rr : L.ny - 1 - rr;
    const bool has_py = rr > 0, has_ny = rr < L.ny - 1;
    bool failed = false, timeout = false;
    if (warp == 1) {
      // ---- helper: records of steps 0 .. nsteps-1 ----
      const bool south = q > 0 && has_py;   // the first row's previous-row neighbour is in strip q - 1
      for (int t = 0; t < nsteps && !failed; ++t) {
        const int b = t & 1;
        if ((used >> b) & 1u) {   // the critical warp is done with step t - 2
          for (int it = 0;; ++it) {
            int ok = 0;
            if (lane == 0) ok = bl_mbar_try_wait(&bar[2 + b], (pe >> b) & 1u) ? 1 : 0;
            if (__shfl_sync(full, ok, 0)) break;
            int f = 0;
            if (lane == 0) f = bl_lds_vol(&ctl[1]);
            if (__shfl_sync(full, f, 0)) { failed = true; break; }
            if (it + 1 >= spin_limit) { failed = timeout = true; break; }
          }
          if (failed) break;
          pe ^= 1u << b;
        }
        used |= 1u << b;
        const int c = t - grp;
        const bool act = row_ok && c >= 0 && c < L.nx;
        int kd = 3;
        if (act) {
          const int ix = forward ? c : L.nx - 1 - c;
          const int i = ix + L.nx * iy;
          double ci[NC];
          for (int k = 0; k < NC; ++k) ci[k] = __ldcg(&U[k * n + i]);
          const double zi = z[i];
          const bool has = role == 0 ? c > 0 : role == 1 ? c < L.nx - 1 : role == 2 ? has_py : has_ny;
          const int j = sd == 0 ? i - 1 : sd == 1 ? i + 1 : sd == 2 ? i - L.nx : i + L.nx;
          const double zo = has ? z[j] : zi;
          // this lane's perturbation of the cell (component p - 1 by eps)
          double cp[NC];
          for (int k = 0; k < NC; ++k) cp[k] = (k == p - 1) ? ci[k] + L.eps : ci[k];
          Prim me;
          me.h = cp[0];
          const double qa = axis == 0 ? cp[1] : cp[2], qb = axis == 0 ? cp[2] : cp[1];
          if (ge_pos(cp[0], L.h_eps)) {
            const double r = 1.0 / cp[0];
            me.u = qa * r;
            me.v = qb * r;
          } else {
            me.u = 0.0;
            me.v = 0.0;
          }
          const double za = upper ? zi : zo, zb = upper ? zo : zi;
          const double zs = dmax(za, zb);
          const Half mh = llf_half(L, me, zi, zs);
          if (!has || !newside) {   // an old neighbour or a boundary ghost: the whole G here
            Prim other;
            if (has) {
              double cj[NC];
              for (int k = 0; k < NC; ++k) cj[k] = __ldcg(&U[k * n + j]);
              other = to_prim(cj[0], axis == 0 ? cj[1] : cj[2], axis == 0 ? cj[2] : cj[1], L.h_eps);
            } else {   // precomputed by ghost_prologue
              const long long t3 = ((long long)(sd * glen + (sd < 2 ? iy : ix)) * NP + p) * 3;
              other.h = __ldcg(&gbuf[t3]);
              other.u = __ldcg(&gbuf[t3 + 1]);
              other.v = __ldcg(&gbuf[t3 + 2]);
            }
            const Half oh = llf_half(L, other, zo, zs);
            double G[NC];
            llf_combine<NC>(L, upper ? mh : oh, upper ? oh : mh, axis, upper, G);
            for (int k = 0; k < NC; ++k) rec[b][k][lane] = G[k];
          } else {
            kd = (role == 2 && grp == 0) ? 2 : 0;
            rec[b][0][lane] = mh.h;
            rec[b][1][lane] = mh.c;
            rec[b][2][lane] = mh.q;
            rec[b][3][lane] = mh.f1;
            rec[b][4][lane] = mh.f2;
            rec[b][5][lane] = mh.hv;
            rec[b][6][lane] = mh.s;
            rec[b][7][lane] = mh.src;
            rec[b][8][lane] = zs;
            rec[b][9][lane] = zo;
          }
          for (int k = 0; k < NC; ++k) rec[b][13 + k][lane] = ci[k];
        }
        kind[b][lane] = kd;
        // the previous strip's new value of column c for the first row, once
        // all six words carry this launch's epoch
        if (south && t < L.nx) {
          double sval[NC];
          for (int it = 0;; ++it) {
            unsigned long long w = 0ull;
            if (lane < 6) w = ld_tagged_g(edge + ((long long)(q - 1) * L.nx + t) * 6 + lane);
            const bool ok = lane >= 6 || (unsigned)(w >> 32) == epoch;
            const unsigned lo = __shfl_sync(full, (unsigned)w, 0), hi0 = __shfl_sync(full, (unsigned)w, 1);
            const unsigned lo1 = __shfl_sync(full, (unsigned)w, 2), hi1 = __shfl_sync(full, (unsigned)w, 3);
            const unsigned lo2 = __shfl_sync(full, (unsigned)w, 4), hi2 = __shfl_sync(full, (unsigned)w, 5);
            if (__all_sync(full, ok)) {
              sval[0] = __longlong_as_double((long long)(((unsigned long long)hi0 << 32) | lo));
              sval[1] = __longlong_as_double((long long)(((unsigned long long)hi1 << 32) | lo1));
              sval[2] = __longlong_as_double((long long)(((unsigned long long)hi2 << 32) | lo2));
              break;
            }
            if ((it & 63) == 63) {
              int f = 0;
              if (lane == 0) f = bl_lds_vol(&ctl[1]) || bl_ld_vol(sync + 1);
              if (__shfl_sync(full, f, 0)) { failed = true; break; }
            }
            if (it + 1 >= spin_limit) { failed = timeout = true; break; }
          }
          if (failed) break;
          if (kd == 2)
            for (int k = 0; k < NC; ++k) rec[b][10 + k][lane] = sval[k];
        }
        __syncwarp();
        if (lane == 0) bl_mbar_arrive(&bar[b]);
      }
    } else {
      // ---- critical: the cell updates of steps 0 .. nsteps-1 ----
      double prevx[NC] = {0.0, 0.0, 0.0};   // the group's last result (new)
      for (int t = 0; t < nsteps; ++t) {
        const int b = t & 1;
        for (int it = 0;; ++it) {   // step t's record
          if (__all_sync(full, bl_mbar_try_wait(&bar[b], (pf >> b) & 1u))) break;
          int f = 0;
          if (lane == 0) f = bl_lds_vol(&ctl[1]);
          if (__shfl_sync(full, f, 0)) { failed = true; break; }
          if (it + 1 >= spin_limit) { failed = timeout = true; break; }
        }
        if (failed) break;
        pf ^= 1u << b;
        const int c = t - grp;
        const bool act = row_ok && c >= 0 && c < L.nx;
        const int kd = kind[b][lane];
        double f8[8], zs = 0.0, zo = 0.0, sn[NC], ci[NC];
        for (int e = 0; e < 8; ++e) f8[e] = rec[b][e][lane];
        if (kd != 3) {
          zs = rec[b][8][lane];
          zo = rec[b][9][lane];
        }
        for (int k = 0; k < NC; ++k) {
          sn[k] = kd == 2 ? rec[b][10 + k][lane] : 0.0;
          ci[k] = rec[b][13 + k][lane];
        }
        __syncwarp();
        if (lane == 0) bl_mbar_arrive(&bar[2 + b]);   // the record goes back to the helper
        // the previous row's new values: the group below
        double py[NC];
        for (int k = 0; k < NC; ++k) py[k] = __shfl_up_sync(full, prevx[k], GRP);
        double G[NC] = {0.0, 0.0, 0.0};
        if (act) {
          if (kd == 3) {
            for (int k = 0; k < NC; ++k) G[k] = f8[k];
          } else {   // a new neighbour: its half and the combination
            double cn[NC];
            for (int k = 0; k < NC; ++k) cn[k] = kd == 2 ? sn[k] : (role == 0 ? prevx[k] : py[k]);
            const Prim other = to_prim(cn[0], axis == 0 ? cn[1] : cn[2], axis == 0 ? cn[2] : cn[1], L.h_eps);
            const Half oh = llf_half(L, other, zo, zs);
            Half mh;
            mh.h = f8[0]; mh.c = f8[1]; mh.q = f8[2]; mh.f1 = f8[3];
            mh.f2 = f8[4]; mh.hv = f8[5]; mh.s = f8[6]; mh.src = f8[7];
            llf_combine<NC>(L, upper ? mh : oh, upper ? oh : mh, axis, upper, G);
          }
        }
        // p = 0 lanes hold |e| G, p = k+1 lanes column k of |e| dG/dU_i
        for (int k = 0; k < NC; ++k) {
          const double gb = __shfl_sync(full, G[k], src0);
          sv[grp][g][k] = len * ((p == 0) ? G[k] : (G[k] - gb) * L.reps);   // |e| G, or |e| (G - G_0) / eps
        }
        __syncwarp();
        if (g < NC * NP) {   // entry (component g / NP, perturbation g % NP): sides in W, E, S, N order
          const int es = g / NP, ep = g % NP;
          double acc = 0.0;
          for (int qs = 0; qs < 4; ++qs) acc = acc + sv[grp][qs * NP + ep][es];
          ss[grp][g] = acc;
        }
        __syncwarp();
        double un[NC] = {0.0, 0.0, 0.0};
        if (act && g == 0) {
          const int ix = forward ? c : L.nx - 1 - c;
          const int i = ix + L.nx * iy;
          double Rs[NC], D[NC * NC];
          for (int k = 0; k < NC; ++k) {
            Rs[k] = ss[grp][k * NP];
            for (int pp = 1; pp < NP; ++pp) D[k * NC + (pp - 1)] = ss[grp][k * NP + pp];
          }
          if (gt_zero(L.t_ka)) {   // time step (Remark 2.6): the step's residual and diagonal block
            const double ka = tka(L, i);
            for (int k = 0; k < NC; ++k) Rs[k] = (L.t_omb * Rs[k] + ka * ci[k]) - L.t_src[k * n + i];
            for (int e = 0; e < NC * NC; ++e) D[e] = L.t_omb * D[e];
            for (int k = 0; k < NC; ++k) D[k * NC + k] = D[k * NC + k] + ka;
          }
          double m = fabs(Rs[0]) + fabs(Rs[1]);
          m = m + fabs(Rs[2]);
          const double am = L.alpha * m;
          for (int k = 0; k < NC; ++k) D[k * NC + k] = D[k * NC + k] + am;
          double x[NC];
          small_solve<NC>(D, Rs, x);
          if (lt_pos(ci[0], L.h_eps))   // dry at the start: momentum stays zero (Remark 2.5)
            for (int k = 1; k < NC; ++k) x[k] = 0.0;
          for (int k = 0; k < NC; ++k) un[k] = ci[k] - x[k];
          if (lt_pos(un[0], L.h_eps))
            for (int k = 0; k < NC; ++k) un[k] = 0.0;
          for (int k = 0; k < NC; ++k) U[k * n + i] = un[k];
          if (grp == rows - 1 && q + 1 < nstrips) {   // the last row's new value for the next strip, tagged
            unsigned long long* e = edge + ((long long)q * L.nx + c) * 6;
            for (int k = 0; k < NC; ++k) {
              const unsigned long long u = (unsigned long long)__double_as_longlong(un[k]);
              st_tagged_g(e + 2 * k, ((unsigned long long)epoch << 32) | (u & 0xffffffffull));
              st_tagged_g(e + 2 * k + 1, ((unsigned long long)epoch << 32) | (u >> 32));
            }
          }
        }
        for (int k = 0; k < NC; ++k) {
          const double v = __shfl_sync(full, un[k], grp * GRP);
          if (act) prevx[k] = v;
        }
      }
    }
    if (failed && lane == 0) {
      if (timeout) atomicOr(sticky_err, 1);
      bl_sts_vol(&ctl[1], 1);
      st_rel(sync + 1, 1);
    }
    __syncthreads();
    if (ctl[1]) return;
  }
}

// ---- adjoint: lambda^T dR/dz and lambda^T dR/dq --------------------------------
// Central differences (step delta) of the edge terms with respect to the bed of
// either cell, contracted with lambda of both cells: cz[e] for the left cell's
// bed, cz[n_e + e] for the right cell's.  A boundary ghost's bed is the
// interior bed, so it moves with it.
template <int NC>
__global__ void k_adj_z_edges(DevLevel L, const double* __restrict__ z, const double* __restrict__ U,
                              const double* __restrict__ lam, double delta, double* __restrict__ cz,
                              int n_xe, int n_e) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_e) return;
  int axis, iL, iR;
  double len;
  edge_cells(L, e, n_xe, axis, iL, iR, len);
  double cL[NC], cR[NC], lL[NC], lR[NC];
  if (iL >= 0) { load_c<NC>(U, L.n, iL, cL); load_c<NC>(lam, L.n, iL, lL); }
  if (iR >= 0) { load_c<NC>(U, L.n, iR, cR); load_c<NC>(lam, L.n, iR, lR); }
  const double zL = iL >= 0 ? z[iL] : 0.0, zR = iR >= 0 ? z[iR] : 0.0;
  const double* pL = iL >= 0 ? cL : nullptr;
  const double* pR = iR >= 0 ? cR : nullptr;
  const double r2d = 1.0 / (2.0 * delta);
  for (int which = 0; which < 2; ++which) {
    const int cell = which == 0 ? iL : iR;
    double acc = 0.0;
    if (cell >= 0) {
      double GLp[NC], GRp[NC], GLm[NC], GRm[NC];
      if (which == 0) {
        eval_edge_states<NC>(L, axis, pL, zL + delta, pR, zR, GLp, GRp);
        eval_edge_states<NC>(L, axis, pL, zL - delta, pR, zR, GLm, GRm);
      } else {
        eval_edge_states<NC>(L, axis, pL, zL, pR, zR + delta, GLp, GRp);
        eval_edge_states<NC>(L, axis, pL, zL, pR, zR - delta, GLm, GRm);
      }
      for (int s = 0; s < NC; ++s) {
        if (iL >= 0) acc += lL[s] * (len * ((GLp[s] - GLm[s]) * r2d));
        if (iR >= 0) acc += lR[s] * (len * ((GRp[s] - GRm[s]) * r2d));
      }
    }
    cz[(long long)which * n_e + e] = acc;
  }
}

// gz[i] = -lambda^T dR/dz_i (the implicit-function part of dL/dz_i); the
// negation is exact, so gz is bitwise -(lambda^T dR/dz)
__global__ void k_adj_z_cells(DevLevel L, const double* __restrict__ cz, double* __restrict__ gz, int n_xe,
                              int n_e) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L.n) return;
  int eW, eE, eS, eN;
  cell_edges(L, i, n_xe, eW, eE, eS, eN);
  double a = cz[(long long)n_e + eW] + cz[eE];
  if (L.dim == 2) a = a + cz[(long long)n_e + eS] + cz[eN];
  gz[i] = -a;
}

// per boundary cell of `side`: -lambda . |e| (G(q + delta) - G(q - delta)) / (2 delta)
// (negated, so that the sum over the side is -lambda^T dR/dq)
template <int NC>
__global__ void k_adj_q_cells(DevLevel Lp, DevLevel Lm, int side, const double* __restrict__ z,
                              const double* __restrict__ U, const double* __restrict__ lam, double delta,
                              double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Lp.n) return;
  const int ix = i % Lp.nx, iy = i / Lp.nx;
  const bool on = (side == 0 && ix == 0) || (side == 1 && ix == Lp.nx - 1) ||
                  (side == 2 && iy == 0) || (side == 3 && iy == Lp.ny - 1);
  double acc = 0.0;
  if (on) {
    const int axis = side >> 1, upper = side & 1;
    const double len = axis == 0 ? Lp.ex : Lp.ey;
    double c[NC], l[NC], GLp[NC], GRp[NC], GLm[NC], GRm[NC];
    load_c<NC>(U, Lp.n, i, c);
    load_c<NC>(lam, Lp.n, i, l);
    if (upper) {
      eval_edge_states<NC>(Lp, axis, c, z[i], nullptr, 0.0, GLp, GRp);
      eval_edge_states<NC>(Lm, axis, c, z[i], nullptr, 0.0, GLm, GRm);
    } else {
      eval_edge_states<NC>(Lp, axis, nullptr, 0.0, c, z[i], GLp, GRp);
      eval_edge_states<NC>(Lm, axis, nullptr, 0.0, c, z[i], GLm, GRm);
    }
    const double r2d = 1.0 / (2.0 * delta);
    for (int s = 0; s < NC; ++s) {
      const double gp = upper ? GLp[s] : GRp[s], gm = upper ? GLm[s] : GRm[s];
      acc += l[s] * (len * ((gp - gm) * r2d));
    }
  }
  out[i] = -acc;
}

// U += tau dU with the dry rules of Remark 2.5 (eq. NewtonREG-12)
template <typename T>
__device__ __forceinline__ void newton_update_cell(int nx, int ny, int nc, double tau, double h_eps,
                                                   double* __restrict__ U, const T* __restrict__ dU, int i) {
  // dU is a multigrid vector: strip-skewed, nc x skew_slots(nx, ny)
  const long long n = (long long)nx * ny, P = skew_slots(nx, ny), si = skew_pos(i % nx, i / nx, nx);
  const double h0 = U[i];
  double v[3];
  for (int s = 0; s < nc; ++s) {
    double d = static_cast<double>(dU[(long long)s * P + si]);
    if (s > 0 && h0 < h_eps) d = 0.0;
    v[s] = U[(long long)s * n + i] + tau * d;
  }
  if (v[0] < h_eps)
    for (int s = 0; s < nc; ++s) v[s] = 0.0;
  for (int s = 0; s < nc; ++s) U[(long long)s * n + i] = v[s];
}

template <typename T>
__global__ void k_newton_update(int nx, int ny, int nc, double tau, double h_eps, double* __restrict__ U,
                                const T* __restrict__ dU) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nx * ny) newton_update_cell<T>(nx, ny, nc, tau, h_eps, U, dU, i);
}

// t_src = ka U^n - beta R(U^n) (Remark 2.6)
__global__ void k_time_source(long long m, double ka, double beta, const double* __restrict__ U,
                              const double* __restrict__ R, double* __restrict__ src) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e < m) src[e] = ka * U[e] - beta * R[e];
}

// coarse value = mean of the children (child order 00, 10, 01, 11)
__device__ __forceinline__ void average_cell(int dim, int nxf, int nyf, int ncomp, const double* __restrict__ vf,
                                             double* __restrict__ vc, int I) {
  const int nxc = nxf / 2, nyc = dim == 2 ? nyf / 2 : 1, nc_cells = nxc * nyc;
  const long long nf = (long long)nxf * (dim == 2 ? nyf : 1);
  const int Ix = I % nxc, Iy = I / nxc;
  for (int s = 0; s < ncomp; ++s) {
    const double* v = vf + s * nf;
    double a;
    if (dim == 1) {
      a = v[2 * Ix];
      a = a + v[2 * Ix + 1];
      a = a * 0.5;
    } else {
      const int f = 2 * Ix + nxf * 2 * Iy;
      a = v[f];
      a = a + v[f + 1];
      a = a + v[f + nxf];
      a = a + v[f + nxf + 1];
      a = a * 0.25;
    }
    vc[(long long)s * nc_cells + I] = a;
  }
}

__global__ void k_average(int dim, int nxf, int nyf, int ncomp, const double* __restrict__ vf,
                          double* __restrict__ vc) {
  const int nc_cells = (nxf / 2) * (dim == 2 ? nyf / 2 : 1);
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I < nc_cells) average_cell(dim, nxf, nyf, ncomp, vf, vc, I);
}

// curvilinear mesh: the children weighted by their areas (the cell average
// over their union), sum_q |K_q| v_q / sum_q |K_q|, children in the order 00,
// 10, 01, 11
__global__ void k_average_area(int nxf, int nyf, int ncomp, const double* __restrict__ area_f,
                               const double* __restrict__ vf, double* __restrict__ vc) {
  const int nxc = nxf / 2, nc_cells = nxc * (nyf / 2);
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nc_cells) return;
  const long long nf = (long long)nxf * nyf;
  const int f = 2 * (I % nxc) + nxf * 2 * (I / nxc);
  const int ch[4] = {f, f + 1, f + nxf, f + nxf + 1};
  double ar[4], tot = 0.0;
  for (int q = 0; q < 4; ++q) {
    ar[q] = area_f[ch[q]];
    tot = tot + ar[q];
  }
  for (int s = 0; s < ncomp; ++s) {
    double a = 0.0;
    for (int q = 0; q < 4; ++q) a = a + ar[q] * vf[s * nf + ch[q]];
    vc[(long long)s * nc_cells + I] = a / tot;
  }
}

// time step on a curvilinear mesh: t_src = |K_i|/dt U^n - beta R(U^n), per cell
__global__ void k_time_source_cells(long long m, long long n, const double* __restrict__ kai, double beta,
                                    const double* __restrict__ U, const double* __restrict__ R,
                                    double* __restrict__ src) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e < m) src[e] = kai[e % n] * U[e] - beta * R[e];
}

// ---- curvilinear mesh geometry --------------------------------------------------
// Level l of a mesh with vertex (a, b) at (vx, vy)[a + vrow b] is the mesh of
// every step-th vertex, step = 2^l.  Edge e (x-edges first, edge_cells'
// numbering) runs from vertex (a, b) to (a, b + 1) (x-edges) or to (a + 1, b)
// (y-edges); with t their difference, |e| = sqrt(t.t) and n is t turned by
// -90 degrees (x-edges) or +90 degrees (y-edges), divided by |e|.  |K_i| is
// half the cross product of the quadrilateral's diagonals.  A degenerate edge
// or a cell of non-positive area sets *bad.
__device__ __forceinline__ void mesh_vertex(const double* vx, const double* vy, int vrow, int step, int a, int b,
                                            double& x, double& y) {
  const long long k = (long long)a * step + (long long)vrow * ((long long)b * step);
  x = vx[k];
  y = vy[k];
}

__global__ void k_edge_geometry(int nx, int ny, int vrow, int step, const double* __restrict__ vx,
                                const double* __restrict__ vy, double* __restrict__ geo, int* bad) {
  const long long n_xe = (long long)(nx + 1) * ny, ne = n_xe + (long long)nx * (ny + 1);
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const bool xe = e < n_xe;
  int a0, b0, a1, b1;
  if (xe) {
    a0 = (int)(e % (nx + 1));
    b0 = (int)(e / (nx + 1));
    a1 = a0;
    b1 = b0 + 1;
  } else {
    const long long f = e - n_xe;
    a0 = (int)(f % nx);
    b0 = (int)(f / nx);
    a1 = a0 + 1;
    b1 = b0;
  }
  double xa, ya, xb, yb;
  mesh_vertex(vx, vy, vrow, step, a0, b0, xa, ya);
  mesh_vertex(vx, vy, vrow, step, a1, b1, xb, yb);
  const double tx = xb - xa, ty = yb - ya;
  const double l = sqrt(tx * tx + ty * ty);
  geo[e] = l;
  geo[ne + e] = xe ? ty / l : -ty / l;
  geo[2 * ne + e] = xe ? -tx / l : tx / l;
  if (!(l > 0.0)) atomicOr(bad, 1);
}

__global__ void k_cell_area(int nx, int ny, int vrow, int step, const double* __restrict__ vx,
                            const double* __restrict__ vy, double* __restrict__ area, int* bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nx * ny) return;
  const int ix = i % nx, iy = i / nx;
  double x00, y00, x10, y10, x11, y11, x01, y01;
  mesh_vertex(vx, vy, vrow, step, ix, iy, x00, y00);
  mesh_vertex(vx, vy, vrow, step, ix + 1, iy, x10, y10);
  mesh_vertex(vx, vy, vrow, step, ix + 1, iy + 1, x11, y11);
  mesh_vertex(vx, vy, vrow, step, ix, iy + 1, x01, y01);
  const double a = 0.5 * ((x11 - x00) * (y01 - y10) - (x01 - x10) * (y11 - y00));
  area[i] = a;
  if (!(a > 0.0)) atomicOr(bad, 1);
}

__global__ void k_time_ka(int n, const double* __restrict__ area, double dt, double* __restrict__ kai) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) kai[i] = area[i] / dt;
}

// piecewise-constant injection of a coarse solution (Algorithm 1, Step 1)
__device__ __forceinline__ void inject_cell(int dim, int nxf, int nyf, int ncomp, const double* __restrict__ vc,
                                            double* __restrict__ vf, int i) {
  const int nf_cells = nxf * (dim == 2 ? nyf : 1);
  const int ix = i % nxf, iy = i / nxf, nxc = nxf / 2;
  const int nc_cells = nxc * (dim == 2 ? nyf / 2 : 1);
  const int I = (ix / 2) + nxc * (dim == 2 ? iy / 2 : 0);
  for (int s = 0; s < ncomp; ++s) vf[(long long)s * nf_cells + i] = vc[(long long)s * nc_cells + I];
}

__global__ void k_inject(int dim, int nxf, int nyf, int ncomp, const double* __restrict__ vc,
                         double* __restrict__ vf) {
  const int nf_cells = nxf * (dim == 2 ? nyf : 1);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nf_cells) inject_cell(dim, nxf, nyf, ncomp, vc, vf, i);
}

// ---- batched forms -------------------------------------------------------------
// The same per-edge / per-cell bodies; the block's problem comes from the
// launch's block table (blocks of 128 threads), so every problem of a batch
// gets exactly the arithmetic of its own single-problem launch.
#define BATCH_PROLOGUE(bl)                                        \
  const int p_ = batch_find((bl).bstart, (bl).B, blockIdx.x);     \
  if (!(bl).mask[p_]) return;                                     \
  const BItem* it = (bl).items + p_;                              \
  const int idx = (blockIdx.x - (bl).bstart[p_]) * 128 + threadIdx.x;

template <int NC>
__global__ void __launch_bounds__(128) kb_res_edges(BLaunch bl) {
  BATCH_PROLOGUE(bl)
  if (idx >= it->n_e) return;
  const DevLevel L = it->L;
  res_edge<NC>(L, it->z, it->U, it->eb, it->n_xe, it->n_e, idx, it->n_e, idx);
}

template <int NC>
__global__ void __launch_bounds__(128) kb_res_cells(BLaunch bl) {
  BATCH_PROLOGUE(bl)
  const DevLevel L = it->L;
  if (idx >= L.n) return;
  int eW, eE, eS, eN;
  cell_edges(L, idx, it->n_xe, eW, eE, eS, eN);
  res_cell<NC>(L, it->eb, it->U, it->R, it->rn, it->n_xe, it->n_e, idx, it->n_e, eW, eE, eS, eN);
}

template <int NC, typename T>
__global__ void __launch_bounds__(128) kb_jac_edges(BLaunch bl) {
  BATCH_PROLOGUE(bl)
  if (idx >= it->n_e) return;
  const DevLevel L = it->L;
  jac_edge<NC, T>(L, it->z, it->U, it->eb, it->blk, it->n_xe, it->n_e, idx, it->n_e, idx);
}

template <int NC, typename T>
__global__ void __launch_bounds__(128) kb_jac_cells(BLaunch bl) {
  BATCH_PROLOGUE(bl)
  const DevLevel L = it->L;
  if (idx >= L.n) return;
  int eW, eE, eS, eN;
  cell_edges(L, idx, it->n_xe, eW, eE, eS, eN);
  jac_cell<NC, T>(L, it->eb, it->U, it->R, it->rn, it->blk, it->n_xe, it->n_e, idx, it->n_e, eW, eE, eS, eN);
}

template <typename T>
__global__ void __launch_bounds__(128) kb_newton_update(BLaunch bl, double tau, double h_eps) {
  BATCH_PROLOGUE(bl)
  if (idx >= it->L.n) return;
  newton_update_cell<T>(it->L.nx, it->L.ny, it->L.nc, tau, h_eps, it->U, static_cast<const T*>(it->x), idx);
}

__global__ void __launch_bounds__(128) kb_average(BLaunch bl, const BItem* fine) {
  BATCH_PROLOGUE(bl)
  if (idx >= it->L.n) return;
  const BItem* f = fine + p_;
  average_cell(2, f->L.nx, f->L.ny, f->L.nc, f->U, it->U, idx);
}

__global__ void __launch_bounds__(128) kb_inject(BLaunch bl, const BItem* coarse) {
  BATCH_PROLOGUE(bl)
  if (idx >= it->L.n) return;
  inject_cell(2, it->L.nx, it->L.ny, it->L.nc, coarse[p_].U, it->U, idx);
}
#undef BATCH_PROLOGUE

// BLU-SGS half-sweep over a batch: step q updates diagonal q (forward) of
// every masked problem that has one; the diagonals' cells are concatenated
// in problem order and dealt to the warps, then the grid meets at the same
// bounded barrier as the single-problem sweep.
template <int NC, int NS, int GRP>
__global__ void __launch_bounds__(128) kb_blusgs_sweep(const BItem* __restrict__ items,
                                                       const int* __restrict__ mask, int B, int nsteps,
                                                       int forward, int* sync, int* sticky_err,
                                                       int spin_limit) {
  __shared__ int s_off[BATCH_MAX + 1];
  __shared__ int s_cnt[BATCH_MAX], s_d[BATCH_MAX], s_ix0[BATCH_MAX];
  const unsigned full = 0xffffffffu;
  const int wpb = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // warp-major numbering: consecutive cell pairs go to different SMs first,
  // so a short diagonal puts one warp per SM (GB300 issues about two FP64
  // operations per clock per SM; four warps of one SM would queue on it)
  const int gw = warp * gridDim.x + blockIdx.x, nw = gridDim.x * wpb;
  const int cpw = 32 / GRP;
  for (int p = 0; p < B; ++p)
    if (mask[p])
      ghost_prologue<NC, NS>(items[p].L, items[p].U, items[p].ghost, blockIdx.x * blockDim.x + threadIdx.x,
                             gridDim.x * blockDim.x);
  if (!grid_barrier(sync, 0, sticky_err, spin_limit)) return;
  for (int q = 0; q < nsteps; ++q) {
    for (int p = threadIdx.x; p < B; p += blockDim.x) {
      int cnt = 0, d = 0, ix0 = 0;
      if (mask[p]) {
        const int nx = items[p].L.nx, ny = items[p].L.ny, ndiag = nx + ny - 1;
        if (q < ndiag) {
          d = forward ? q : ndiag - 1 - q;
          ix0 = d - (ny - 1) > 0 ? d - (ny - 1) : 0;
          const int ix1 = d < nx - 1 ? d : nx - 1;
          cnt = ix1 - ix0 + 1;
        }
      }
      s_cnt[p] = cnt;
      s_d[p] = d;
      s_ix0[p] = ix0;
    }
    __syncthreads();
    if (warp == 0) {   // exclusive prefix of the counts
      const int per = (B + 31) / 32;
      int loc = 0;
      for (int k = 0; k < per; ++k) {
        const int p = lane * per + k;
        if (p < B) loc += s_cnt[p];
      }
      int inc = loc;
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(full, inc, o);
        if (lane >= o) inc += v;
      }
      int run = inc - loc;
      for (int k = 0; k < per; ++k) {
        const int p = lane * per + k;
        if (p < B) {
          s_off[p] = run;
          run += s_cnt[p];
        }
      }
      if (lane == 31) s_off[B] = inc;
    }
    __syncthreads();
    const int total = s_off[B];
    for (int c0 = gw * cpw; c0 < total; c0 += nw * cpw) {   // warp-uniform loop
      const int flat = c0 + lane / GRP;
      int p = 0, cell = 0, ncell = 0;
      if (flat < total) {
        int lo = 0, hi = B - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (s_off[mid] <= flat) lo = mid;
          else hi = mid - 1;
        }
        p = lo;
        cell = flat - s_off[p];
        ncell = s_cnt[p];
      }
      blusgs_group<NC, NS, GRP, true>(items[p].L, items[p].z, items[p].U, items[p].ghost, s_d[p], s_ix0[p],
                                      ncell, cell, lane % GRP);
    }
    if (!grid_barrier(sync, q + 1, sticky_err, spin_limit)) return;
  }
}

inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

// ---- launch wrappers ---------------------------------------------------------

static void edge_counts(const DevLevel& L, int& n_xe, int& n_e) {
  n_xe = (L.nx + 1) * L.ny;
  n_e = n_xe + (L.dim == 2 ? L.nx * (L.ny + 1) : 0);
}

// tile shapes of the fused 2D residual and Jacobian
constexpr int RT_X = 32, RT_Y = 8, RT_T = 288;
constexpr int JT_X = 32, JT_Y = 8, JT_T = 288;

void launch_residual(const DevLevel& L, const double* z, const double* U, double* R, double* rn,
                     double* eb, cudaStream_t st) {
  count_launches(2);
  int n_xe, n_e;
  edge_counts(L, n_xe, n_e);
  if (L.nc == 3) {   // 2D: fused tiles, the edge pieces stay in shared memory (eb unused)
    count_launches(-1);
    const dim3 grid((L.nx + RT_X - 1) / RT_X, (L.ny + RT_Y - 1) / RT_Y);
    k_res_tile<3, RT_X, RT_Y, RT_T><<<grid, RT_T, 0, st>>>(L, z, U, R, rn, n_xe, n_e);
  } else {
    k_res_edges<2><<<nblk(n_e, 128), 128, 0, st>>>(L, z, U, eb, n_xe, n_e);
    k_res_cells<2><<<nblk(L.n, 256), 256, 0, st>>>(L, eb, U, R, rn, n_xe, n_e);
  }
}

void launch_jacobian(const DevLevel& L, const double* z, const double* U, double* R, double* rn,
                     double* eb, void* blk, int fp32, cudaStream_t st) {
  count_launches(2);
  int n_xe, n_e;
  edge_counts(L, n_xe, n_e);
  if (L.nc == 3) {   // 2D: fused tiles, the edge pieces stay in shared memory (eb unused)
    count_launches(-1);
    const dim3 grid((L.nx + JT_X - 1) / JT_X, (L.ny + JT_Y - 1) / JT_Y);
    constexpr size_t smem = (size_t)(2 * 3 + 2 * 9) * tile_edges<JT_X, JT_Y>() * sizeof(double);
    static bool attr_set = false;
    if (!attr_set) {
      cudaFuncSetAttribute(k_jac_tile<3, float, JT_X, JT_Y, JT_T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      cudaFuncSetAttribute(k_jac_tile<3, double, JT_X, JT_Y, JT_T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      attr_set = true;
    }
    if (fp32) k_jac_tile<3, float, JT_X, JT_Y, JT_T><<<grid, JT_T, smem, st>>>(L, z, U, R, rn, blk, n_xe, n_e);
    else k_jac_tile<3, double, JT_X, JT_Y, JT_T><<<grid, JT_T, smem, st>>>(L, z, U, R, rn, blk, n_xe, n_e);
  } else {
    if (fp32) {
      k_jac_edges<2, float><<<nblk(n_e, 128), 128, 0, st>>>(L, z, U, eb, blk, n_xe, n_e);
      k_jac_cells<2, float><<<nblk(L.n, 128), 128, 0, st>>>(L, eb, U, R, rn, blk, n_xe, n_e);
    } else {
      k_jac_edges<2, double><<<nblk(n_e, 128), 128, 0, st>>>(L, z, U, eb, blk, n_xe, n_e);
      k_jac_cells<2, double><<<nblk(L.n, 128), 128, 0, st>>>(L, eb, U, R, rn, blk, n_xe, n_e);
    }
  }
}

// strip-pipelined half-sweep: ghosts, then one warp per strip in flight;
// sync holds 2 + ceil(ny / R) ints, R = 2 (2D) or 4 (1D) rows per strip
void launch_blusgs_strip(const DevLevel& L, const double* z, double* U, double* gbuf, int forward, int* sync,
                         unsigned long long* edge, unsigned epoch, int* sticky_err, cudaStream_t st) {
  count_launches(2);
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  }
  const int R = L.nc == 3 ? 2 : 4;
  const int nstrips = (L.ny + R - 1) / R;
  cudaMemsetAsync(sync, 0, (2 + nstrips) * sizeof(int), st);
  const int glen = L.nx > L.ny ? L.nx : L.ny;
  const int gthreads = 4 * glen * (L.nc + 1);
  const int gblocks = (gthreads + 127) / 128;
  // at most 16 warps per SM: more strips than that queue on the ticket
  const int grid = nstrips < 16 * nsm ? nstrips : 16 * nsm;
  const int spin = wait_limit();
  if (L.nc == 3 && L.geo == nullptr) {   // 2D uniform mesh: the lean kernel, flux fixed at compile time
    k_ghost_prologue<3, 4><<<gblocks, 128, 0, st>>>(L, U, gbuf);
    if (L.flux == FX_LLF && edge)   // the two-warp kernel
      k_blusgs_ws<<<grid, 64, 0, st>>>(L, z, U, gbuf, forward, sync, edge, epoch, sticky_err, spin);
    else if (L.flux == FX_LLF) k_blusgs_lean<FX_LLF><<<grid, 32, 0, st>>>(L, z, U, gbuf, forward, sync, sticky_err, spin);
    else if (L.flux == FX_HLLC) k_blusgs_lean<FX_HLLC><<<grid, 32, 0, st>>>(L, z, U, gbuf, forward, sync, sticky_err, spin);
    else if (L.flux == FX_ROE) k_blusgs_lean<FX_ROE><<<grid, 32, 0, st>>>(L, z, U, gbuf, forward, sync, sticky_err, spin);
    else k_blusgs_lean<FX_HLL><<<grid, 32, 0, st>>>(L, z, U, gbuf, forward, sync, sticky_err, spin);
  } else if (L.nc == 3) {
    k_ghost_prologue<3, 4><<<gblocks, 128, 0, st>>>(L, U, gbuf);
    k_blusgs_strip<3, 4, 16><<<grid, 32, 0, st>>>(L, z, U, gbuf, forward, sync, sticky_err, spin);
  } else {
    k_ghost_prologue<2, 2><<<gblocks, 128, 0, st>>>(L, U, gbuf);
    k_blusgs_strip<2, 2, 8><<<grid, 32, 0, st>>>(L, z, U, gbuf, forward, sync, sticky_err, spin);
  }
}

void launch_blusgs_sweep(const DevLevel& L, const double* z, double* U, double* gbuf, int forward, int* sync,
                         int* sticky_err, cudaStream_t st) {
  count_launches(1);
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  }
  cudaMemsetAsync(sync, 0, 2 * sizeof(int), st);
  // one block of 4 warps per SM (co-resident by cooperative launch); a
  // diagonal's cells are dealt to the warps in rounds
  int fw = forward;
  int spin = wait_limit();
  DevLevel Lc = L;
  void* args[] = {(void*)&Lc, (void*)&z, (void*)&U, (void*)&gbuf, (void*)&fw, (void*)&sync, (void*)&sticky_err,
                  (void*)&spin};
  if (L.nc == 3)
    cudaLaunchCooperativeKernel((const void*)k_blusgs_sweep<3, 4, 16>, dim3(nsm), dim3(128), args, 0, st);
  else
    cudaLaunchCooperativeKernel((const void*)k_blusgs_sweep<2, 2, 8>, dim3(nsm), dim3(128), args, 0, st);
}

void launch_adjoint_z(const DevLevel& L, const double* z, const double* U, const double* lam, double delta,
                      double* cz, double* dRz, cudaStream_t st) {
  count_launches(2);
  int n_xe, n_e;
  edge_counts(L, n_xe, n_e);
  if (L.nc == 3) k_adj_z_edges<3><<<nblk(n_e, 128), 128, 0, st>>>(L, z, U, lam, delta, cz, n_xe, n_e);
  else k_adj_z_edges<2><<<nblk(n_e, 128), 128, 0, st>>>(L, z, U, lam, delta, cz, n_xe, n_e);
  k_adj_z_cells<<<nblk(L.n, 256), 256, 0, st>>>(L, cz, dRz, n_xe, n_e);
}

void launch_adjoint_q(const DevLevel& L, int side, const double* z, const double* U, const double* lam,
                      double delta, double* out, cudaStream_t st) {
  count_launches(1);
  DevLevel Lp = L, Lm = L;
  Lp.bc[side].q = L.bc[side].q + delta;
  Lm.bc[side].q = L.bc[side].q - delta;
  if (L.nc == 3) k_adj_q_cells<3><<<nblk(L.n, 128), 128, 0, st>>>(Lp, Lm, side, z, U, lam, delta, out);
  else k_adj_q_cells<2><<<nblk(L.n, 128), 128, 0, st>>>(Lp, Lm, side, z, U, lam, delta, out);
}

void launch_newton_update(int nx, int ny, int nc, double tau, double h_eps, double* U, const void* dU,
                          int dU_fp32, cudaStream_t st) {
  count_launches(1);
  const int n = nx * ny;
  if (dU_fp32)
    k_newton_update<float><<<nblk(n, 256), 256, 0, st>>>(nx, ny, nc, tau, h_eps, U, (const float*)dU);
  else
    k_newton_update<double><<<nblk(n, 256), 256, 0, st>>>(nx, ny, nc, tau, h_eps, U, (const double*)dU);
}

void launch_time_source(long long m, double ka, double beta, const double* U, const double* R, double* src,
                        cudaStream_t st) {
  count_launches(1);
  k_time_source<<<nblk(m, 256), 256, 0, st>>>(m, ka, beta, U, R, src);
}

void launch_average_area(int nxf, int nyf, int ncomp, const double* area_f, const double* vf, double* vc,
                         cudaStream_t st) {
  count_launches(1);
  const int ncells = (nxf / 2) * (nyf / 2);
  k_average_area<<<nblk(ncells, 256), 256, 0, st>>>(nxf, nyf, ncomp, area_f, vf, vc);
}

void launch_time_source_cells(long long m, long long n, const double* kai, double beta, const double* U,
                              const double* R, double* src, cudaStream_t st) {
  count_launches(1);
  k_time_source_cells<<<nblk(m, 256), 256, 0, st>>>(m, n, kai, beta, U, R, src);
}

void launch_mesh_level(int nx, int ny, int vrow, int step, const double* vx, const double* vy, double* geo,
                       double* area, int* bad, cudaStream_t st) {
  count_launches(2);
  const long long ne = (long long)(nx + 1) * ny + (long long)nx * (ny + 1);
  k_edge_geometry<<<nblk(ne, 256), 256, 0, st>>>(nx, ny, vrow, step, vx, vy, geo, bad);
  k_cell_area<<<nblk((long long)nx * ny, 256), 256, 0, st>>>(nx, ny, vrow, step, vx, vy, area, bad);
}

void launch_time_ka(int n, const double* area, double dt, double* kai, cudaStream_t st) {
  count_launches(1);
  k_time_ka<<<nblk(n, 256), 256, 0, st>>>(n, area, dt, kai);
}

void launch_average(int dim, int nxf, int nyf, int ncomp, const double* vf, double* vc,
                    cudaStream_t st) {
  count_launches(1);
  const int ncells = (nxf / 2) * (dim == 2 ? nyf / 2 : 1);
  k_average<<<nblk(ncells, 256), 256, 0, st>>>(dim, nxf, nyf, ncomp, vf, vc);
}

void launch_inject(int dim, int nxf, int nyf, int ncomp, const double* vc, double* vf,
                   cudaStream_t st) {
  count_launches(1);
  const int ncells = nxf * (dim == 2 ? nyf : 1);
  k_inject<<<nblk(ncells, 256), 256, 0, st>>>(dim, nxf, nyf, ncomp, vc, vf);
}

// ---- batched launchers ----------------------------------------------------------

void launch_b_residual(const BLaunch& edges, const BLaunch& cells, cudaStream_t st) {
  count_launches(2);
  if (edges.nblocks > 0) kb_res_edges<3><<<edges.nblocks, 128, 0, st>>>(edges);
  if (cells.nblocks > 0) kb_res_cells<3><<<cells.nblocks, 128, 0, st>>>(cells);
}

void launch_b_jacobian(const BLaunch& edges, const BLaunch& cells, int fp32, cudaStream_t st) {
  count_launches(2);
  if (fp32) {
    if (edges.nblocks > 0) kb_jac_edges<3, float><<<edges.nblocks, 128, 0, st>>>(edges);
    if (cells.nblocks > 0) kb_jac_cells<3, float><<<cells.nblocks, 128, 0, st>>>(cells);
  } else {
    if (edges.nblocks > 0) kb_jac_edges<3, double><<<edges.nblocks, 128, 0, st>>>(edges);
    if (cells.nblocks > 0) kb_jac_cells<3, double><<<cells.nblocks, 128, 0, st>>>(cells);
  }
}

void launch_b_newton_update(const BLaunch& cells, double tau, double h_eps, int fp32, cudaStream_t st) {
  count_launches(1);
  if (cells.nblocks <= 0) return;
  if (fp32) kb_newton_update<float><<<cells.nblocks, 128, 0, st>>>(cells, tau, h_eps);
  else kb_newton_update<double><<<cells.nblocks, 128, 0, st>>>(cells, tau, h_eps);
}

void launch_b_average(const BLaunch& coarse, const BItem* fine_items, cudaStream_t st) {
  count_launches(1);
  if (coarse.nblocks > 0) kb_average<<<coarse.nblocks, 128, 0, st>>>(coarse, fine_items);
}

void launch_b_inject(const BLaunch& fine, const BItem* coarse_items, cudaStream_t st) {
  count_launches(1);
  if (fine.nblocks > 0) kb_inject<<<fine.nblocks, 128, 0, st>>>(fine, coarse_items);
}

// Batched strip-pipelined BLU-SGS: the schedule of k_blusgs_strip, one
// (problem, strip) ticket at a time; problems outside the mask are skipped
// whole.  Tickets list strip 0 of every problem first, then strip 1, ..., so
// a strip only waits for one that a running warp owns.  sync: [0] ticket,
// [1] abort, [2 + bstrip0(p) + q] columns completed by strip q's last row.
template <int NC, int NS>
__global__ void __launch_bounds__(128) kb_ghost_prologue(const BItem* __restrict__ items,
                                                         const int* __restrict__ mask, int B) {
  for (int p = 0; p < B; ++p)
    if (mask[p])
      ghost_prologue<NC, NS>(items[p].L, items[p].U, items[p].ghost, blockIdx.x * blockDim.x + threadIdx.x,
                             gridDim.x * blockDim.x);
}

template <int NC, int NS, int GRP>
__global__ void __launch_bounds__(32) kb_blusgs_strip(const BItem* __restrict__ items,
                                                      const int2* __restrict__ tickets, int ntickets,
                                                      const int* __restrict__ mask, int forward, int* sync,
                                                      int* sticky_err, int spin_limit) {
  constexpr int R = 32 / GRP;
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  for (;;) {
    int tid = 0;
    if (lane == 0) tid = atomicAdd(&sync[0], 1);
    tid = __shfl_sync(full, tid, 0);
    if (tid >= ntickets) return;
    const int2 tk = tickets[tid];
    const int p = tk.x, q = tk.y;
    if (!mask[p]) continue;
    const BItem& it = items[p];
    const DevLevel L = it.L;
    const int nstrips = (L.ny + R - 1) / R;
    int* prog = sync + 2 + it.bstrip0;
    const int rows = (L.ny - q * R < R) ? L.ny - q * R : R;
    const int nsteps = L.nx + rows - 1;
    int known = 0;
    for (int t = 0; t < nsteps; ++t) {
      if (q > 0 && t < L.nx && known < t + 1) {
        int pg = 0, n_it = 0;
        do {
          if (lane == 0) {
            pg = ld_acq(&prog[q - 1]);
            if (pg < t + 1 && ld_acq(&sync[1])) pg = -1;
          }
          pg = __shfl_sync(full, pg, 0);
          if (pg >= t + 1 || pg < 0) break;
          __nanosleep(32);
        } while (++n_it < spin_limit);
        if (pg < t + 1) {
          if (lane == 0) {
            if (pg >= 0) atomicOr(sticky_err, 1);
            atomicExch(&sync[1], 1);
          }
          return;
        }
        known = pg;
      }
      __syncwarp();
      const int c_lo = t - rows + 1 > 0 ? t - rows + 1 : 0;
      const int c_hi = t < L.nx - 1 ? t : L.nx - 1;
      const int ncell = c_hi - c_lo + 1;
      int d, ix0;
      if (forward) {
        d = q * R + t;
        ix0 = c_lo;
      } else {
        d = (L.nx - 1) + (L.ny - 1) - (q * R + t);
        ix0 = L.nx - 1 - c_hi;
      }
      blusgs_group<NC, NS, GRP, true>(L, it.z, it.U, it.ghost, d, ix0, ncell, lane / GRP, lane % GRP);
      __syncwarp();
      const int done = t - rows + 2;
      if (q + 1 < nstrips && done >= 1 && done <= L.nx) {
        const int rel = forward ? 0 : (ncell - 1) * GRP;
        if (lane == rel) st_rel(&prog[q], done);
      }
    }
  }
}

void launch_b_blusgs_strip(const BItem* items, const int2* tickets, int ntickets, int nslots, const int* mask,
                           int B, int forward, int grid, int* sync, int* sticky_err, cudaStream_t st) {
  if (ntickets <= 0) return;
  count_launches(2);
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  }
  cudaMemsetAsync(sync, 0, (2 + nslots) * sizeof(int), st);
  kb_ghost_prologue<3, 4><<<4 * nsm, 128, 0, st>>>(items, mask, B);
  const int g = grid < ntickets ? grid : ntickets;
  kb_blusgs_strip<3, 4, 16><<<g > 0 ? g : 1, 32, 0, st>>>(items, tickets, ntickets, mask, forward, sync, sticky_err,
                                                         1 << 22);
}

void launch_b_blusgs_sweep(const BItem* items, const int* mask, int B, int nsteps, int forward, int blocks,
                           int* sync, int* sticky_err, cudaStream_t st) {
  count_launches(1);
  cudaMemsetAsync(sync, 0, 2 * sizeof(int), st);
  int b = B, ns = nsteps, fw = forward, spin = wait_limit();
  void* args[] = {(void*)&items, (void*)&mask, (void*)&b, (void*)&ns, (void*)&fw, (void*)&sync,
                  (void*)&sticky_err, (void*)&spin};
  cudaLaunchCooperativeKernel((const void*)kb_blusgs_sweep<3, 4, 16>, dim3(blocks), dim3(128), args, 0, st);
}

int b_blusgs_max_blocks_per_sm() {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kb_blusgs_sweep<3, 4, 16>, 128, 0);
  return nb;
}

}  // namespace swnmg
