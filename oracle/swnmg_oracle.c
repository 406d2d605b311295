/*
 * swnmg_oracle.c -- TEST INFRASTRUCTURE, not part of the library.
 *
 * A plain, slow, single-threaded FP64 CPU restatement of the Newton multigrid
 * method (NMGM) of Wu & Tang, "A Newton multigrid method for steady-state
 * shallow water equations with topography and dry areas" (arXiv:1608.06721),
 * written from the paper's equations in the paper's order.  It exists only to
 * check the CUDA library: tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline are the only callers.  It shares no code, header or table with the
 * CUDA path.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no FMA contraction, so every
 * a*b+c rounds twice; the flux arithmetic is written in one fixed order that
 * the CUDA flux code also follows, which makes residuals and finite-difference
 * Jacobians comparable bit for bit).
 *
 * Layouts (shared with the library's interface, not its code):
 *   cell index      i = ix + nx*iy (x fastest)
 *   mesh            uniform Cartesian, or (2D) structured curvilinear with
 *                   vertex (a, b) at (mesh_x, mesh_y)[a + (nx+1)*b]
 *   state / vectors SoA: comp c of cell i at v[c*n + i]; 1D: (h, hu), 2D: (h, hu, hv)
 *   blocks          blk[((i*5 + b)*nc + s)*nc + k], b = 0 diag, 1 W, 2 E, 3 S, 4 N;
 *                   block b maps the neighbour's unknown k to equation s of cell i.
 *
 * Readings of the paper that this file fixes (the paper is silent there) are
 * named where they are used: edge orientation, the dry-velocity rule, the
 * inflow ghost solve, the Galerkin/restriction summation order, the coarse
 * solve, the smoothing counts and the stop test.
 *
 * Parity status: pinned by tests/test_oracle_*.py (lake at rest, Bernoulli
 * closed form, flux properties, dense-matrix restatements of Algorithm 0,
 * central-difference Jacobian, the paper's Newton counts and spectral radii;
 * on curvilinear meshes: the Cartesian special case, rotation invariance,
 * free-stream preservation, and the oblique-jump plateau heights of
 * Example 3.4).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---- configuration (mirrors the C-ABI structs field for field) ---------- */
enum { BC_WALL_REFLECT = 0, BC_WALL_SLIP = 1, BC_INFLOW_DISCHARGE = 2,
       BC_OUTFLOW_DEPTH = 3, BC_SUPER_INFLOW = 4, BC_SUPER_OUTFLOW = 5, BC_AUTO_FROUDE = 6 };
enum { FLUX_HLL = 0, FLUX_HLLC = 1, FLUX_LLF = 2, FLUX_ROE = 3 };
enum { INIT_CASCADE = 0, INIT_NONE = 1 };
enum { ST_OK = 0, ST_ARG = 1, ST_NOT_CONVERGED = 3, ST_NONFINITE = 4, ST_DIVERGED = 5 };

typedef struct { int kind; double h, q, ut; } orc_bc;   /* q: discharge along +axis */

typedef struct {
  int dim, nx, ny;
  double x0, x1, y0, y1, g;
  orc_bc bc[4];                       /* sides W, E, S, N */
  int flux, llf_wetdry;
  double alpha, fd_eps, tau, h_eps, eps_r, eps_p, tol;
  int n_levels, n_mg, nu1, nu2, gamma, coarse_sweeps, max_newton, max_blusgs, init_mode;
  double eps_f;                       /* Harten's entropy-fix width of the Roe flux */
  /* implicit time step (Remark 2.6), active when t_ka > 0: the level-0
   * residual becomes (1 - beta) R(U) + |K_i|/dt U - t_src with
   * t_src = |K_i|/dt U^n - beta R(U^n), t_ka = |K_i|/dt, t_omb = 1 - beta */
  double t_ka, t_omb;
  const double* t_src;
  /* structured curvilinear quadrilateral mesh (2D; both NULL: the uniform
   * Cartesian mesh of [x0,x1] x [y0,y1]).  Vertex (a, b), 0 <= a <= nx,
   * 0 <= b <= ny, lies at (mesh_x, mesh_y)[a + (nx + 1) b]; cell (ix, iy) has
   * the corners (ix, iy), (ix+1, iy), (ix+1, iy+1), (ix, iy+1).  The coarse
   * mesh of level l is that of every 2^l-th vertex. */
  const double* mesh_x;
  const double* mesh_y;
  const double* t_kai;                /* per-cell |K_i|/dt of a time step on such a mesh */
  int smoother;                       /* block SGS order: 0 lexicographic (the paper's), 1 two colours */
} orc_cfg;

#define ORC_HIST 512
typedef struct {
  int status, n_newton, n_vcycles;
  int blusgs_sweeps[16];
  double init_res, final_res;
  double res_hist[ORC_HIST];          /* sum ||R_i||_1 after Newton step n+1 */
} orc_stats;

typedef struct {
  int nx, ny, n;
  double ex, ey;                      /* Cartesian: ex = |x-edge|, ey = |y-edge| */
  const double* vx;                   /* curvilinear: the finest vertices, NULL otherwise */
  const double* vy;
  int vrow, vstep;                    /* vertex row length (nx + 1) and 2^l */
} lvl;

static int ncomp(const orc_cfg* c) { return c->dim == 2 ? 3 : 2; }

static lvl level_geom(const orc_cfg* c, int l) {
  lvl L;
  L.vx = L.vy = NULL;
  L.vrow = c->nx + 1;
  L.vstep = 1 << l;
  if (c->dim == 2 && c->mesh_x && c->mesh_y) { L.vx = c->mesh_x; L.vy = c->mesh_y; }
  L.nx = c->nx >> l;
  L.ny = (c->dim == 2) ? (c->ny >> l) : 1;
  L.n = L.nx * L.ny;
  if (c->dim == 2) {
    double s = (double)(1 << l);
    double dx = (c->x1 - c->x0) / c->nx, dy = (c->y1 - c->y0) / c->ny;
    L.ex = dy * s;                      /* x-edges (W/E) are vertical: length dy */
    L.ey = dx * s;
  } else {                              /* 1D: R_i = F_{i+1/2} - F_{i-1/2} - S_i (Remark 2.1) */
    L.ex = 1.0;
    L.ey = 0.0;
  }
  return L;
}

/* neighbour of cell i across side (0 W, 1 E, 2 S, 3 N), -1 on the boundary */
static int nbr(const lvl* L, int i, int side) {
  int ix = i % L->nx, iy = i / L->nx;
  switch (side) {
    case 0: return ix > 0 ? i - 1 : -1;
    case 1: return ix < L->nx - 1 ? i + 1 : -1;
    case 2: return iy > 0 ? i - L->nx : -1;
    default: return iy < L->ny - 1 ? i + L->nx : -1;
  }
}

/* ---- structured curvilinear meshes (Examples 3.4, 3.5) --------------------
 * Every quantity of eq. totalFlux that depends on the mesh -- |e_ij|, n_ij and
 * |K_i| -- is taken from the straight segments between a cell's four
 * vertices. */
static int curvilinear(const lvl* L) { return L->vx != NULL; }

static void vertex(const lvl* L, int a, int b, double* x, double* y) {
  size_t k = (size_t)a * L->vstep + (size_t)L->vrow * ((size_t)b * L->vstep);
  *x = L->vx[k];
  *y = L->vy[k];
}

/* Edge `side` (0 W, 1 E, 2 S, 3 N) of cell i: its length |e| and its unit
 * normal n, oriented from the lower-index cell to the higher-index one (the
 * +i direction on W/E edges, +j on S/N edges, as on the Cartesian mesh).
 * t = the edge's vertex difference, from (a, b) to (a, b+1) on W/E edges and
 * from (a, b) to (a+1, b) on S/N edges; n is t turned by -90 degrees on W/E
 * edges and by +90 degrees on S/N edges. */
static void edge_frame(const lvl* L, int i, int side, double* len, double* nx, double* ny) {
  int ix = i % L->nx, iy = i / L->nx;
  int a0 = ix, b0 = iy, a1, b1;
  if (side < 2) { a0 = ix + (side & 1); a1 = a0; b1 = iy + 1; }
  else { b0 = iy + (side & 1); b1 = b0; a1 = ix + 1; }
  double xa, ya, xb, yb;
  vertex(L, a0, b0, &xa, &ya);
  vertex(L, a1, b1, &xb, &yb);
  double tx = xb - xa, ty = yb - ya;
  double l = sqrt(tx * tx + ty * ty);
  *len = l;
  if (side < 2) { *nx = ty / l; *ny = -tx / l; }
  else { *nx = -ty / l; *ny = tx / l; }
}

/* |K_i| of the quadrilateral (shoelace form: half the cross product of its
 * diagonals); positive for a mesh whose i and j directions are
 * counter-clockwise */
static double cell_area(const lvl* L, int i) {
  int ix = i % L->nx, iy = i / L->nx;
  double x00, y00, x10, y10, x11, y11, x01, y01;
  vertex(L, ix, iy, &x00, &y00);
  vertex(L, ix + 1, iy, &x10, &y10);
  vertex(L, ix + 1, iy + 1, &x11, &y11);
  vertex(L, ix, iy + 1, &x01, &y01);
  return 0.5 * ((x11 - x00) * (y01 - y10) - (x01 - x10) * (y11 - y00));
}

static double mn(double a, double b) { return (a < b) ? a : b; }
static double mx(double a, double b) { return (a > b) ? a : b; }

/* velocities of a cell: u = hu/h, v = hv/h evaluated as hu*(1/h), hv*(1/h);
 * both taken as 0 where h < h_eps (the paper treats such cells as dry,
 * Remark 2.5; u is undefined at h = 0). */
static void vels(double h, double qa, double qb, double h_eps, double* ua, double* ub) {
  if (h >= h_eps) { double r = 1.0 / h; *ua = qa * r; *ub = qb * r; }
  else { *ua = 0.0; *ub = 0.0; }
}

/* ---- Section 2.1: fluxes ------------------------------------------------ */

/* physical flux F(U).n in the edge frame: U = (h, h u_n, h u_t) */
static void phys_flux(double half_g, double h, double un, double ut, double F[3]) {
  double qn = h * un;
  F[0] = qn;
  F[1] = qn * un + half_g * (h * h);
  F[2] = qn * ut;
}

/* HLL flux, Remark 2.2 (eq. HLLflux, wet/dry wave speeds s_L, s_R with
 * u_*, h_*); with hllc != 0 the third component is replaced by the HLLC
 * contact choice u_tau,-/+ * f1 selected by s_M. */
static void flux_hll(const orc_cfg* c, double hl, double ul, double vl,
                     double hr, double ur, double vr, int hllc, double F[3]) {
  double g = c->g, half_g = 0.5 * c->g;
  if (hl == 0.0 && hr == 0.0) { F[0] = F[1] = F[2] = 0.0; return; }
  double cl = sqrt(g * hl), cr = sqrt(g * hr);
  double us = ((ul + ur) * 0.5 + cl) - cr;
  /* h_* = (t)^2/(4g) with t = sqrt(g h-) + sqrt(g h+) + (u- - u+)/2, so
   * sqrt(g h_*) = |t|/2 exactly; it is evaluated in that form. */
  double t = (cl + cr) + (ul - ur) * 0.5;
  double cs = fabs(t) * 0.5;
  double sL = (hl == 0.0) ? ur - 2.0 * cr : mn(ul - cl, us - cs);
  double sR = (hr == 0.0) ? ul + 2.0 * cl : mx(ur + cr, us + cs);
  double FL[3], FR[3];
  phys_flux(half_g, hl, ul, vl, FL);
  phys_flux(half_g, hr, ur, vr, FR);
  if (sL >= 0.0) { F[0] = FL[0]; F[1] = FL[1]; F[2] = FL[2]; return; }
  if (sR <= 0.0) { F[0] = FR[0]; F[1] = FR[1]; F[2] = FR[2]; return; }
  double UL[3] = { hl, hl * ul, hl * vl };
  double UR[3] = { hr, hr * ur, hr * vr };
  double rden = 1.0 / (sR - sL), p = sL * sR;
  for (int k = 0; k < 3; ++k)
    F[k] = ((sR * FL[k] - sL * FR[k]) + p * (UR[k] - UL[k])) * rden;
  if (hllc) {
    double a = hr * (ur - sR), b = hl * (ul - sL);
    double sM = (sL * a - sR * b) / (a - b);
    F[2] = (sM >= 0.0) ? vl * F[0] : vr * F[0];   /* s_L<0<=s_M: left; s_M<0<s_R: right */
  }
}

/* local Lax-Friedrichs flux, eq. LLFflux, with the wet/dry speed increase
 * eps_r*sqrt(g*max(h-,h+)) applied on every edge when llf_wetdry is set. */
static void flux_llf(const orc_cfg* c, double hl, double ul, double vl,
                     double hr, double ur, double vr, double F[3]) {
  double g = c->g, half_g = 0.5 * c->g;
  if (hl == 0.0 && hr == 0.0) { F[0] = F[1] = F[2] = 0.0; return; }
  double cl = sqrt(g * hl), cr = sqrt(g * hr);
  double smax = mx(fabs(ul) + cl, fabs(ur) + cr);
  if (c->llf_wetdry) smax = smax + c->eps_r * sqrt(g * mx(hl, hr));
  double FL[3], FR[3];
  phys_flux(half_g, hl, ul, vl, FL);
  phys_flux(half_g, hr, ur, vr, FR);
  double UL[3] = { hl, hl * ul, hl * vl };
  double UR[3] = { hr, hr * ur, hr * vr };
  for (int k = 0; k < 3; ++k)
    F[k] = ((FL[k] + FR[k]) - smax * (UR[k] - UL[k])) * 0.5;
}

/* Harten's entropy fix of the Roe flux (Remark 2.2): |x| replaced by
 * x^2/(4 eps_f) + eps_f when |x| < 2 eps_f. */
static double harten_q(double x, double ef) {
  double a = fabs(x);
  return (a < 2.0 * ef) ? (x * x) / (4.0 * ef) + ef : a;
}

/* Roe flux with Harten's entropy fix, eq. ROEflux.  The Roe matrix of the
 * shallow water equations: mean depth h^ = (h- + h+)/2 and sqrt(h)-weighted
 * velocities u^, v^, c^ = sqrt(g h^); eigenvalues u^ - c^, u^, u^ + c^ with
 * right eigenvectors (1, u^ - c^, v^), (0, 0, 1), (1, u^ + c^, v^); the wave
 * strengths chi_k solve U+ - U- = sum chi_k r_k.  In 1D the middle wave has
 * zero strength (no tangential momentum), which leaves the m = 2 form.  Both
 * depths zero: zero flux. */
static void flux_roe(const orc_cfg* c, double hl, double ul, double vl,
                     double hr, double ur, double vr, double F[3]) {
  double g = c->g, half_g = 0.5 * c->g, ef = c->eps_f;
  if (hl == 0.0 && hr == 0.0) { F[0] = F[1] = F[2] = 0.0; return; }
  double sl = sqrt(hl), sr = sqrt(hr);
  double rs = 1.0 / (sl + sr);
  double uh = (sl * ul + sr * ur) * rs;
  double vh = (sl * vl + sr * vr) * rs;
  double ch = sqrt(g * ((hl + hr) * 0.5));
  double FL[3], FR[3];
  phys_flux(half_g, hl, ul, vl, FL);
  phys_flux(half_g, hr, ur, vr, FR);
  double dh = hr - hl, dq = hr * ur - hl * ul, dp = hr * vr - hl * vl;
  double l1 = uh - ch, l3 = uh + ch;
  double r2c = 1.0 / (2.0 * ch);
  double a1 = (l3 * dh - dq) * r2c;   /* chi_1 */
  double a3 = (dq - l1 * dh) * r2c;   /* chi_3 */
  double a2 = dp - vh * dh;           /* chi_2 */
  double w1 = harten_q(l1, ef) * a1, w2 = harten_q(uh, ef) * a2, w3 = harten_q(l3, ef) * a3;
  double D0 = w1 + w3;
  double D1 = w1 * l1 + w3 * l3;
  double D2 = (w1 * vh + w2) + w3 * vh;
  F[0] = ((FL[0] + FR[0]) - D0) * 0.5;
  F[1] = ((FL[1] + FR[1]) - D1) * 0.5;
  F[2] = ((FL[2] + FR[2]) - D2) * 0.5;
}

/* One edge, eq. totalFlux with the hydrostatic reconstruction of section 2.1.
 * Inputs are the two cell states in the edge frame (depth, normal velocity,
 * tangential velocity, bed), the left one being the cell on the lower-index
 * side.  out = (F0, F1, F2, sL, sR) with sL = g/2 h_{e,-}^2, sR = g/2 h_{e,+}^2:
 * the left cell receives F - sL n, the right cell -(F - sR n). */
static void edge_eval(const orc_cfg* c, double hL, double uL, double vL, double zL,
                      double hR, double uR, double vR, double zR, double out[5]) {
  double zs = mx(zL, zR);
  double tl = (hL + zL) - zs, tr = (hR + zR) - zs;
  double hl = (tl > 0.0) ? tl : 0.0, hr = (tr > 0.0) ? tr : 0.0;
  double F[3];
  if (c->flux == FLUX_LLF) flux_llf(c, hl, uL, vL, hr, uR, vR, F);
  else if (c->flux == FLUX_ROE) flux_roe(c, hl, uL, vL, hr, uR, vR, F);
  else flux_hll(c, hl, uL, vL, hr, uR, vR, c->flux == FLUX_HLLC, F);
  double half_g = 0.5 * c->g;
  out[0] = F[0]; out[1] = F[1]; out[2] = F[2];
  out[3] = half_g * (hl * hl);
  out[4] = half_g * (hr * hr);
}

/* ---- Remark 2.3: ghost states ------------------------------------------ */

/* Subcritical inflow with prescribed outward discharge qn (< 0): the ghost
 * celerity c = sqrt(g h_g) solves qn/h_g + 2c = R_I, i.e.
 * f(c) = 2c^3 - R_I c^2 + g qn = 0.  f is convex and increasing right of its
 * largest root, so Newton's method started right of the root (c = R_I, or 1,
 * doubled until f > 0) decreases monotonically; it stops when an iterate no
 * longer decreases (or after 60 steps). */
static double inflow_celerity(double g, double RI, double qn) {
  double gq = g * qn;
  double c = (RI > 0.0) ? RI : 1.0;
  for (int k = 0; k < 200; ++k) {
    double f = ((2.0 * c - RI) * c) * c + gq;
    if (f > 0.0) break;
    c = 2.0 * c;
  }
  for (int it = 0; it < 60; ++it) {
    double f = ((2.0 * c - RI) * c) * c + gq;
    double fp = (6.0 * c - 2.0 * RI) * c;
    if (!(fp > 0.0)) break;
    double cn = c - f / fp;
    if (!(cn < c)) break;
    c = cn;
  }
  return c;
}

/* ghost state for the interior state (hI, uI, vI) in the edge frame; u is the
 * velocity along +axis, v the tangential one; sigma = -1 on W/S, +1 on E/N
 * (so sigma*u is the outward normal velocity u_n of Remark 2.3). */
static void ghost(const orc_cfg* c, const orc_bc* b, double sigma, double hI, double uI,
                  double vI, double* hg, double* ug, double* vg) {
  double g = c->g;
  int kind = b->kind;
  if (kind == BC_AUTO_FROUDE) {
    /* Remark 2.3's choice by the interior's local Froude number |u|/sqrt(g h)
     * (compared as |u|^2 >= g h: supercritical, a dry cell included) and the
     * sign of the outward normal velocity (u_n < 0: inflow) */
    int super = (uI * uI + vI * vI) >= g * hI;
    int in = (sigma * uI) < 0.0;
    kind = super ? (in ? BC_SUPER_INFLOW : BC_SUPER_OUTFLOW) : (in ? BC_INFLOW_DISCHARGE : BC_OUTFLOW_DEPTH);
  }
  switch (kind) {
    case BC_WALL_SLIP: *hg = hI; *ug = 0.0; *vg = vI; break;
    case BC_INFLOW_DISCHARGE: {
      double qn = sigma * b->q;
      double RI = sigma * uI + 2.0 * sqrt(g * hI);
      double cg = inflow_celerity(g, RI, qn);
      double h = (cg * cg) / g;
      double un = (h > 0.0) ? qn / h : 0.0;
      *hg = h; *ug = sigma * un; *vg = b->ut;
      break;
    }
    case BC_OUTFLOW_DEPTH: {
      double un = (sigma * uI + 2.0 * sqrt(g * hI)) - 2.0 * sqrt(g * b->h);
      *hg = b->h; *ug = sigma * un; *vg = vI;
      break;
    }
    case BC_SUPER_INFLOW:
      *hg = b->h; *ug = (b->h > 0.0) ? b->q / b->h : 0.0; *vg = b->ut; break;
    case BC_SUPER_OUTFLOW: *hg = hI; *ug = uI; *vg = vI; break;
    default: /* reflective wall */
      *hg = hI; *ug = -uI; *vg = vI; break;
  }
}

/* ---- per-cell edge term G (the piece of R_i contributed by one edge) ----- */

/* conserved state of cell idx, with comp pk of cell pc raised by eps */
static void load_state(const double* U, int n, int nc, int idx, int pc, int pk, double eps,
                       double q[3]) {
  q[2] = 0.0;
  for (int k = 0; k < nc; ++k) q[k] = U[k * n + idx];
  if (idx == pc) q[pk] = q[pk] + eps;
}

/* G received by cell i from its edge `side`, in global components; the state
 * of cell pc (i or its neighbour) has component pk perturbed by eps.  The
 * edge is always evaluated with its lower-index cell on the left. */
static void cell_G_curv(const orc_cfg* c, const lvl* L, const double* z, const double* U, int i,
                        int side, int pc, int pk, double eps, double G[3]);

static void cell_G(const orc_cfg* c, const lvl* L, const double* z, const double* U, int i,
                   int side, int pc, int pk, double eps, double G[3]) {
  if (curvilinear(L)) { cell_G_curv(c, L, z, U, i, side, pc, pk, eps, G); return; }
  int nc = ncomp(c), n = L->n;
  int axis = side >> 1, upper = side & 1;
  int j = nbr(L, i, side);
  double qi[3], hi, ui, vi, hj, uj, vj, zj;
  load_state(U, n, nc, i, pc, pk, eps, qi);
  hi = qi[0];
  if (axis == 0) vels(hi, qi[1], qi[2], c->h_eps, &ui, &vi);
  else vels(hi, qi[2], qi[1], c->h_eps, &ui, &vi);
  if (j >= 0) {
    double qj[3];
    load_state(U, n, nc, j, pc, pk, eps, qj);
    hj = qj[0];
    if (axis == 0) vels(hj, qj[1], qj[2], c->h_eps, &uj, &vj);
    else vels(hj, qj[2], qj[1], c->h_eps, &uj, &vj);
    zj = z[j];
  } else {
    ghost(c, &c->bc[side], upper ? 1.0 : -1.0, hi, ui, vi, &hj, &uj, &vj);
    zj = z[i];                                  /* ghost bed = interior bed */
  }
  double o[5], Ge[3];
  if (upper) {                                  /* cell i is the left state */
    edge_eval(c, hi, ui, vi, z[i], hj, uj, vj, zj, o);
    Ge[0] = o[0]; Ge[1] = o[1] - o[3]; Ge[2] = o[2];
  } else {                                      /* cell i is the right state */
    edge_eval(c, hj, uj, vj, zj, hi, ui, vi, z[i], o);
    Ge[0] = -o[0]; Ge[1] = -(o[1] - o[4]); Ge[2] = -o[2];
  }
  if (axis == 0) { G[0] = Ge[0]; G[1] = Ge[1]; G[2] = Ge[2]; }
  else { G[0] = Ge[0]; G[1] = Ge[2]; G[2] = Ge[1]; }
}

/* cell_G on a curvilinear mesh.  The states are taken to the edge frame
 * (h, u_n, u_tau) with u_n = u.n and u_tau = u.tau, tau being n turned by
 * +90 degrees on W/E edges and by -90 degrees on S/N edges (so that on a
 * Cartesian mesh the frame is the one above: u_tau is v on W/E edges and u
 * on S/N edges; a boundary's discharge q is along n and its u_tau along tau).
 * The flux is taken back to global components, F_n = F_1 n + F_2 tau, and the
 * source term of eq. totalFlux, g/2 h_{e,-}^2 (n^x, n^y), is subtracted there. */
static void cell_G_curv(const orc_cfg* c, const lvl* L, const double* z, const double* U, int i,
                        int side, int pc, int pk, double eps, double G[3]) {
  int n = L->n, upper = side & 1;
  int j = nbr(L, i, side);
  double len, nx, ny;
  edge_frame(L, i, side, &len, &nx, &ny);
  double tx = (side < 2) ? -ny : ny, ty = (side < 2) ? nx : -nx;
  double qi[3], u, v, hi, ui, vi, hj, uj, vj, zj;
  load_state(U, n, 3, i, pc, pk, eps, qi);
  hi = qi[0];
  vels(hi, qi[1], qi[2], c->h_eps, &u, &v);
  ui = u * nx + v * ny;
  vi = u * tx + v * ty;
  if (j >= 0) {
    double qj[3];
    load_state(U, n, 3, j, pc, pk, eps, qj);
    hj = qj[0];
    vels(hj, qj[1], qj[2], c->h_eps, &u, &v);
    uj = u * nx + v * ny;
    vj = u * tx + v * ty;
    zj = z[j];
  } else {
    ghost(c, &c->bc[side], upper ? 1.0 : -1.0, hi, ui, vi, &hj, &uj, &vj);
    zj = z[i];                                  /* ghost bed = interior bed */
  }
  double o[5];
  if (upper) edge_eval(c, hi, ui, vi, z[i], hj, uj, vj, zj, o);
  else edge_eval(c, hj, uj, vj, zj, hi, ui, vi, z[i], o);
  double fx = o[1] * nx + o[2] * tx, fy = o[1] * ny + o[2] * ty;
  double s = upper ? o[3] : o[4];
  double G0 = o[0], G1 = fx - s * nx, G2 = fy - s * ny;
  if (upper) { G[0] = G0; G[1] = G1; G[2] = G2; }
  else { G[0] = -G0; G[1] = -G1; G[2] = -G2; }
}

static int nsides(const orc_cfg* c) { return c->dim == 2 ? 4 : 2; }

/* |e| of edge `side` of cell i */
static double edge_len(const lvl* L, int i, int side) {
  if (!curvilinear(L)) return side < 2 ? L->ex : L->ey;
  double len, nx, ny;
  edge_frame(L, i, side, &len, &nx, &ny);
  return len;
}

static double l1norm(const double* r, int nc) {
  double s = fabs(r[0]) + fabs(r[1]);
  if (nc == 3) s = s + fabs(r[2]);
  return s;
}

/* |K_i|/dt of a time step: one value on the uniform mesh, per cell on a curvilinear one */
static double time_ka(const orc_cfg* c, int i) { return c->t_kai ? c->t_kai[i] : c->t_ka; }

/* Remark 2.6: the time-step residual of cell i on level 0 from its flux sum R */
static void time_residual(const orc_cfg* c, const lvl* L, const double* U, int i, double R[3]) {
  int nc = ncomp(c), n = L->n;
  for (int s = 0; s < nc; ++s)
    R[s] = (c->t_omb * R[s] + time_ka(c, i) * U[s * n + i]) - c->t_src[s * n + i];
}

static int time_mode(const orc_cfg* c, const lvl* L) { return c->t_ka > 0.0 && L->nx == c->nx; }

/* eq. Res: R_i = sum_e |e| F_hat(...), edges in the order W, E, S, N */
static void cell_residual(const orc_cfg* c, const lvl* L, const double* z, const double* U,
                          int i, double R[3]) {
  int nc = ncomp(c);
  R[0] = R[1] = R[2] = 0.0;
  for (int side = 0; side < nsides(c); ++side) {
    double G[3], len = edge_len(L, i, side);
    cell_G(c, L, z, U, i, side, -1, 0, 0.0, G);
    for (int s = 0; s < nc; ++s) R[s] = R[s] + len * G[s];
  }
  if (time_mode(c, L)) time_residual(c, L, U, i, R);
}

/* eq. NumerDiff plus eq. NewtonREG: the diagonal block
 * D_i = sum_e |e| (G(U_i + eps e_k) - G(U_i))/eps  +  alpha ||R_i||_1 I
 * (the quotient by eps is taken as a product with 1/eps)
 * (boundary edges recompute the ghost from the perturbed U_i), and optionally
 * the off-diagonal blocks |e| (G(U_j + eps e_k) - G(U_j))/eps. */
static void cell_jacobian(const orc_cfg* c, const lvl* L, const double* z, const double* U,
                          int i, double R[3], double* rn, double D[9], double* offd /*4x9 or NULL*/) {
  int nc = ncomp(c);
  double eps = c->fd_eps, reps = 1.0 / c->fd_eps;
  for (int e = 0; e < 9; ++e) D[e] = 0.0;
  if (offd) for (int e = 0; e < 36; ++e) offd[e] = 0.0;
  R[0] = R[1] = R[2] = 0.0;
  for (int side = 0; side < nsides(c); ++side) {
    double len = edge_len(L, i, side), Gb[3], Gp[3];
    cell_G(c, L, z, U, i, side, -1, 0, 0.0, Gb);
    for (int s = 0; s < nc; ++s) R[s] = R[s] + len * Gb[s];
    for (int k = 0; k < nc; ++k) {
      cell_G(c, L, z, U, i, side, i, k, eps, Gp);
      for (int s = 0; s < nc; ++s) D[s * nc + k] = D[s * nc + k] + len * ((Gp[s] - Gb[s]) * reps);
    }
    int j = nbr(L, i, side);
    if (offd && j >= 0) {
      for (int k = 0; k < nc; ++k) {
        cell_G(c, L, z, U, i, side, j, k, eps, Gp);
        for (int s = 0; s < nc; ++s) offd[side * 9 + s * nc + k] = len * ((Gp[s] - Gb[s]) * reps);
      }
    }
  }
  if (time_mode(c, L)) {   /* d/dU of (1 - beta) R + |K|/dt U: scaled blocks, |K|/dt on the diagonal */
    time_residual(c, L, U, i, R);
    for (int e = 0; e < nc * nc; ++e) D[e] = c->t_omb * D[e];
    for (int s = 0; s < nc; ++s) D[s * nc + s] = D[s * nc + s] + time_ka(c, i);
    if (offd) for (int e = 0; e < 36; ++e) offd[e] = c->t_omb * offd[e];
  }
  *rn = l1norm(R, nc);
  for (int s = 0; s < nc; ++s) D[s * nc + s] = D[s * nc + s] + c->alpha * (*rn);
}

/* ---- 3x3 / 2x2 block LU with partial pivoting and a singular guard ------- */
typedef struct { double m[9]; int perm[3]; int sing[3]; } blu;

/* Gaussian elimination with partial pivoting (largest |entry|, lowest row on
 * ties).  A pivot with |p| <= 1e-14 max|D| marks its unknown singular: the
 * solve sets that unknown to zero (wet/dry blocks are singular, Example 3.3). */
static void lu_factor(int n, const double* A, blu* f) {
  double amax = 0.0;
  for (int e = 0; e < n * n; ++e) { double a = fabs(A[e]); if (a > amax) amax = a; }
  double tiny = 1e-14 * amax;
  for (int e = 0; e < n * n; ++e) f->m[e] = A[e];
  for (int r = 0; r < n; ++r) { f->perm[r] = r; f->sing[r] = 0; }
  for (int col = 0; col < n; ++col) {
    int p = col; double best = fabs(f->m[col * n + col]);
    for (int r = col + 1; r < n; ++r) { double a = fabs(f->m[r * n + col]); if (a > best) { best = a; p = r; } }
    if (p != col) {
      for (int k = 0; k < n; ++k) { double t = f->m[col * n + k]; f->m[col * n + k] = f->m[p * n + k]; f->m[p * n + k] = t; }
      int t = f->perm[col]; f->perm[col] = f->perm[p]; f->perm[p] = t;
    }
    if (!(best > tiny)) {
      f->sing[col] = 1;
      for (int r = col + 1; r < n; ++r) f->m[r * n + col] = 0.0;
      continue;
    }
    for (int r = col + 1; r < n; ++r) {
      double l = f->m[r * n + col] / f->m[col * n + col];
      f->m[r * n + col] = l;
      for (int k = col + 1; k < n; ++k) f->m[r * n + k] = f->m[r * n + k] - l * f->m[col * n + k];
    }
  }
}

static void lu_solve(int n, const blu* f, const double* b, double* x) {
  double y[3];
  for (int r = 0; r < n; ++r) y[r] = b[f->perm[r]];
  for (int r = 0; r < n; ++r)
    for (int k = 0; k < r; ++k) y[r] = y[r] - f->m[r * n + k] * y[k];
  for (int r = n - 1; r >= 0; --r) {
    if (f->sing[r]) { x[r] = 0.0; continue; }
    double s = y[r];
    for (int k = r + 1; k < n; ++k) s = s - f->m[r * n + k] * x[k];
    x[r] = s / f->m[r * n + r];
  }
}

/* ---- public: residual / Jacobian on level l ----------------------------- */

static int check_cfg(const orc_cfg* c) {
  if (!c || (c->dim != 1 && c->dim != 2) || c->nx < 1 || (c->dim == 2 && c->ny < 1)) return ST_ARG;
  if (c->n_levels < 0 || c->n_levels > 12) return ST_ARG;
  if (c->smoother < 0 || c->smoother > 1) return ST_ARG;
  if (c->flux < 0 || c->flux > FLUX_ROE || (c->flux == FLUX_ROE && !(c->eps_f > 0.0))) return ST_ARG;
  int m = 1 << c->n_levels;
  if (c->nx % m) return ST_ARG;
  if (c->dim == 2 && c->ny % m) return ST_ARG;
  if ((c->mesh_x != NULL) != (c->mesh_y != NULL)) return ST_ARG;
  if (c->mesh_x) {                    /* every level's cells positive and their edges non-degenerate */
    if (c->dim != 2) return ST_ARG;
    for (int l = 0; l <= c->n_levels; ++l) {
      lvl L = level_geom(c, l);
      for (int i = 0; i < L.n; ++i) {
        if (!(cell_area(&L, i) > 0.0)) return ST_ARG;
        for (int side = 0; side < 4; ++side) if (!(edge_len(&L, i, side) > 0.0)) return ST_ARG;
      }
    }
  }
  return ST_OK;
}

int orc_level_cells(const orc_cfg* c, int l) { lvl L = level_geom(c, l); return L.n; }

/* |K_i| of every cell of level l (curvilinear meshes; ST_ARG otherwise) */
int orc_cell_areas(const orc_cfg* c, int l, double* out) {
  lvl L = level_geom(c, l);
  if (!curvilinear(&L)) return ST_ARG;
  for (int i = 0; i < L.n; ++i) out[i] = cell_area(&L, i);
  return ST_OK;
}

int orc_residual(const orc_cfg* c, int l, const double* z, const double* U, double* R, double* rn) {
  lvl L = level_geom(c, l);
  int nc = ncomp(c);
  for (int i = 0; i < L.n; ++i) {
    double r[3];
    cell_residual(c, &L, z, U, i, r);
    for (int s = 0; s < nc; ++s) R[s * L.n + i] = r[s];
    if (rn) rn[i] = l1norm(r, nc);
  }
  return ST_OK;
}

double orc_residual_sum(const orc_cfg* c, int l, const double* z, const double* U) {
  lvl L = level_geom(c, l);
  double s = 0.0;
  for (int i = 0; i < L.n; ++i) {
    double r[3];
    cell_residual(c, &L, z, U, i, r);
    s = s + l1norm(r, ncomp(c));
  }
  return s;
}

/* blocks in the export layout (see header comment), D includes alpha*||R_i||_1 */
int orc_jacobian(const orc_cfg* c, int l, const double* z, const double* U, double* R, double* rn,
                 double* blk) {
  lvl L = level_geom(c, l);
  int nc = ncomp(c), bs = nc * nc;
  for (int i = 0; i < L.n; ++i) {
    double r[3], D[9], off[36], rni;
    cell_jacobian(c, &L, z, U, i, r, &rni, D, off);
    if (R) for (int s = 0; s < nc; ++s) R[s * L.n + i] = r[s];
    if (rn) rn[i] = rni;
    double* b = blk + (size_t)i * 5 * bs;
    for (int e = 0; e < bs; ++e) b[e] = D[e];
    for (int side = 0; side < 4; ++side)
      for (int s = 0; s < nc; ++s)
        for (int k = 0; k < nc; ++k)
          b[(1 + side) * bs + s * nc + k] = (side < nsides(c)) ? off[side * 9 + s * nc + k] : 0.0;
  }
  return ST_OK;
}

/* single-edge flux, for unit tests: states in the edge frame */
void orc_edge_flux(const orc_cfg* c, double hL, double uL, double vL, double zL,
                   double hR, double uR, double vR, double zR, double* out5) {
  edge_eval(c, hL, uL, vL, zL, hR, uR, vR, zR, out5);
}

void orc_ghost(const orc_cfg* c, int side, double hI, double uI, double vI, double* out3) {
  ghost(c, &c->bc[side], (side & 1) ? 1.0 : -1.0, hI, uI, vI, &out3[0], &out3[1], &out3[2]);
}

/* ---- Section 2.3: multigrid pieces --------------------------------------- */

/* children of coarse cell I in the order (0,0), (1,0), (0,1), (1,1); 1D: (0), (1) */
static int children(const orc_cfg* c, const lvl* Lf, const lvl* Lc, int I, int ch[4]) {
  int Ix = I % Lc->nx, Iy = I / Lc->nx;
  if (c->dim == 1) { ch[0] = 2 * Ix; ch[1] = 2 * Ix + 1; return 2; }
  int fx = 2 * Ix, fy = 2 * Iy;
  ch[0] = fx + Lf->nx * fy;       ch[1] = fx + 1 + Lf->nx * fy;
  ch[2] = fx + Lf->nx * (fy + 1); ch[3] = fx + 1 + Lf->nx * (fy + 1);
  return 4;
}

static void badd(double* dst, const double* a, int bs) { for (int e = 0; e < bs; ++e) dst[e] = dst[e] + a[e]; }

/* eq. ProjectAR, first half: A_{IJ,l+1} = sum_{i in I} sum_{j in J} A_{ij,l}.
 * Diagonal: children's diagonals in child order, then the couplings between
 * children 00->10, 10->00, 00->01, 01->00, 10->11, 11->10, 01->11, 11->01.
 * Off-diagonals: the two couplings that cross the coarse edge, lower child first. */
int orc_galerkin(const orc_cfg* c, int l, const double* bf, double* bc_out) {
  lvl Lf = level_geom(c, l), Lc = level_geom(c, l + 1);
  int nc = ncomp(c), bs = nc * nc;
  for (int I = 0; I < Lc.n; ++I) {
    int ch[4];
    children(c, &Lf, &Lc, I, ch);
    double* o = bc_out + (size_t)I * 5 * bs;
    for (int e = 0; e < 5 * bs; ++e) o[e] = 0.0;
#define FB(cell, b) (bf + ((size_t)(cell) * 5 + (b)) * bs)
    if (c->dim == 1) {
      badd(o, FB(ch[0], 0), bs); badd(o, FB(ch[1], 0), bs);
      badd(o, FB(ch[0], 2), bs); badd(o, FB(ch[1], 1), bs);
      badd(o + 1 * bs, FB(ch[0], 1), bs);
      badd(o + 2 * bs, FB(ch[1], 2), bs);
    } else {
      for (int q = 0; q < 4; ++q) badd(o, FB(ch[q], 0), bs);
      badd(o, FB(ch[0], 2), bs); badd(o, FB(ch[1], 1), bs);   /* 00 <-> 10 */
      badd(o, FB(ch[0], 4), bs); badd(o, FB(ch[2], 3), bs);   /* 00 <-> 01 */
      badd(o, FB(ch[1], 4), bs); badd(o, FB(ch[3], 3), bs);   /* 10 <-> 11 */
      badd(o, FB(ch[2], 2), bs); badd(o, FB(ch[3], 1), bs);   /* 01 <-> 11 */
      badd(o + 1 * bs, FB(ch[0], 1), bs); badd(o + 1 * bs, FB(ch[2], 1), bs);   /* W */
      badd(o + 2 * bs, FB(ch[1], 2), bs); badd(o + 2 * bs, FB(ch[3], 2), bs);   /* E */
      badd(o + 3 * bs, FB(ch[0], 3), bs); badd(o + 3 * bs, FB(ch[1], 3), bs);   /* S */
      badd(o + 4 * bs, FB(ch[2], 4), bs); badd(o + 4 * bs, FB(ch[3], 4), bs);   /* N */
    }
#undef FB
  }
  return ST_OK;
}

/* fine-level residual of the linear system at cell i: r = b - D x_i - sum_nbr A x_j */
static void lin_resid(const orc_cfg* c, const lvl* L, const double* blk, const double* b,
                      const double* x, int i, double r[3]) {
  int nc = ncomp(c), bs = nc * nc, n = L->n;
  const double* D = blk + (size_t)i * 5 * bs;
  for (int s = 0; s < nc; ++s) {
    r[s] = b[s * n + i];
    for (int k = 0; k < nc; ++k) r[s] = r[s] - D[s * nc + k] * x[k * n + i];
  }
  for (int side = 0; side < nsides(c); ++side) {
    int j = nbr(L, i, side);
    if (j < 0) continue;
    const double* A = blk + ((size_t)i * 5 + 1 + side) * bs;
    for (int s = 0; s < nc; ++s)
      for (int k = 0; k < nc; ++k) r[s] = r[s] - A[s * nc + k] * x[k * n + j];
  }
}

/* eq. ProjectAR, second half.  With b = -R the coarse right-hand side is
 * -R_{I,l+1} = sum_{j in I} (b_j - (A x)_j), children summed in child order. */
int orc_restrict(const orc_cfg* c, int l, const double* blk, const double* b, const double* x,
                 double* bc_out) {
  lvl Lf = level_geom(c, l), Lc = level_geom(c, l + 1);
  int nc = ncomp(c);
  for (int I = 0; I < Lc.n; ++I) {
    int ch[4], m = children(c, &Lf, &Lc, I, ch);
    double acc[3] = { 0.0, 0.0, 0.0 }, r[3];
    for (int q = 0; q < m; ++q) {
      lin_resid(c, &Lf, blk, b, x, ch[q], r);
      for (int s = 0; s < nc; ++s) acc[s] = (q == 0) ? r[s] : acc[s] + r[s];
    }
    for (int s = 0; s < nc; ++s) bc_out[s * Lc.n + I] = acc[s];
  }
  return ST_OK;
}

/* eq. correction with piecewise-constant prolongation: x_j += x_I for j in I */
int orc_prolong(const orc_cfg* c, int l, const double* xc, double* xf) {
  lvl Lf = level_geom(c, l), Lc = level_geom(c, l + 1);
  int nc = ncomp(c);
  for (int I = 0; I < Lc.n; ++I) {
    int ch[4], m = children(c, &Lf, &Lc, I, ch);
    for (int q = 0; q < m; ++q)
      for (int s = 0; s < nc; ++s) xf[s * Lf.n + ch[q]] = xf[s * Lf.n + ch[q]] + xc[s * Lc.n + I];
  }
  return ST_OK;
}

static void factor_level(const orc_cfg* c, int n, const double* blk, blu* f) {
  int nc = ncomp(c), bs = nc * nc;
  for (int i = 0; i < n; ++i) lu_factor(nc, blk + (size_t)i * 5 * bs, &f[i]);
}

/* the block Gauss-Seidel update of cell i:
 *   x_i <- D_i^{-1} (b_i - sum_{j != i} A_ij x_j) */
static void gs_cell(const orc_cfg* c, const lvl* L, const double* blk, const blu* f,
                    const double* b, double* x, int i) {
  int nc = ncomp(c), bs = nc * nc, n = L->n;
  double r[3], xi[3];
  for (int s = 0; s < nc; ++s) r[s] = b[s * n + i];
  for (int side = 0; side < nsides(c); ++side) {
    int j = nbr(L, i, side);
    if (j < 0) continue;
    const double* A = blk + ((size_t)i * 5 + 1 + side) * bs;
    for (int s = 0; s < nc; ++s)
      for (int k = 0; k < nc; ++k) r[s] = r[s] - A[s * nc + k] * x[k * n + j];
  }
  lu_solve(nc, &f[i], r, xi);
  for (int s = 0; s < nc; ++s) x[s * n + i] = xi[s];
}

/* one block Gauss-Seidel sweep, forward or backward.  smoother 0 (the
 * paper's): lexicographic order, x fastest, or its reverse.  smoother 1 (a
 * variant, not in the paper): two colours, cell i = (ix, iy) of colour
 * (ix + iy) mod 2; the forward sweep updates every cell of colour 0, then
 * every cell of colour 1, the backward sweep colour 1 then colour 0.  Cells
 * of one colour only couple to the other colour (5-point stencil), so the
 * order inside a colour does not matter. */
static void sgs_half(const orc_cfg* c, const lvl* L, const double* blk, const blu* f,
                     const double* b, double* x, int forward) {
  int n = L->n;
  if (c->smoother == 1) {
    for (int pass = 0; pass < 2; ++pass) {
      int colour = forward ? pass : 1 - pass;
      for (int i = 0; i < n; ++i)
        if (((i % L->nx) + (i / L->nx)) % 2 == colour) gs_cell(c, L, blk, f, b, x, i);
    }
    return;
  }
  for (int t = 0; t < n; ++t) gs_cell(c, L, blk, f, b, x, forward ? t : n - 1 - t);
}

int orc_sgs(const orc_cfg* c, int l, const double* blk, const double* b, double* x, int forward) {
  lvl L = level_geom(c, l);
  blu* f = (blu*)malloc(sizeof(blu) * L.n);
  if (!f) return ST_ARG;
  factor_level(c, L.n, blk, f);
  sgs_half(c, &L, blk, f, b, x, forward);
  free(f);
  return ST_OK;
}

/* exact solve by dense Gaussian elimination with partial pivoting, unknowns
 * ordered cell-major (i*nc + s); a pivot <= 1e-14 max|A| sets its unknown to 0. */
static void dense_solve(const orc_cfg* c, const lvl* L, const double* blk, const double* b,
                        double* x) {
  int nc = ncomp(c), bs = nc * nc, n = L->n, m = n * nc;
  double* A = (double*)calloc((size_t)m * m, sizeof(double));
  double* y = (double*)malloc(sizeof(double) * m);
  int* sing = (int*)calloc(m, sizeof(int));
  for (int i = 0; i < n; ++i) {
    for (int s = 0; s < nc; ++s) {
      y[i * nc + s] = b[s * n + i];
      for (int k = 0; k < nc; ++k) A[(size_t)(i * nc + s) * m + i * nc + k] = blk[(size_t)i * 5 * bs + s * nc + k];
    }
    for (int side = 0; side < nsides(c); ++side) {
      int j = nbr(L, i, side);
      if (j < 0) continue;
      for (int s = 0; s < nc; ++s)
        for (int k = 0; k < nc; ++k)
          A[(size_t)(i * nc + s) * m + j * nc + k] = blk[((size_t)i * 5 + 1 + side) * bs + s * nc + k];
    }
  }
  double amax = 0.0;
  for (size_t e = 0; e < (size_t)m * m; ++e) if (fabs(A[e]) > amax) amax = fabs(A[e]);
  double tiny = 1e-14 * amax;
  for (int col = 0; col < m; ++col) {
    int p = col; double best = fabs(A[(size_t)col * m + col]);
    for (int r = col + 1; r < m; ++r) if (fabs(A[(size_t)r * m + col]) > best) { best = fabs(A[(size_t)r * m + col]); p = r; }
    if (p != col) {
      for (int k = 0; k < m; ++k) { double t = A[(size_t)col * m + k]; A[(size_t)col * m + k] = A[(size_t)p * m + k]; A[(size_t)p * m + k] = t; }
      double t = y[col]; y[col] = y[p]; y[p] = t;
    }
    if (!(best > tiny)) { sing[col] = 1; continue; }
    for (int r = col + 1; r < m; ++r) {
      double l = A[(size_t)r * m + col] / A[(size_t)col * m + col];
      if (l == 0.0) continue;
      for (int k = col; k < m; ++k) A[(size_t)r * m + k] = A[(size_t)r * m + k] - l * A[(size_t)col * m + k];
      y[r] = y[r] - l * y[col];
    }
  }
  double* xs = (double*)malloc(sizeof(double) * m);
  for (int r = m - 1; r >= 0; --r) {
    if (sing[r]) { xs[r] = 0.0; continue; }
    double s = y[r];
    for (int k = r + 1; k < m; ++k) s = s - A[(size_t)r * m + k] * xs[k];
    xs[r] = s / A[(size_t)r * m + r];
  }
  for (int i = 0; i < n; ++i) for (int s = 0; s < nc; ++s) x[s * n + i] = xs[i * nc + s];
  free(A); free(y); free(sing); free(xs);
}

/* coarsest level: 1D exact elimination (the paper solves it exactly); 2D
 * coarse_sweeps symmetric block Gauss-Seidel sweeps from the current x, or an
 * exact solve when coarse_sweeps <= 0. */
static void coarse_solve(const orc_cfg* c, const lvl* L, const double* blk, const blu* f,
                         const double* b, double* x) {
  if (c->dim == 1 || c->coarse_sweeps <= 0) { dense_solve(c, L, blk, b, x); return; }
  for (int k = 0; k < c->coarse_sweeps; ++k) {
    sgs_half(c, L, blk, f, b, x, 1);
    sgs_half(c, L, blk, f, b, x, 0);
  }
}

int orc_coarse_solve(const orc_cfg* c, int l, const double* blk, const double* b, double* x) {
  lvl L = level_geom(c, l);
  blu* f = (blu*)malloc(sizeof(blu) * L.n);
  factor_level(c, L.n, blk, f);
  coarse_solve(c, &L, blk, f, b, x);
  free(f);
  return ST_OK;
}

/* the operator hierarchy of one Newton step */
typedef struct {
  int nl;
  lvl L[13];
  double* blk[13];
  blu* lu[13];
  double* b[13];
  double* x[13];
} hier;

static void hier_free(hier* H) {
  for (int l = 0; l <= H->nl; ++l) { free(H->blk[l]); free(H->lu[l]); free(H->b[l]); free(H->x[l]); }
}

/* levels 1..N_L by eq. ProjectAR from the level-0 blocks; LU of every diagonal */
static void hier_build(const orc_cfg* c, const double* blk0, hier* H) {
  int nc = ncomp(c), bs = nc * nc;
  H->nl = c->n_levels;
  for (int l = 0; l <= H->nl; ++l) {
    H->L[l] = level_geom(c, l);
    int n = H->L[l].n;
    H->blk[l] = (double*)malloc(sizeof(double) * (size_t)n * 5 * bs);
    H->lu[l] = (blu*)malloc(sizeof(blu) * n);
    H->b[l] = (double*)calloc((size_t)n * nc, sizeof(double));
    H->x[l] = (double*)calloc((size_t)n * nc, sizeof(double));
  }
  memcpy(H->blk[0], blk0, sizeof(double) * (size_t)H->L[0].n * 5 * bs);
  for (int l = 0; l < H->nl; ++l) orc_galerkin(c, l, H->blk[l], H->blk[l + 1]);
  for (int l = 0; l <= H->nl; ++l) factor_level(c, H->L[l].n, H->blk[l], H->lu[l]);
}

/* Algorithm 0: x_l <- MG_l^gamma(x_l, b_l) */
static void mg_cycle(const orc_cfg* c, hier* H, int l) {
  int nc = ncomp(c);
  lvl* L = &H->L[l];
  if (l == H->nl) { coarse_solve(c, L, H->blk[l], H->lu[l], H->b[l], H->x[l]); return; }
  for (int k = 0; k < c->nu1; ++k) {
    sgs_half(c, L, H->blk[l], H->lu[l], H->b[l], H->x[l], 1);
    sgs_half(c, L, H->blk[l], H->lu[l], H->b[l], H->x[l], 0);
  }
  orc_restrict(c, l, H->blk[l], H->b[l], H->x[l], H->b[l + 1]);
  memset(H->x[l + 1], 0, sizeof(double) * (size_t)H->L[l + 1].n * nc);
  int gam = (l == 0) ? 1 : c->gamma;
  for (int k = 0; k < gam; ++k) mg_cycle(c, H, l + 1);
  orc_prolong(c, l, H->x[l + 1], H->x[l]);
  for (int k = 0; k < c->nu2; ++k) {
    sgs_half(c, L, H->blk[l], H->lu[l], H->b[l], H->x[l], 1);
    sgs_half(c, L, H->blk[l], H->lu[l], H->b[l], H->x[l], 0);
  }
}

/* ncycles of Algorithm 0 on A x = b at level 0, A given by its level-0 blocks */
int orc_vcycle(const orc_cfg* c, const double* blk0, const double* b, double* x, int ncycles) {
  if (check_cfg(c)) return ST_ARG;
  hier H;
  hier_build(c, blk0, &H);
  int n = H.L[0].n, nc = ncomp(c);
  memcpy(H.b[0], b, sizeof(double) * (size_t)n * nc);
  memcpy(H.x[0], x, sizeof(double) * (size_t)n * nc);
  for (int k = 0; k < ncycles; ++k) mg_cycle(c, &H, 0);
  memcpy(x, H.x[0], sizeof(double) * (size_t)n * nc);
  hier_free(&H);
  return ST_OK;
}

/* coarse blocks of every level, concatenated (level 0 first) */
int orc_hierarchy(const orc_cfg* c, const double* blk0, double* out) {
  if (check_cfg(c)) return ST_ARG;
  hier H;
  hier_build(c, blk0, &H);
  int bs = ncomp(c) * ncomp(c);
  size_t off = 0;
  for (int l = 0; l <= H.nl; ++l) {
    memcpy(out + off, H.blk[l], sizeof(double) * (size_t)H.L[l].n * 5 * bs);
    off += (size_t)H.L[l].n * 5 * bs;
  }
  hier_free(&H);
  return ST_OK;
}

/* ---- Section 2.4: BLU-SGS and Algorithm 1 --------------------------------- */

static void dry_reset(int nc, int n, double* U, int i, double h_eps) {
  if (U[i] < h_eps) for (int s = 0; s < nc; ++s) U[s * n + i] = 0.0;
}

/* BLU-SGS cell update (Algorithm 1, Steps 1 and 2.1):
 * U_i <- U_i - (alpha ||R_i||_1 I + dR_i/dU_i)^{-1} R_i, with R_i from the
 * current neighbours, followed by the dry-cell reset of Remark 2.5.
 * A cell that is dry when its update starts (h_i < h_eps) has zero velocity,
 * so R does not depend on its momentum (those Jacobian columns vanish and
 * only the regularisation fixes that correction); it keeps zero momentum in
 * this update and only its depth changes ("temporarily regarded as a dry
 * cell", Remark 2.5). */
static void blusgs_cell(const orc_cfg* c, const lvl* L, const double* z, double* U, int i) {
  int nc = ncomp(c), n = L->n;
  double R[3], D[9], rn, x[3];
  blu f;
  cell_jacobian(c, L, z, U, i, R, &rn, D, NULL);
  lu_factor(nc, D, &f);
  lu_solve(nc, &f, R, x);
  if (U[i] < c->h_eps) for (int s = 1; s < nc; ++s) x[s] = 0.0;
  for (int s = 0; s < nc; ++s) U[s * n + i] = U[s * n + i] - x[s];
  dry_reset(nc, n, U, i, c->h_eps);
}

/* nsweeps symmetric BLU-SGS sweeps (forward then backward) on level l */
int orc_blusgs(const orc_cfg* c, int l, const double* z, double* U, int nsweeps) {
  lvl L = level_geom(c, l);
  for (int k = 0; k < nsweeps; ++k) {
    for (int i = 0; i < L.n; ++i) blusgs_cell(c, &L, z, U, i);
    for (int i = L.n - 1; i >= 0; --i) blusgs_cell(c, &L, z, U, i);
  }
  return ST_OK;
}

/* average the children of every coarse cell (child order), for z and U: the
 * cell average over the coarse cell (Algorithm 1, Step 1) from the children's
 * averages.  On a curvilinear mesh the children are weighted by their areas,
 * sum_q |K_q| v_q / sum_q |K_q|. */
int orc_average(const orc_cfg* c, int l, int ncomp_v, const double* vf, double* vc) {
  lvl Lf = level_geom(c, l), Lc = level_geom(c, l + 1);
  double w = (c->dim == 2) ? 0.25 : 0.5;
  for (int I = 0; I < Lc.n; ++I) {
    int ch[4], m = children(c, &Lf, &Lc, I, ch);
    if (curvilinear(&Lf)) {
      double ar[4], tot = 0.0;
      for (int q = 0; q < m; ++q) { ar[q] = cell_area(&Lf, ch[q]); tot = tot + ar[q]; }
      for (int s = 0; s < ncomp_v; ++s) {
        double a = 0.0;
        for (int q = 0; q < m; ++q) a = a + ar[q] * vf[s * Lf.n + ch[q]];
        vc[s * Lc.n + I] = a / tot;
      }
      continue;
    }
    for (int s = 0; s < ncomp_v; ++s) {
      double a = vf[s * Lf.n + ch[0]];
      for (int q = 1; q < m; ++q) a = a + vf[s * Lf.n + ch[q]];
      vc[s * Lc.n + I] = a * w;
    }
  }
  return ST_OK;
}

static int finite_vec(const double* v, size_t m) {
  for (size_t e = 0; e < m; ++e) if (!isfinite(v[e])) return 0;
  return 1;
}

/* Algorithm 1 (NMGM).  U (level 0) is the initial data on entry and the
 * computed steady state on return. */
int orc_solve(const orc_cfg* c, const double* z0, double* U0, orc_stats* st) {
  if (check_cfg(c)) return ST_ARG;
  int nc = ncomp(c), bs = nc * nc, NL = c->n_levels;
  memset(st, 0, sizeof(*st));
  lvl L0 = level_geom(c, 0);
  double* zl[13] = { 0 }; double* Ul[13] = { 0 };
  for (int l = 0; l <= NL; ++l) {
    lvl L = level_geom(c, l);
    zl[l] = (double*)malloc(sizeof(double) * L.n);
    Ul[l] = (double*)malloc(sizeof(double) * (size_t)L.n * nc);
  }
  memcpy(zl[0], z0, sizeof(double) * L0.n);
  for (int l = 0; l < NL; ++l) orc_average(c, l, 1, zl[l], zl[l + 1]);

  /* Step 1: initial guess by BLU-SGS from the coarsest level up to level 1.
   * eps_p < 0 selects the paper's rule for it (its remark on Step 1: about
   * one percent of the residual of the initial data): |eps_p| times
   * sum_i ||R_i||_1 of the initial data on the finest mesh. */
  double eps_p = c->eps_p;
  if (c->init_mode == INIT_CASCADE && NL > 0 && eps_p < 0.0) eps_p = -eps_p * orc_residual_sum(c, 0, zl[0], U0);
  if (c->init_mode == INIT_CASCADE && NL > 0) {
    memcpy(Ul[0], U0, sizeof(double) * (size_t)L0.n * nc);
    for (int l = 0; l < NL; ++l) orc_average(c, l, nc, Ul[l], Ul[l + 1]);
    for (int l = NL; l >= 1; --l) {
      double thr = eps_p / (double)(1 << l);
      double res = orc_residual_sum(c, l, zl[l], Ul[l]);
      int nsw = 0;
      while (res >= thr && nsw < c->max_blusgs && isfinite(res)) {
        orc_blusgs(c, l, zl[l], Ul[l], 1);
        ++nsw;
        res = orc_residual_sum(c, l, zl[l], Ul[l]);
      }
      st->blusgs_sweeps[l] = nsw;
      lvl Lc = level_geom(c, l), Lf = level_geom(c, l - 1);
      for (int I = 0; I < Lc.n; ++I) {          /* U_{j,l-1} = U_{I,l}, j in I */
        int ch[4], m = children(c, &Lf, &Lc, I, ch);
        for (int q = 0; q < m; ++q)
          for (int s = 0; s < nc; ++s) Ul[l - 1][s * Lf.n + ch[q]] = Ul[l][s * Lc.n + I];
      }
    }
    memcpy(U0, Ul[0], sizeof(double) * (size_t)L0.n * nc);
  }

  /* Steps 2-3: Newton multigrid iteration */
  int n = L0.n;
  double* R = (double*)malloc(sizeof(double) * (size_t)n * nc);
  double* blk = (double*)malloc(sizeof(double) * (size_t)n * 5 * bs);
  double res = orc_residual_sum(c, 0, zl[0], U0);
  double best = res;
  st->init_res = res;
  int status = ST_NOT_CONVERGED, it = 0;
  if (!isfinite(res) || !finite_vec(U0, (size_t)n * nc)) status = ST_NONFINITE;
  while (status == ST_NOT_CONVERGED && it < c->max_newton) {
    if (res < c->tol) { status = ST_OK; break; }
    orc_blusgs(c, 0, zl[0], U0, 1);                         /* Step 2.1 */
    orc_jacobian(c, 0, zl[0], U0, R, NULL, blk);            /* eq. NewtonREG */
    hier H;
    hier_build(c, blk, &H);
    for (int e = 0; e < n * nc; ++e) { H.b[0][e] = -R[e]; H.x[0][e] = 0.0; }
    for (int k = 0; k < c->n_mg; ++k) mg_cycle(c, &H, 0);   /* Step 2.2 */
    /* Step 2.3 + Remark 2.5; cells dry at the linearisation point keep zero
     * momentum (see blusgs_cell) */
    for (int i = 0; i < n; ++i)
      if (U0[i] < c->h_eps) for (int s = 1; s < nc; ++s) H.x[0][s * n + i] = 0.0;
    for (int i = 0; i < n; ++i) {
      for (int s = 0; s < nc; ++s) U0[s * n + i] = U0[s * n + i] + c->tau * H.x[0][s * n + i];
      dry_reset(nc, n, U0, i, c->h_eps);
    }
    hier_free(&H);
    ++it;
    st->n_vcycles += c->n_mg;
    res = orc_residual_sum(c, 0, zl[0], U0);                /* Step 3 */
    if (it <= ORC_HIST) st->res_hist[it - 1] = res;
    if (!isfinite(res) || !finite_vec(U0, (size_t)n * nc)) { status = ST_NONFINITE; break; }
    if (res < best) best = res;
    if (res > 1e6 * best) { status = ST_DIVERGED; break; }
  }
  if (status == ST_NOT_CONVERGED && res < c->tol) status = ST_OK;
  st->n_newton = it;
  st->final_res = res;
  st->status = status;
  free(R); free(blk);
  for (int l = 0; l <= NL; ++l) { free(zl[l]); free(Ul[l]); }
  return status;
}

/* ---- discrete adjoint (not in the paper) ---------------------------------
 * At a steady state U_s (R(U_s, z, q) = 0) and for a loss L(U, z), the
 * implicit function theorem gives the derivative of U_s with respect to z as
 * -J^{-1} dR/dz with J = dR/dU, so
 *   dL/dz = dL/dz|_direct - lambda^T dR/dz,   dL/dq = -lambda^T dR/dq,
 *   J^T lambda = (dL/dU)^T.
 * J is the finite-difference Jacobian of eq. NumerDiff with its
 * regularisation (negligible at a steady state).  lambda solves the
 * transposed system with the same multigrid: the transposed operator's
 * Galerkin hierarchy is the transpose of the forward one (P^T A^T P =
 * (P^T A P)^T) and its smoother is block Gauss-Seidel on A^T.  dR/dz and
 * dR/dq are central differences with step ADJ_DELTA, contracted with lambda
 * (these derivatives are not part of the paper's method; the central form
 * keeps their error near 1e-10 where a forward difference would leave 1e-8
 * per term, which cancellation in lambda^T dR/dz magnifies).
 */
#define ADJ_DELTA 1e-6

/* transposed blocks: D'_i = D_i^T, and the block of cell i towards its
 * neighbour j in A^T is the transpose of cell j's block towards i in A */
static void transpose_blocks(const orc_cfg* c, const lvl* L, const double* blk, double* out) {
  int nc = ncomp(c), bs = nc * nc;
  for (int i = 0; i < L->n; ++i) {
    double* o = out + (size_t)i * 5 * bs;
    const double* D = blk + (size_t)i * 5 * bs;
    for (int s = 0; s < nc; ++s)
      for (int k = 0; k < nc; ++k) o[s * nc + k] = D[k * nc + s];
    for (int side = 0; side < 4; ++side) {
      double* ob = o + (1 + side) * bs;
      int j = (side < nsides(c)) ? nbr(L, i, side) : -1;
      if (j < 0) { for (int e = 0; e < bs; ++e) ob[e] = 0.0; continue; }
      const double* A = blk + ((size_t)j * 5 + 1 + (side ^ 1)) * bs;   /* j's block towards i */
      for (int s = 0; s < nc; ++s)
        for (int k = 0; k < nc; ++k) ob[s * nc + k] = A[k * nc + s];
    }
  }
}

int orc_transpose_blocks(const orc_cfg* c, int l, const double* blk, double* out) {
  lvl L = level_geom(c, l);
  transpose_blocks(c, &L, blk, out);
  return ST_OK;
}

/* lambda^T dR/dz (n values) and lambda^T dR/dq (per side, inflow sides only) */
static void adjoint_vjp(const orc_cfg* c, const lvl* L, const double* z, const double* U,
                        const double* lam, double* dRz, double* dRq) {
  int nc = ncomp(c), n = L->n;
  double d = ADJ_DELTA, r2d = 1.0 / (2.0 * ADJ_DELTA);
  double* zp = (double*)malloc(sizeof(double) * n);
  double* zm = (double*)malloc(sizeof(double) * n);
  memcpy(zp, z, sizeof(double) * n);
  memcpy(zm, z, sizeof(double) * n);
  for (int j = 0; j < n; ++j) {
    double acc = 0.0;
    zp[j] = z[j] + d;
    zm[j] = z[j] - d;
    for (int side = 0; side < nsides(c); ++side) {
      double len = edge_len(L, j, side), Gm[3], Gp[3];
      cell_G(c, L, zm, U, j, side, -1, 0, 0.0, Gm);          /* the cell itself */
      cell_G(c, L, zp, U, j, side, -1, 0, 0.0, Gp);
      for (int s = 0; s < nc; ++s) acc = acc + lam[s * n + j] * (len * ((Gp[s] - Gm[s]) * r2d));
      int k = nbr(L, j, side);
      if (k >= 0) {                                            /* the neighbour across it */
        cell_G(c, L, zm, U, k, side ^ 1, -1, 0, 0.0, Gm);
        cell_G(c, L, zp, U, k, side ^ 1, -1, 0, 0.0, Gp);
        for (int s = 0; s < nc; ++s) acc = acc + lam[s * n + k] * (len * ((Gp[s] - Gm[s]) * r2d));
      }
    }
    zp[j] = z[j];
    zm[j] = z[j];
    dRz[j] = acc;
  }
  free(zp);
  free(zm);
  for (int side = 0; side < 4; ++side) {
    dRq[side] = 0.0;
    if (side >= nsides(c) || c->bc[side].kind != BC_INFLOW_DISCHARGE) continue;
    orc_cfg cp = *c, cm = *c;
    cp.bc[side].q = c->bc[side].q + d;
    cm.bc[side].q = c->bc[side].q - d;
    double acc = 0.0;
    for (int i = 0; i < n; ++i) {
      if (nbr(L, i, side) >= 0) continue;
      double Gm[3], Gp[3], len = edge_len(L, i, side);
      cell_G(&cm, L, z, U, i, side, -1, 0, 0.0, Gm);
      cell_G(&cp, L, z, U, i, side, -1, 0, 0.0, Gp);
      for (int s = 0; s < nc; ++s) acc = acc + lam[s * n + i] * (len * ((Gp[s] - Gm[s]) * r2d));
    }
    dRq[side] = acc;
  }
}

/* lambda (nc*n), lambda^T dR/dz (n) and lambda^T dR/dq (4) at U for the
 * right-hand side g = (dL/dU)^T; ncycles > 0: that many cycles of Algorithm 0
 * on A^T from lambda = 0, ncycles <= 0: exact dense solve. */
int orc_adjoint(const orc_cfg* c, const double* z, const double* U, const double* g, double* lam,
                double* dRz, double* dRq, int ncycles) {
  if (check_cfg(c)) return ST_ARG;
  lvl L = level_geom(c, 0);
  int nc = ncomp(c), bs = nc * nc, n = L.n;
  double* R = (double*)malloc(sizeof(double) * (size_t)n * nc);
  double* blk = (double*)malloc(sizeof(double) * (size_t)n * 5 * bs);
  double* blkT = (double*)malloc(sizeof(double) * (size_t)n * 5 * bs);
  orc_jacobian(c, 0, z, U, R, NULL, blk);
  transpose_blocks(c, &L, blk, blkT);
  for (int e = 0; e < n * nc; ++e) lam[e] = 0.0;
  if (ncycles <= 0) dense_solve(c, &L, blkT, g, lam);
  else orc_vcycle(c, blkT, g, lam, ncycles);
  adjoint_vjp(c, &L, z, U, lam, dRz, dRq);
  free(R); free(blk); free(blkT);
  return ST_OK;
}

/* ---- Remark 2.6: one implicit (beta = 0) or semi-implicit time step -------
 * |K_i| (U^{n+1} - U^n)/dt + beta R(U^n) + (1 - beta) R(U^{n+1}) = 0 solved by
 * Steps 2-3 of Algorithm 1 from U^{n+1} = U^n (no Step 1); the Jacobian is
 * |K_i|/dt I + (1 - beta) J, regularised by alpha ||R_i||_1 of the time-step
 * residual.  U holds U^n on entry and U^{n+1} on return. */
int orc_time_step(const orc_cfg* c, const double* z, double* U, double dt, double beta, orc_stats* st) {
  if (check_cfg(c) || !(dt > 0.0) || !(beta >= 0.0 && beta < 1.0)) return ST_ARG;
  lvl L = level_geom(c, 0);
  int nc = ncomp(c), n = L.n;
  double dx = (c->x1 - c->x0) / c->nx;
  double area = (c->dim == 2) ? dx * ((c->y1 - c->y0) / c->ny) : dx;
  double ka = area / dt;
  orc_cfg cs = *c;
  cs.t_ka = 0.0;
  cs.t_kai = NULL;
  double* Rn = (double*)malloc(sizeof(double) * (size_t)n * nc);
  double* S = (double*)malloc(sizeof(double) * (size_t)n * nc);
  double* kai = NULL;
  if (curvilinear(&L)) {              /* |K_i|/dt per cell */
    kai = (double*)malloc(sizeof(double) * (size_t)n);
    for (int i = 0; i < n; ++i) kai[i] = cell_area(&L, i) / dt;
  }
  orc_residual(&cs, 0, z, U, Rn, NULL);
  for (int e = 0; e < n * nc; ++e) S[e] = (kai ? kai[e % n] : ka) * U[e] - beta * Rn[e];
  orc_cfg ct = *c;
  ct.t_ka = kai ? 1.0 : ka;           /* > 0: time mode; the values come from t_kai */
  ct.t_kai = kai;
  ct.t_omb = 1.0 - beta;
  ct.t_src = S;
  ct.init_mode = INIT_NONE;
  int status = orc_solve(&ct, z, U, st);
  free(Rn);
  free(S);
  free(kai);
  return status;
}
