// api.cu -- the C ABI (include/swnmg.h): context, operator hierarchy and the
// host side of Algorithm 1 (NMGM) and Algorithm 0 (gamma-cycle).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>
#include <cstdio>
#include <cstring>
#include <string>

#include "ctx.cuh"

using namespace swnmg;

namespace {


const char* status_text(swnmg_status s) {
  switch (s) {
    case SWNMG_OK: return "ok";
    case SWNMG_ERR_ARG: return "invalid argument";
    case SWNMG_ERR_CUDA: return "CUDA error";
    case SWNMG_ERR_NOT_CONVERGED: return "not converged";
    case SWNMG_ERR_NONFINITE: return "non-finite state or residual";
    case SWNMG_ERR_DIVERGED: return "diverged";
    case SWNMG_ERR_TIMEOUT: return "device wait timed out";
    case SWNMG_ERR_OOM: return "out of device memory";
  }
  return "unknown";
}

char g_err[512] = "";

// A multigrid operator hierarchy (the Jacobian's, or its transpose's)
struct Hier {
  Level* lv;
  int nl, fp32;
  bool coarse_exact, coarse_inverse;
  void* cinv;
  void* caug;
  int* csing;
  double* band;
};

}  // namespace

void swnmg::set_static_error(const char* msg) { snprintf(g_err, sizeof g_err, "%s", msg); }


namespace {

Hier fwd_hier(swnmg_ctx* c) {
  return Hier{c->lv, c->nl, c->fp32, c->coarse_exact, c->coarse_inverse, c->cinv, c->caug, c->csing, c->band};
}

Hier adj_hier(swnmg_ctx* c) {
  return Hier{c->alv, c->nl, 0, c->coarse_exact, c->coarse_inverse, c->acinv, c->acaug, c->acsing, c->aband};
}

swnmg_status fail(swnmg_ctx* c, swnmg_status s, const std::string& msg) {
  std::string m = std::string(status_text(s)) + ": " + msg;
  if (c) c->err = m;
  snprintf(g_err, sizeof g_err, "%s", m.c_str());
  return s;
}

#define CUDA_TRY(ctx, expr)                                                          \
  do {                                                                               \
    cudaError_t e_ = (expr);                                                         \
    if (e_ != cudaSuccess)                                                           \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? SWNMG_ERR_OOM : SWNMG_ERR_CUDA, \
                  std::string(#expr) + " -> " + cudaGetErrorString(e_));              \
  } while (0)

#define LAUNCH_CHECK(ctx) CUDA_TRY(ctx, cudaGetLastError())

DevLevel dev_level(const swnmg_ctx* c, int l) {
  DevLevel L;
  L.dim = c->prob.dim;
  L.nc = c->nc;
  L.nx = c->lv[l].nx;
  L.ny = c->lv[l].ny;
  L.n = c->lv[l].n;
  L.ex = c->lv[l].ex;
  L.ey = c->lv[l].ey;
  L.flux = c->prm.flux;
  L.llf_wetdry = c->prm.llf_wetdry;
  L.g = c->prob.g;
  L.half_g = 0.5 * c->prob.g;
  L.h_eps = c->prm.h_eps;
  L.eps_r = c->prm.eps_r;
  L.alpha = c->prm.alpha;
  L.eps = c->prm.fd_eps;
  L.eps_f = c->prm.eps_f;
  L.t_ka = (l == 0 && c->t_on) ? c->t_ka : 0.0;   // implicit time step (Remark 2.6)
  L.t_omb = c->t_omb;
  L.t_src = c->t_src;
  L.reps = 1.0 / c->prm.fd_eps;
  if (c->curv) {
    L.geo = c->lv[l].geo;
    L.area = c->lv[l].area;
    L.t_kai = (l == 0 && c->t_on) ? c->kai : nullptr;
  }
  for (int s = 0; s < 4; ++s) {
    L.bc[s].kind = c->prob.bc[s].kind;
    L.bc[s].h = c->prob.bc[s].h;
    L.bc[s].q = c->prob.bc[s].q;
    L.bc[s].ut = c->prob.bc[s].ut;
  }
  return L;
}

swnmg_status check_params(const swnmg_problem* p, const swnmg_params* q) {
  if (q->flux < 0 || q->flux > 3) return SWNMG_ERR_ARG;
  if (q->smoother != SWNMG_SMOOTH_LEX && q->smoother != SWNMG_SMOOTH_COLOUR) return SWNMG_ERR_ARG;
  if (q->flux == SWNMG_FLUX_ROE && !(q->eps_f > 0)) return SWNMG_ERR_ARG;
  if (p->dim == 1 && q->flux == SWNMG_FLUX_HLLC) return SWNMG_ERR_ARG;
  if (!(q->fd_eps > 0) || !(q->h_eps > 0) || q->alpha < 0) return SWNMG_ERR_ARG;
  if (q->n_levels < 0 || q->n_levels > 12 || q->n_mg < 0 || q->nu1 < 0 || q->nu2 < 0) return SWNMG_ERR_ARG;
  if (q->gamma < 1 || q->gamma > 2 || q->max_newton < 0 || q->max_blusgs < 0) return SWNMG_ERR_ARG;
  if (q->precision != SWNMG_PREC_FP64 && q->precision != SWNMG_PREC_MIXED && q->precision != SWNMG_PREC_MIXED_STEP1)
    return SWNMG_ERR_ARG;
  if (q->init_mode != SWNMG_INIT_CASCADE && q->init_mode != SWNMG_INIT_NONE) return SWNMG_ERR_ARG;
  const int m = 1 << q->n_levels;
  if (p->nx % m) return SWNMG_ERR_ARG;
  if (p->dim == 2 && p->ny % m) return SWNMG_ERR_ARG;
  return SWNMG_OK;
}

// ---- kernel timing ------------------------------------------------------------
void timing_resolve(swnmg_ctx* c) {
  if (c->ev_used == 0) return;
  cudaEventSynchronize(c->ev_pool[2 * (c->ev_used - 1) + 1]);
  for (int k = 0; k < c->ev_used; ++k) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev_pool[2 * k], c->ev_pool[2 * k + 1]) == cudaSuccess) {
      c->t_ms[c->ev_class[k]] += ms;
      c->t_n[c->ev_class[k]] += 1;
      c->t_cells[c->ev_class[k]] += c->ev_cells[k];
    }
  }
  c->ev_used = 0;
}

// RAII scope: records start/stop events around the launches of one class
struct TimedScope {
  swnmg_ctx* c;
  int k = -1;
  TimedScope(swnmg_ctx* ctx, int cls, double cells = 0.0) : c(ctx) {
    if (!c->timing) return;
    if (c->ev_used * 2 + 2 > (int)c->ev_pool.size()) timing_resolve(c);
    k = c->ev_used++;
    c->ev_class[k] = cls;
    c->ev_cells[k] = cells;
    cudaEventRecord(c->ev_pool[2 * k], c->st);
  }
  ~TimedScope() {
    if (k >= 0) cudaEventRecord(c->ev_pool[2 * k + 1], c->st);
  }
};

// sum_i v_i over n doubles (fixed-order device reduction), synchronises
swnmg_status device_sum(swnmg_ctx* c, const double* v, int n, double* out) {
  launch_sum(v, n, c->red, c->red + 1024, c->st);
  LAUNCH_CHECK(c);
  CUDA_TRY(c, cudaMemcpyAsync(c->hbuf, c->red + 1024, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  *out = *c->hbuf;
  return SWNMG_OK;
}

// reports a device-side wait that ran out of its bound (the wavefront sweeps)
swnmg_status check_sticky(swnmg_ctx* c) {
  int* h = reinterpret_cast<int*>(c->hbuf + 1);
  CUDA_TRY(c, cudaMemcpyAsync(h, c->sticky, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  if (*h) {
    cudaMemsetAsync(c->sticky, 0, sizeof(int), c->st);
    return fail(c, SWNMG_ERR_TIMEOUT, "a wavefront sweep waited past its bound");
  }
  return SWNMG_OK;
}

swnmg_status level_residual_sum(swnmg_ctx* c, int l, const double* U, double* out) {
  DevLevel L = dev_level(c, l);
  {
    TimedScope ts(c, SWNMG_T_RESIDUAL, L.n);
    launch_residual(L, c->lv[l].z, U, c->R, c->rn, c->eb, c->st);
  }
  LAUNCH_CHECK(c);
  return device_sum(c, c->rn, L.n, out);
}

// the epoch of the next launch that hands values between strips through tagged
// words: never 0, the tag of the zero-filled words before the first launch
unsigned next_epoch(unsigned& e) {
  if (++e == 0u) e = 1u;
  return e;
}

// one block SGS half-sweep of level l in the order the parameters select
void sgs_launch(swnmg_ctx* c, const Level& v, int fp32, int forward) {
  if (c->prm.smoother == SWNMG_SMOOTH_COLOUR)
    launch_sgs_colour_sweep(c->nc, v.nx, v.ny, v.blk, v.lu, v.piv, v.b, v.x, forward, fp32, c->st);
  else
    launch_sgs_sweep(c->nc, v.nx, v.ny, v.blk, v.lu, v.piv, v.b, v.x, forward, fp32, c->sgs_sync, c->sgs_edge,
                     next_epoch(c->sgs_epoch), c->sticky, c->st);
}

void sgs_half(swnmg_ctx* c, const Hier& H, int l, int forward) {
  Level& v = H.lv[l];
  TimedScope ts(c, l == 0 ? SWNMG_T_SGS_FINE : SWNMG_T_SGS_COARSE, v.n);
  sgs_launch(c, v, H.fp32, forward);
}

void blusgs_half(swnmg_ctx* c, int l, double* U, int forward) {
  DevLevel L = dev_level(c, l);
  TimedScope ts(c, l == 0 ? SWNMG_T_BLUSGS : SWNMG_T_BLUSGS_COARSE, L.n);
  if (l >= 1 && c->prm.precision == SWNMG_PREC_MIXED_STEP1)   // Step 1's coarse levels in FP32
    launch_blusgs32_strip(L, c->lv[l].z, U, reinterpret_cast<float*>(c->ghost), forward, c->blu_sync, c->sticky,
                          c->st);
  else
    launch_blusgs_strip(L, c->lv[l].z, U, c->ghost, forward, c->blu_sync, c->blu_edge, next_epoch(c->blu_epoch),
                        c->sticky, c->st);
}

// Algorithm 0 on level l of hierarchy H (lv[l].b, lv[l].x)
swnmg_status coarse_solve(swnmg_ctx* c, const Hier& H, int l) {
  Level& v = H.lv[l];
  if (H.coarse_inverse) {
    TimedScope ts(c, SWNMG_T_COARSE_EXACT);
    launch_coarse_apply(c->nc, v.nx, v.ny, H.cinv, v.b, v.x, H.fp32, c->st);
    LAUNCH_CHECK(c);
    return SWNMG_OK;
  }
  if (H.coarse_exact) {
    TimedScope ts(c, SWNMG_T_COARSE_EXACT);
    launch_coarse_exact(c->nc, v.nx, v.ny, v.blk, v.b, v.x, H.band, c->derr, H.fp32, c->st);
    LAUNCH_CHECK(c);
    return SWNMG_OK;
  }
  for (int k = 0; k < c->prm.coarse_sweeps; ++k) {
    sgs_half(c, H, l, 1);
    sgs_half(c, H, l, 0);
  }
  LAUNCH_CHECK(c);
  return SWNMG_OK;
}

swnmg_status smooth(swnmg_ctx* c, const Hier& H, int l, int nsym) {
  for (int k = 0; k < nsym; ++k) {
    sgs_half(c, H, l, 1);
    sgs_half(c, H, l, 0);
  }
  LAUNCH_CHECK(c);
  return SWNMG_OK;
}

swnmg_status mg_cycle(swnmg_ctx* c, const Hier& H, int l) {
  if (l == H.nl) return coarse_solve(c, H, l);
  swnmg_status s;
  if ((s = smooth(c, H, l, c->prm.nu1)) != SWNMG_OK) return s;
  Level& v = H.lv[l];
  Level& w = H.lv[l + 1];
  {
    TimedScope ts(c, SWNMG_T_TRANSFER);
    launch_restrict(c->prob.dim, c->nc, v.nx, v.ny, v.blk, v.b, v.x, w.b, H.fp32, c->st);
    launch_fill(w.x, H.fp32, (long long)c->nc * skew_slots(w.nx, w.ny), c->st);
  }
  LAUNCH_CHECK(c);
  const int gam = (l == 0) ? 1 : c->prm.gamma;
  for (int k = 0; k < gam; ++k)
    if ((s = mg_cycle(c, H, l + 1)) != SWNMG_OK) return s;
  {
    TimedScope ts(c, SWNMG_T_TRANSFER);
    launch_prolong(c->prob.dim, c->nc, v.nx, v.ny, w.x, v.x, H.fp32, c->st);
  }
  LAUNCH_CHECK(c);
  return smooth(c, H, l, c->prm.nu2);
}

// Galerkin coarse operators, block LU factors and the coarse inverse of H
// from its level-0 blocks
void build_hier(swnmg_ctx* c, const Hier& H) {
  TimedScope ts(c, SWNMG_T_GALERKIN);
  for (int l = 0; l < H.nl; ++l)
    launch_galerkin(c->prob.dim, c->nc, H.lv[l].nx, H.lv[l].ny, H.lv[l].blk, H.lv[l + 1].blk, H.fp32,
                    c->st);
  for (int l = 0; l <= H.nl; ++l)
    launch_lu_factor(H.lv[l].nx, H.lv[l].ny, c->nc, H.lv[l].blk, H.lv[l].lu, H.lv[l].piv, H.fp32, c->st);
  if (H.coarse_inverse) {
    const Level& vc = H.lv[H.nl];
    launch_coarse_inverse(c->nc, vc.nx, vc.ny, vc.blk, H.caug, H.cinv, H.csing, H.fp32, c->st);
  }
}

swnmg_status assemble(swnmg_ctx* c, const double* U) {
  DevLevel L = dev_level(c, 0);
  {
    TimedScope ts(c, SWNMG_T_JACOBIAN, L.n);
    launch_jacobian(L, c->lv[0].z, U, c->R, c->rn, c->eb, c->lv[0].blk, c->fp32, c->st);
  }
  LAUNCH_CHECK(c);
  build_hier(c, fwd_hier(c));
  LAUNCH_CHECK(c);
  return SWNMG_OK;
}

void free_ctx(swnmg_ctx* c) {
  for (auto& v : c->alv) {
    if (v.blk) cudaFree(v.blk);
    if (v.lu) cudaFree(v.lu);
    if (v.piv) cudaFree(v.piv);
    if (v.b) cudaFree(v.b);
    if (v.x) cudaFree(v.x);
  }
  if (c->acinv) cudaFree(c->acinv);
  if (c->acaug) cudaFree(c->acaug);
  if (c->acsing) cudaFree(c->acsing);
  if (c->aband) cudaFree(c->aband);
  if (c->adj_cz) cudaFree(c->adj_cz);
  if (c->adj_A) cudaFree(c->adj_A);
  if (c->adj_cell) cudaFree(c->adj_cell);
  for (auto& v : c->lv) {
    if (v.z) cudaFree(v.z);
    if (v.U) cudaFree(v.U);
    if (v.blk) cudaFree(v.blk);
    if (v.lu) cudaFree(v.lu);
    if (v.piv) cudaFree(v.piv);
    if (v.b) cudaFree(v.b);
    if (v.x) cudaFree(v.x);
    if (v.geo) cudaFree(v.geo);
    if (v.area) cudaFree(v.area);
  }
  if (c->mesh) cudaFree(c->mesh);
  if (c->kai) cudaFree(c->kai);
  if (c->R) cudaFree(c->R);
  if (c->rn) cudaFree(c->rn);
  if (c->eb) cudaFree(c->eb);
  if (c->red) cudaFree(c->red);
  if (c->band) cudaFree(c->band);
  if (c->cinv) cudaFree(c->cinv);
  if (c->caug) cudaFree(c->caug);
  if (c->csing) cudaFree(c->csing);
  if (c->derr) cudaFree(c->derr);
  if (c->sgs_sync) cudaFree(c->sgs_sync);
  if (c->sgs_edge) cudaFree(c->sgs_edge);
  if (c->blu_sync) cudaFree(c->blu_sync);
  if (c->blu_edge) cudaFree(c->blu_edge);
  if (c->sticky) cudaFree(c->sticky);
  if (c->ghost) cudaFree(c->ghost);
  if (c->t_src) cudaFree(c->t_src);
  if (c->hbuf) cudaFreeHost(c->hbuf);
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  c->ev_pool.clear();
}

}  // namespace

// ============================== C ABI =========================================

SWNMG_API swnmg_status swnmg_default_params(int32_t dim, swnmg_params* o) {
  if (!o || (dim != 1 && dim != 2)) return fail(nullptr, SWNMG_ERR_ARG, "dim must be 1 or 2");
  memset(o, 0, sizeof *o);
  o->flux = dim == 2 ? SWNMG_FLUX_HLLC : SWNMG_FLUX_HLL;
  o->llf_wetdry = 0;
  o->alpha = 3.0;
  o->fd_eps = 1e-8;
  o->tau = 1.0;
  o->h_eps = 1e-6;
  o->eps_r = 0.03;
  o->eps_p = 0.2;
  o->tol = 1e-10;
  o->n_levels = 3;
  o->n_mg = dim == 2 ? 3 : 2;
  o->nu1 = 1;
  o->nu2 = 1;
  o->gamma = 1;
  o->coarse_sweeps = 8;
  o->max_newton = 200;
  o->max_blusgs = 1000;
  o->init_mode = SWNMG_INIT_CASCADE;
  o->precision = SWNMG_PREC_FP64;
  o->eps_f = 0.4;
  o->smoother = SWNMG_SMOOTH_LEX;
  return SWNMG_OK;
}

SWNMG_API const char* swnmg_last_error(const swnmg_ctx* c) { return c ? c->err.c_str() : g_err; }

SWNMG_API int64_t swnmg_level_cells(const swnmg_ctx* c, int32_t l) {
  if (!c || l < 0 || l > c->nl) return 0;
  return c->lv[l].n;
}

SWNMG_API swnmg_status swnmg_create(const swnmg_problem* p, const swnmg_params* q,
                                    const double* z_dev, void* stream, swnmg_ctx** out) {
  if (!p || !q || !z_dev || !out) return fail(nullptr, SWNMG_ERR_ARG, "null pointer");
  *out = nullptr;
  if ((p->dim != 1 && p->dim != 2) || p->nx < 1 || (p->dim == 2 && p->ny < 1) || !(p->g > 0) ||
      !(p->x1 > p->x0) || (p->dim == 2 && !(p->y1 > p->y0)))
    return fail(nullptr, SWNMG_ERR_ARG, "bad mesh or gravity");
  if ((long long)p->nx * (p->dim == 2 ? p->ny : 1) > (1LL << 28))
    return fail(nullptr, SWNMG_ERR_ARG, "more than 2^28 cells");
  for (int s = 0; s < 4; ++s)
    if (p->bc[s].kind < 0 || p->bc[s].kind > 6) return fail(nullptr, SWNMG_ERR_ARG, "bad boundary kind");
  if (check_params(p, q) != SWNMG_OK)
    return fail(nullptr, SWNMG_ERR_ARG, "bad parameters or mesh not divisible by 2^n_levels");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(nullptr, SWNMG_ERR_CUDA, "no CUDA device");
  swnmg_ctx* c = new swnmg_ctx();
  c->prob = *p;
  if (p->dim == 1) c->prob.ny = 1;
  c->prm = *q;
  c->nc = p->dim == 2 ? 3 : 2;
  c->nl = q->n_levels;
  c->fp32 = q->precision != SWNMG_PREC_FP64;
  c->wsz = c->fp32 ? 4 : 8;
  c->st = (cudaStream_t)stream;
  const double dx = (p->x1 - p->x0) / p->nx;
  const double dy = p->dim == 2 ? (p->y1 - p->y0) / p->ny : 0.0;
  swnmg_status rc = SWNMG_OK;
#define ALLOC(ptr, bytes)                                                             \
  do {                                                                                \
    cudaError_t e_ = cudaMalloc((void**)&(ptr), (bytes));                             \
    if (e_ != cudaSuccess) {                                                          \
      rc = fail(c, SWNMG_ERR_OOM, std::string("cudaMalloc ") + cudaGetErrorString(e_)); \
      goto fail_out;                                                                  \
    }                                                                                 \
  } while (0)
  for (int l = 0; l <= c->nl; ++l) {
    Level& v = c->lv[l];
    v.nx = p->nx >> l;
    v.ny = p->dim == 2 ? (p->ny >> l) : 1;
    v.n = v.nx * v.ny;
    if (p->dim == 2) {
      const double s = (double)(1 << l);
      v.ex = dy * s;
      v.ey = dx * s;
    } else {
      v.ex = 1.0;
      v.ey = 0.0;
    }
    const size_t n = v.n;
    const size_t P = (size_t)skew_slots(v.nx, v.ny);   // strip-skewed operator slots
    ALLOC(v.z, n * sizeof(double));
    if (l > 0) ALLOC(v.U, n * c->nc * sizeof(double));
    ALLOC(v.blk, P * 5 * c->nc * c->nc * c->wsz);
    ALLOC(v.lu, P * LU_E * c->wsz);
    ALLOC(v.piv, P);
    if (cudaMemset(v.blk, 0, P * 5 * c->nc * c->nc * c->wsz) != cudaSuccess ||
        cudaMemset(v.lu, 0, P * LU_E * c->wsz) != cudaSuccess || cudaMemset(v.piv, 0, P) != cudaSuccess) {
      rc = fail(c, SWNMG_ERR_CUDA, "memset of the operator arrays");
      goto fail_out;
    }
    ALLOC(v.b, P * c->nc * c->wsz);   // multigrid vectors: strip-skewed like the operator
    ALLOC(v.x, P * c->nc * c->wsz);
  }
  {
    const Level& v0 = c->lv[0];
    const size_t n_e = (size_t)(v0.nx + 1) * v0.ny + (p->dim == 2 ? (size_t)v0.nx * (v0.ny + 1) : 0);
    ALLOC(c->R, (size_t)v0.n * c->nc * sizeof(double));
    ALLOC(c->rn, (size_t)v0.n * sizeof(double));
    ALLOC(c->eb, n_e * (2 * c->nc + 2 * c->nc * c->nc) * sizeof(double));
    ALLOC(c->red, 1032 * sizeof(double));
    ALLOC(c->derr, sizeof(int));
    ALLOC(c->sgs_sync, sizeof(int) * (2 + (v0.ny + 31) / 32 + 8));
    ALLOC(c->sgs_edge, sizeof(unsigned long long) * (size_t)((v0.ny + 31) / 32) * v0.nx * c->nc * 2);
    if (cudaMemset(c->sgs_edge, 0, sizeof(unsigned long long) * (size_t)((v0.ny + 31) / 32) * v0.nx * c->nc * 2) !=
        cudaSuccess) {
      rc = fail(c, SWNMG_ERR_CUDA, "memset of the SGS hand-off words");
      goto fail_out;
    }
    ALLOC(c->blu_sync, sizeof(int) * (2 + (v0.ny + 1) / 2 + 8));   // 2-row strips
    ALLOC(c->blu_edge, sizeof(unsigned long long) * (size_t)((v0.ny + 1) / 2) * v0.nx * 6);
    if (cudaMemset(c->blu_edge, 0, sizeof(unsigned long long) * (size_t)((v0.ny + 1) / 2) * v0.nx * 6) !=
        cudaSuccess) {
      rc = fail(c, SWNMG_ERR_CUDA, "memset of the BLU-SGS hand-off words");
      goto fail_out;
    }
    ALLOC(c->sticky, sizeof(int));
    ALLOC(c->ghost, sizeof(double) * 4 * (size_t)std::max(v0.nx, v0.ny) * (c->nc + 1) * 3);
  }
  {
    const Level& vc = c->lv[c->nl];
    c->coarse_exact = (p->dim == 1) || (q->coarse_sweeps <= 0);
    const long long mc = (long long)vc.n * c->nc;
    c->coarse_inverse = c->coarse_exact && mc <= 384;
    if (c->coarse_inverse) {
      ALLOC(c->cinv, (size_t)(mc * mc) * c->wsz);
      ALLOC(c->caug, (size_t)(2 * mc * mc) * c->wsz);
      ALLOC(c->csing, (size_t)mc * sizeof(int));
    } else if (c->coarse_exact) {
      const long long m = (long long)vc.n * c->nc;
      const long long ml = c->nc * (vc.ny > 1 ? vc.nx : 1) + c->nc - 1;
      const long long words = m * (3 * ml + 1) + 2 * m;
      if (words > (16LL << 20)) {
        rc = fail(c, SWNMG_ERR_ARG, "coarsest level too large for the exact solve; use more levels "
                                    "or coarse_sweeps > 0");
        goto fail_out;
      }
      ALLOC(c->band, (size_t)words * sizeof(double));
    }
  }
  if (cudaMemsetAsync(c->sticky, 0, sizeof(int), c->st) != cudaSuccess) {
    rc = fail(c, SWNMG_ERR_CUDA, "memset");
    goto fail_out;
  }
  if (cudaMallocHost((void**)&c->hbuf, 32) != cudaSuccess) {
    rc = fail(c, SWNMG_ERR_OOM, "cudaMallocHost");
    goto fail_out;
  }
#undef ALLOC
  if (cudaMemcpyAsync(c->lv[0].z, z_dev, (size_t)c->lv[0].n * sizeof(double), cudaMemcpyDeviceToDevice,
                      c->st) != cudaSuccess) {
    rc = fail(c, SWNMG_ERR_CUDA, "copy of z");
    goto fail_out;
  }
  for (int l = 0; l < c->nl; ++l)
    launch_average(p->dim, c->lv[l].nx, c->lv[l].ny, 1, c->lv[l].z, c->lv[l + 1].z, c->st);
  if (cudaStreamSynchronize(c->st) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    rc = fail(c, SWNMG_ERR_CUDA, "bed averaging");
    goto fail_out;
  }
  *out = c;
  return SWNMG_OK;
fail_out:
  snprintf(g_err, sizeof g_err, "%s", c->err.c_str());
  free_ctx(c);
  delete c;
  return rc;
}

SWNMG_API swnmg_status swnmg_destroy(swnmg_ctx* c) {
  if (!c) return SWNMG_ERR_ARG;
  cudaStreamSynchronize(c->st);
  free_ctx(c);
  delete c;
  return SWNMG_OK;
}

SWNMG_API swnmg_status swnmg_set_params(swnmg_ctx* c, const swnmg_params* q) {
  if (!c || !q) return fail(c, SWNMG_ERR_ARG, "null pointer");
  if (q->n_levels != c->prm.n_levels || q->precision != c->prm.precision)
    return fail(c, SWNMG_ERR_ARG, "n_levels and precision are fixed at create");
  if (check_params(&c->prob, q) != SWNMG_OK) return fail(c, SWNMG_ERR_ARG, "bad parameters");
  const bool exact = (c->prob.dim == 1) || (q->coarse_sweeps <= 0);
  if (exact != c->coarse_exact) return fail(c, SWNMG_ERR_ARG, "coarse-solve kind is fixed at create");
  c->prm = *q;
  return SWNMG_OK;
}

SWNMG_API swnmg_status swnmg_set_mesh(swnmg_ctx* c, const double* vx, const double* vy) {
  if (!c || !vx || !vy) return fail(c, SWNMG_ERR_ARG, "null pointer");
  if (c->prob.dim != 2) return fail(c, SWNMG_ERR_ARG, "curvilinear meshes are two-dimensional");
  const int nx = c->prob.nx, ny = c->prob.ny;
  const size_t nv = (size_t)(nx + 1) * (ny + 1);
  if (!c->mesh) {
    CUDA_TRY(c, cudaMalloc((void**)&c->mesh, 2 * nv * sizeof(double)));
    CUDA_TRY(c, cudaMalloc((void**)&c->kai, (size_t)c->lv[0].n * sizeof(double)));
    for (int l = 0; l <= c->nl; ++l) {
      Level& v = c->lv[l];
      const size_t ne = (size_t)(v.nx + 1) * v.ny + (size_t)v.nx * (v.ny + 1);
      CUDA_TRY(c, cudaMalloc((void**)&v.geo, 3 * ne * sizeof(double)));
      CUDA_TRY(c, cudaMalloc((void**)&v.area, (size_t)v.n * sizeof(double)));
    }
  }
  c->curv = false;
  CUDA_TRY(c, cudaMemcpyAsync(c->mesh, vx, nv * sizeof(double), cudaMemcpyHostToDevice, c->st));
  CUDA_TRY(c, cudaMemcpyAsync(c->mesh + nv, vy, nv * sizeof(double), cudaMemcpyHostToDevice, c->st));
  CUDA_TRY(c, cudaMemsetAsync(c->derr, 0, sizeof(int), c->st));
  for (int l = 0; l <= c->nl; ++l) {
    Level& v = c->lv[l];
    launch_mesh_level(v.nx, v.ny, nx + 1, 1 << l, c->mesh, c->mesh + nv, v.geo, v.area, c->derr, c->st);
  }
  LAUNCH_CHECK(c);
  int bad = 0;
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  CUDA_TRY(c, cudaMemcpy(&bad, c->derr, sizeof(int), cudaMemcpyDeviceToHost));
  if (bad) {   // back to the uniform mesh's coarse beds (a replaced mesh may have changed them)
    for (int l = 0; l < c->nl; ++l)
      launch_average(2, c->lv[l].nx, c->lv[l].ny, 1, c->lv[l].z, c->lv[l + 1].z, c->st);
    LAUNCH_CHECK(c);
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    return fail(c, SWNMG_ERR_ARG, "degenerate mesh: an edge of zero length or a cell of non-positive area");
  }
  c->curv = true;
  for (int l = 0; l < c->nl; ++l)   // coarse beds: the children weighted by their areas
    launch_average_area(c->lv[l].nx, c->lv[l].ny, 1, c->lv[l].area, c->lv[l].z, c->lv[l + 1].z, c->st);
  LAUNCH_CHECK(c);
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  return SWNMG_OK;
}

SWNMG_API swnmg_status swnmg_residual(swnmg_ctx* c, const double* U, double* R, double* rn,
                                      double* l1_host) {
  if (!c || !U || !R) return fail(c, SWNMG_ERR_ARG, "null pointer");
  DevLevel L = dev_level(c, 0);
  double* rnp = rn ? rn : c->rn;
  launch_residual(L, c->lv[0].z, U, R, rnp, c->eb, c->st);
  LAUNCH_CHECK(c);
  if (l1_host) return device_sum(c, rnp, L.n, l1_host);
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  return SWNMG_OK;
}

SWNMG_API swnmg_status swnmg_jacobian(swnmg_ctx* c, const double* U) {
  if (!c || !U) return fail(c, SWNMG_ERR_ARG, "null pointer");
  swnmg_status s = assemble(c, U);
  if (s != SWNMG_OK) return s;
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  return SWNMG_OK;
}

SWNMG_API swnmg_status swnmg_get_blocks(swnmg_ctx* c, int32_t level, double* host_out) {
  if (!c || !host_out || level < 0 || level > c->nl) return fail(c, SWNMG_ERR_ARG, "bad level");
  const Level& v = c->lv[level];
  const size_t cnt = (size_t)v.n * 5 * c->nc * c->nc;
  double* tmp = nullptr;
  CUDA_TRY(c, cudaMalloc((void**)&tmp, cnt * sizeof(double)));
  launch_blocks_export(v.nx, v.ny, c->nc, v.blk, c->fp32, tmp, c->st);
  cudaError_t e1 = cudaGetLastError();
  cudaError_t e2 = cudaMemcpyAsync(host_out, tmp, cnt * sizeof(double), cudaMemcpyDeviceToHost, c->st);
  cudaError_t e3 = cudaStreamSynchronize(c->st);
  cudaFree(tmp);
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess)
    return fail(c, SWNMG_ERR_CUDA, "block export");
  return SWNMG_OK;
}

SWNMG_API swnmg_status swnmg_vcycle(swnmg_ctx* c, const double* rhs, double* dU, int32_t ncycles) {
  if (!c || !rhs || !dU || ncycles < 0) return fail(c, SWNMG_ERR_ARG, "bad argument");
  Level& v = c->lv[0];
  launch_to_skew(rhs, 0, v.b, c->fp32, c->nc, v.nx, v.ny, 1.0, c->st);
  launch_to_skew(dU, 0, v.x, c->fp32, c->nc, v.nx, v.ny, 1.0, c->st);
  LAUNCH_CHECK(c);
  const Hier H = fwd_hier(c);
  for (int k = 0; k < ncycles; ++k) {
    swnmg_status s = mg_cycle(c, H, 0);
    if (s != SWNMG_OK) return s;
  }
  launch_from_skew(v.x, c->fp32, dU, 0, c->nc, v.nx, v.ny, 1.0, c->st);
  LAUNCH_CHECK(c);
  return check_sticky(c);
}

SWNMG_API swnmg_status swnmg_sgs_sweep(swnmg_ctx* c, int32_t level, const double* rhs, double* x,
                                       int32_t forward) {
  if (!c || !rhs || !x || level < 0 || level > c->nl) return fail(c, SWNMG_ERR_ARG, "bad argument");
  Level& v = c->lv[level];
  launch_to_skew(rhs, 0, v.b, c->fp32, c->nc, v.nx, v.ny, 1.0, c->st);
  launch_to_skew(x, 0, v.x, c->fp32, c->nc, v.nx, v.ny, 1.0, c->st);
  sgs_launch(c, v, c->fp32, forward ? 1 : 0);
  launch_from_skew(v.x, c->fp32, x, 0, c->nc, v.nx, v.ny, 1.0, c->st);
  LAUNCH_CHECK(c);
  return check_sticky(c);
}

SWNMG_API swnmg_status swnmg_blusgs(swnmg_ctx* c, double* U, int32_t level, int32_t nsweeps) {
  if (!c || !U || level < 0 || level > c->nl || nsweeps < 0) return fail(c, SWNMG_ERR_ARG, "bad argument");
  DevLevel L = dev_level(c, level);
  (void)L;
  for (int k = 0; k < nsweeps; ++k) {
    blusgs_half(c, level, U, 1);
    blusgs_half(c, level, U, 0);
  }
  LAUNCH_CHECK(c);
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  return check_sticky(c);
}

SWNMG_API swnmg_status swnmg_solve(swnmg_ctx* c, double* U, swnmg_stats* stats) {
  if (!c || !U) return fail(c, SWNMG_ERR_ARG, "null pointer");
  swnmg_stats local;
  swnmg_stats* st = stats ? stats : &local;
  memset(st, 0, sizeof *st);
  const int nc = c->nc, NL = c->nl;
  using clk = std::chrono::steady_clock;
  auto t0 = clk::now();
  swnmg_status s;
  // Step 1: BLU-SGS from the coarsest level to level 1, piecewise-constant
  // prolongation of the solution (Algorithm 1)
  if (c->prm.init_mode == SWNMG_INIT_CASCADE && NL > 0) {
    // eps_p < 0: the paper's rule, |eps_p| x sum_i ||R_i||_1 of the initial data
    double eps_p = c->prm.eps_p;
    if (eps_p < 0.0) {
      double r0;
      if ((s = level_residual_sum(c, 0, U, &r0)) != SWNMG_OK) return s;
      eps_p = -eps_p * r0;
    }
    const double* src = U;
    for (int l = 0; l < NL; ++l) {
      if (c->curv)   // the children weighted by their areas
        launch_average_area(c->lv[l].nx, c->lv[l].ny, nc, c->lv[l].area, src, c->lv[l + 1].U, c->st);
      else
        launch_average(c->prob.dim, c->lv[l].nx, c->lv[l].ny, nc, src, c->lv[l + 1].U, c->st);
      src = c->lv[l + 1].U;
    }
    LAUNCH_CHECK(c);
    for (int l = NL; l >= 1; --l) {
      const double thr = eps_p / (double)(1 << l);
      double res;
      if ((s = level_residual_sum(c, l, c->lv[l].U, &res)) != SWNMG_OK) return s;
      int nsw = 0;
      DevLevel L = dev_level(c, l);
      (void)L;
      while (res >= thr && nsw < c->prm.max_blusgs && std::isfinite(res)) {
        blusgs_half(c, l, c->lv[l].U, 1);
        blusgs_half(c, l, c->lv[l].U, 0);
        LAUNCH_CHECK(c);
        ++nsw;
        if ((s = level_residual_sum(c, l, c->lv[l].U, &res)) != SWNMG_OK) return s;
      }
      if (l < 16) st->blusgs_sweeps[l] = nsw;
      double* dst = (l - 1 == 0) ? U : c->lv[l - 1].U;
      launch_inject(c->prob.dim, c->lv[l - 1].nx, c->lv[l - 1].ny, nc, c->lv[l].U, dst, c->st);
      LAUNCH_CHECK(c);
    }
  }
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  auto t1 = clk::now();
  // Steps 2-3: Newton multigrid iteration
  Level& v0 = c->lv[0];
  double res;
  if ((s = level_residual_sum(c, 0, U, &res)) != SWNMG_OK) return s;
  st->init_res = res;
  double best = res;
  swnmg_status status = std::isfinite(res) ? SWNMG_ERR_NOT_CONVERGED : SWNMG_ERR_NONFINITE;
  int it = 0;
  while (status == SWNMG_ERR_NOT_CONVERGED && it < c->prm.max_newton) {
    if (res < c->prm.tol) { status = SWNMG_OK; break; }
    blusgs_half(c, 0, U, 1);                                       // Step 2.1
    blusgs_half(c, 0, U, 0);
    LAUNCH_CHECK(c);
    if ((s = assemble(c, U)) != SWNMG_OK) return s;                // eq. NewtonREG
    launch_to_skew(c->R, 0, v0.b, c->fp32, nc, v0.nx, v0.ny, -1.0, c->st);   // b = -R
    launch_fill(v0.x, c->fp32, (long long)nc * skew_slots(v0.nx, v0.ny), c->st);
    LAUNCH_CHECK(c);
    for (int k = 0; k < c->prm.n_mg; ++k)                          // Step 2.2
      if ((s = mg_cycle(c, fwd_hier(c), 0)) != SWNMG_OK) return s;
    {
      TimedScope ts(c, SWNMG_T_UPDATE);                            // Step 2.3
      launch_newton_update(v0.nx, v0.ny, nc, c->prm.tau, c->prm.h_eps, U, v0.x, c->fp32, c->st);
    }
    LAUNCH_CHECK(c);
    ++it;
    st->n_vcycles += c->prm.n_mg;
    if ((s = check_sticky(c)) != SWNMG_OK) return s;
    if ((s = level_residual_sum(c, 0, U, &res)) != SWNMG_OK) return s;   // Step 3
    if (it <= SWNMG_HIST) st->res_hist[it - 1] = res;
    if (!std::isfinite(res)) { status = SWNMG_ERR_NONFINITE; break; }
    if (res < best) best = res;
    if (res > 1e6 * best) { status = SWNMG_ERR_DIVERGED; break; }
  }
  if (status == SWNMG_ERR_NOT_CONVERGED && res < c->prm.tol) status = SWNMG_OK;
  auto t2 = clk::now();
  st->n_newton = it;
  st->final_res = res;
  st->status = status;
  st->ms_step1 = std::chrono::duration<double, std::milli>(t1 - t0).count();
  st->ms_newton = std::chrono::duration<double, std::milli>(t2 - t1).count();
  if (status != SWNMG_OK) return fail(c, status, "after " + std::to_string(it) + " Newton steps");
  return SWNMG_OK;
}

SWNMG_API swnmg_status swnmg_time_step(swnmg_ctx* c, double* U, double dt, double beta, swnmg_stats* st) {
  if (!c || !U) return fail(c, SWNMG_ERR_ARG, "null pointer");
  if (!(dt > 0) || !(beta >= 0 && beta < 1)) return fail(c, SWNMG_ERR_ARG, "need dt > 0 and 0 <= beta < 1");
  const Level& v0 = c->lv[0];
  const long long m = (long long)v0.n * c->nc;
  if (!c->t_src) CUDA_TRY(c, cudaMalloc((void**)&c->t_src, sizeof(double) * m));
  const double dx = (c->prob.x1 - c->prob.x0) / c->prob.nx;
  const double area = c->prob.dim == 2 ? dx * ((c->prob.y1 - c->prob.y0) / c->prob.ny) : dx;
  const double ka = area / dt;
  c->t_on = false;
  const DevLevel L = dev_level(c, 0);
  launch_residual(L, v0.z, U, c->R, c->rn, c->eb, c->st);   // R(U^n)
  if (c->curv) {   // |K_i|/dt per cell
    launch_time_ka(v0.n, v0.area, dt, c->kai, c->st);
    launch_time_source_cells(m, v0.n, c->kai, beta, U, c->R, c->t_src, c->st);
  } else {
    launch_time_source(m, ka, beta, U, c->R, c->t_src, c->st);
  }
  LAUNCH_CHECK(c);
  c->t_on = true;
  c->t_ka = c->curv ? 1.0 : ka;   // > 0 switches the time step on; a curvilinear mesh reads kai
  c->t_omb = 1.0 - beta;
  const int32_t im = c->prm.init_mode;
  c->prm.init_mode = SWNMG_INIT_NONE;
  const swnmg_status s = swnmg_solve(c, U, st);
  c->prm.init_mode = im;
  c->t_on = false;
  return s;
}

namespace {

// FP64 transposed hierarchy and adjoint scratch, allocated on first use
swnmg_status adjoint_alloc(swnmg_ctx* c) {
  if (c->adj_ready) return SWNMG_OK;
  const int nc = c->nc, bs = nc * nc;
#define AALLOC(ptr, bytes)                                                                   \
  do {                                                                                       \
    cudaError_t e_ = cudaMalloc((void**)&(ptr), (bytes));                                    \
    if (e_ != cudaSuccess) return fail(c, SWNMG_ERR_OOM, std::string("adjoint cudaMalloc ") + \
                                                              cudaGetErrorString(e_));       \
  } while (0)
  for (int l = 0; l <= c->nl; ++l) {
    const Level& f = c->lv[l];
    Level& v = c->alv[l];
    v.nx = f.nx;
    v.ny = f.ny;
    v.n = f.n;
    v.ex = f.ex;
    v.ey = f.ey;
    const size_t P = (size_t)skew_slots(v.nx, v.ny);
    if (!v.blk) AALLOC(v.blk, P * 5 * bs * sizeof(double));
    if (!v.lu) AALLOC(v.lu, P * LU_E * sizeof(double));
    if (!v.piv) AALLOC(v.piv, P);
    if (!v.b) AALLOC(v.b, P * nc * sizeof(double));
    if (!v.x) AALLOC(v.x, P * nc * sizeof(double));
    CUDA_TRY(c, cudaMemset(v.blk, 0, P * 5 * bs * sizeof(double)));
    CUDA_TRY(c, cudaMemset(v.lu, 0, P * LU_E * sizeof(double)));
    CUDA_TRY(c, cudaMemset(v.piv, 0, P));
  }
  const Level& v0 = c->lv[0];
  const size_t P0 = (size_t)skew_slots(v0.nx, v0.ny);
  if (!c->adj_A) AALLOC(c->adj_A, P0 * 5 * bs * sizeof(double));
  CUDA_TRY(c, cudaMemset(c->adj_A, 0, P0 * 5 * bs * sizeof(double)));
  const size_t n_e = (size_t)(v0.nx + 1) * v0.ny + (c->prob.dim == 2 ? (size_t)v0.nx * (v0.ny + 1) : 0);
  if (!c->adj_cz) AALLOC(c->adj_cz, 2 * n_e * sizeof(double));
  if (!c->adj_cell) AALLOC(c->adj_cell, (size_t)v0.n * sizeof(double));
  const Level& vc = c->lv[c->nl];
  const long long mc = (long long)vc.n * nc;
  if (c->coarse_inverse) {
    if (!c->acinv) AALLOC(c->acinv, (size_t)(mc * mc) * sizeof(double));
    if (!c->acaug) AALLOC(c->acaug, (size_t)(2 * mc * mc) * sizeof(double));
    if (!c->acsing) AALLOC(c->acsing, (size_t)mc * sizeof(int));
  } else if (c->coarse_exact) {
    const long long ml = nc * (vc.ny > 1 ? vc.nx : 1) + nc - 1;
    const long long words = mc * (3 * ml + 1) + 2 * mc;
    if (!c->aband) AALLOC(c->aband, (size_t)words * sizeof(double));
  }
#undef AALLOC
  c->adj_ready = true;
  return SWNMG_OK;
}

}  // namespace

SWNMG_API swnmg_status swnmg_adjoint(swnmg_ctx* c, const double* U, const double* g, double* lam,
                                     double* gz, double* gq_host, int32_t max_cycles, double rtol,
                                     int32_t* cycles_out) {
  if (!c || !U || !g || !lam || !gz || max_cycles < 1) return fail(c, SWNMG_ERR_ARG, "bad argument");
  if (!(rtol == rtol)) return fail(c, SWNMG_ERR_ARG, "rtol is NaN");
  if (c->curv) return fail(c, SWNMG_ERR_ARG, "the adjoint is built for uniform meshes only");
  if (cycles_out) *cycles_out = 0;
  swnmg_status s = adjoint_alloc(c);
  if (s != SWNMG_OK) return s;
  const int nc = c->nc;
  const DevLevel L = dev_level(c, 0);
  Level& a0 = c->alv[0];
  // J at U* in FP64, then J^T in the strip-skewed layout and its hierarchy
  {
    TimedScope ts(c, SWNMG_T_JACOBIAN, L.n);
    launch_jacobian(L, c->lv[0].z, U, c->R, c->rn, c->eb, c->adj_A, 0, c->st);
    launch_transpose_blocks(nc, a0.nx, a0.ny, c->adj_A, 0, (double*)a0.blk, c->st);
  }
  LAUNCH_CHECK(c);
  const Hier H = adj_hier(c);
  build_hier(c, H);
  LAUNCH_CHECK(c);
  launch_to_skew(g, 0, a0.b, 0, nc, a0.nx, a0.ny, 1.0, c->st);
  launch_fill(a0.x, 0, (long long)nc * skew_slots(a0.nx, a0.ny), c->st);
  LAUNCH_CHECK(c);
  double gnorm = 0.0, rnorm = 0.0;
  if (rtol > 0) {
    launch_abs_cells(a0.n, nc, g, c->adj_cell, c->st);
    LAUNCH_CHECK(c);
    if ((s = device_sum(c, c->adj_cell, a0.n, &gnorm)) != SWNMG_OK) return s;
    if (!std::isfinite(gnorm)) return fail(c, SWNMG_ERR_NONFINITE, "adjoint: g is not finite");
  }
  int k = 0;
  swnmg_status status = SWNMG_OK;
  while (k < max_cycles) {
    if ((s = mg_cycle(c, H, 0)) != SWNMG_OK) return s;
    ++k;
    if (rtol > 0) {
      if ((s = check_sticky(c)) != SWNMG_OK) return s;
      launch_lin_resid_abs(c->prob.dim, nc, a0.nx, a0.ny, a0.blk, a0.b, a0.x, 0, c->adj_cell, c->st);
      LAUNCH_CHECK(c);
      if ((s = device_sum(c, c->adj_cell, a0.n, &rnorm)) != SWNMG_OK) return s;
      if (!std::isfinite(rnorm)) { status = SWNMG_ERR_NONFINITE; break; }
      if (rnorm <= rtol * gnorm) break;
      if (k == max_cycles) status = SWNMG_ERR_NOT_CONVERGED;
    }
  }
  if (cycles_out) *cycles_out = k;
  if ((s = check_sticky(c)) != SWNMG_OK) return s;
  launch_from_skew(a0.x, 0, lam, 0, nc, a0.nx, a0.ny, 1.0, c->st);
  // -lambda^T dR/dz and -lambda^T dR/dq (central differences of the edge terms)
  const double delta = 1e-6;
  launch_adjoint_z(L, c->lv[0].z, U, lam, delta, c->adj_cz, gz, c->st);
  LAUNCH_CHECK(c);
  if (gq_host) {
    const int nsides = c->prob.dim == 2 ? 4 : 2;
    for (int side = 0; side < 4; ++side) {
      gq_host[side] = 0.0;
      if (side >= nsides || c->prob.bc[side].kind != SWNMG_BC_INFLOW_DISCHARGE) continue;
      launch_adjoint_q(L, side, c->lv[0].z, U, lam, delta, c->adj_cell, c->st);
      LAUNCH_CHECK(c);
      if ((s = device_sum(c, c->adj_cell, L.n, &gq_host[side])) != SWNMG_OK) return s;
    }
  }
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  if (status != SWNMG_OK)
  {
    char msg[160];
    snprintf(msg, sizeof msg, "adjoint: after %d cycles sum ||g - J^T lambda||_1 = %.3e, sum ||g||_1 = %.3e", k,
             rnorm, gnorm);
    return fail(c, status, msg);
  }
  return SWNMG_OK;
}

SWNMG_API swnmg_status swnmg_set_timing(swnmg_ctx* c, int32_t enable) {
  if (!c) return fail(c, SWNMG_ERR_ARG, "null context");
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  c->ev_used = 0;
  for (int k = 0; k < SWNMG_T_COUNT; ++k) { c->t_ms[k] = 0; c->t_n[k] = 0; c->t_cells[k] = 0; }
  if (enable && c->ev_pool.empty()) {
    const int pairs = 4096;
    c->ev_pool.resize(2 * pairs);
    c->ev_class.resize(pairs);
    c->ev_cells.resize(pairs);
    for (auto& e : c->ev_pool) CUDA_TRY(c, cudaEventCreate(&e));
  }
  c->timing = enable != 0;
  return SWNMG_OK;
}

SWNMG_API swnmg_status swnmg_get_timing(swnmg_ctx* c, double* ms_out, int64_t* n_out,
                                        double* cells_out) {
  if (!c || !ms_out || !n_out || !cells_out) return fail(c, SWNMG_ERR_ARG, "null pointer");
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  timing_resolve(c);
  for (int k = 0; k < SWNMG_T_COUNT; ++k) {
    ms_out[k] = c->t_ms[k];
    n_out[k] = c->t_n[k];
    cells_out[k] = c->t_cells[k];
  }
  return SWNMG_OK;
}

SWNMG_API int64_t swnmg_launch_count(void) { return launches_total(); }

SWNMG_API int32_t swnmg_set_wait_limit(int32_t polls) {
  const int old = wait_limit();
  set_wait_limit(polls);
  return old;
}

DevLevel swnmg::ctx_dev_level(const swnmg_ctx* c, int l) { return dev_level(c, l); }
