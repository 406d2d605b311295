// noalloc.cu -- residual entry point that allocates no device memory.
//
// swnmg_residual() keeps its per-edge pieces and reduction partials in the
// context's workspace, which swnmg_create allocates with cudaMalloc.  Some
// callers cannot allocate: code embedded in a runtime that owns every byte
// of device memory through its own pool, and latency-critical loops that
// cannot afford cudaMalloc/cudaFree's implicit device-wide synchronisation.
// swnmg_residual_noalloc evaluates the same residual with the same kernels,
// taking its scratch from one fixed array in device global memory instead.
// It enqueues kernels, so (like every CUDA call) it is not for stream or
// host-function callbacks.
//
// That array lives for the whole process on every GPU that loads the
// library.  Host code cannot use the array's name as a device address (in
// host code it names a host-side stand-in), so the address is looked up once
// per device with cudaGetSymbolAddress while that device is current.  With
// lazy module loading that first lookup is also what loads the module and
// commits the array, so the first call per device is the warm-up; the cached
// address does not survive cudaDeviceReset.
#include <cstdio>
#include <mutex>

#include "common.cuh"
#include "../../include/swnmg.h"

using namespace swnmg;

namespace {

// 2^20 doubles = 8 MiB of scratch per device
constexpr long long kScratchWords = 1LL << 20;
static __device__ __align__(256) double g_residual_scratch[kScratchWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_ptr[kMaxDevices] = {nullptr};

// the text is returned by swnmg_last_error(NULL)
swnmg_status noalloc_fail(swnmg_status s, const char* msg) {
  set_static_error(msg);
  return s;
}

// device address of the scratch array on the current device (looked up once)
swnmg_status scratch_ptr(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return noalloc_fail(SWNMG_ERR_CUDA, "residual_noalloc: no usable CUDA device");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_residual_scratch);
    if (e != cudaSuccess || !p) {
      char msg[256];
      snprintf(msg, sizeof msg, "residual_noalloc: cudaGetSymbolAddress failed: %s",
               cudaGetErrorString(e));
      // the lookup loads the module and commits the array: a shortage of
      // device memory is reported as such
      return noalloc_fail(e == cudaErrorMemoryAllocation ? SWNMG_ERR_OOM : SWNMG_ERR_CUDA, msg);
    }
    g_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_ptr[dev];
  return SWNMG_OK;
}

}  // namespace

SWNMG_API swnmg_status swnmg_residual_noalloc(const swnmg_problem* p, const swnmg_params* q,
                                              const double* z, const double* U, double* R,
                                              double* rnorm, double* l1_dev, void* stream) {
  if (!p || !q || !z || !U || !R) return noalloc_fail(SWNMG_ERR_ARG, "residual_noalloc: null pointer");
  if ((p->dim != 1 && p->dim != 2) || p->nx < 1 || (p->dim == 2 && p->ny < 1) || !(p->g > 0) ||
      !(p->x1 > p->x0) || (p->dim == 2 && !(p->y1 > p->y0)))
    return noalloc_fail(SWNMG_ERR_ARG, "residual_noalloc: bad mesh or gravity");
  for (int s = 0; s < 4; ++s)
    if (p->bc[s].kind < 0 || p->bc[s].kind > 6)
      return noalloc_fail(SWNMG_ERR_ARG, "residual_noalloc: bad boundary kind");
  if (q->flux < 0 || q->flux > 3 || (p->dim == 1 && q->flux == SWNMG_FLUX_HLLC) || !(q->h_eps > 0) ||
      (q->flux == SWNMG_FLUX_ROE && !(q->eps_f > 0)))
    return noalloc_fail(SWNMG_ERR_ARG, "residual_noalloc: bad flux parameters");
  const int nc = p->dim == 2 ? 3 : 2;
  const int ny = p->dim == 2 ? p->ny : 1;
  const long long n = (long long)p->nx * ny;
  const long long n_e = (long long)(p->nx + 1) * ny + (p->dim == 2 ? (long long)p->nx * (ny + 1) : 0);
  // scratch: edge pieces (2*nc per edge), ||R_i||_1 when rnorm is NULL, 1024
  // reduction partials
  const long long words = 2LL * nc * n_e + (rnorm ? 0 : n) + 1024;
  if (n > (1LL << 28) || words > kScratchWords) {
    char msg[256];
    snprintf(msg, sizeof msg,
             "residual_noalloc: %lld cells need %lld scratch doubles, more than the %lld available",
             n, words, kScratchWords);
    return noalloc_fail(SWNMG_ERR_ARG, msg);
  }
  double* scratch = nullptr;
  swnmg_status s = scratch_ptr(&scratch);
  if (s != SWNMG_OK) return s;

  DevLevel L;
  L.dim = p->dim;
  L.nc = nc;
  L.nx = p->nx;
  L.ny = ny;
  L.n = (int)n;
  if (p->dim == 2) {
    L.ex = (p->y1 - p->y0) / p->ny;
    L.ey = (p->x1 - p->x0) / p->nx;
  } else {
    L.ex = 1.0;
    L.ey = 0.0;
  }
  L.flux = q->flux;
  L.llf_wetdry = q->llf_wetdry;
  L.g = p->g;
  L.half_g = 0.5 * p->g;
  L.h_eps = q->h_eps;
  L.eps_r = q->eps_r;
  L.alpha = q->alpha;
  L.eps = q->fd_eps;
  L.reps = 1.0 / q->fd_eps;
  L.eps_f = q->eps_f;
  L.t_ka = 0.0;   // steady residual
  L.t_omb = 1.0;
  L.t_src = nullptr;
  for (int k = 0; k < 4; ++k) {
    L.bc[k].kind = p->bc[k].kind;
    L.bc[k].h = p->bc[k].h;
    L.bc[k].q = p->bc[k].q;
    L.bc[k].ut = p->bc[k].ut;
  }
  double* eb = scratch;
  double* rn = rnorm ? rnorm : scratch + 2LL * nc * n_e;
  double* part = scratch + 2LL * nc * n_e + (rnorm ? 0 : n);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // every scratch word these kernels read is written earlier in the same call
  // (all edge pieces, all ||R_i||_1, all partials), so nothing is cleared
  launch_residual(L, z, U, R, rn, eb, st);
  if (l1_dev) launch_sum(rn, (int)n, part, l1_dev, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    char msg[256];
    snprintf(msg, sizeof msg, "residual_noalloc: launch failed: %s", cudaGetErrorString(e));
    return noalloc_fail(SWNMG_ERR_CUDA, msg);
  }
  return SWNMG_OK;
}
