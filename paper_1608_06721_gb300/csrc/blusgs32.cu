// blusgs32.cu -- the BLU-SGS cell update of Algorithm 1, Step 1, in FP32
// (precision SWNMG_PREC_MIXED_STEP1).
//
// Step 1 only has to bring each coarse level below eps_p 2^-l, a threshold
// far above FP32 rounding, and GB300 issues FP32 arithmetic at about 58 times
// its FP64 rate.  This unit restates the flux of Remark 2.2 (eq. HLLflux,
// HLLC, eq. LLFflux, eq. ROEflux), the ghosts of Remark 2.3, the hydrostatic
// reconstruction and the regularised block update in float.  The state stays
// FP64 in memory: a cell's FP64 state is rounded to float, the update is
// computed in float and subtracted in FP64, and the dry reset of Remark 2.5
// is applied in FP64.  Two quantities cannot keep their FP64 values:
//   * the finite-difference step of eq. NumerDiff is 2^-12 (about the square
//     root of FP32's unit roundoff, which balances rounding against
//     truncation), not 1e-8, which FP32 cannot resolve;
//   * the singular-pivot guard of the 3x3 elimination is 1e-6 max|D|.
// The iterates therefore differ from the FP64 path; the Newton iteration
// that follows Step 1 is unchanged (FP64 residual and update).
#include "common.cuh"
#include "flux32.cuh"

namespace swnmg {

namespace {

using namespace f32;

// the edge frame of side sd of cell (ix, iy): (n, tau) on a curvilinear mesh
// (tau = n turned by +90 degrees on W/E edges, -90 degrees on S/N edges),
// the axis frame otherwise (returned as n = e_axis, tau = the other axis)
struct F32 { float nx, ny, tx, ty; bool curv; };

__device__ __forceinline__ F32 frame32(const DevLevel& L, int ix, int iy, int sd) {
  F32 f;
  f.curv = L.geo != nullptr;
  const int axis = sd >> 1;
  if (!f.curv) {
    f.nx = axis == 0 ? 1.0f : 0.0f;
    f.ny = axis == 0 ? 0.0f : 1.0f;
    f.tx = axis == 0 ? 0.0f : 1.0f;
    f.ty = axis == 0 ? 1.0f : 0.0f;
    return f;
  }
  const long long n_xe = (long long)(L.nx + 1) * L.ny, ne = n_xe + (long long)L.nx * (L.ny + 1);
  long long e;
  switch (sd) {
    case 0: e = ix + (long long)(L.nx + 1) * iy; break;
    case 1: e = ix + 1 + (long long)(L.nx + 1) * iy; break;
    case 2: e = n_xe + ix + (long long)L.nx * iy; break;
    default: e = n_xe + ix + (long long)L.nx * (iy + 1); break;
  }
  f.nx = (float)L.geo[ne + e];
  f.ny = (float)L.geo[2 * ne + e];
  if (axis == 0) { f.tx = -f.ny; f.ty = f.nx; }
  else { f.tx = f.ny; f.ty = -f.nx; }
  return f;
}

__device__ __forceinline__ float len32(const DevLevel& L, int ix, int iy, int sd) {
  if (!L.geo) return (float)((sd >> 1) == 0 ? L.ex : L.ey);
  const long long n_xe = (long long)(L.nx + 1) * L.ny;
  switch (sd) {
    case 0: return (float)L.geo[ix + (long long)(L.nx + 1) * iy];
    case 1: return (float)L.geo[ix + 1 + (long long)(L.nx + 1) * iy];
    case 2: return (float)L.geo[n_xe + ix + (long long)L.nx * iy];
    default: return (float)L.geo[n_xe + ix + (long long)L.nx * (iy + 1)];
  }
}

// a cell's (possibly perturbed) float state c in the frame of side sd
template <int NC>
__device__ __forceinline__ P32 frame_prim32(const DevLevel& L, const float c[NC], const F32& f, float h_eps) {
  if (NC == 2) return prim32(c[0], c[1], 0.0f, h_eps);
  const P32 gl = prim32(c[0], c[1], c[NC - 1], h_eps);
  P32 p;
  p.h = gl.h;
  p.u = gl.u * f.nx + gl.v * f.ny;
  p.v = gl.u * f.tx + gl.v * f.ty;
  return p;
}


// Gaussian elimination with partial pivoting, the guard at 1e-6 max|D|
template <int NC>
__device__ __forceinline__ void small_solve32(float m[NC * NC], const float b[NC], float x[NC]) {
  float amax = 0.0f;
#pragma unroll
  for (int e = 0; e < NC * NC; ++e) amax = fmax2(amax, fabsf(m[e]));
  const float tiny = 1e-6f * amax;
  int perm[NC];
  bool sing[NC];
#pragma unroll
  for (int r = 0; r < NC; ++r) { perm[r] = r; sing[r] = false; }
#pragma unroll
  for (int col = 0; col < NC; ++col) {
    int p = col;
    float best = fabsf(m[col * NC + col]);
#pragma unroll
    for (int r = col + 1; r < NC; ++r)
      if (fabsf(m[r * NC + col]) > best) { best = fabsf(m[r * NC + col]); p = r; }
#pragma unroll
    for (int r = col + 1; r < NC; ++r)
      if (r == p) {
#pragma unroll
        for (int k = 0; k < NC; ++k) {
          const float t = m[col * NC + k];
          m[col * NC + k] = m[r * NC + k];
          m[r * NC + k] = t;
        }
        const int t = perm[col]; perm[col] = perm[r]; perm[r] = t;
      }
    if (!(best > tiny)) {
      sing[col] = true;
#pragma unroll
      for (int r = col + 1; r < NC; ++r) m[r * NC + col] = 0.0f;
    } else {
#pragma unroll
      for (int r = col + 1; r < NC; ++r) {
        const float l = m[r * NC + col] / m[col * NC + col];
        m[r * NC + col] = l;
#pragma unroll
        for (int k = col + 1; k < NC; ++k) m[r * NC + k] = m[r * NC + k] - l * m[col * NC + k];
      }
    }
  }
  float y[NC];
#pragma unroll
  for (int r = 0; r < NC; ++r) {
    float v = b[0];
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
    float s = y[r];
#pragma unroll
    for (int k = r + 1; k < NC; ++k) s = s - m[r * NC + k] * x[k];
    x[r] = sing[r] ? 0.0f : s / m[r * NC + r];
  }
}

// a cell state rounded to float, with component p-1 raised by the FD step
template <int NC>
__device__ __forceinline__ void load32(const double* U, long long n, long long i, int p, float c[NC]) {
#pragma unroll
  for (int s = 0; s < NC; ++s) c[s] = (float)__ldcg(&U[s * n + i]);
  if (p > 0) c[p - 1] = c[p - 1] + FD32;
}

// ghosts of every boundary cell for the base state and each perturbation,
// before a half-sweep (a cell's state does not change before its update)
// gbuf[((side * glen + k) * NP + p) * 3 + {h, u, v}]
template <int NC, int NS>
__global__ void __launch_bounds__(128) k_ghost32(DevLevel L, const double* __restrict__ U, float* gbuf) {
  constexpr int NP = NC + 1;
  const int glen = L.nx > L.ny ? L.nx : L.ny;
  const int total = NS * glen * NP;
  const float h_eps = (float)L.h_eps;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int p = t % NP, k = (t / NP) % glen, sd = t / (NP * glen);
    if (k >= (sd < 2 ? L.ny : L.nx)) continue;
    const int ix = sd == 0 ? 0 : (sd == 1 ? L.nx - 1 : k);
    const int iy = sd < 2 ? k : (sd == 2 ? 0 : L.ny - 1);
    float c[NC];
    load32<NC>(U, L.n, ix + (long long)L.nx * iy, p, c);
    const P32 gh = ghost32(L, sd, frame_prim32<NC>(L, c, frame32(L, ix, iy, sd), h_eps));
    gbuf[(long long)t * 3 + 0] = gh.h;
    gbuf[(long long)t * 3 + 1] = gh.u;
    gbuf[(long long)t * 3 + 2] = gh.v;
  }
}

// One cell per group of GRP lanes, lane g = (side, perturbation p): p = 0
// evaluates the side's edge term at the cell's state, p = k + 1 with
// component k raised by the FD step.  The group's first lanes sum the sides
// per entry; its first lane solves (alpha ||R_i||_1 I + dR_i/dU_i) x = R_i
// and stores U_i - x in FP64, with Remark 2.5's dry rules.
template <int NC, int NS, int GRP>
__device__ __forceinline__ void group32(const DevLevel& L, const double* __restrict__ z, double* U,
                                        const float* gbuf, int d, int ix0, int ncell, int cell, int g) {
  constexpr int NP = NC + 1;
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int side = g / NP, p = g % NP, gbase = lane - g;
  const bool cell_ok = cell < ncell, act = cell_ok && side < NS;
  const int ix = ix0 + (cell_ok ? cell : 0), iy = d - ix;
  const long long i = ix + (long long)L.nx * iy, n = L.n;
  const int sd = side < NS ? side : 0, upper = sd & 1;
  const float h_eps = (float)L.h_eps;
  long long j = -1;
  if (act) {
    if (sd == 0 && ix > 0) j = i - 1;
    if (sd == 1 && ix < L.nx - 1) j = i + 1;
    if (sd == 2 && iy > 0) j = i - L.nx;
    if (sd == 3 && iy < L.ny - 1) j = i + L.nx;
  }
  float G[NC];
#pragma unroll
  for (int s = 0; s < NC; ++s) G[s] = 0.0f;
  if (act) {
    const F32 fr = frame32(L, ix, iy, sd);
    float c[NC];
    load32<NC>(U, n, i, p, c);
    const P32 me = frame_prim32<NC>(L, c, fr, h_eps);
    P32 other;
    if (j >= 0) {
      float cj[NC];
      load32<NC>(U, n, j, 0, cj);
      other = frame_prim32<NC>(L, cj, fr, h_eps);
    } else {
      const int glen = L.nx > L.ny ? L.nx : L.ny;
      const long long t = ((long long)(sd * glen + (sd < 2 ? iy : ix)) * NP + p) * 3;
      other.h = __ldcg(&gbuf[t]);
      other.u = __ldcg(&gbuf[t + 1]);
      other.v = __ldcg(&gbuf[t + 2]);
    }
    const float zi = (float)z[i], zo = (j >= 0) ? (float)z[j] : zi;
    float o[5];
    if (upper) edge_eval32(L, me, zi, other, zo, o);
    else edge_eval32(L, other, zo, me, zi, o);
    const float sgn = upper ? 1.0f : -1.0f, sc = upper ? o[3] : o[4];
    G[0] = sgn * o[0];
    if (NC == 2) {
      G[1] = sgn * (o[1] - sc);
    } else {
      const float fx = o[1] * fr.nx + o[2] * fr.tx, fy = o[1] * fr.ny + o[2] * fr.ty;
      G[1] = sgn * (fx - sc * fr.nx);
      G[NC - 1] = sgn * (fy - sc * fr.ny);
    }
    const float len = len32(L, ix, iy, sd);
#pragma unroll
    for (int s = 0; s < NC; ++s) G[s] = len * G[s];
  }
  // p = 0: |e| G; p = k + 1: column k of |e| dG/dU_i
  const int src0 = gbase + sd * NP;
  float v[NC];
#pragma unroll
  for (int s = 0; s < NC; ++s) {
    const float gb = __shfl_sync(full, G[s], src0);
    v[s] = (p == 0) ? G[s] : (G[s] - gb) * (1.0f / FD32);
  }
  const int es = g / NP < NC ? g / NP : 0, ep = g % NP;
  float acc = 0.0f;
  for (int q = 0; q < NS; ++q) {
    float w = 0.0f;
#pragma unroll
    for (int s = 0; s < NC; ++s) {
      const float t = __shfl_sync(full, v[s], gbase + q * NP + ep);
      if (s == es) w = t;
    }
    acc = acc + w;
  }
  float Rs[NC], D[NC * NC];
#pragma unroll
  for (int s = 0; s < NC; ++s)
#pragma unroll
    for (int pp = 0; pp < NP; ++pp) {
      const float t = __shfl_sync(full, acc, gbase + s * NP + pp);
      if (pp == 0) Rs[s] = t;
      else D[s * NC + (pp - 1)] = t;
    }
  if (!cell_ok || g != 0) return;
  float m = fabsf(Rs[0]) + fabsf(Rs[1]);
  if (NC == 3) m = m + fabsf(Rs[NC - 1]);
  const float am = (float)L.alpha * m;
#pragma unroll
  for (int s = 0; s < NC; ++s) D[s * NC + s] = D[s * NC + s] + am;
  float x[NC];
  small_solve32<NC>(D, Rs, x);
  double ci[NC];
#pragma unroll
  for (int s = 0; s < NC; ++s) ci[s] = __ldcg(&U[s * n + i]);
  if (ci[0] < L.h_eps)   // dry at the start: momentum stays zero (Remark 2.5)
#pragma unroll
    for (int s = 1; s < NC; ++s) x[s] = 0.0f;
  double un[NC];
#pragma unroll
  for (int s = 0; s < NC; ++s) un[s] = ci[s] - (double)x[s];
  if (un[0] < L.h_eps)
#pragma unroll
    for (int s = 0; s < NC; ++s) un[s] = 0.0;
#pragma unroll
  for (int s = 0; s < NC; ++s) U[s * n + i] = un[s];
}

__device__ __forceinline__ int ld_acq32(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_rel32(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// The strip-pipelined half-sweep of flux.cu's k_blusgs_strip (same schedule,
// waits and publication) with the FP32 cell update.
// sync: [0] ticket, [1] abort, [2 + q] columns completed by strip q's last row.
template <int NC, int NS, int GRP>
__global__ void __launch_bounds__(32) k_blusgs32_strip(DevLevel L, const double* __restrict__ z, double* U,
                                                       const float* gbuf, int forward, int* sync,
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
      if (q > 0 && t < L.nx && known < t + 1) {
        int pg = 0, it = 0;
        do {
          if (lane == 0) {
            pg = ld_acq32(&prog[q - 1]);
            if (pg < t + 1 && ld_acq32(&sync[1])) pg = -1;
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
      group32<NC, NS, GRP>(L, z, U, gbuf, d, ix0, ncell, lane / GRP, lane % GRP);
      __syncwarp();
      const int done = t - rows + 2;
      if (q + 1 < nstrips && done >= 1 && done <= L.nx) {
        const int rel = forward ? 0 : (ncell - 1) * GRP;
        if (lane == rel) st_rel32(&prog[q], done);
      }
    }
  }
}

}  // namespace

// FP32 BLU-SGS half-sweep: ghosts, then the strip sweep.  gbuf holds
// 4 * max(nx, ny) * (nc + 1) * 3 floats, sync 2 + ceil(ny / R) ints.
void launch_blusgs32_strip(const DevLevel& L, const double* z, double* U, float* gbuf, int forward, int* sync,
                           int* sticky_err, cudaStream_t st) {
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
  const int gblocks = (4 * glen * (L.nc + 1) + 127) / 128;
  const int grid = nstrips < 16 * nsm ? nstrips : 16 * nsm;
  const int spin = wait_limit();
  if (L.nc == 3) {
    k_ghost32<3, 4><<<gblocks, 128, 0, st>>>(L, U, gbuf);
    k_blusgs32_strip<3, 4, 16><<<grid, 32, 0, st>>>(L, z, U, gbuf, forward, sync, sticky_err, spin);
  } else {
    k_ghost32<2, 2><<<gblocks, 128, 0, st>>>(L, U, gbuf);
    k_blusgs32_strip<2, 2, 8><<<grid, 32, 0, st>>>(L, z, U, gbuf, forward, sync, sticky_err, spin);
  }
}

}  // namespace swnmg
