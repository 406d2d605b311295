// mg.cu -- geometric multigrid pieces of Section 2.3 (eq. MatrixForm,
// ProjectAR, Project, correction; Algorithm 0's smoother and coarse solve),
// templated on the working precision (double, or float in the mixed mode).
#include <atomic>

#include "common.cuh"

namespace swnmg {

namespace {

inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }

template <typename T> __device__ __forceinline__ T tabs(T a) { return a < T(0) ? -a : a; }

// ---- block LU of every diagonal block of a level ------------------------------
// Partial pivoting (largest |entry|, lowest row on ties); a pivot below
// 1e-14 max|D| marks a singular unknown (its reciprocal pivot is stored as 0,
// so its correction is 0).
template <int NC, typename T>
__device__ __forceinline__ void lu_factor_slot(int nx, int ny, const T* __restrict__ blk, T* __restrict__ lu,
                                               int8_t* __restrict__ piv, long long slot) {
  const long long P = skew_slots(nx, ny);
  // slot -> cell: lane k of strip t on skewed diagonal d is (d - k, 32 t + k)
  const int k = (int)(slot & 31);
  const long long line = slot >> 5;
  const int t = (int)(line / (nx + 31)), d = (int)(line % (nx + 31));
  const int ix = d - k, iy = 32 * t + k;
  if (ix < 0 || ix >= nx || iy >= ny) return;
  const long long i = slot;
  T m[NC][NC];
  T amax = T(0);
  for (int s = 0; s < NC; ++s)
    for (int q = 0; q < NC; ++q) {
      m[s][q] = blk[(long long)(s * NC + q) * P + i];
      amax = tabs(m[s][q]) > amax ? tabs(m[s][q]) : amax;
    }
  const T tiny = T(1e-14) * amax;
  int perm[3] = {0, 1, 2};
  T inv[3] = {T(0), T(0), T(0)};
  for (int c = 0; c < NC; ++c) {
    int p = c;
    T best = tabs(m[c][c]);
    for (int r = c + 1; r < NC; ++r)
      if (tabs(m[r][c]) > best) { best = tabs(m[r][c]); p = r; }
    if (p != c) {
      for (int q = 0; q < NC; ++q) { T tt = m[c][q]; m[c][q] = m[p][q]; m[p][q] = tt; }
      int tt = perm[c]; perm[c] = perm[p]; perm[p] = tt;
    }
    if (!(best > tiny)) {
      for (int r = c + 1; r < NC; ++r) m[r][c] = T(0);
      inv[c] = T(0);
      continue;
    }
    inv[c] = T(1) / m[c][c];
    for (int r = c + 1; r < NC; ++r) {
      const T l = m[r][c] * inv[c];
      m[r][c] = l;
      for (int q = c + 1; q < NC; ++q) m[r][q] = m[r][q] - l * m[c][q];
    }
  }
  if (NC == 3) {
    lu[0 * P + i] = m[1][0]; lu[1 * P + i] = m[2 % NC][0]; lu[2 * P + i] = m[2 % NC][1];
    lu[3 * P + i] = m[0][1]; lu[4 * P + i] = m[0][2 % NC]; lu[5 * P + i] = m[1][2 % NC];
    lu[6 * P + i] = inv[0]; lu[7 * P + i] = inv[1]; lu[8 * P + i] = inv[2];
    piv[i] = (int8_t)(perm[0] | (perm[1] << 2) | (perm[2] << 4));
  } else {
    lu[0 * P + i] = m[1][0]; lu[1 * P + i] = T(0); lu[2 * P + i] = T(0);
    lu[3 * P + i] = m[0][1]; lu[4 * P + i] = T(0); lu[5 * P + i] = T(0);
    lu[6 * P + i] = inv[0]; lu[7 * P + i] = inv[1]; lu[8 * P + i] = T(0);
    piv[i] = (int8_t)(perm[0] | (perm[1] << 2));
  }
}

template <int NC, typename T>
__global__ void k_lu_factor(int nx, int ny, const T* __restrict__ blk, T* __restrict__ lu,
                            int8_t* __restrict__ piv) {
  const long long slot = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (slot < skew_slots(nx, ny)) lu_factor_slot<NC, T>(nx, ny, blk, lu, piv, slot);
}

// explicit fused multiply-add: the smoother's rounding does not depend on how
// the compiler contracts a given call site
template <typename T> __device__ __forceinline__ T tfma(T a, T b, T c);
template <> __device__ __forceinline__ float tfma<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <> __device__ __forceinline__ double tfma<double>(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename T> __device__ __forceinline__ T pick3(const T* r, int p) {
  return p == 0 ? r[0] : (p == 1 ? r[1] : r[2]);
}

// LU solve with the factors of one cell read from 9 values L[e*ls]
template <int NC, typename T>
__device__ __forceinline__ void lu_apply_v(const T* __restrict__ L, int ls, int8_t pv, const T r[NC],
                                           T x[NC]) {
  const int p0 = pv & 3, p1 = (pv >> 2) & 3, p2 = (pv >> 4) & 3;
  if (NC == 3) {
    const T y0 = pick3(r, p0);
    const T y1 = tfma(-L[0 * ls], y0, pick3(r, p1));
    const T y2 = tfma(-L[2 * ls], y1, tfma(-L[1 * ls], y0, pick3(r, p2)));
    const T x2 = y2 * L[8 * ls];
    const T x1 = tfma(-L[5 * ls], x2, y1) * L[7 * ls];
    const T x0 = tfma(-L[4 * ls], x2, tfma(-L[3 * ls], x1, y0)) * L[6 * ls];
    x[0] = x0; x[1 % NC] = x1; x[2 % NC] = x2;
  } else {
    const T y0 = p0 == 0 ? r[0] : r[1 % NC];
    const T y1 = tfma(-L[0 * ls], y0, p1 == 0 ? r[0] : r[1 % NC]);
    const T x1 = y1 * L[7 * ls];
    const T x0 = tfma(-L[3 * ls], x1, y0) * L[6 * ls];
    x[0] = x0; x[1 % NC] = x1;
  }
}

// One block Gauss-Seidel cell update, x_i = D_i^-1 (b_i - A_W x_W - A_E x_E -
// A_S x_S - A_N x_N) in logical directions (the sweep's own west / south are
// the new values): the old east and north terms first, then the new west and
// south terms.  A* point at a block's entry (s, k) = A*[(s NC + k) * es]; lu
// at the 9 LU values (stride es).  Explicit FMAs fix its rounding wherever it
// is inlined.
template <int NC, typename T>
__device__ __forceinline__ void sgs_cell(const T* AW, const T* AE, const T* AS, const T* AN, int es,
                                         const T* lu, int8_t pv, const T bb[NC], bool hW, const T xw[NC],
                                         bool hE, const T xe[NC], bool hS, const T xs[NC], bool hN,
                                         const T xn[NC], T res[NC]) {
  T r[NC];
#pragma unroll
  for (int s2 = 0; s2 < NC; ++s2) {
    T a = bb[s2];
    if (hE)
#pragma unroll
      for (int k = 0; k < NC; ++k) a = tfma(-AE[(s2 * NC + k) * es], xe[k], a);
    if (hN)
#pragma unroll
      for (int k = 0; k < NC; ++k) a = tfma(-AN[(s2 * NC + k) * es], xn[k], a);
    T w = T(0), so = T(0);
    if (hW)
#pragma unroll
      for (int k = 0; k < NC; ++k) w = tfma(AW[(s2 * NC + k) * es], xw[k], w);
    if (hS)
#pragma unroll
      for (int k = 0; k < NC; ++k) so = tfma(AS[(s2 * NC + k) * es], xs[k], so);
    r[s2] = (a - w) - so;
  }
  lu_apply_v<NC, T>(lu, es, pv, r, res);
}

// sgs_cell in two parts, with its operations in its order: the old east and
// north terms (known a step ahead), then the new west and south terms and the
// LU solve on operands held in registers (blocks row-major, entry s NC + k).
// A neighbour that does not exist contributes through a zero sum, as in
// sgs_cell, so the two parts together give sgs_cell's bits.
template <int NC, typename T>
__device__ __forceinline__ void sgs_cell_old(const T* AE, const T* AN, int es, const T bb[NC], bool hE,
                                             const T xe[NC], bool hN, const T xn[NC], T a[NC]) {
#pragma unroll
  for (int s2 = 0; s2 < NC; ++s2) {
    T v = bb[s2], ve = bb[s2];
#pragma unroll
    for (int k = 0; k < NC; ++k) ve = tfma(-AE[(s2 * NC + k) * es], xe[k], ve);
    v = hE ? ve : v;
    T vn = v;
#pragma unroll
    for (int k = 0; k < NC; ++k) vn = tfma(-AN[(s2 * NC + k) * es], xn[k], vn);
    a[s2] = hN ? vn : v;
  }
}

template <int NC, typename T>
__device__ __forceinline__ void sgs_cell_new(const T aw[NC * NC], const T as[NC * NC], const T lu[LU_E],
                                             int8_t pv, const T a[NC], bool hW, const T xw[NC], bool hS,
                                             const T xs[NC], T res[NC]) {
  T r[NC];
#pragma unroll
  for (int s2 = 0; s2 < NC; ++s2) {
    T w = T(0), so = T(0);
#pragma unroll
    for (int k = 0; k < NC; ++k) w = tfma(aw[s2 * NC + k], xw[k], w);
#pragma unroll
    for (int k = 0; k < NC; ++k) so = tfma(as[s2 * NC + k], xs[k], so);
    r[s2] = (a[s2] - (hW ? w : T(0))) - (hS ? so : T(0));
  }
  lu_apply_v<NC, T>(lu, 1, pv, r, res);
}

// ---- Galerkin coarse operator: A_{IJ,l+1} = sum_{i in I} sum_{j in J} A_ij ---
// children 00, 10, 01, 11; diagonal = children's diagonals plus the 8
// couplings between children; W/E/S/N = the two couplings crossing that side.
template <int NC, typename T>
__device__ __forceinline__ void galerkin_cell(int dim, int nxf, int nyf, const T* __restrict__ bf,
                                              T* __restrict__ bc, int I) {
  const int nxc = nxf / 2, nyc = dim == 2 ? nyf / 2 : 1;
  const int nyff = dim == 2 ? nyf : 1;
  const long long Pf = skew_slots(nxf, nyff), Pc = skew_slots(nxc, nyc);
  const int BS = NC * NC;
  const int Ix = I % nxc, Iy = I / nxc;
  const long long sc = skew_pos(Ix, Iy, nxc);
#define FB(pos, b, e) bf[((long long)(b) * BS + (e)) * Pf + (pos)]
#define CB(b, e) bc[((long long)(b) * BS + (e)) * Pc + sc]
  if (dim == 1) {
    const long long c0 = skew_pos(2 * Ix, 0, nxf), c1 = skew_pos(2 * Ix + 1, 0, nxf);
    for (int e = 0; e < BS; ++e) {
      CB(0, e) = ((FB(c0, 0, e) + FB(c1, 0, e)) + FB(c0, 2, e)) + FB(c1, 1, e);
      CB(1, e) = FB(c0, 1, e);
      CB(2, e) = FB(c1, 2, e);
      CB(3, e) = T(0);
      CB(4, e) = T(0);
    }
    return;
  }
  const long long c00 = skew_pos(2 * Ix, 2 * Iy, nxf), c10 = skew_pos(2 * Ix + 1, 2 * Iy, nxf);
  const long long c01 = skew_pos(2 * Ix, 2 * Iy + 1, nxf), c11 = skew_pos(2 * Ix + 1, 2 * Iy + 1, nxf);
  for (int e = 0; e < BS; ++e) {
    T d = FB(c00, 0, e) + FB(c10, 0, e);
    d = d + FB(c01, 0, e);
    d = d + FB(c11, 0, e);
    d = d + FB(c00, 2, e); d = d + FB(c10, 1, e);
    d = d + FB(c00, 4, e); d = d + FB(c01, 3, e);
    d = d + FB(c10, 4, e); d = d + FB(c11, 3, e);
    d = d + FB(c01, 2, e); d = d + FB(c11, 1, e);
    CB(0, e) = d;
    CB(1, e) = FB(c00, 1, e) + FB(c01, 1, e);
    CB(2, e) = FB(c10, 2, e) + FB(c11, 2, e);
    CB(3, e) = FB(c00, 3, e) + FB(c10, 3, e);
    CB(4, e) = FB(c01, 4, e) + FB(c11, 4, e);
  }
#undef FB
#undef CB
}

template <int NC, typename T>
__global__ void k_galerkin(int dim, int nxf, int nyf, const T* __restrict__ bf, T* __restrict__ bc) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I < (nxf / 2) * (dim == 2 ? nyf / 2 : 1)) galerkin_cell<NC, T>(dim, nxf, nyf, bf, bc, I);
}

// linear residual of the fine system at cell i: r = b - D x_i - sum A x_j
template <int NC, typename T>
__device__ __forceinline__ void lin_resid(int dim, int nx, int ny, const T* __restrict__ blk,
                                          const T* __restrict__ b, const T* __restrict__ x, int i,
                                          T r[NC]) {
  const long long n = (long long)nx * ny, P = skew_slots(nx, ny);
  const int BS = NC * NC;
  const int ix = i % nx, iy = i / nx;
  const long long si = skew_pos(ix, iy, nx);
  // neighbours' slots (b and x are strip-skewed like the operator)
  const long long nb[4] = {ix > 0 ? skew_pos(ix - 1, iy, nx) : -1, ix < nx - 1 ? skew_pos(ix + 1, iy, nx) : -1,
                           iy > 0 ? skew_pos(ix, iy - 1, nx) : -1, iy < ny - 1 ? skew_pos(ix, iy + 1, nx) : -1};
  (void)n;
  T xi[NC];
  for (int k = 0; k < NC; ++k) xi[k] = x[k * P + si];
  for (int s = 0; s < NC; ++s) {
    T a = b[s * P + si];
    for (int k = 0; k < NC; ++k) a = a - blk[(long long)(s * NC + k) * P + si] * xi[k];
    r[s] = a;
  }
  const int nsd = dim == 2 ? 4 : 2;
  for (int side = 0; side < nsd; ++side) {
    const long long j = nb[side];
    if (j < 0) continue;
    T xj[NC];
    for (int k = 0; k < NC; ++k) xj[k] = x[k * P + j];
    for (int s = 0; s < NC; ++s)
      for (int k = 0; k < NC; ++k)
        r[s] = r[s] - blk[((long long)(1 + side) * BS + s * NC + k) * P + si] * xj[k];
  }
}

// coarse right-hand side = sum over children of (b - A x)  (eq. ProjectAR)
template <int NC, typename T>
__device__ __forceinline__ void restrict_cell(int dim, int nxf, int nyf, const T* __restrict__ blk,
                                              const T* __restrict__ b, const T* __restrict__ x,
                                              T* __restrict__ bc, int I) {
  const int nxc = nxf / 2, nyc = dim == 2 ? nyf / 2 : 1, ncc = nxc * nyc;
  const int Ix = I % nxc, Iy = I / nxc;
  const int ny = dim == 2 ? nyf : 1;
  int ch[4];
  int m;
  if (dim == 1) { ch[0] = 2 * Ix; ch[1] = ch[0] + 1; m = 2; }
  else {
    ch[0] = 2 * Ix + nxf * 2 * Iy; ch[1] = ch[0] + 1; ch[2] = ch[0] + nxf; ch[3] = ch[2] + 1;
    m = 4;
  }
  T acc[NC], r[NC];
  for (int q = 0; q < m; ++q) {
    lin_resid<NC, T>(dim, nxf, ny, blk, b, x, ch[q], r);
    for (int s = 0; s < NC; ++s) acc[s] = q == 0 ? r[s] : acc[s] + r[s];
  }
  const long long Pc = skew_slots(nxc, nyc), sc = skew_pos(Ix, Iy, nxc);
  (void)ncc;
  for (int s = 0; s < NC; ++s) bc[(long long)s * Pc + sc] = acc[s];
}

template <int NC, typename T>
__global__ void k_restrict(int dim, int nxf, int nyf, const T* __restrict__ blk,
                           const T* __restrict__ b, const T* __restrict__ x, T* __restrict__ bc) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I < (nxf / 2) * (dim == 2 ? nyf / 2 : 1)) restrict_cell<NC, T>(dim, nxf, nyf, blk, b, x, bc, I);
}

// restrict_cell in 2D with a lane per child: lane 4 I + q forms child q's
// residual, lane 4 I sums the four in child order (the same operations)
template <int NC, typename T>
__global__ void k_restrict4(int nxf, int nyf, const T* __restrict__ blk, const T* __restrict__ b,
                            const T* __restrict__ x, T* __restrict__ bc) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int nxc = nxf / 2, nyc = nyf / 2;
  const int I = t >> 2, q = t & 3;
  const bool ok = I < nxc * nyc;
  T r[NC];
#pragma unroll
  for (int s = 0; s < NC; ++s) r[s] = T(0);
  if (ok) {
    const int Ix = I % nxc, Iy = I / nxc;
    const int ch = 2 * Ix + nxf * 2 * Iy + (q & 1) + (q >> 1) * nxf;   // children 00, 10, 01, 11
    lin_resid<NC, T>(2, nxf, nyf, blk, b, x, ch, r);
  }
  T acc[NC];
#pragma unroll
  for (int s = 0; s < NC; ++s) {
    const T r1 = __shfl_down_sync(0xffffffffu, r[s], 1), r2 = __shfl_down_sync(0xffffffffu, r[s], 2),
            r3 = __shfl_down_sync(0xffffffffu, r[s], 3);
    acc[s] = r[s];
    acc[s] = acc[s] + r1;
    acc[s] = acc[s] + r2;
    acc[s] = acc[s] + r3;
  }
  if (ok && q == 0) {
    const long long Pc = skew_slots(nxc, nyc), sc = skew_pos(I % nxc, I / nxc, nxc);
#pragma unroll
    for (int s = 0; s < NC; ++s) bc[(long long)s * Pc + sc] = acc[s];
  }
}

// x_j += x_I for every child j of I  (eq. correction, piecewise constant)
template <typename T>
__device__ __forceinline__ void prolong_cell(int dim, int nc, int nxf, int nyf, const T* __restrict__ xc,
                                             T* __restrict__ xf, int i) {
  const int nyf1 = dim == 2 ? nyf : 1;
  const int ix = i % nxf, iy = i / nxf, nxc = nxf / 2, nyc = dim == 2 ? nyf / 2 : 1;
  const long long Pf = skew_slots(nxf, nyf1), Pc = skew_slots(nxc, nyc);
  const long long sf = skew_pos(ix, iy, nxf), sc = skew_pos(ix / 2, dim == 2 ? iy / 2 : 0, nxc);
  for (int s = 0; s < nc; ++s) xf[(long long)s * Pf + sf] = xf[(long long)s * Pf + sf] + xc[(long long)s * Pc + sc];
}

template <typename T>
__global__ void k_prolong(int dim, int nc, int nxf, int nyf, const T* __restrict__ xc,
                          T* __restrict__ xf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nxf * (dim == 2 ? nyf : 1)) prolong_cell<T>(dim, nc, nxf, nyf, xc, xf, i);
}

// ---- block Gauss-Seidel sweep: strip-pipelined wavefront ---------------------
// x_i <- D_i^{-1} (b_i - A_W x_W - A_E x_E - A_S x_S - A_N x_N) in lexicographic
// order (forward) or its reverse (backward).  One warp owns a strip of 32 rows;
// lane k handles row k of the strip and runs k columns behind lane k-1, so a
// warp step updates one skewed diagonal of the strip: the "new" west value is
// the lane's own previous result, the "new" south value comes from the lane
// below by shuffle, and the "old" east / north values have not been written
// yet.  Strip q starts a column once strip q-1 has published that its last
// row passed it (progress counter, release/acquire).  Strips are claimed in
// order through an atomic ticket, so a strip only ever waits for one that a
// running warp already owns.
//
// The operator of a warp step is one contiguous line per entry in the
// strip-skewed layout; lane 0 streams chunks of S lines of all entries into a
// double-buffered shared-memory ring with cp.async.bulk (completion on an
// mbarrier) while the warp computes the previous chunk.
//
// Every wait is bounded.  When one expires the kernel sets the sticky error
// word and the abort flag, waits (bounded) for its own copies in flight, and
// returns; the other strips see the abort flag and return as well.
// sync layout: [0] ticket, [1] abort, [2 .. 2+nstrips) progress.
constexpr int SGS_PUBLISH = 8;
constexpr int SGS_PREFETCH = 4;   // columns of b / old x values loaded ahead

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// default lines per staged chunk: the largest that fits twice in shared memory
template <typename T> struct SgsChunk { static constexpr int S = sizeof(T) == 4 ? 16 : 8; };

template <int NC, typename T>
__host__ __device__ constexpr int sgs_entries() { return 4 * NC * NC + LU_E + 2 * NC; }   // W, E, S, N, LU, b, old x

template <int NC, typename T, int S>
__host__ __device__ constexpr size_t sgs_stage_bytes() {
  return (size_t)sgs_entries<NC, T>() * S * 32 * sizeof(T) + S * 32;
}

template <int NC, typename T, int S>
size_t sgs_smem_bytes() {   // barriers, two staging buffers, two groups of the previous strip's row
  return 128 + 2 * sgs_stage_bytes<NC, T, S>() + 2 * SGS_PUBLISH * NC * sizeof(T);
}

// bounded wait of every lane for one chunk; warp-uniform result, false when
// the bound expired for some lane
__device__ __forceinline__ bool chunk_wait(uint64_t* bar, unsigned parity, int limit) {
  bool ok = false;
  for (int it = 0; it < limit && !ok; ++it) ok = mbar_try_wait(bar, parity);
  return __all_sync(0xffffffffu, ok) != 0;
}

// One strip (processing index q of nstrips) of one sweep; lane 0 stages the
// operator through the warp's two shared-memory buffers.  prog[q - 1] is the
// previous strip's progress, prog[q] this strip's.  Returns false when a wait
// ran out (the abort flag and the sticky error are then set).
template <int NC, typename T, bool FWD, int S>
__device__ __forceinline__ bool sgs_strip_run(int nx, int ny, const T* __restrict__ blk,
                                              const T* __restrict__ lu, const int8_t* __restrict__ piv,
                                              const T* __restrict__ b, T* x, int* prog, int* abort_flag,
                                              int* sticky_err, int q, int nstrips, int spin_limit,
                                              unsigned char* smem, unsigned parity[2]) {
  constexpr int BS = NC * NC;
  constexpr int NOFF = 4 * BS;
  constexpr int EB = NOFF + LU_E;         // stage entries: b, then the old x line
  constexpr int EX = EB + NC;
  constexpr int NE = EX + NC;
  constexpr size_t STAGE = sgs_stage_bytes<NC, T, S>();
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  // staging buffer st at smem + 128 + st * STAGE: values, then the pivot codes.
  // Addresses are formed by arithmetic on the shared array (not picked from an
  // array of pointers), so every operand read stays a shared-memory load.
  auto vals = [&](int st) { return reinterpret_cast<T*>(smem + 128 + (size_t)st * STAGE); };
  auto pvs = [&](int st) {
    return reinterpret_cast<int8_t*>(smem + 128 + (size_t)st * STAGE + (size_t)NE * S * 32 * sizeof(T));
  };
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x;
  const long long P = skew_slots(nx, ny);
  const int oW = (FWD ? 0 : 1) * BS, oE = (FWD ? 1 : 0) * BS, oS = (FWD ? 2 : 3) * BS,
            oN = (FWD ? 3 : 2) * BS;
  const int lagk = FWD ? lane : 31 - lane;
  const int nsteps_full = nx + 31;
  const int wait_limit = spin_limit;
  const int ps = FWD ? q : nstrips - 1 - q;
  const long long line_base = (long long)ps * (nx + 31);
  // the strip's valid rows; in a forward sweep its last valid lane finishes
  // at step nx + rows - 2, in a backward sweep the leading lane is lane 31
  // (lag 0) only when it is valid, so short strips keep the full skew there
  const int rows = min(32, ny - ps * 32);
  const int nsteps = FWD ? nx + rows - 1 : nsteps_full;
  const int nchunks = (nsteps + S - 1) / S;
  // The step on skewed diagonal d updates line d; its "old" east and north
  // values are line d + 1 (forward) or d - 1 (backward): the same lane and
  // the lane above (below).  Lane 0 stages chunk j (S lines) of the operator,
  // LU factors, b and those old x lines into buffer st.  Old lines outside
  // the strip are never used (they belong to the edge lanes' neighbours,
  // which come from global memory) and are not copied.
  auto issue = [&](int j, int st) {
    const int s0 = j * S, cnt = min(S, nsteps - s0);
    const int dlo = FWD ? s0 : nsteps_full - s0 - cnt;
    const long long off = (line_base + dlo) * 32;
    const unsigned vb = (unsigned)(cnt * 32 * sizeof(T));
    const int xlo = dlo + (FWD ? 1 : -1);
    const int xa = max(xlo, 0), xb = min(xlo + cnt, nsteps_full);
    const unsigned xbytes = xb > xa ? (unsigned)((xb - xa) * 32 * sizeof(T)) : 0u;
    fence_proxy_async();
    mbar_expect_tx(&bar[st], vb * EX + xbytes * NC + (unsigned)(cnt * 32));
    for (int e = 0; e < NOFF; ++e)
      bulk_g2s(vals(st) + (size_t)e * S * 32, blk + (long long)(BS + e) * P + off, vb, &bar[st]);
    for (int e = 0; e < LU_E; ++e)
      bulk_g2s(vals(st) + (size_t)(NOFF + e) * S * 32, lu + (long long)e * P + off, vb, &bar[st]);
    for (int k = 0; k < NC; ++k)
      bulk_g2s(vals(st) + (size_t)(EB + k) * S * 32, b + (long long)k * P + off, vb, &bar[st]);
    if (xbytes)
      for (int k = 0; k < NC; ++k)
        bulk_g2s(vals(st) + (size_t)(EX + k) * S * 32 + (size_t)(xa - xlo) * 32,
                 x + (long long)k * P + (line_base + xa) * 32, xbytes, &bar[st]);
    bulk_g2s(pvs(st), piv + off, (unsigned)(cnt * 32), &bar[st]);
  };
  bool inflight[2] = {false, false};
  if (lane == 0) {
    issue(0, 0);
    if (nchunks > 1) issue(1, 1);
  }
  inflight[0] = true;
  inflight[1] = nchunks > 1;
  const int y = ps * 32 + lane;
  const bool rowok = y < ny;
  const int yS = FWD ? y - 1 : y + 1, yN = FWD ? y + 1 : y - 1;
  const bool hasS = FWD ? (y > 0) : (y < ny - 1);
  const bool hasN = FWD ? (y < ny - 1) : (y > 0);
  // the lane whose north neighbour lies in the next strip (in processing order)
  const bool nedge = FWD ? (lane == 31) : (lane == 0);
  int known = 0;
  bool failed = false;
  T xprev[NC], res[NC];
#pragma unroll
  for (int k = 0; k < NC; ++k) { xprev[k] = T(0); res[k] = T(0); }
  // old north values of the edge lane, SGS_PREFETCH columns ahead
  T rn[SGS_PREFETCH][NC];
  auto load_north = [&](int c, T* xn) {
    const int px = FWD ? c : nx - 1 - c;
    const long long jj = skew_pos(px, yN, nx);
#pragma unroll
    for (int k = 0; k < NC; ++k) xn[k] = x[k * P + jj];
  };
#pragma unroll
  for (int t = 0; t < SGS_PREFETCH; ++t) {
#pragma unroll
    for (int k = 0; k < NC; ++k) rn[t][k] = T(0);
    if (nedge && rowok && hasN && t - lagk >= 0 && t - lagk < nx) load_north(t - lagk, rn[t]);
  }
  // the previous strip's last row for the lag-0 lane, SGS_PUBLISH columns at
  // a time: the current group and, once published, the next one, in two
  // shared-memory buffers after the staging ring.  That lane alone writes
  // and reads them, and a column's values are picked by index (not by a
  // chain of selections).
  T* sgrp = reinterpret_cast<T*>(smem + 128 + 2 * STAGE);
  int gcur = 0;
  bool have_next = false;
  const int poller = FWD ? 0 : 31;   // the lag-0 lane
  auto load_group = [&](int c0, int buf) {
#pragma unroll
    for (int t = 0; t < SGS_PUBLISH; ++t)
      if (c0 + t < nx) {
        const int pxt = FWD ? c0 + t : nx - 1 - (c0 + t);
        const long long jj = skew_pos(pxt, yS, nx);
#pragma unroll
        for (int k = 0; k < NC; ++k) sgrp[(buf * SGS_PUBLISH + t) * NC + k] = __ldcg(&x[k * P + jj]);
      }
  };
  for (int j = 0; j < nchunks && !failed; ++j) {
    const int st = j & 1;
    if (!chunk_wait(&bar[st], parity[st], wait_limit)) {
      if (lane == 0) atomicOr(sticky_err, 1);
      failed = true;
      break;
    }
    parity[st] ^= 1u;
    inflight[st] = false;
    const T* V = vals(st);
    const int8_t* PV = pvs(st);
    const int s0 = j * S, cnt = min(S, nsteps - s0);
    const long long dbase = line_base + (FWD ? s0 : nsteps_full - s0 - cnt);
    for (int s = s0; s < s0 + cnt; ++s) {
      const int line = FWD ? s - s0 : cnt - 1 - (s - s0);
      const int c = s - lagk;
      const bool act = rowok && c >= 0 && c < nx;
      T xS[NC];
#pragma unroll
      for (int k = 0; k < NC; ++k)
        xS[k] = FWD ? __shfl_up_sync(FULL, res[k], 1) : __shfl_down_sync(FULL, res[k], 1);
      if (q > 0 && s < nx && (s & (SGS_PUBLISH - 1)) == 0) {
        // group start of the lag-0 lane (column s): its south values
        if (have_next) {
          gcur ^= 1;
          have_next = false;
        } else {
          const int need = min(s + SGS_PUBLISH, nx);
          if (known < need) {
            int pg = 0, it = 0;
            do {
              if (lane == poller) {
                pg = ld_acquire(&prog[q - 1]);
                if (pg < need && ld_acquire(abort_flag)) pg = -1;
              }
              pg = __shfl_sync(FULL, pg, poller);
              if (pg >= need || pg < 0) break;
              __nanosleep(32);
            } while (++it < spin_limit);
            if (pg < need) {
              if (lane == poller && pg >= 0) atomicOr(sticky_err, 1);
              failed = true;
              break;
            }
            known = pg;
          }
          if (lane == poller && hasS) load_group(s, gcur);
        }
        // the next group too, if the previous strip has already published it
        const int need2 = min(s + 2 * SGS_PUBLISH, nx);
        if (s + SGS_PUBLISH < nx) {
          if (known < need2) {
            int pg = 0;
            if (lane == poller) pg = ld_acquire(&prog[q - 1]);
            pg = __shfl_sync(FULL, pg, poller);
            if (pg > known) known = pg;
          }
          if (known >= need2) {
            if (lane == poller && hasS) load_group(s + SGS_PUBLISH, gcur ^ 1);
            have_next = true;
          }
        }
      }
      if (act) {
        if (lagk == 0 && hasS) {   // south value from the previous strip
#pragma unroll
          for (int k = 0; k < NC; ++k) xS[k] = sgrp[(gcur * SGS_PUBLISH + (c & (SGS_PUBLISH - 1))) * NC + k];
        }
        const T* Vl = V + line * 32 + lane;
        const int ES = S * 32;   // stride between entries in the stage
        T xe[NC], xn[NC];
#pragma unroll
        for (int k = 0; k < NC; ++k) {
          xe[k] = Vl[(EX + k) * ES];
          xn[k] = nedge ? rn[0][k] : Vl[(EX + k) * ES + (FWD ? 1 : -1)];
        }
        T bb[NC];
#pragma unroll
        for (int k = 0; k < NC; ++k) bb[k] = Vl[(EB + k) * ES];
        sgs_cell<NC, T>(Vl + oW * ES, Vl + oE * ES, Vl + oS * ES, Vl + oN * ES, ES, Vl + (size_t)NOFF * ES,
                        PV[line * 32 + lane], bb, c > 0, xprev, c < nx - 1, xe, hasS, xS, hasN, xn, res);
        const long long slot = (dbase + line) * 32 + lane;   // coalesced: one line per step
#pragma unroll
        for (int k = 0; k < NC; ++k) {
          x[k * P + slot] = res[k];
          xprev[k] = res[k];
        }
      }
      if (nedge) {   // advance the edge lane's ring, fetch column c + SGS_PREFETCH
#pragma unroll
        for (int t = 0; t + 1 < SGS_PREFETCH; ++t)
#pragma unroll
          for (int k = 0; k < NC; ++k) rn[t][k] = rn[t + 1][k];
        const int cf = c + SGS_PREFETCH;
#pragma unroll
        for (int k = 0; k < NC; ++k) rn[SGS_PREFETCH - 1][k] = T(0);
        if (rowok && hasN && cf >= 0 && cf < nx) load_north(cf, rn[SGS_PREFETCH - 1]);
      }
      __syncwarp();
      if (lagk == 31 && act && q + 1 < nstrips && ((c + 1) % SGS_PUBLISH == 0 || c == nx - 1))
        st_release(&prog[q], c + 1);   // orders this lane's earlier stores and loads
    }
    __syncwarp();
    if (!failed && j + 2 < nchunks) {
      if (lane == 0) issue(j + 2, st);
      inflight[st] = true;
    }
  }
  if (failed) {
    // stop the other strips, then let this warp's copies land before leaving;
    // the drain has its own bound: a bulk copy that was issued completes, so
    // it must not inherit a wait limit shortened for failure tests
    if (lane == 0) st_release(abort_flag, 1);
    for (int st = 0; st < 2; ++st)
      if (inflight[st]) chunk_wait(&bar[st], parity[st], kDrainLimit);
    return false;
  }
  return true;
}

// barriers of the warp's two staging buffers
__device__ __forceinline__ void sgs_init_bars(unsigned char* smem) {
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  if (threadIdx.x == 0) {
    mbar_init(&bar[0]);
    mbar_init(&bar[1]);
    fence_proxy_async();
  }
  __syncwarp();
}

// one problem: strips claimed through the ticket sync[0]; sync[1] abort,
// sync[2 + q] progress of the strip processed q-th
template <int NC, typename T, bool FWD, int S>
__global__ void __launch_bounds__(32, 1) k_sgs_strip(int nx, int ny, const T* __restrict__ blk,
                                                  const T* __restrict__ lu, const int8_t* __restrict__ piv,
                                                  const T* __restrict__ b, T* x, int* sync, int* sticky_err,
                                                  int nstrips, int spin_limit) {
  extern __shared__ __align__(128) unsigned char smem[];
  sgs_init_bars(smem);
  unsigned parity[2] = {0u, 0u};
  for (;;) {
    int q = 0;
    if (threadIdx.x == 0) q = atomicAdd(&sync[0], 1);
    q = __shfl_sync(0xffffffffu, q, 0);
    if (q >= nstrips) return;
    if (!sgs_strip_run<NC, T, FWD, S>(nx, ny, blk, lu, piv, b, x, sync + 2, sync + 1, sticky_err, q, nstrips,
                                      spin_limit, smem, parity))
      return;
  }
}

// ---- block SGS half-sweep, warp-specialised strip kernel -------------------
// The sweep, the cell order and the cell arithmetic (sgs_cell) of k_sgs_strip,
// with everything that is not on the sweep's dependency chain taken off the
// warp that updates the cells.  One CTA of three warps per strip in flight:
//   warp 0 (compute) updates the strip's 32 rows, one skewed line per step,
//     reading its operands from shared memory only;
//   warp 1 moves the previous strip's new last-row values into a shared ring;
//   warp 2 stages the operator chunks into the two shared buffers
//     (cp.async.bulk, mbarrier completion; the compute warp hands a buffer
//     back through a second mbarrier) and, once a chunk has landed, forms the
//     old east / north part of every step of it (a third mbarrier), so that
//     a step of warp 0 is only the new west / south terms and the LU solve.
// Ring words carry the strip and column they hold, so the compute warp needs
// no fence to read them (a fence would wait for its own stores in flight);
// it reports the columns it is done with through a plain counter that only
// paces warp 1.
// Hand-off between strips without fences: the strip's last lane writes every
// new value of its row as 64-bit words, each holding 32 bits of the value and
// the launch's epoch (a counter that differs between launches).  The next
// strip's loader polls these words and takes a column once all of its words
// carry the current epoch; a word is written and read in one access, so a
// value never arrives without its tag.  On a GB300 a release store costs about
// a microsecond, several cell updates of this kernel.
// Every wait is bounded.  On expiry the kernel sets the sticky error word and
// the abort word, lets its own bulk copies in flight land (bounded), and
// returns; the other CTAs see the abort word and return as well.
// sync: [0] ticket, [1] abort.  edge: (strip q, column c, word w) at
// (q * nx + c) * WPC + w, WPC = NC * sizeof(T) / 4.
constexpr int SGS_RING = 32;   // columns held by each shared ring

// plain (volatile) shared-memory words: the progress counters between the two
// warps only pace the rings; the data in the rings carries its own tag
__device__ __forceinline__ int lds_vol(const int* p) {
  int v;
  asm volatile("ld.volatile.shared.s32 %0, [%1];" : "=r"(v) : "r"(smem_addr(p)) : "memory");
  return v;
}
__device__ __forceinline__ void sts_vol(int* p, int v) {
  asm volatile("st.volatile.shared.s32 [%0], %1;" ::"r"(smem_addr(p)), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long lds64_vol(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.volatile.shared.u64 %0, [%1];" : "=l"(v) : "r"(smem_addr(p)) : "memory");
  return v;
}
__device__ __forceinline__ void sts64_vol(unsigned long long* p, unsigned long long v) {
  asm volatile("st.volatile.shared.u64 [%0], %1;" ::"r"(smem_addr(p)), "l"(v) : "memory");
}
// predicated forms: the lane-specific accesses of a warp step without a branch
__device__ __forceinline__ unsigned long long lds64_vol_if(const unsigned long long* p, bool c) {
  unsigned long long v = 0ull;
  asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %2, 0;\n @q ld.volatile.shared.u64 %0, [%1];\n}"
               : "+l"(v)
               : "r"(smem_addr(p)), "r"((unsigned)c)
               : "memory");
  return v;
}
__device__ __forceinline__ void sts_vol_if(int* p, int v, bool c) {
  asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %2, 0;\n @q st.volatile.shared.s32 [%0], %1;\n}" ::"r"(smem_addr(p)),
               "r"(v), "r"((unsigned)c)
               : "memory");
}
__device__ __forceinline__ void st_tagged_if(unsigned long long* p, unsigned long long v, bool c) {
  asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %2, 0;\n @q st.relaxed.gpu.global.u64 [%0], %1;\n}" ::"l"(p), "l"(v),
               "r"((unsigned)c)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive_if(uint64_t* bar, bool c) {
  asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %1, 0;\n @q mbarrier.arrive.shared::cta.b64 _, [%0];\n}" ::"r"(
                   smem_addr(bar)),
               "r"((unsigned)c)
               : "memory");
}
__device__ __forceinline__ int ldg_vol(const int* p) {
  int v;
  asm volatile("ld.volatile.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_tagged(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// 32-bit pieces of a value: one for float, two (low, high) for double
template <typename T> struct Words;
template <> struct Words<float> {
  static constexpr int N = 1;
  __device__ static unsigned get(float v, int) { return __float_as_uint(v); }
  __device__ static float make(const unsigned* w) { return __uint_as_float(w[0]); }
};
template <> struct Words<double> {
  static constexpr int N = 2;
  __device__ static unsigned get(double v, int h) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    return h ? (unsigned)(u >> 32) : (unsigned)u;
  }
  __device__ static double make(const unsigned* w) {
    return __longlong_as_double((long long)(((unsigned long long)w[1] << 32) | w[0]));
  }
};

__host__ __device__ constexpr int pow2_floor(int v) { return v >= 32 ? 32 : v >= 16 ? 16 : v >= 8 ? 8 : v >= 4 ? 4 : v >= 2 ? 2 : 1; }

template <int NC, typename T>
struct SgsWs {
  static constexpr int WPC = NC * Words<T>::N;         // tagged words per column
  static constexpr int GS = pow2_floor(32 / WPC);      // previous-strip columns polled at once
  // control block (the first 128 bytes): mbarriers full[2] (a chunk's bulk
  // copies landed), empty[2] (the compute warp is done with a buffer),
  // afull[2] (the chunk's old east / north parts are written) in bytes 0-47,
  // then these int slots (indices into the block as int[32])
  static constexpr int Q = 12, LEAD = 13, FAIL = 14, ISSUED = 15;
  static_assert(Q * 4 >= 48 && ISSUED * 4 + 4 <= 128, "control slots must sit between the barriers and byte 128");
  static_assert(GS * WPC <= 32 && 2 * GS <= SGS_RING, "ring groups");
};

// Shared memory of k_sgs_ws: control block, two staging buffers, two buffers
// of the old east / north parts (S lines x NC x 32 lanes), the north values of
// a chunk (S x NC), the south ring.  The ring holds 64-bit words: 32 bits of a
// value and, above them, the tag q * nx + c of the strip q and column c it
// belongs to (all ones: empty).
template <int NC, typename T, int S>
struct SgsWsLayout {
  static constexpr size_t STAGE = sgs_stage_bytes<NC, T, S>();
  static constexpr size_t ABUF = (size_t)S * NC * 32 * sizeof(T);
  static constexpr size_t OFF_A = 128 + 2 * STAGE;
  static constexpr size_t OFF_N = OFF_A + 2 * ABUF;
  static constexpr size_t OFF_R = OFF_N + ((S * NC * sizeof(T) + 15) / 16) * 16;
  static constexpr size_t BYTES = OFF_R + (size_t)SGS_RING * SgsWs<NC, T>::WPC * 8;
};

template <int NC, typename T, int S>
size_t sgs_ws_smem_bytes() { return SgsWsLayout<NC, T, S>::BYTES; }

// warp 0 of k_sgs_ws: the strip's cell updates.  Per step it reads the new
// west (its own last result) and south (the lane below; for the lane of lag
// 0 the previous strip, through the south ring) values, the W and S blocks,
// the LU factors and the old east / north part that warp 2 formed for the
// chunk, and finishes the cell (sgs_cell_new).  waited counts the chunks
// whose staging completed.  Returns false when a wait ran out (sticky error
// and abort word set here) or another warp failed.
template <int NC, typename T, bool FWD, int S>
__device__ __forceinline__ bool sgs_ws_compute(int nx, int ny, T* x, unsigned long long* edge, unsigned epoch,
                                               int* abort_flag, int* sticky_err, int q, int nstrips,
                                               int spin_limit, unsigned char* smem, unsigned& parity_f,
                                               unsigned& parity_a, int& waited) {
  using W = SgsWs<NC, T>;
  using LY = SgsWsLayout<NC, T, S>;
  constexpr int BS = NC * NC;
  constexpr int NOFF = 4 * BS;
  constexpr int EX = NOFF + LU_E + NC;
  constexpr int NE = EX + NC;
  constexpr int ES = S * 32;   // stride between entries in a stage
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);   // full[0..1], empty[2..3], afull[4..5]
  int* ctl = reinterpret_cast<int*>(smem);
  const unsigned long long* ring_s = reinterpret_cast<const unsigned long long*>(smem + LY::OFF_R);
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const long long P = skew_slots(nx, ny);
  const unsigned tag0 = (unsigned)q * (unsigned)nx;   // ring tag of column c: tag0 + c
  const int oW = (FWD ? 0 : 1) * BS, oS = (FWD ? 2 : 3) * BS;
  const int lagk = FWD ? lane : 31 - lane;
  const int nsteps_full = nx + 31;
  const int ps = FWD ? q : nstrips - 1 - q;
  const long long line_base = (long long)ps * (nx + 31);
  const int rows = min(32, ny - ps * 32);
  const int nsteps = FWD ? nx + rows - 1 : nsteps_full;
  const int nchunks = (nsteps + S - 1) / S;
  const int y = ps * 32 + lane;
  const bool rowok = y < ny;
  const bool hasS = FWD ? (y > 0) : (y < ny - 1);
  const int lead = FWD ? 0 : 31;   // the lane of lag 0
  const bool need_s = q > 0 && __shfl_sync(FULL, (int)(rowok && hasS), lead) != 0;
  const bool publish = q + 1 < nstrips;
  bool timeout = false, failed = false;
  int bad = 0;   // this lane's ring wait: 1 another warp failed, 2 ran out
  // bounded wait for a barrier phase (warp-uniform), watching the fail word
  auto wait_bar = [&](uint64_t* b, unsigned par) -> bool {
    for (int it = 0;; ++it) {
      if (__all_sync(FULL, mbar_try_wait(b, par))) return true;
      int f = 0;
      if (lane == 0) f = lds_vol(&ctl[W::FAIL]);
      if (__shfl_sync(FULL, f, 0)) return false;
      if (it + 1 >= spin_limit) {
        timeout = true;
        return false;
      }
    }
  };
  T xprev[NC], res[NC];
#pragma unroll
  for (int k = 0; k < NC; ++k) { xprev[k] = T(0); res[k] = T(0); }
  for (int j = 0; j < nchunks; ++j) {
    const int st = j & 1;
    if (!wait_bar(&bar[st], (parity_f >> st) & 1u)) { failed = true; break; }
    parity_f ^= 1u << st;
    ++waited;
    if (!wait_bar(&bar[4 + st], (parity_a >> st) & 1u)) { failed = true; break; }
    parity_a ^= 1u << st;
    const T* V = reinterpret_cast<const T*>(smem + 128 + (size_t)st * LY::STAGE) + lane;
    const int8_t* PV = reinterpret_cast<const int8_t*>(smem + 128 + (size_t)st * LY::STAGE +
                                                       (size_t)NE * S * 32 * sizeof(T)) + lane;
    const T* A = reinterpret_cast<const T*>(smem + LY::OFF_A + (size_t)st * LY::ABUF) + lane;
    const int s0 = j * S, cnt = min(S, nsteps - s0);
#pragma unroll 2
    for (int i = 0; i < cnt; ++i) {
      const int s = s0 + i;
      const int line = FWD ? i : cnt - 1 - i;
      const T* Vl = V + line * 32;
      const int c = s - lagk;
      const bool act = rowok && (unsigned)c < (unsigned)nx;
      T aw[BS], as[BS], lu[LU_E], a[NC];
#pragma unroll
      for (int e = 0; e < BS; ++e) {
        aw[e] = Vl[(oW + e) * ES];
        as[e] = Vl[(oS + e) * ES];
      }
#pragma unroll
      for (int e = 0; e < LU_E; ++e) lu[e] = Vl[(NOFF + e) * ES];
      const int8_t pv = PV[line * 32];
#pragma unroll
      for (int k = 0; k < NC; ++k) a[k] = A[(line * NC + k) * 32];
      // the lead lane's south value of column s, once its ring words carry
      // this strip's and column's tag (the wait is warp-uniform)
      const bool want = lagk == 0 && need_s && s < nx;
      T rv[NC];
      {
        const unsigned long long* r = ring_s + (s & (SGS_RING - 1)) * W::WPC;
        const unsigned tg = tag0 + (unsigned)s;
        unsigned bits[W::WPC];
        bool ok = true;
#pragma unroll
        for (int w = 0; w < W::WPC; ++w) {
          const unsigned long long v64 = lds64_vol_if(r + w, want);
          bits[w] = (unsigned)v64;
          ok = ok && (unsigned)(v64 >> 32) == tg;
        }
        ok = ok || !want;
        if (__any_sync(FULL, !ok)) {
          for (int it = 1; !ok && !bad; ++it) {
            ok = true;
#pragma unroll
            for (int w = 0; w < W::WPC; ++w) {
              const unsigned long long v64 = lds64_vol(r + w);
              bits[w] = (unsigned)v64;
              ok = ok && (unsigned)(v64 >> 32) == tg;
            }
            if (!ok && (it & 63) == 63 && lds_vol(&ctl[W::FAIL])) bad = 1;
            else if (!ok && it + 1 >= spin_limit) bad = 2;
          }
          if (__any_sync(FULL, bad != 0)) { failed = true; break; }
        }
#pragma unroll
        for (int k = 0; k < NC; ++k) rv[k] = Words<T>::make(bits + k * Words<T>::N);
      }
      T xS[NC], rnew[NC];
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        xS[k] = FWD ? __shfl_up_sync(FULL, res[k], 1) : __shfl_down_sync(FULL, res[k], 1);
        if (lagk == 0) xS[k] = rv[k];
      }
      sgs_cell_new<NC, T>(aw, as, lu, pv, a, c > 0, xprev, hasS, xS, rnew);
      const long long slot = (line_base + (FWD ? s : nsteps_full - 1 - s)) * 32 + lane;
      const bool pub = lagk == 31 && publish && act;
      unsigned long long* e = edge + ((long long)q * nx + (pub ? c : 0)) * W::WPC;
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        if (act) x[k * P + slot] = rnew[k];
        xprev[k] = act ? rnew[k] : xprev[k];
        res[k] = rnew[k];
#pragma unroll
        for (int h = 0; h < Words<T>::N; ++h)   // the new last-row value for the next strip, tagged
          st_tagged_if(e + k * Words<T>::N + h, ((unsigned long long)epoch << 32) | Words<T>::get(rnew[k], h), pub);
      }
      // south ring slots the lead lane is done with (pace the poller)
      sts_vol_if(&ctl[W::LEAD], s + 1, lagk == 0 && s < nx && (((s + 1) & (W::GS - 1)) == 0 || s == nx - 1));
    }
    if (failed) break;
    __syncwarp();
    mbar_arrive_if(&bar[2 + st], lane == 0);   // the buffer goes back to warp 2
  }
  if (failed && lane == 0) {
    if (timeout) atomicOr(sticky_err, 1);
    sts_vol(&ctl[W::FAIL], 1);
    st_release(abort_flag, 1);
  }
  if (failed && __any_sync(FULL, bad == 2) && lane == 0) atomicOr(sticky_err, 1);
  return !failed;
}

// warps 1 and 2 of k_sgs_ws.  Role 1 fills the south ring from the previous
// strip's tagged words.  Role 2 stages the operator chunks and, once a chunk
// has landed, forms its old east / north part for every line and lane
// (sgs_cell_old, the north values of the strip's last lane loaded from the
// next strip's first row, which that strip cannot have updated yet: it waits
// for this strip's last row, which needs these values first).  One pass of
// the loop looks at each of the role's tasks once and blocks on none.
// Returns false when its wait ran out (sticky error and abort word set here)
// or another warp or CTA failed.
template <int NC, typename T, bool FWD, int S>
__device__ __forceinline__ bool sgs_ws_helper(int nx, int ny, const T* __restrict__ blk,
                                              const T* __restrict__ lu, const int8_t* __restrict__ piv,
                                              const T* __restrict__ b, const T* x,
                                              const unsigned long long* edge, unsigned epoch, int* abort_flag,
                                              int* sticky_err, int q, int nstrips, int spin_limit,
                                              unsigned char* smem, unsigned& parity_e, unsigned& parity_f2,
                                              unsigned& used, int role) {
  using W = SgsWs<NC, T>;
  using LY = SgsWsLayout<NC, T, S>;
  constexpr int BS = NC * NC;
  constexpr int NOFF = 4 * BS;
  constexpr int EB = NOFF + LU_E;
  constexpr int EX = EB + NC;
  constexpr int NE = EX + NC;
  constexpr int ES = S * 32;
  constexpr size_t STAGE = LY::STAGE;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  int* ctl = reinterpret_cast<int*>(smem);
  auto vals = [&](int st) { return reinterpret_cast<T*>(smem + 128 + (size_t)st * STAGE); };
  auto pvs = [&](int st) {
    return reinterpret_cast<int8_t*>(smem + 128 + (size_t)st * STAGE + (size_t)NE * S * 32 * sizeof(T));
  };
  unsigned long long* ring_s = reinterpret_cast<unsigned long long*>(smem + LY::OFF_R);
  T* nbuf = reinterpret_cast<T*>(smem + LY::OFF_N);
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const long long P = skew_slots(nx, ny);
  const unsigned tag0 = (unsigned)q * (unsigned)nx;
  const int oE = (FWD ? 1 : 0) * BS, oN = (FWD ? 3 : 2) * BS;
  const int lagk = FWD ? lane : 31 - lane;
  const int nsteps_full = nx + 31;
  const int ps = FWD ? q : nstrips - 1 - q;
  const long long line_base = (long long)ps * (nx + 31);
  const int rows = min(32, ny - ps * 32);
  const int nsteps = FWD ? nx + rows - 1 : nsteps_full;
  const int nchunks = (nsteps + S - 1) / S;
  const int y = ps * 32 + lane;
  const bool hasN = FWD ? (y < ny - 1) : (y > 0);
  // chunk j (S lines) of the operator, LU factors, b and the old x lines one
  // step ahead, copies spread over the warp's lanes
  auto issue = [&](int j, int st) {
    const int s0 = j * S, cnt = min(S, nsteps - s0);
    const int dlo = FWD ? s0 : nsteps_full - s0 - cnt;
    const long long off = (line_base + dlo) * 32;
    const unsigned vb = (unsigned)(cnt * 32 * sizeof(T));
    const int xlo = dlo + (FWD ? 1 : -1);
    const int xa = max(xlo, 0), xb = min(xlo + cnt, nsteps_full);
    const unsigned xbytes = xb > xa ? (unsigned)((xb - xa) * 32 * sizeof(T)) : 0u;
    if (lane == 0) {
      fence_proxy_async();
      mbar_expect_tx(&bar[st], vb * EX + xbytes * NC + (unsigned)(cnt * 32));
    }
    __syncwarp();
    const int ncopy = EX + (xbytes ? NC : 0) + 1;   // operator, LU, b, old x, pivot codes
    for (int e = lane; e < ncopy; e += 32) {
      if (e < NOFF)
        bulk_g2s(vals(st) + (size_t)e * S * 32, blk + (long long)(BS + e) * P + off, vb, &bar[st]);
      else if (e < NOFF + LU_E)
        bulk_g2s(vals(st) + (size_t)e * S * 32, lu + (long long)(e - NOFF) * P + off, vb, &bar[st]);
      else if (e < EX)
        bulk_g2s(vals(st) + (size_t)e * S * 32, b + (long long)(e - EB) * P + off, vb, &bar[st]);
      else if (e < ncopy - 1)
        bulk_g2s(vals(st) + (size_t)e * S * 32 + (size_t)(xa - xlo) * 32,
                 x + (long long)(e - EX) * P + (line_base + xa) * 32, xbytes, &bar[st]);
      else
        bulk_g2s(pvs(st), piv + off, (unsigned)(cnt * 32), &bar[st]);
    }
  };
  // the old east / north part of every step of chunk j into its buffer
  auto old_part = [&](int j) {
    const int st = j & 1;
    const int s0 = j * S, cnt = min(S, nsteps - s0);
    // north values of the last lane's columns s - 31, s in the chunk
    const int ytrail = ps * 32 + (FWD ? 31 : 0);
    const bool need_n = ytrail < ny && (FWD ? ytrail < ny - 1 : ytrail > 0);
    const int yN = FWD ? ytrail + 1 : ytrail - 1;
    for (int idx = lane; idx < cnt * NC; idx += 32) {
      const int t = idx / NC, k = idx - t * NC, c = s0 + t - 31;
      T v = T(0);
      if (need_n && c >= 0 && c < nx) v = __ldcg(&x[k * P + skew_pos(FWD ? c : nx - 1 - c, yN, nx)]);
      nbuf[idx] = v;
    }
    __syncwarp();
    const T* V = vals(st) + lane;
    T* A = reinterpret_cast<T*>(smem + LY::OFF_A + (size_t)st * LY::ABUF) + lane;
    for (int line = 0; line < cnt; ++line) {
      const int i = FWD ? line : cnt - 1 - line;   // the chunk step of this line
      const int c = s0 + i - lagk;
      const T* Vl = V + line * 32;
      T xe[NC], xn[NC], bb[NC], a[NC];
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        xe[k] = Vl[(EX + k) * ES];
        xn[k] = lagk == 31 ? nbuf[i * NC + k] : Vl[(EX + k) * ES + (FWD ? 1 : -1)];
        bb[k] = Vl[(EB + k) * ES];
      }
      sgs_cell_old<NC, T>(Vl + oE * ES, Vl + oN * ES, ES, bb, c < nx - 1, xe, hasN, xn, a);
#pragma unroll
      for (int k = 0; k < NC; ++k) A[(line * NC + k) * 32] = a[k];
    }
    __syncwarp();
    mbar_arrive_if(&bar[4 + st], lane == 0);
  };
  const int ylead = ps * 32 + (FWD ? 0 : 31);
  const bool need_s = q > 0 && ylead < ny && (FWD ? ylead > 0 : ylead < ny - 1);
  int next = role == 2 ? 0 : nchunks;      // chunks issued
  int next_a = role == 2 ? 0 : nchunks;    // chunks whose old part is written
  int s_loaded = role == 1 && need_s ? 0 : nx;
  bool failed = false, timeout = false;
  for (int idle = 0;;) {
    bool prog = false;
    if (s_loaded < nx) {   // the previous strip's new last row, up to GS columns at a time
      int ldone = 0;
      if (lane == 0) ldone = lds_vol(&ctl[W::LEAD]);
      ldone = __shfl_sync(FULL, ldone, 0);
      if (s_loaded + W::GS <= ldone + SGS_RING) {
        const int t = lane / W::WPC, w = lane % W::WPC, c = s_loaded + t;
        const bool mine = lane < W::GS * W::WPC && c < nx;
        unsigned long long word = 0ull;
        bool ok = true;
        if (mine) {
          word = ld_tagged(edge + ((long long)(q - 1) * nx + c) * W::WPC + w);
          ok = (unsigned)(word >> 32) == epoch;
        }
        const unsigned stale = __ballot_sync(FULL, mine && !ok);
        int nv = stale ? (__ffs(stale) - 1) / W::WPC : W::GS;   // columns before the first stale word
        nv = min(nv, nx - s_loaded);
        if (nv > 0) {
          if (mine && t < nv)
            sts64_vol(ring_s + (c & (SGS_RING - 1)) * W::WPC + w,
                      ((unsigned long long)(tag0 + (unsigned)c) << 32) | (unsigned)word);
          s_loaded += nv;
          prog = true;
        }
      }
    }
    if (next_a < next) {   // a landed chunk's old part
      int ok = 0;
      if (lane == 0) ok = mbar_try_wait(&bar[next_a & 1], (parity_f2 >> (next_a & 1)) & 1u) ? 1 : 0;
      if (__shfl_sync(FULL, ok, 0)) {
        parity_f2 ^= 1u << (next_a & 1);
        old_part(next_a);
        ++next_a;
        prog = true;
      }
    }
    if (next < nchunks) {   // the next chunk, once its buffer is free
      const int st = next & 1;
      bool free_buf = true;
      if ((used >> st) & 1u) {
        int ok = 0;
        if (lane == 0) ok = mbar_try_wait(&bar[2 + st], (parity_e >> st) & 1u) ? 1 : 0;
        free_buf = __shfl_sync(FULL, ok, 0) != 0;
      }
      if (free_buf) {
        if ((used >> st) & 1u) parity_e ^= 1u << st;
        used |= 1u << st;
        issue(next, st);
        ++next;
        prog = true;
      }
    }
    if (next >= nchunks && next_a >= nchunks && s_loaded >= nx) break;
    if (prog) {
      idle = 0;
      continue;
    }
    int stop = 0;
    if (lane == 0) stop = (lds_vol(&ctl[W::FAIL]) || ldg_vol(abort_flag)) ? 1 : 0;
    if (__shfl_sync(FULL, stop, 0)) {
      failed = true;
      break;
    }
    if (++idle >= spin_limit) {
      failed = timeout = true;
      break;
    }
    __nanosleep(20);
  }
  if (lane == 0) {
    if (role == 2) ctl[W::ISSUED] = next;
    if (failed) {
      if (timeout) atomicOr(sticky_err, 1);
      sts_vol(&ctl[W::FAIL], 1);
      st_release(abort_flag, 1);
    }
  }
  return !failed;
}

template <int NC, typename T, bool FWD, int S>
__global__ void __launch_bounds__(96, 1) k_sgs_ws(int nx, int ny, const T* __restrict__ blk,
                                                  const T* __restrict__ lu, const int8_t* __restrict__ piv,
                                                  const T* __restrict__ b, T* x, int* sync,
                                                  unsigned long long* edge, unsigned epoch, int* sticky_err,
                                                  int nstrips, int spin_limit) {
  using W = SgsWs<NC, T>;
  using LY = SgsWsLayout<NC, T, S>;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  int* ctl = reinterpret_cast<int*>(smem);
  if (threadIdx.x == 0) {
    for (int k = 0; k < 6; ++k) mbar_init(&bar[k]);
    ctl[W::FAIL] = 0;
    fence_proxy_async();
  }
  {   // empty ring words: a tag no column has
    unsigned long long* ring = reinterpret_cast<unsigned long long*>(smem + LY::OFF_R);
    for (int i = threadIdx.x; i < SGS_RING * W::WPC; i += blockDim.x) ring[i] = ~0ull;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5;
  // per stage st (bit st): phase parities of full (warps 0 and 2 each keep
  // their own), afull, empty; buffers used once
  unsigned parity_f = 0u, parity_a = 0u, parity_e = 0u, used = 0u;
  for (;;) {
    if (threadIdx.x == 0) {
      ctl[W::Q] = atomicAdd(&sync[0], 1);
      ctl[W::LEAD] = 0;
      ctl[W::ISSUED] = 0;
    }
    __syncthreads();
    const int q = ctl[W::Q];
    if (q >= nstrips) return;
    int waited = 0;
    if (warp == 0)
      sgs_ws_compute<NC, T, FWD, S>(nx, ny, x, edge, epoch, sync + 1, sticky_err, q, nstrips, spin_limit, smem,
                                    parity_f, parity_a, waited);
    else
      sgs_ws_helper<NC, T, FWD, S>(nx, ny, blk, lu, piv, b, x, edge, epoch, sync + 1, sticky_err, q, nstrips,
                                   spin_limit, smem, parity_e, parity_f, used, warp);
    __syncthreads();
    if (ctl[W::FAIL]) {
      // the bulk copies in flight land before the CTA's shared memory goes
      // away; the drain has its own bound (an issued copy completes)
      if (warp == 0) {
        const int issued = ctl[W::ISSUED];
        for (int j = waited; j < issued; ++j) {
          chunk_wait(&bar[j & 1], (parity_f >> (j & 1)) & 1u, kDrainLimit);
          parity_f ^= 1u << (j & 1);
        }
      }
      return;
    }
  }
}

// ---- block Gauss-Seidel, two-colour variant (SWNMG_SMOOTH_COLOUR) ----------
// Not the paper's smoother (Section 2.3 sweeps lexicographically): a variant
// whose iterates differ, reported separately.  Cell (ix, iy) has colour
// (ix + iy) & 1.  In the strip-skewed layout line d of strip s holds the
// cells with ix + (iy & 31) = d, of colour (d + 32 s) & 1 = d & 1, so every
// line is one colour.  One warp per line of the colour being updated: lane k
// is row k of the strip; its west and east neighbours are lane k of lines
// d - 1 and d + 1, its south and north neighbours lanes k - 1 and k + 1 of
// those lines (across a strip edge: the neighbouring strip's edge row).
// Every neighbour has the other colour, so the lines of one colour are
// independent; each operator entry, b and x is read and x written as one
// coalesced line.  The cell update is sgs_cell, the lexicographic
// smoother's.
template <int NC, typename T>
__global__ void __launch_bounds__(256) k_sgs_colour(int nx, int ny, const T* __restrict__ blk,
                                                    const T* __restrict__ lu, const int8_t* __restrict__ piv,
                                                    const T* __restrict__ b, T* __restrict__ x, int colour,
                                                    long long nlines) {
  const long long w = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w >= nlines) return;
  constexpr int BS = NC * NC;
  const int lane = threadIdx.x & 31;
  const int per = nx + 31;                    // lines per strip
  const int half = (per - colour + 1) / 2;    // lines d = colour, colour + 2, ... of one strip
  const int strip = (int)(w / half);
  const int d = colour + 2 * (int)(w % half);
  const int ix = d - lane, iy = strip * 32 + lane;
  if (ix < 0 || ix >= nx || iy >= ny) return;
  const long long P = skew_slots(nx, ny);
  const long long slot = ((long long)strip * per + d) * 32 + lane;
  const bool hW = ix > 0, hE = ix < nx - 1, hS = iy > 0, hN = iy < ny - 1;
  T xw[NC], xe[NC], xs[NC], xn[NC], bb[NC], res[NC];
  const long long sW = slot - 32, sE = slot + 32;
  const long long sS = hS ? skew_pos(ix, iy - 1, nx) : slot, sN = hN ? skew_pos(ix, iy + 1, nx) : slot;
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    const T* xk = x + (long long)k * P;
    xw[k] = hW ? xk[sW] : T(0);
    xe[k] = hE ? xk[sE] : T(0);
    xs[k] = hS ? xk[sS] : T(0);
    xn[k] = hN ? xk[sN] : T(0);
    bb[k] = b[(long long)k * P + slot];
  }
  const int es = (int)P;
  sgs_cell<NC, T>(blk + (long long)BS * P + slot, blk + 2LL * BS * P + slot, blk + 3LL * BS * P + slot,
                  blk + 4LL * BS * P + slot, es, lu + slot, piv[slot], bb, hW, xw, hE, xe, hS, xs, hN, xn, res);
#pragma unroll
  for (int k = 0; k < NC; ++k) x[(long long)k * P + slot] = res[k];
}

// ---- exact coarse solve: banded Gaussian elimination, partial pivoting -------
// Unknowns cell-major (i*NC + s); lower bandwidth ml = NC*nx + NC - 1, upper
// ml (mu) plus ml fill.  One CTA; a pivot <= 1e-14 max|A| leaves its unknown
// at zero.  band: m * (2*ml + mu + 1) doubles of scratch.
template <int NC, typename T>
__global__ void k_coarse_exact(int nx, int ny, const T* __restrict__ blk, const T* __restrict__ b,
                               T* __restrict__ x, double* __restrict__ band, int* err) {
  const int n = nx * ny, m = n * NC;
  const int ml = NC * (ny > 1 ? nx : 1) + NC - 1, mu = ml, ldab = 2 * ml + mu + 1;
  const int BS = NC * NC;
  // row-major band: A(r, c), c - r in [-ml, ml + mu], at band[r * ldab + (c - r + ml)]
  auto AB = [&](int r, int c) -> double& { return band[(long long)r * ldab + (c - r + ml)]; };
  double* rhs = band + (long long)m * ldab;
  int* sing = reinterpret_cast<int*>(rhs + m);
  __shared__ double s_amax;
  for (long long e = threadIdx.x; e < (long long)m * ldab; e += blockDim.x) band[e] = 0.0;
  __syncthreads();
  const long long P = skew_slots(nx, ny);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int ix = i % nx, iy = i / nx;
    const long long si = skew_pos(ix, iy, nx);
    int nb[4] = {ix > 0 ? i - 1 : -1, ix < nx - 1 ? i + 1 : -1, iy > 0 ? i - nx : -1,
                 iy < ny - 1 ? i + nx : -1};
    for (int s = 0; s < NC; ++s) {
      rhs[i * NC + s] = (double)b[(long long)s * P + si];
      sing[i * NC + s] = 0;
      for (int k = 0; k < NC; ++k) AB(i * NC + s, i * NC + k) = (double)blk[(long long)(s * NC + k) * P + si];
      for (int side = 0; side < 4; ++side) {
        const int j = nb[side];
        if (j < 0) continue;
        for (int k = 0; k < NC; ++k)
          AB(i * NC + s, j * NC + k) = (double)blk[((long long)(1 + side) * BS + s * NC + k) * P + si];
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (long long e = 0; e < (long long)m * ldab; ++e) a = fabs(band[e]) > a ? fabs(band[e]) : a;
    s_amax = a;
  }
  __syncthreads();
  const double tiny = 1e-14 * s_amax;
  __shared__ int s_p, s_sing;
  for (int c = 0; c < m; ++c) {
    const int rend = c + ml < m - 1 ? c + ml : m - 1;
    if (threadIdx.x == 0) {
      int p = c;
      double best = fabs(AB(c, c));
      for (int r = c + 1; r <= rend; ++r)
        if (fabs(AB(r, c)) > best) { best = fabs(AB(r, c)); p = r; }
      s_p = p;
      s_sing = !(best > tiny);
      if (s_sing) sing[c] = 1;
    }
    __syncthreads();
    const int p = s_p;
    const int cend = c + ml + mu < m - 1 ? c + ml + mu : m - 1;
    if (p != c) {
      for (int k = c + threadIdx.x; k <= cend; k += blockDim.x) {
        const double t = AB(c, k); AB(c, k) = AB(p, k); AB(p, k) = t;
      }
      if (threadIdx.x == 0) { const double t = rhs[c]; rhs[c] = rhs[p]; rhs[p] = t; }
    }
    __syncthreads();
    if (s_sing) continue;   // uniform: the unknown keeps the value 0
    const double piv = AB(c, c);
    for (int r = c + 1 + threadIdx.x; r <= rend; r += blockDim.x) {
      const double l = AB(r, c) / piv;
      if (l == 0.0) continue;
      for (int k = c; k <= cend; ++k) AB(r, k) = AB(r, k) - l * AB(c, k);
      rhs[r] = rhs[r] - l * rhs[c];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    for (int r = m - 1; r >= 0; --r) {
      double v;
      if (sing[r]) v = 0.0;
      else {
        double s = rhs[r];
        const int cend = r + ml + mu < m - 1 ? r + ml + mu : m - 1;
        for (int k = r + 1; k <= cend; ++k) s = s - AB(r, k) * rhs[k];
        v = s / AB(r, r);
      }
      rhs[r] = v;   // rhs now holds the solution from r on
    }
    for (int r = 0; r < m; ++r) {
      const int cell = r / NC;
      x[(long long)(r % NC) * P + skew_pos(cell % nx, cell / nx, nx)] = (T)rhs[r];
    }
    if (err) *err = 0;
  }
}

// ---- exact coarse solve: guarded inverse -------------------------------------
// For a small coarsest level (m = NC*n unknowns, cell-major i*NC + s) the
// solve of Algorithm 0 is x = X b with X the "guarded inverse": Gaussian
// elimination with partial pivoting (largest |entry|, lowest row on ties) on
// [A | I], a pivot <= 1e-14 max|A| leaving its unknown at zero, then back
// substitution for every unit right-hand side.  The solve is linear in b, so
// X b equals that elimination applied to b.  X is formed once per Newton step
// (one CTA) and applied at every visit of the coarsest level.
// aug: m x 2m working array (row-major), X: m x m column-major.
template <int NC, typename T>
__device__ __forceinline__ void coarse_inverse_cta(int nx, int ny, const T* __restrict__ blk, T* __restrict__ aug,
                                                   T* __restrict__ X, int* __restrict__ sing) {
  const int n = nx * ny, m = n * NC, w = 2 * m;
  const long long P = skew_slots(nx, ny);
  const int BS = NC * NC;
  __shared__ T s_amax[32];
  __shared__ int s_p, s_sing;
  for (long long e = threadIdx.x; e < (long long)m * w; e += blockDim.x) aug[e] = T(0);
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int ix = i % nx, iy = i / nx;
    const long long si = skew_pos(ix, iy, nx);
    int nb[4] = {ix > 0 ? i - 1 : -1, ix < nx - 1 ? i + 1 : -1, iy > 0 ? i - nx : -1,
                 iy < ny - 1 ? i + nx : -1};
    for (int s = 0; s < NC; ++s) {
      const long long row = (long long)(i * NC + s) * w;
      for (int k = 0; k < NC; ++k) aug[row + i * NC + k] = blk[(long long)(s * NC + k) * P + si];
      for (int side = 0; side < 4; ++side) {
        const int j = nb[side];
        if (j < 0) continue;
        for (int k = 0; k < NC; ++k)
          aug[row + j * NC + k] = blk[((long long)(1 + side) * BS + s * NC + k) * P + si];
      }
      aug[row + m + i * NC + s] = T(1);
      sing[i * NC + s] = 0;
    }
  }
  __syncthreads();
  // max |A| (A part only)
  T a = T(0);
  for (long long e = threadIdx.x; e < (long long)m * m; e += blockDim.x) {
    const T v = tabs(aug[(e / m) * w + (e % m)]);
    a = v > a ? v : a;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const T b2 = __shfl_down_sync(0xffffffffu, a, o);
    a = b2 > a ? b2 : a;
  }
  if ((threadIdx.x & 31) == 0) s_amax[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    T mx = T(0);
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) mx = s_amax[q] > mx ? s_amax[q] : mx;
    s_amax[0] = mx;
  }
  __syncthreads();
  const T tiny = T(1e-14) * s_amax[0];
  for (int c = 0; c < m; ++c) {
    if (threadIdx.x < 32) {
      // the pivot row of the scan "if (|a| > best)" from row c down, by the
      // first warp: each lane scans every 32nd row, then the largest value
      // wins, the lower row on ties (the first one the scan meets); NaN
      // entries never win, and a NaN in row c keeps the scan there
      const int ln = (int)threadIdx.x;
      T best = T(-1);
      int p = m;
      for (int r = c + ln; r < m; r += 32) {
        const T v = tabs(aug[(long long)r * w + c]);
        if (v > best) { best = v; p = r; }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const T ob = __shfl_down_sync(0xffffffffu, best, off);
        const int op = __shfl_down_sync(0xffffffffu, p, off);
        if (ob > best || (ob == best && op < p)) { best = ob; p = op; }
      }
      if (ln == 0) {
        const T d = tabs(aug[(long long)c * w + c]);
        if (d != d) { best = d; p = c; }
        s_p = p;
        s_sing = !(best > tiny);
        if (s_sing) sing[c] = 1;
      }
    }
    __syncthreads();
    const int p = s_p;
    if (p != c)
      for (int k = threadIdx.x; k < w; k += blockDim.x) {
        const T t = aug[(long long)c * w + k];
        aug[(long long)c * w + k] = aug[(long long)p * w + k];
        aug[(long long)p * w + k] = t;
      }
    __syncthreads();
    if (!s_sing) {
      // multipliers first (kept in column c below the pivot, which the back
      // substitution never reads), then the row updates
      const T piv = aug[(long long)c * w + c];
      for (int r = c + 1 + threadIdx.x; r < m; r += blockDim.x) aug[(long long)r * w + c] /= piv;
      __syncthreads();
      // a warp per row, its lanes along the row (no index division)
      const int nwarps = (int)(blockDim.x >> 5), wid = (int)(threadIdx.x >> 5), ln = (int)(threadIdx.x & 31);
      const T* prow = aug + (long long)c * w;
      for (int r = c + 1 + wid; r < m; r += nwarps) {
        T* row = aug + (long long)r * w;
        const T l = row[c];
        for (int k = c + 1 + ln; k < w; k += 32) row[k] -= l * prow[k];
      }
    }
    __syncthreads();
  }
  // back substitution, one unit right-hand side per thread
  for (int jcol = threadIdx.x; jcol < m; jcol += blockDim.x) {
    for (int r = m - 1; r >= 0; --r) {
      T v;
      if (sing[r]) v = T(0);
      else {
        T acc = aug[(long long)r * w + m + jcol];
#pragma unroll 8
        for (int k = r + 1; k < m; ++k) acc -= aug[(long long)r * w + k] * X[(long long)jcol * m + k];
        v = acc / aug[(long long)r * w + r];
      }
      X[(long long)jcol * m + r] = v;
    }
  }
}

template <int NC, typename T>
__global__ void k_coarse_inverse(int nx, int ny, const T* __restrict__ blk, T* __restrict__ aug,
                                 T* __restrict__ X, int* __restrict__ sing) {
  coarse_inverse_cta<NC, T>(nx, ny, blk, aug, X, sing);
}

// x = X b on the coarsest level (SoA vectors, cell-major unknowns)
template <int NC, typename T>
__device__ __forceinline__ void coarse_apply_block(int nx, int ny, const T* __restrict__ X,
                                                   const T* __restrict__ b, T* __restrict__ x) {
  // b gathered once per block into unknown order (m <= 384), then one row per thread
  __shared__ __align__(16) unsigned char sraw[384 * sizeof(T)];
  T* sb = reinterpret_cast<T*>(sraw);
  const int n = nx * ny, m = n * NC;
  const long long P = skew_slots(nx, ny);
  for (int u = threadIdx.x; u < m; u += blockDim.x) {
    const int cell = u / NC;
    sb[u] = b[(long long)(u % NC) * P + skew_pos(cell % nx, cell / nx, nx)];
  }
  __syncthreads();
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= m) return;
  T acc = T(0);
#pragma unroll 16
  for (int jcol = 0; jcol < m; ++jcol) acc += X[(long long)jcol * m + u] * sb[jcol];   // in column order
  const int cell = u / NC;
  x[(long long)(u % NC) * P + skew_pos(cell % nx, cell / nx, nx)] = acc;
}

template <int NC, typename T>
__global__ void k_coarse_apply(int nx, int ny, const T* __restrict__ X, const T* __restrict__ b,
                               T* __restrict__ x) {
  coarse_apply_block<NC, T>(nx, ny, X, b, x);
}

// ---- adjoint support ----------------------------------------------------------
// Transposed block operator (FP64): D'_i = D_i^T, and the block of cell i
// towards neighbour j is the transpose of j's block towards i.
template <int NC, typename T>
__global__ void k_transpose_blocks(int nx, int ny, const T* __restrict__ src, double* __restrict__ dst) {
  const int n = nx * ny;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long P = skew_slots(nx, ny);
  const int BS = NC * NC;
  const int ix = i % nx, iy = i / nx;
  const long long si = skew_pos(ix, iy, nx);
  for (int s = 0; s < NC; ++s)
    for (int k = 0; k < NC; ++k) dst[(long long)(s * NC + k) * P + si] = (double)src[(long long)(k * NC + s) * P + si];
  const int nb[4] = {ix > 0 ? i - 1 : -1, ix < nx - 1 ? i + 1 : -1, iy > 0 ? i - nx : -1,
                     iy < ny - 1 ? i + nx : -1};
  for (int side = 0; side < 4; ++side) {
    const int j = nb[side];
    const long long sj = j >= 0 ? skew_pos(j % nx, j / nx, nx) : 0;
    const int back = side ^ 1;   // j's side facing i
    for (int s = 0; s < NC; ++s)
      for (int k = 0; k < NC; ++k)
        dst[((long long)(1 + side) * BS + s * NC + k) * P + si] =
            j >= 0 ? (double)src[((long long)(1 + back) * BS + k * NC + s) * P + sj] : 0.0;
  }
}

// ||b - A x||_1 per cell
template <int NC, typename T>
__global__ void k_lin_resid_abs(int dim, int nx, int ny, const T* __restrict__ blk, const T* __restrict__ b,
                                const T* __restrict__ x, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nx * ny) return;
  T r[NC];
  lin_resid<NC, T>(dim, nx, ny, blk, b, x, i, r);
  double a = 0.0;
  for (int s = 0; s < NC; ++s) a += fabs((double)r[s]);
  out[i] = a;
}

// sum_s |v_s| per cell (SoA, nc components)
__global__ void k_abs_cells(int n, int nc, const double* __restrict__ v, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a = 0.0;
  for (int s = 0; s < nc; ++s) a += fabs(v[(long long)s * n + i]);
  out[i] = a;
}

// fixed-order sum: per-block tree partials, then one block over the partials
__global__ void k_sum_partial(const double* __restrict__ v, int n, double* __restrict__ part) {
  __shared__ double sh[256];
  double a = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a += v[i];
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_sum_final(const double* __restrict__ part, int np, double* __restrict__ out) {
  __shared__ double sh[256];
  double a = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) a += part[i];
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

template <typename S, typename D>
__global__ void k_convert(const S* __restrict__ s, D* __restrict__ d, long long n, double scale) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    d[i] = static_cast<D>(scale * static_cast<double>(s[i]));
}

// natural SoA vector (nc x n) <-> strip-skewed vector (nc x P), scaled
template <typename S, typename D>
__global__ void k_to_skew(const S* __restrict__ s, D* __restrict__ d, int nc, int nx, int ny, double scale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = nx * ny;
  if (i >= n) return;
  const long long P = skew_slots(nx, ny), si = skew_pos(i % nx, i / nx, nx);
  for (int k = 0; k < nc; ++k) d[k * P + si] = static_cast<D>(scale * static_cast<double>(s[(long long)k * n + i]));
}

template <typename S, typename D>
__global__ void k_from_skew(const S* __restrict__ s, D* __restrict__ d, int nc, int nx, int ny, double scale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = nx * ny;
  if (i >= n) return;
  const long long P = skew_slots(nx, ny), si = skew_pos(i % nx, i / nx, nx);
  for (int k = 0; k < nc; ++k) d[(long long)k * n + i] = static_cast<D>(scale * static_cast<double>(s[k * P + si]));
}

template <typename T>
__global__ void k_fill0(T* __restrict__ d, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    d[i] = T(0);
}

template <typename T>
__global__ void k_export(int nx, int ny, int nc, const T* __restrict__ blk, double* __restrict__ out) {
  const int n = nx * ny;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long P = skew_slots(nx, ny), si = skew_pos(i % nx, i / nx, nx);
  const int BS = nc * nc;
  for (int b = 0; b < 5; ++b)
    for (int e = 0; e < BS; ++e)
      out[((long long)i * 5 + b) * BS + e] = (double)blk[((long long)b * BS + e) * P + si];
}

// ---- batched forms -------------------------------------------------------------
// Same bodies as the single-problem kernels; problem from the block table.
#define BATCH_PROLOGUE(bl)                                        \
  const int p_ = batch_find((bl).bstart, (bl).B, blockIdx.x);     \
  if (!(bl).mask[p_]) return;                                     \
  const BItem* it = (bl).items + p_;                              \
  const int idx = (blockIdx.x - (bl).bstart[p_]) * 128 + threadIdx.x;

template <int NC, typename T>
__global__ void __launch_bounds__(128) kb_lu_factor(BLaunch bl) {
  BATCH_PROLOGUE(bl)
  const int nx = it->L.nx, ny = it->L.ny;
  if (idx < skew_slots(nx, ny))
    lu_factor_slot<NC, T>(nx, ny, static_cast<const T*>(it->blk), static_cast<T*>(it->lu), it->piv, idx);
}

template <int NC, typename T>
__global__ void __launch_bounds__(128) kb_galerkin(BLaunch bl, const BItem* fine) {
  BATCH_PROLOGUE(bl)
  if (idx >= it->L.n) return;
  const BItem* f = fine + p_;
  galerkin_cell<NC, T>(2, f->L.nx, f->L.ny, static_cast<const T*>(f->blk), static_cast<T*>(it->blk), idx);
}

template <int NC, typename T>
__global__ void __launch_bounds__(128) kb_restrict(BLaunch bl, const BItem* fine) {
  BATCH_PROLOGUE(bl)
  if (idx >= it->L.n) return;
  const BItem* f = fine + p_;
  restrict_cell<NC, T>(2, f->L.nx, f->L.ny, static_cast<const T*>(f->blk), static_cast<const T*>(f->b),
                       static_cast<const T*>(f->x), static_cast<T*>(it->b), idx);
}

template <typename T>
__global__ void __launch_bounds__(128) kb_prolong(BLaunch bl, const BItem* coarse) {
  BATCH_PROLOGUE(bl)
  if (idx >= it->L.n) return;
  prolong_cell<T>(2, it->L.nc, it->L.nx, it->L.ny, static_cast<const T*>(coarse[p_].x), static_cast<T*>(it->x),
                  idx);
}

template <typename T>
__global__ void __launch_bounds__(128) kb_fill_x(BLaunch bl) {
  BATCH_PROLOGUE(bl)
  const int n = it->L.n;
  if (idx >= n) return;
  T* x = static_cast<T*>(it->x);
  const long long P = skew_slots(it->L.nx, it->L.ny), si = skew_pos(idx % it->L.nx, idx / it->L.nx, it->L.nx);
  for (int s = 0; s < it->L.nc; ++s) x[(long long)s * P + si] = T(0);
}

template <typename T>
__global__ void __launch_bounds__(128) kb_neg_residual(BLaunch bl) {
  BATCH_PROLOGUE(bl)
  const int n = it->L.n;
  if (idx >= n) return;
  T* b = static_cast<T*>(it->b);
  const long long P = skew_slots(it->L.nx, it->L.ny), si = skew_pos(idx % it->L.nx, idx / it->L.nx, it->L.nx);
  for (int s = 0; s < it->L.nc; ++s)
    b[(long long)s * P + si] = static_cast<T>(-1.0 * it->R[(long long)s * n + idx]);
}
#undef BATCH_PROLOGUE

// per-problem fixed-order sums of ||R_i||_1: the partial / final trees of
// launch_sum with the problem's own partial count (blockIdx.y = problem)
__device__ __forceinline__ int sum_partials(int n) {
  int g = (n + 255) / 256;
  return g > 1024 ? 1024 : (g < 1 ? 1 : g);
}

__global__ void kb_sum_partial(const BItem* items, const int* mask) {
  const int p = blockIdx.y;
  if (!mask[p]) return;
  const int n = items[p].L.n, g = sum_partials(n);
  if ((int)blockIdx.x >= g) return;
  const double* v = items[p].rn;
  __shared__ double sh[256];
  double a = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += g * blockDim.x) a += v[i];
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) items[p].red[blockIdx.x] = sh[0];
}

__global__ void kb_sum_final(const BItem* items, const int* mask, double* out) {
  const int p = blockIdx.x;
  if (!mask[p]) return;
  const int np = sum_partials(items[p].L.n);
  const double* part = items[p].red;
  __shared__ double sh[256];
  double a = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) a += part[i];
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[p] = sh[0];
}

// SGS over a batch: warps claim (problem, strip) tickets in order (strip
// index first), so a strip only ever waits for the previous strip of its own
// problem, which a running warp already owns.  sync: [0] ticket, [1] abort,
// [2 + strip0 + q] progress.
template <int NC, typename T, bool FWD, int S>
__global__ void __launch_bounds__(32, 1) kb_sgs_strip(const BItem* __restrict__ items,
                                                      const int2* __restrict__ tickets, int ntickets,
                                                      const int* __restrict__ mask, int* sync, int* sticky_err,
                                                      int spin_limit) {
  extern __shared__ __align__(128) unsigned char smem[];
  sgs_init_bars(smem);
  unsigned parity[2] = {0u, 0u};
  for (;;) {
    int t = 0;
    if (threadIdx.x == 0) t = atomicAdd(&sync[0], 1);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= ntickets) return;
    const int2 tk = tickets[t];
    if (!mask[tk.x]) continue;
    const BItem* it = items + tk.x;
    const int nx = it->L.nx, ny = it->L.ny;
    if (!sgs_strip_run<NC, T, FWD, S>(nx, ny, static_cast<const T*>(it->blk), static_cast<const T*>(it->lu),
                                      it->piv, static_cast<const T*>(it->b), static_cast<T*>(it->x),
                                      sync + 2 + it->strip0, sync + 1, sticky_err, tk.y, (ny + 31) / 32,
                                      spin_limit, smem, parity))
      return;
  }
}

template <int NC, typename T>
__global__ void __launch_bounds__(1024) kb_coarse_inverse(const BItem* items, const int* mask) {
  const int p = blockIdx.x;
  if (!mask[p]) return;
  const BItem* it = items + p;
  coarse_inverse_cta<NC, T>(it->L.nx, it->L.ny, static_cast<const T*>(it->blk), static_cast<T*>(it->caug),
                            static_cast<T*>(it->cinv), it->csing);
}

template <int NC, typename T>
__global__ void __launch_bounds__(128) kb_coarse_apply(const BItem* items, const int* mask) {
  const int p = blockIdx.y;
  if (!mask[p]) return;
  const BItem* it = items + p;
  if ((int)(blockIdx.x * blockDim.x) >= it->L.n * NC) return;   // whole block idle
  coarse_apply_block<NC, T>(it->L.nx, it->L.ny, static_cast<const T*>(it->cinv), static_cast<const T*>(it->b),
                            static_cast<T*>(it->x));
}

}  // namespace

// ---- launch wrappers ----------------------------------------------------------

static std::atomic<long long> g_launches{0};
void count_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launches_total() { return g_launches.load(std::memory_order_relaxed); }

static std::atomic<int> g_wait_limit{kDefaultWaitLimit};
int wait_limit() { return g_wait_limit.load(std::memory_order_relaxed); }
void set_wait_limit(int polls) {
  g_wait_limit.store(polls > 0 ? polls : kDefaultWaitLimit, std::memory_order_relaxed);
}

void launch_lu_factor(int nx, int ny, int nc, const void* blk, void* lu, int8_t* piv, int fp32,
                      cudaStream_t st) {
  count_launches(1);
  const int g = nblk(skew_slots(nx, ny), 128);
  if (nc == 3) {
    if (fp32) k_lu_factor<3, float><<<g, 128, 0, st>>>(nx, ny, (const float*)blk, (float*)lu, piv);
    else k_lu_factor<3, double><<<g, 128, 0, st>>>(nx, ny, (const double*)blk, (double*)lu, piv);
  } else {
    if (fp32) k_lu_factor<2, float><<<g, 128, 0, st>>>(nx, ny, (const float*)blk, (float*)lu, piv);
    else k_lu_factor<2, double><<<g, 128, 0, st>>>(nx, ny, (const double*)blk, (double*)lu, piv);
  }
}

void launch_galerkin(int dim, int nc, int nxf, int nyf, const void* bf, void* bc, int fp32,
                     cudaStream_t st) {
  count_launches(1);
  const int ncc = (nxf / 2) * (dim == 2 ? nyf / 2 : 1);
  const int g = nblk(ncc, 128);
  if (nc == 3) {
    if (fp32) k_galerkin<3, float><<<g, 128, 0, st>>>(dim, nxf, nyf, (const float*)bf, (float*)bc);
    else k_galerkin<3, double><<<g, 128, 0, st>>>(dim, nxf, nyf, (const double*)bf, (double*)bc);
  } else {
    if (fp32) k_galerkin<2, float><<<g, 128, 0, st>>>(dim, nxf, nyf, (const float*)bf, (float*)bc);
    else k_galerkin<2, double><<<g, 128, 0, st>>>(dim, nxf, nyf, (const double*)bf, (double*)bc);
  }
}

void launch_restrict(int dim, int nc, int nxf, int nyf, const void* blk, const void* b,
                     const void* x, void* bcoarse, int fp32, cudaStream_t st) {
  count_launches(1);
  const int ncc = (nxf / 2) * (dim == 2 ? nyf / 2 : 1);
  const int g = nblk(ncc, 128);
  if (dim == 2) {   // a lane per child
    const int g4 = nblk(4LL * ncc, 128);
    if (nc == 3) {
      if (fp32) k_restrict4<3, float><<<g4, 128, 0, st>>>(nxf, nyf, (const float*)blk, (const float*)b,
                                                          (const float*)x, (float*)bcoarse);
      else k_restrict4<3, double><<<g4, 128, 0, st>>>(nxf, nyf, (const double*)blk, (const double*)b,
                                                      (const double*)x, (double*)bcoarse);
      return;
    }
  }
#define RL(NC, T) k_restrict<NC, T><<<g, 128, 0, st>>>(dim, nxf, nyf, (const T*)blk, (const T*)b, \
                                                        (const T*)x, (T*)bcoarse)
  if (nc == 3) { if (fp32) RL(3, float); else RL(3, double); }
  else { if (fp32) RL(2, float); else RL(2, double); }
#undef RL
}

void launch_prolong(int dim, int nc, int nxf, int nyf, const void* xc, void* xf, int fp32,
                    cudaStream_t st) {
  count_launches(1);
  const int nf = nxf * (dim == 2 ? nyf : 1);
  if (fp32) k_prolong<float><<<nblk(nf, 256), 256, 0, st>>>(dim, nc, nxf, nyf, (const float*)xc, (float*)xf);
  else k_prolong<double><<<nblk(nf, 256), 256, 0, st>>>(dim, nc, nxf, nyf, (const double*)xc, (double*)xf);
}

template <int NC, typename T, bool F>
static void sgs_launch(int nx, int ny, const void* blk, const void* lu, const int8_t* piv,
                       const void* b, void* x, int* sync, int* sticky, cudaStream_t st) {
  constexpr int S = SgsChunk<T>::S;
  const int nstrips = (ny + 31) / 32;
  const size_t smem = sgs_smem_bytes<NC, T, S>();
  static bool configured = false;   // per template instance
  if (!configured) {
    cudaFuncSetAttribute(k_sgs_strip<NC, T, F, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    configured = true;
  }
  k_sgs_strip<NC, T, F, S><<<nstrips, 32, smem, st>>>(nx, ny, (const T*)blk, (const T*)lu, piv,
                                                       (const T*)b, (T*)x, sync, sticky, nstrips, wait_limit());
}

template <int NC, typename T, bool F>
static void sgs_ws_launch(int nx, int ny, const void* blk, const void* lu, const int8_t* piv, const void* b,
                          void* x, int* sync, unsigned long long* edge, unsigned epoch, int* sticky,
                          cudaStream_t st) {
  constexpr int S = SgsChunk<T>::S;
  const int nstrips = (ny + 31) / 32;
  const size_t smem = sgs_ws_smem_bytes<NC, T, S>();
  static bool configured = false;   // per template instance
  if (!configured) {
    cudaFuncSetAttribute(k_sgs_ws<NC, T, F, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    configured = true;
  }
  k_sgs_ws<NC, T, F, S><<<nstrips, 96, smem, st>>>(nx, ny, (const T*)blk, (const T*)lu, piv, (const T*)b,
                                                    (T*)x, sync, edge, epoch, sticky, nstrips, wait_limit());
}

void launch_sgs_sweep(int nc, int nx, int ny, const void* blk, const void* lu, const int8_t* piv,
                      const void* b, void* x, int forward, int fp32, int* sync, unsigned long long* edge,
                      unsigned epoch, int* sticky_err, cudaStream_t st) {
  count_launches(1);
  const int nstrips = (ny + 31) / 32;
  cudaMemsetAsync(sync, 0, sizeof(int) * (2 + nstrips), st);
  if (edge) {   // the warp-specialised kernel
#define WL(NC, T, F) sgs_ws_launch<NC, T, F>(nx, ny, blk, lu, piv, b, x, sync, edge, epoch, sticky_err, st)
    if (nc == 3) {
      if (fp32) { if (forward) WL(3, float, true); else WL(3, float, false); }
      else { if (forward) WL(3, double, true); else WL(3, double, false); }
    } else {
      if (fp32) { if (forward) WL(2, float, true); else WL(2, float, false); }
      else { if (forward) WL(2, double, true); else WL(2, double, false); }
    }
#undef WL
    return;
  }
#define SL(NC, T, F) sgs_launch<NC, T, F>(nx, ny, blk, lu, piv, b, x, sync, sticky_err, st)
  if (nc == 3) {
    if (fp32) { if (forward) SL(3, float, true); else SL(3, float, false); }
    else { if (forward) SL(3, double, true); else SL(3, double, false); }
  } else {
    if (fp32) { if (forward) SL(2, float, true); else SL(2, float, false); }
    else { if (forward) SL(2, double, true); else SL(2, double, false); }
  }
#undef SL
}

void launch_sgs_colour_sweep(int nc, int nx, int ny, const void* blk, const void* lu, const int8_t* piv,
                             const void* b, void* x, int forward, int fp32, cudaStream_t st) {
  const int nstrips = (ny + 31) / 32, per = nx + 31;
  for (int pass = 0; pass < 2; ++pass) {
    count_launches(1);
    const int colour = forward ? pass : 1 - pass;
    const long long nlines = (long long)nstrips * ((per - colour + 1) / 2);
    const int grid = (int)((nlines + 7) / 8);
#define CL(NC, T) k_sgs_colour<NC, T><<<grid, 256, 0, st>>>(nx, ny, (const T*)blk, (const T*)lu, piv, \
                                                             (const T*)b, (T*)x, colour, nlines)
    if (nc == 3) { if (fp32) CL(3, float); else CL(3, double); }
    else { if (fp32) CL(2, float); else CL(2, double); }
#undef CL
  }
}

void launch_coarse_exact(int nc, int nx, int ny, const void* blk, const void* b, void* x,
                         double* band, int* err, int fp32, cudaStream_t st) {
  count_launches(1);
#define CL(NC, T) k_coarse_exact<NC, T><<<1, 256, 0, st>>>(nx, ny, (const T*)blk, (const T*)b, (T*)x, band, err)
  if (nc == 3) { if (fp32) CL(3, float); else CL(3, double); }
  else { if (fp32) CL(2, float); else CL(2, double); }
#undef CL
}

void launch_coarse_inverse(int nc, int nx, int ny, const void* blk, void* aug, void* X, int* sing,
                           int fp32, cudaStream_t st) {
  count_launches(1);
#define CI(NC, T) k_coarse_inverse<NC, T><<<1, 1024, 0, st>>>(nx, ny, (const T*)blk, (T*)aug, (T*)X, sing)
  if (nc == 3) { if (fp32) CI(3, float); else CI(3, double); }
  else { if (fp32) CI(2, float); else CI(2, double); }
#undef CI
}

void launch_coarse_apply(int nc, int nx, int ny, const void* X, const void* b, void* x, int fp32,
                         cudaStream_t st) {
  count_launches(1);
  const int m = nx * ny * nc;
#define CA(NC, T) k_coarse_apply<NC, T><<<nblk(m, 128), 128, 0, st>>>(nx, ny, (const T*)X, (const T*)b, (T*)x)
  if (nc == 3) { if (fp32) CA(3, float); else CA(3, double); }
  else { if (fp32) CA(2, float); else CA(2, double); }
#undef CA
}

void launch_transpose_blocks(int nc, int nx, int ny, const void* src, int src_fp32, double* dst,
                             cudaStream_t st) {
  count_launches(1);
  const int g = nblk(nx * ny, 128);
#define TB(NC, T) k_transpose_blocks<NC, T><<<g, 128, 0, st>>>(nx, ny, (const T*)src, dst)
  if (nc == 3) { if (src_fp32) TB(3, float); else TB(3, double); }
  else { if (src_fp32) TB(2, float); else TB(2, double); }
#undef TB
}

void launch_lin_resid_abs(int dim, int nc, int nx, int ny, const void* blk, const void* b, const void* x,
                          int fp32, double* out, cudaStream_t st) {
  count_launches(1);
  const int g = nblk(nx * ny, 128);
#define LR(NC, T) k_lin_resid_abs<NC, T><<<g, 128, 0, st>>>(dim, nx, ny, (const T*)blk, (const T*)b, (const T*)x, out)
  if (nc == 3) { if (fp32) LR(3, float); else LR(3, double); }
  else { if (fp32) LR(2, float); else LR(2, double); }
#undef LR
}

void launch_abs_cells(int n, int nc, const double* v, double* out, cudaStream_t st) {
  count_launches(1);
  k_abs_cells<<<nblk(n, 256), 256, 0, st>>>(n, nc, v, out);
}

void launch_sum(const double* v, int n, double* partial, double* out, cudaStream_t st) {
  count_launches(2);
  int g = nblk(n, 256);
  if (g > 1024) g = 1024;
  if (g < 1) g = 1;
  k_sum_partial<<<g, 256, 0, st>>>(v, n, partial);
  k_sum_final<<<1, 256, 0, st>>>(partial, g, out);
}

void launch_convert(const void* src, int src_fp32, void* dst, int dst_fp32, long long n,
                    double scale, cudaStream_t st) {
  count_launches(1);
  const int g = (int)(n / 256 + 1 > 4096 ? 4096 : n / 256 + 1);
  if (src_fp32 && dst_fp32) k_convert<float, float><<<g, 256, 0, st>>>((const float*)src, (float*)dst, n, scale);
  else if (src_fp32) k_convert<float, double><<<g, 256, 0, st>>>((const float*)src, (double*)dst, n, scale);
  else if (dst_fp32) k_convert<double, float><<<g, 256, 0, st>>>((const double*)src, (float*)dst, n, scale);
  else k_convert<double, double><<<g, 256, 0, st>>>((const double*)src, (double*)dst, n, scale);
}

void launch_to_skew(const void* src, int src_fp32, void* dst, int dst_fp32, int nc, int nx, int ny, double scale,
                    cudaStream_t st) {
  count_launches(1);
  const int g = nblk((long long)nx * ny, 256);
  if (src_fp32 && dst_fp32) k_to_skew<float, float><<<g, 256, 0, st>>>((const float*)src, (float*)dst, nc, nx, ny, scale);
  else if (src_fp32) k_to_skew<float, double><<<g, 256, 0, st>>>((const float*)src, (double*)dst, nc, nx, ny, scale);
  else if (dst_fp32) k_to_skew<double, float><<<g, 256, 0, st>>>((const double*)src, (float*)dst, nc, nx, ny, scale);
  else k_to_skew<double, double><<<g, 256, 0, st>>>((const double*)src, (double*)dst, nc, nx, ny, scale);
}

void launch_from_skew(const void* src, int src_fp32, void* dst, int dst_fp32, int nc, int nx, int ny, double scale,
                      cudaStream_t st) {
  count_launches(1);
  const int g = nblk((long long)nx * ny, 256);
  if (src_fp32 && dst_fp32) k_from_skew<float, float><<<g, 256, 0, st>>>((const float*)src, (float*)dst, nc, nx, ny, scale);
  else if (src_fp32) k_from_skew<float, double><<<g, 256, 0, st>>>((const float*)src, (double*)dst, nc, nx, ny, scale);
  else if (dst_fp32) k_from_skew<double, float><<<g, 256, 0, st>>>((const double*)src, (float*)dst, nc, nx, ny, scale);
  else k_from_skew<double, double><<<g, 256, 0, st>>>((const double*)src, (double*)dst, nc, nx, ny, scale);
}

void launch_fill(void* dst, int fp32, long long n, cudaStream_t st) {
  count_launches(1);
  const int g = (int)(n / 256 + 1 > 4096 ? 4096 : n / 256 + 1);
  if (fp32) k_fill0<float><<<g, 256, 0, st>>>((float*)dst, n);
  else k_fill0<double><<<g, 256, 0, st>>>((double*)dst, n);
}

void launch_blocks_export(int nx, int ny, int nc, const void* blk, int fp32, double* out,
                          cudaStream_t st) {
  count_launches(1);
  const int n = nx * ny;
  if (fp32) k_export<float><<<nblk(n, 128), 128, 0, st>>>(nx, ny, nc, (const float*)blk, out);
  else k_export<double><<<nblk(n, 128), 128, 0, st>>>(nx, ny, nc, (const double*)blk, out);
}

// ---- batched launchers ----------------------------------------------------------

void launch_b_sum(const BItem* items, const int* mask, int B, int max_n, double* out, cudaStream_t st) {
  count_launches(2);
  int gmax = nblk(max_n, 256);
  gmax = gmax > 1024 ? 1024 : (gmax < 1 ? 1 : gmax);
  kb_sum_partial<<<dim3(gmax, B), 256, 0, st>>>(items, mask);
  kb_sum_final<<<B, 256, 0, st>>>(items, mask, out);
}

void launch_b_lu_factor(const BLaunch& slots, int fp32, cudaStream_t st) {
  count_launches(1);
  if (slots.nblocks <= 0) return;
  if (fp32) kb_lu_factor<3, float><<<slots.nblocks, 128, 0, st>>>(slots);
  else kb_lu_factor<3, double><<<slots.nblocks, 128, 0, st>>>(slots);
}

void launch_b_galerkin(const BLaunch& coarse, const BItem* fine_items, int fp32, cudaStream_t st) {
  count_launches(1);
  if (coarse.nblocks <= 0) return;
  if (fp32) kb_galerkin<3, float><<<coarse.nblocks, 128, 0, st>>>(coarse, fine_items);
  else kb_galerkin<3, double><<<coarse.nblocks, 128, 0, st>>>(coarse, fine_items);
}

void launch_b_restrict(const BLaunch& coarse, const BItem* fine_items, int fp32, cudaStream_t st) {
  count_launches(1);
  if (coarse.nblocks <= 0) return;
  if (fp32) kb_restrict<3, float><<<coarse.nblocks, 128, 0, st>>>(coarse, fine_items);
  else kb_restrict<3, double><<<coarse.nblocks, 128, 0, st>>>(coarse, fine_items);
}

void launch_b_prolong(const BLaunch& fine, const BItem* coarse_items, int fp32, cudaStream_t st) {
  count_launches(1);
  if (fine.nblocks <= 0) return;
  if (fp32) kb_prolong<float><<<fine.nblocks, 128, 0, st>>>(fine, coarse_items);
  else kb_prolong<double><<<fine.nblocks, 128, 0, st>>>(fine, coarse_items);
}

void launch_b_fill_x(const BLaunch& cells, int fp32, cudaStream_t st) {
  count_launches(1);
  if (cells.nblocks <= 0) return;
  if (fp32) kb_fill_x<float><<<cells.nblocks, 128, 0, st>>>(cells);
  else kb_fill_x<double><<<cells.nblocks, 128, 0, st>>>(cells);
}

void launch_b_neg_residual(const BLaunch& cells, int fp32, cudaStream_t st) {
  count_launches(1);
  if (cells.nblocks <= 0) return;
  if (fp32) kb_neg_residual<float><<<cells.nblocks, 128, 0, st>>>(cells);
  else kb_neg_residual<double><<<cells.nblocks, 128, 0, st>>>(cells);
}

template <typename T, bool F, int S>
static void b_sgs_launch(const BItem* items, const int2* tickets, int ntickets, const int* mask, int* sync,
                         int* sticky, cudaStream_t st) {
  const size_t smem = sgs_smem_bytes<3, T, S>();
  static int per_sm = 0;   // per template instance
  static int nsm = 0;
  if (per_sm == 0) {
    cudaFuncSetAttribute(kb_sgs_strip<3, T, F, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kb_sgs_strip<3, T, F, S>, 32, smem);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (per_sm < 1) per_sm = 1;
  }
  // warps resident at once (each loops over tickets), never more than tickets
  const int grid = ntickets < per_sm * nsm ? ntickets : per_sm * nsm;
  kb_sgs_strip<3, T, F, S><<<grid, 32, smem, st>>>(items, tickets, ntickets, mask, sync, sticky, wait_limit());
}

size_t b_sgs_smem_bytes(int fp32, int chunk) {
  if (fp32) return chunk == 4 ? sgs_smem_bytes<3, float, 4>() : chunk == 8 ? sgs_smem_bytes<3, float, 8>()
                                                                           : sgs_smem_bytes<3, float, 16>();
  return chunk == 2 ? sgs_smem_bytes<3, double, 2>() : chunk == 4 ? sgs_smem_bytes<3, double, 4>()
                                                                  : sgs_smem_bytes<3, double, 8>();
}

void launch_b_sgs_sweep(const BItem* items, const int2* tickets, int ntickets, int nslots, const int* mask,
                        int forward, int fp32, int chunk, int* sync, int* sticky_err, cudaStream_t st) {
  count_launches(1);
  if (ntickets <= 0) return;
  cudaMemsetAsync(sync, 0, sizeof(int) * (2 + nslots), st);
#define BS_(T, F, S) b_sgs_launch<T, F, S>(items, tickets, ntickets, mask, sync, sticky_err, st)
  if (fp32) {
    if (forward) { if (chunk == 4) BS_(float, true, 4); else if (chunk == 8) BS_(float, true, 8); else BS_(float, true, 16); }
    else { if (chunk == 4) BS_(float, false, 4); else if (chunk == 8) BS_(float, false, 8); else BS_(float, false, 16); }
  } else {
    if (forward) { if (chunk == 2) BS_(double, true, 2); else if (chunk == 4) BS_(double, true, 4); else BS_(double, true, 8); }
    else { if (chunk == 2) BS_(double, false, 2); else if (chunk == 4) BS_(double, false, 4); else BS_(double, false, 8); }
  }
#undef BS_
}

void launch_b_coarse_inverse(const BItem* items, const int* mask, int B, int fp32, cudaStream_t st) {
  count_launches(1);
  if (fp32) kb_coarse_inverse<3, float><<<B, 1024, 0, st>>>(items, mask);
  else kb_coarse_inverse<3, double><<<B, 1024, 0, st>>>(items, mask);
}

void launch_b_coarse_apply(const BItem* items, const int* mask, int B, int max_m, int fp32, cudaStream_t st) {
  count_launches(1);
  const dim3 g(nblk(max_m > 0 ? max_m : 1, 128), B);
  if (fp32) kb_coarse_apply<3, float><<<g, 128, 0, st>>>(items, mask);
  else kb_coarse_apply<3, double><<<g, 128, 0, st>>>(items, mask);
}

}  // namespace swnmg
