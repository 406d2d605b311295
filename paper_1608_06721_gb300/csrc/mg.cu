// mg.cu -- geometric multigrid pieces of Section 2.3 (eq. MatrixForm,
// ProjectAR, Project, correction; Algorithm 0's smoother and coarse solve),
// templated on the working precision (double, or float in the mixed mode).
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
__global__ void k_lu_factor(int n, const T* __restrict__ blk, T* __restrict__ lu,
                            int8_t* __restrict__ piv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  T m[NC][NC];
  T amax = T(0);
  for (int s = 0; s < NC; ++s)
    for (int k = 0; k < NC; ++k) {
      m[s][k] = blk[(long long)(s * NC + k) * n + i];
      amax = tabs(m[s][k]) > amax ? tabs(m[s][k]) : amax;
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
      for (int k = 0; k < NC; ++k) { T t = m[c][k]; m[c][k] = m[p][k]; m[p][k] = t; }
      int t = perm[c]; perm[c] = perm[p]; perm[p] = t;
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
      for (int k = c + 1; k < NC; ++k) m[r][k] = m[r][k] - l * m[c][k];
    }
  }
  const long long N = n;
  if (NC == 3) {
    lu[0 * N + i] = m[1][0]; lu[1 * N + i] = m[2][0]; lu[2 * N + i] = m[2][1];
    lu[3 * N + i] = m[0][1]; lu[4 * N + i] = m[0][2]; lu[5 * N + i] = m[1][2];
    lu[6 * N + i] = inv[0]; lu[7 * N + i] = inv[1]; lu[8 * N + i] = inv[2];
    piv[i] = (int8_t)(perm[0] + 3 * perm[1] + 9 * perm[2]);
  } else {
    lu[0 * N + i] = m[1][0]; lu[1 * N + i] = T(0); lu[2 * N + i] = T(0);
    lu[3 * N + i] = m[0][1]; lu[4 * N + i] = T(0); lu[5 * N + i] = T(0);
    lu[6 * N + i] = inv[0]; lu[7 * N + i] = inv[1]; lu[8 * N + i] = T(0);
    piv[i] = (int8_t)(perm[0] + 3 * perm[1]);
  }
}

template <int NC, typename T>
__device__ __forceinline__ void lu_apply(const T* __restrict__ lu, int8_t pv, long long N, int i,
                                         const T r[NC], T x[NC]) {
  const int p0 = pv % 3, p1 = (pv / 3) % 3, p2 = pv / 9;
  if (NC == 3) {
    T y0 = r[p0], y1 = r[p1], y2 = r[p2 % NC];
    y1 = y1 - lu[0 * N + i] * y0;
    y2 = y2 - lu[1 * N + i] * y0 - lu[2 * N + i] * y1;
    const T x2 = y2 * lu[8 * N + i];
    const T x1 = (y1 - lu[5 * N + i] * x2) * lu[7 * N + i];
    const T x0 = (y0 - lu[3 * N + i] * x1 - lu[4 * N + i] * x2) * lu[6 * N + i];
    x[0] = x0; x[1 % NC] = x1; x[2 % NC] = x2;
  } else {
    T y0 = r[p0], y1 = r[p1 % NC];
    y1 = y1 - lu[0 * N + i] * y0;
    const T x1 = y1 * lu[7 * N + i];
    const T x0 = (y0 - lu[3 * N + i] * x1) * lu[6 * N + i];
    x[0] = x0; x[1 % NC] = x1;
  }
}

// ---- Galerkin coarse operator: A_{IJ,l+1} = sum_{i in I} sum_{j in J} A_ij ---
// children 00, 10, 01, 11; diagonal = children's diagonals plus the 8
// couplings between children; W/E/S/N = the two couplings crossing that side.
template <int NC, typename T>
__global__ void k_galerkin(int dim, int nxf, int nyf, const T* __restrict__ bf, T* __restrict__ bc) {
  const int nxc = nxf / 2, nyc = dim == 2 ? nyf / 2 : 1, ncc = nxc * nyc;
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= ncc) return;
  const long long nf = (long long)nxf * (dim == 2 ? nyf : 1), nc_ = ncc;
  const int BS = NC * NC;
  const int Ix = I % nxc, Iy = I / nxc;
#define FB(cell, b, e) bf[((long long)(b) * BS + (e)) * nf + (cell)]
#define CB(b, e) bc[((long long)(b) * BS + (e)) * nc_ + I]
  if (dim == 1) {
    const int c0 = 2 * Ix, c1 = c0 + 1;
    for (int e = 0; e < BS; ++e) {
      CB(0, e) = ((FB(c0, 0, e) + FB(c1, 0, e)) + FB(c0, 2, e)) + FB(c1, 1, e);
      CB(1, e) = FB(c0, 1, e);
      CB(2, e) = FB(c1, 2, e);
      CB(3, e) = T(0);
      CB(4, e) = T(0);
    }
    return;
  }
  const int c00 = 2 * Ix + nxf * 2 * Iy, c10 = c00 + 1, c01 = c00 + nxf, c11 = c01 + 1;
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

// linear residual of the fine system at cell i: r = b - D x_i - sum A x_j
template <int NC, typename T>
__device__ __forceinline__ void lin_resid(int dim, int nx, int ny, const T* __restrict__ blk,
                                          const T* __restrict__ b, const T* __restrict__ x, int i,
                                          T r[NC]) {
  const long long n = (long long)nx * ny;
  const int BS = NC * NC;
  const int ix = i % nx, iy = i / nx;
  int nb[4] = {ix > 0 ? i - 1 : -1, ix < nx - 1 ? i + 1 : -1, iy > 0 ? i - nx : -1,
               iy < ny - 1 ? i + nx : -1};
  T xi[NC];
  for (int k = 0; k < NC; ++k) xi[k] = x[k * n + i];
  for (int s = 0; s < NC; ++s) {
    T a = b[s * n + i];
    for (int k = 0; k < NC; ++k) a = a - blk[(long long)(s * NC + k) * n + i] * xi[k];
    r[s] = a;
  }
  const int nsd = dim == 2 ? 4 : 2;
  for (int side = 0; side < nsd; ++side) {
    const int j = nb[side];
    if (j < 0) continue;
    T xj[NC];
    for (int k = 0; k < NC; ++k) xj[k] = x[k * n + j];
    for (int s = 0; s < NC; ++s)
      for (int k = 0; k < NC; ++k)
        r[s] = r[s] - blk[((long long)(1 + side) * BS + s * NC + k) * n + i] * xj[k];
  }
}

// coarse right-hand side = sum over children of (b - A x)  (eq. ProjectAR)
template <int NC, typename T>
__global__ void k_restrict(int dim, int nxf, int nyf, const T* __restrict__ blk,
                           const T* __restrict__ b, const T* __restrict__ x, T* __restrict__ bc) {
  const int nxc = nxf / 2, nyc = dim == 2 ? nyf / 2 : 1, ncc = nxc * nyc;
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= ncc) return;
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
  for (int s = 0; s < NC; ++s) bc[(long long)s * ncc + I] = acc[s];
}

// x_j += x_I for every child j of I  (eq. correction, piecewise constant)
template <typename T>
__global__ void k_prolong(int dim, int nc, int nxf, int nyf, const T* __restrict__ xc,
                          T* __restrict__ xf) {
  const int nf = nxf * (dim == 2 ? nyf : 1);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nf) return;
  const int ix = i % nxf, iy = i / nxf, nxc = nxf / 2;
  const int ncc = nxc * (dim == 2 ? nyf / 2 : 1);
  const int I = (ix / 2) + nxc * (dim == 2 ? iy / 2 : 0);
  for (int s = 0; s < nc; ++s) xf[(long long)s * nf + i] = xf[(long long)s * nf + i] + xc[(long long)s * ncc + I];
}

// ---- block Gauss-Seidel, one anti-diagonal of the lexicographic order --------
// x_i <- D_i^{-1} (b_i - A_W x_W - A_E x_E - A_S x_S - A_N x_N)
template <int NC, typename T>
__global__ void k_sgs_diag(int nx, int ny, const T* __restrict__ blk, const T* __restrict__ lu,
                           const int8_t* __restrict__ piv, const T* __restrict__ b, T* __restrict__ x,
                           int d, int ix0, int ncell) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const int ix = ix0 + c, iy = d - ix, i = ix + nx * iy;
  const long long n = (long long)nx * ny;
  const int BS = NC * NC;
  int nb[4] = {ix > 0 ? i - 1 : -1, ix < nx - 1 ? i + 1 : -1, iy > 0 ? i - nx : -1,
               iy < ny - 1 ? i + nx : -1};
  T r[NC];
  for (int s = 0; s < NC; ++s) r[s] = b[s * n + i];
  for (int side = 0; side < 4; ++side) {
    const int j = nb[side];
    if (j < 0) continue;
    T xj[NC];
    for (int k = 0; k < NC; ++k) xj[k] = x[k * n + j];
    for (int s = 0; s < NC; ++s)
      for (int k = 0; k < NC; ++k)
        r[s] = r[s] - blk[((long long)(1 + side) * BS + s * NC + k) * n + i] * xj[k];
  }
  T xi[NC];
  lu_apply<NC, T>(lu, piv[i], n, i, r, xi);
  for (int s = 0; s < NC; ++s) x[s * n + i] = xi[s];
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
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int ix = i % nx, iy = i / nx;
    int nb[4] = {ix > 0 ? i - 1 : -1, ix < nx - 1 ? i + 1 : -1, iy > 0 ? i - nx : -1,
                 iy < ny - 1 ? i + nx : -1};
    for (int s = 0; s < NC; ++s) {
      rhs[i * NC + s] = (double)b[(long long)s * n + i];
      sing[i * NC + s] = 0;
      for (int k = 0; k < NC; ++k) AB(i * NC + s, i * NC + k) = (double)blk[(long long)(s * NC + k) * n + i];
      for (int side = 0; side < 4; ++side) {
        const int j = nb[side];
        if (j < 0) continue;
        for (int k = 0; k < NC; ++k)
          AB(i * NC + s, j * NC + k) = (double)blk[((long long)(1 + side) * BS + s * NC + k) * n + i];
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
    for (int r = 0; r < m; ++r) x[(long long)(r % NC) * n + r / NC] = (T)rhs[r];
    if (err) *err = 0;
  }
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

template <typename T>
__global__ void k_fill0(T* __restrict__ d, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    d[i] = T(0);
}

template <typename T>
__global__ void k_export(int n, int nc, const T* __restrict__ blk, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int BS = nc * nc;
  for (int b = 0; b < 5; ++b)
    for (int e = 0; e < BS; ++e)
      out[((long long)i * 5 + b) * BS + e] = (double)blk[((long long)b * BS + e) * n + i];
}

}  // namespace

// ---- launch wrappers ----------------------------------------------------------

void launch_lu_factor(int n, int nc, const void* blk, void* lu, int8_t* piv, int fp32,
                      cudaStream_t st) {
  const int g = nblk(n, 128);
  if (nc == 3) {
    if (fp32) k_lu_factor<3, float><<<g, 128, 0, st>>>(n, (const float*)blk, (float*)lu, piv);
    else k_lu_factor<3, double><<<g, 128, 0, st>>>(n, (const double*)blk, (double*)lu, piv);
  } else {
    if (fp32) k_lu_factor<2, float><<<g, 128, 0, st>>>(n, (const float*)blk, (float*)lu, piv);
    else k_lu_factor<2, double><<<g, 128, 0, st>>>(n, (const double*)blk, (double*)lu, piv);
  }
}

void launch_galerkin(int dim, int nc, int nxf, int nyf, const void* bf, void* bc, int fp32,
                     cudaStream_t st) {
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
  const int ncc = (nxf / 2) * (dim == 2 ? nyf / 2 : 1);
  const int g = nblk(ncc, 128);
#define RL(NC, T) k_restrict<NC, T><<<g, 128, 0, st>>>(dim, nxf, nyf, (const T*)blk, (const T*)b, \
                                                        (const T*)x, (T*)bcoarse)
  if (nc == 3) { if (fp32) RL(3, float); else RL(3, double); }
  else { if (fp32) RL(2, float); else RL(2, double); }
#undef RL
}

void launch_prolong(int dim, int nc, int nxf, int nyf, const void* xc, void* xf, int fp32,
                    cudaStream_t st) {
  const int nf = nxf * (dim == 2 ? nyf : 1);
  if (fp32) k_prolong<float><<<nblk(nf, 256), 256, 0, st>>>(dim, nc, nxf, nyf, (const float*)xc, (float*)xf);
  else k_prolong<double><<<nblk(nf, 256), 256, 0, st>>>(dim, nc, nxf, nyf, (const double*)xc, (double*)xf);
}

void launch_sgs_sweep(int nc, int nx, int ny, const void* blk, const void* lu, const int8_t* piv,
                      const void* b, void* x, int forward, int fp32, cudaStream_t st) {
  const int ndiag = nx + ny - 1;
  for (int q = 0; q < ndiag; ++q) {
    const int d = forward ? q : ndiag - 1 - q;
    const int ix0 = d - (ny - 1) > 0 ? d - (ny - 1) : 0;
    const int ix1 = d < nx - 1 ? d : nx - 1;
    const int ncell = ix1 - ix0 + 1;
    const int bs = ncell < 128 ? ((ncell + 31) / 32) * 32 : 128;
    const int g = nblk(ncell, bs);
#define SL(NC, T) k_sgs_diag<NC, T><<<g, bs, 0, st>>>(nx, ny, (const T*)blk, (const T*)lu, piv, \
                                                       (const T*)b, (T*)x, d, ix0, ncell)
    if (nc == 3) { if (fp32) SL(3, float); else SL(3, double); }
    else { if (fp32) SL(2, float); else SL(2, double); }
#undef SL
  }
}

void launch_coarse_exact(int nc, int nx, int ny, const void* blk, const void* b, void* x,
                         double* band, int* err, int fp32, cudaStream_t st) {
#define CL(NC, T) k_coarse_exact<NC, T><<<1, 256, 0, st>>>(nx, ny, (const T*)blk, (const T*)b, (T*)x, band, err)
  if (nc == 3) { if (fp32) CL(3, float); else CL(3, double); }
  else { if (fp32) CL(2, float); else CL(2, double); }
#undef CL
}

void launch_sum(const double* v, int n, double* partial, double* out, cudaStream_t st) {
  int g = nblk(n, 256);
  if (g > 1024) g = 1024;
  if (g < 1) g = 1;
  k_sum_partial<<<g, 256, 0, st>>>(v, n, partial);
  k_sum_final<<<1, 256, 0, st>>>(partial, g, out);
}

void launch_convert(const void* src, int src_fp32, void* dst, int dst_fp32, long long n,
                    double scale, cudaStream_t st) {
  const int g = (int)(n / 256 + 1 > 4096 ? 4096 : n / 256 + 1);
  if (src_fp32 && dst_fp32) k_convert<float, float><<<g, 256, 0, st>>>((const float*)src, (float*)dst, n, scale);
  else if (src_fp32) k_convert<float, double><<<g, 256, 0, st>>>((const float*)src, (double*)dst, n, scale);
  else if (dst_fp32) k_convert<double, float><<<g, 256, 0, st>>>((const double*)src, (float*)dst, n, scale);
  else k_convert<double, double><<<g, 256, 0, st>>>((const double*)src, (double*)dst, n, scale);
}

void launch_fill(void* dst, int fp32, long long n, cudaStream_t st) {
  const int g = (int)(n / 256 + 1 > 4096 ? 4096 : n / 256 + 1);
  if (fp32) k_fill0<float><<<g, 256, 0, st>>>((float*)dst, n);
  else k_fill0<double><<<g, 256, 0, st>>>((double*)dst, n);
}

void launch_blocks_export(int n, int nc, const void* blk, int fp32, double* out, cudaStream_t st) {
  if (fp32) k_export<float><<<nblk(n, 128), 128, 0, st>>>(n, nc, (const float*)blk, out);
  else k_export<double><<<nblk(n, 128), 128, 0, st>>>(n, nc, (const double*)blk, out);
}

}  // namespace swnmg
