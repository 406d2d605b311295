// Internal declarations shared by the CUDA translation units of libswnmg.
//
// Device data layout (SoA, x-fastest cell index i = ix + nx*iy):
//   state U, residual R               : [c*n + i]  (row-major)
//   multigrid vectors b, x of a level : [c*P + spos(i)]  (strip-skewed, below)
//   operator blocks of a level       : blk[(b*nc*nc + s*nc + k)*P + spos(i)]
//        b = 0 diagonal (raw, with alpha||R_i||_1), 1 W, 2 E, 3 S, 4 N
//   LU factors of the diagonal       : lu[e*P + spos(i)], e = 0..8 (LU layout below)
//        + perm code piv[spos(i)] (int8)
//   per-edge Jacobian pieces          : x-edges (nx+1)*ny then y-edges nx*(ny+1)
//
// Strip-skewed operator layout.  Rows are grouped in strips of 32; cell
// (ix, iy) of strip t = iy/32, lane k = iy%32 sits on skewed diagonal
// d = ix + k and is stored at spos = (t*(nx+31) + d)*32 + k.  The block
// Gauss-Seidel wavefront updates one skewed diagonal of a strip per warp
// step (lane k at column d - k), so every step reads one contiguous line of
// 32 values per entry, in either sweep direction.  P = strips*(nx+31)*32
// slots per entry (padding slots are never read as data).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace swnmg {

// boundary kinds / fluxes (same numbering as the public header)
enum { BC_REFLECT = 0, BC_SLIP = 1, BC_INFLOW = 2, BC_OUTFLOW = 3, BC_SUPER_IN = 4, BC_SUPER_OUT = 5,
       BC_AUTO = 6 };
enum { FX_HLL = 0, FX_HLLC = 1, FX_LLF = 2, FX_ROE = 3 };

struct DevBC { int kind; double h, q, ut; };

// Everything a flux / Jacobian kernel needs about one mesh level.
struct DevLevel {
  int dim, nc;            // 1 or 2, components 2 or 3
  int nx, ny, n;          // cells of this level (ny = 1 in 1D)
  double ex, ey;          // |x-edge| (W/E sides), |y-edge| (S/N sides); 1D: 1, 0
  int flux, llf_wetdry;
  double g, half_g, h_eps, eps_r, alpha, eps, reps;   // reps = 1/eps
  double eps_f;           // Harten's entropy-fix width (Roe flux)
  // implicit time step (Remark 2.6), active when t_ka > 0 (level 0 only): the
  // residual becomes (1 - beta) R(U) + |K|/dt U - t_src, t_src = |K|/dt U^n -
  // beta R(U^n) (nc x n), t_ka = |K|/dt, t_omb = 1 - beta
  double t_ka, t_omb;
  const double* t_src;
  DevBC bc[4];            // W, E, S, N
  // structured curvilinear mesh (2D; NULL: the uniform mesh above).  geo per
  // edge e (x-edges first): |e| at geo[e], the unit normal (from the
  // lower-index cell to the higher-index one) at geo[n_e + e], geo[2 n_e + e];
  // area |K_i| per cell; t_kai |K_i|/dt per cell during a time step.
  const double* geo = nullptr;
  const double* area = nullptr;
  const double* t_kai = nullptr;
};

// LU layout of a block (n = 2 or 3), partial pivoting, guard for singular
// pivots.  Solve of D x = b:  y = P b;  y1 -= l10 y0;  y2 -= l20 y0 + l21 y1;
// x2 = y2 inv22; x1 = (y1 - u12 x2) inv11; x0 = (y0 - u01 x1 - u02 x2) inv00.
// Entries: 0 l10, 1 l20, 2 l21, 3 u01, 4 u02, 5 u12, 6 inv00, 7 inv11, 8 inv22
// (inv = 0 marks a singular unknown whose correction is zero).
// piv = p0 | p1 << 2 | p2 << 4 (2-bit fields, decoded with shifts) with
// P b = (b[p0], b[p1], b[p2]).
constexpr int LU_E = 9;

inline int blk_entries(int nc) { return 5 * nc * nc; }

__host__ __device__ __forceinline__ long long skew_pos(int ix, int iy, int nx) {
  return ((long long)(iy >> 5) * (nx + 31) + (ix + (iy & 31))) * 32 + (iy & 31);
}
__host__ __device__ __forceinline__ long long skew_slots(int nx, int ny) {
  return (long long)((ny + 31) >> 5) * (nx + 31) * 32;
}

// ---- batches of independent problems ------------------------------------
// One problem at one level of a batch: what the batched kernels read.  A
// batch keeps one table of these per level (problem p at entry p).
struct BItem {
  DevLevel L;                   // geometry, boundary data, parameters
  const double* z;              // level bed
  double* U;                    // level state (level 0: the caller's state)
  double* R;                    // residual and ||R_i||_1 (problem workspace)
  double* rn;
  double* eb;                   // per-edge scratch (problem workspace)
  double* red;                  // reduction partials (1024 doubles)
  void* blk;                    // level operator, LU factors, MG vectors
  void* lu;
  int8_t* piv;
  void* b;
  void* x;
  double* ghost;                // BLU-SGS ghost scratch (problem workspace)
  void* cinv;                   // coarsest level: guarded inverse and its scratch
  void* caug;
  int* csing;
  int n_xe, n_e;                // x-edges, all edges
  int strip0;                   // first SGS progress slot of this problem
  int bstrip0;                  // first BLU-SGS strip progress slot of this problem
  int has;                      // the problem has this level
};

constexpr int BATCH_MAX = 256;

// problem owning block blk: the largest p with bstart[p] <= blk
__device__ __forceinline__ int batch_find(const int* bstart, int B, int blk) {
  int lo = 0, hi = B - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (bstart[mid] <= blk) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// One batched launch over a per-problem index domain: blocks of 128 threads,
// problem p owns blocks [bstart[p], bstart[p+1]); mask[p] == 0 skips it.
struct BLaunch {
  const BItem* items;
  const int* bstart;
  int nblocks;
  int B;
  const int* mask;
};

// sets the text that swnmg_last_error(NULL) returns
void set_static_error(const char* msg);

// process-wide count of kernel launches issued by the library
void count_launches(long long k);
// Polls a device-side wait makes before it gives up and sets the sticky
// error (swnmg_set_wait_limit); read when a launch is enqueued (or captured).
constexpr int kDefaultWaitLimit = 1 << 22;
int wait_limit();
void set_wait_limit(int polls);
// Bound of the wait for a warp's own in-flight bulk copies before it exits
// after a failure: independent of wait_limit(), since an issued copy lands.
constexpr int kDrainLimit = 1 << 24;
long long launches_total();

// ---- host-side launch wrappers (flux.cu) ---------------------------------
void launch_residual(const DevLevel& L, const double* z, const double* U, double* R, double* rn,
                     double* edge_buf, cudaStream_t st);
void launch_jacobian(const DevLevel& L, const double* z, const double* U, double* R, double* rn,
                     double* edge_buf, void* blk, int fp32, cudaStream_t st);   // blk skewed
// gbuf: 4 * max(nx, ny) * (nc + 1) * 3 doubles of ghost scratch
// FP32 BLU-SGS half-sweep (blusgs32.cu): Step 1 under SWNMG_PREC_MIXED_STEP1
void launch_blusgs32_strip(const DevLevel& L, const double* z, double* U, float* gbuf, int forward, int* sync,
                           int* sticky_err, cudaStream_t st);
// edge: tagged last-row words of the 2-row strips, (ny/2 rounded up) * nx * 6
// entries at least, for the two-warp LLF kernel (NULL: the one-warp kernels);
// epoch: differs from every earlier launch's on the same edge buffer
void launch_blusgs_strip(const DevLevel& L, const double* z, double* U, double* gbuf, int forward, int* sync,
                         unsigned long long* edge, unsigned epoch, int* sticky_err, cudaStream_t st);
void launch_blusgs_sweep(const DevLevel& L, const double* z, double* U, double* gbuf, int forward, int* sync,
                         int* sticky_err, cudaStream_t st);
// dU strip-skewed (a level-0 multigrid iterate)
void launch_newton_update(int nx, int ny, int nc, double tau, double h_eps, double* U, const void* dU,
                          int dU_fp32, cudaStream_t st);
void launch_adjoint_z(const DevLevel& L, const double* z, const double* U, const double* lam, double delta,
                      double* cz, double* dRz, cudaStream_t st);
void launch_adjoint_q(const DevLevel& L, int side, const double* z, const double* U, const double* lam,
                      double delta, double* out, cudaStream_t st);
// curvilinear meshes (Examples 3.4, 3.5)
void launch_average_area(int nxf, int nyf, int ncomp, const double* area_f, const double* vf, double* vc,
                         cudaStream_t st);
void launch_time_source_cells(long long m, long long n, const double* kai, double beta, const double* U,
                              const double* R, double* src, cudaStream_t st);
void launch_mesh_level(int nx, int ny, int vrow, int step, const double* vx, const double* vy, double* geo,
                       double* area, int* bad, cudaStream_t st);
void launch_time_ka(int n, const double* area, double dt, double* kai, cudaStream_t st);
void launch_average(int dim, int nxf, int nyf, int ncomp, const double* vf, double* vc,
                    cudaStream_t st);
// t_src = ka U^n - beta R(U^n) over m values (the time step's fixed part)
void launch_time_source(long long m, double ka, double beta, const double* U, const double* R, double* src,
                        cudaStream_t st);
void launch_inject(int dim, int nxf, int nyf, int ncomp, const double* vc, double* vf,
                   cudaStream_t st);

// batched forms (2D, three components); bl.items is the level's table
void launch_b_residual(const BLaunch& edges, const BLaunch& cells, cudaStream_t st);
void launch_b_jacobian(const BLaunch& edges, const BLaunch& cells, int fp32, cudaStream_t st);
void launch_b_newton_update(const BLaunch& cells, double tau, double h_eps, int fp32, cudaStream_t st);
// coarse cells of level l+1 (bl over the coarse domain, fine table separately)
void launch_b_average(const BLaunch& coarse, const BItem* fine_items, cudaStream_t st);
// fine cells of level l-1 (bl over the fine domain, coarse table separately)
void launch_b_inject(const BLaunch& fine, const BItem* coarse_items, cudaStream_t st);
// one half-sweep over every masked problem's level; nsteps = max diagonals,
// blocks = cooperative grid size, sync: [0] arrivals, [1] abort (zeroed here)
// batched strip-pipelined BLU-SGS half-sweep: (problem, strip) tickets in
// claim order (strip index first), grid warps at most
void launch_b_blusgs_strip(const BItem* items, const int2* tickets, int ntickets, int nslots, const int* mask,
                           int B, int forward, int grid, int* sync, int* sticky_err, cudaStream_t st);
void launch_b_blusgs_sweep(const BItem* items, const int* mask, int B, int nsteps, int forward, int blocks,
                           int* sync, int* sticky_err, cudaStream_t st);
int b_blusgs_max_blocks_per_sm();

// ---- host-side launch wrappers (mg.cu) -----------------------------------
void launch_lu_factor(int nx, int ny, int nc, const void* blk, void* lu, int8_t* piv, int fp32,
                      cudaStream_t st);
void launch_galerkin(int dim, int nc, int nxf, int nyf, const void* bf, void* bc, int fp32,
                     cudaStream_t st);
void launch_restrict(int dim, int nc, int nxf, int nyf, const void* blk, const void* b,
                     const void* x, void* bcoarse, int fp32, cudaStream_t st);
void launch_prolong(int dim, int nc, int nxf, int nyf, const void* xc, void* xf, int fp32,
                    cudaStream_t st);
// edge: tagged last-row words of the strips, (ny/32 rounded up) * nx * nc * 2
// entries at least, for the warp-specialised kernel (NULL: the one-warp strip
// kernel); epoch: differs from every earlier launch's on the same edge buffer
void launch_sgs_sweep(int nc, int nx, int ny, const void* blk, const void* lu, const int8_t* piv,
                      const void* b, void* x, int forward, int fp32, int* sync, unsigned long long* edge,
                      unsigned epoch, int* sticky_err, cudaStream_t st);
void launch_sgs_colour_sweep(int nc, int nx, int ny, const void* blk, const void* lu, const int8_t* piv,
                             const void* b, void* x, int forward, int fp32, cudaStream_t st);
void launch_coarse_exact(int nc, int nx, int ny, const void* blk, const void* b, void* x,
                         double* band, int* err, int fp32, cudaStream_t st);
void launch_coarse_inverse(int nc, int nx, int ny, const void* blk, void* aug, void* X, int* sing,
                           int fp32, cudaStream_t st);
void launch_coarse_apply(int nc, int nx, int ny, const void* X, const void* b, void* x, int fp32,
                         cudaStream_t st);
void launch_sum(const double* v, int n, double* partial, double* out, cudaStream_t st);
void launch_transpose_blocks(int nc, int nx, int ny, const void* src, int src_fp32, double* dst,
                             cudaStream_t st);
void launch_lin_resid_abs(int dim, int nc, int nx, int ny, const void* blk, const void* b, const void* x,
                          int fp32, double* out, cudaStream_t st);
void launch_abs_cells(int n, int nc, const double* v, double* out, cudaStream_t st);
void launch_convert(const void* src, int src_fp32, void* dst, int dst_fp32, long long n,
                    double scale, cudaStream_t st);
void launch_fill(void* dst, int fp32, long long n, cudaStream_t st);
// natural SoA (nc x nx*ny) <-> strip-skewed (nc x skew_slots) vectors, times scale
void launch_to_skew(const void* src, int src_fp32, void* dst, int dst_fp32, int nc, int nx, int ny, double scale,
                    cudaStream_t st);
void launch_from_skew(const void* src, int src_fp32, void* dst, int dst_fp32, int nc, int nx, int ny, double scale,
                      cudaStream_t st);
void launch_blocks_export(int nx, int ny, int nc, const void* blk, int fp32, double* out,
                          cudaStream_t st);

// batched forms (2D, three components)
// sum_i ||R_i||_1 of every masked problem into out[p] (max_n: the table's largest level)
void launch_b_sum(const BItem* items, const int* mask, int B, int max_n, double* out, cudaStream_t st);
void launch_b_lu_factor(const BLaunch& slots, int fp32, cudaStream_t st);
void launch_b_galerkin(const BLaunch& coarse, const BItem* fine_items, int fp32, cudaStream_t st);
void launch_b_restrict(const BLaunch& coarse, const BItem* fine_items, int fp32, cudaStream_t st);
void launch_b_prolong(const BLaunch& fine, const BItem* coarse_items, int fp32, cudaStream_t st);
void launch_b_fill_x(const BLaunch& cells, int fp32, cudaStream_t st);
void launch_b_neg_residual(const BLaunch& cells, int fp32, cudaStream_t st);   // b = -R
// strip tickets (problem, processing index) in claim order; chunk = staged
// lines per buffer (4, 8 or 16); sync: [0] ticket, [1] abort, [2..] progress
void launch_b_sgs_sweep(const BItem* items, const int2* tickets, int ntickets, int nslots, const int* mask,
                        int forward, int fp32, int chunk, int* sync, int* sticky_err, cudaStream_t st);
size_t b_sgs_smem_bytes(int fp32, int chunk);
void launch_b_coarse_inverse(const BItem* items, const int* mask, int B, int fp32, cudaStream_t st);
void launch_b_coarse_apply(const BItem* items, const int* mask, int B, int max_m, int fp32, cudaStream_t st);

}  // namespace swnmg
