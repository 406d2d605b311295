// Internal definition of the solver context (include/swnmg.h declares it
// opaque), shared by the single-problem entry points (api.cu) and the
// batched driver (batch.cu).
#pragma once

#include <string>
#include <vector>

#include "common.cuh"
#include "../../include/swnmg.h"

namespace swnmg {

// one mesh level of a context: bed, Step 1 state, operator and MG vectors
struct Level {
  int nx = 0, ny = 0, n = 0;
  double ex = 0, ey = 0;
  double* z = nullptr;      // bed at cell centres
  double* U = nullptr;      // Step 1 state (levels >= 1)
  void* blk = nullptr;      // 5 blocks (raw diagonal first), working precision
  void* lu = nullptr;       // LU of the diagonal
  int8_t* piv = nullptr;
  void* b = nullptr;        // right-hand side of A x = b
  void* x = nullptr;        // iterate
  double* geo = nullptr;    // curvilinear mesh: per edge |e|, n^x, n^y (3 x n_e)
  double* area = nullptr;   // curvilinear mesh: |K_i|
};

// DevLevel of level l of ctx (api.cu)
DevLevel ctx_dev_level(const swnmg_ctx* c, int l);

}  // namespace swnmg

struct swnmg_ctx {
  swnmg_problem prob;
  swnmg_params prm;
  int nc = 0, nl = 0, fp32 = 0;
  size_t wsz = 8;           // bytes per working-precision value
  cudaStream_t st = nullptr;
  swnmg::Level lv[13];
  double* R = nullptr;      // residual scratch (level-0 size)
  double* rn = nullptr;     // ||R_i||_1
  double* eb = nullptr;     // per-edge Jacobian pieces (level-0 size)
  double* red = nullptr;    // reduction partials (1024) + result
  double* band = nullptr;   // exact coarse-solve scratch (banded elimination, large m)
  void* cinv = nullptr;     // guarded inverse of the coarsest operator (small m)
  void* caug = nullptr;     // its m x 2m elimination array
  int* csing = nullptr;
  int* derr = nullptr;
  double* ghost = nullptr;  // BLU-SGS boundary ghost states (4 * max(nx, ny) * (nc + 1) * 3)
  // implicit time step (Remark 2.6): on during swnmg_time_step only
  bool t_on = false;
  double t_ka = 0.0, t_omb = 1.0;
  double* t_src = nullptr;  // |K|/dt U^n - beta R(U^n), nc x n
  // structured curvilinear mesh (swnmg_set_mesh): finest vertices x then y,
  // (nx + 1)(ny + 1) each; per-cell |K_i|/dt of a time step
  bool curv = false;
  double* mesh = nullptr;
  double* kai = nullptr;
  int* sgs_sync = nullptr;  // ticket / abort / per-strip progress of the wavefront sweeps
  // tagged last-row words of the SGS strips (level-0 strips x nx x nc x 2) and
  // the epoch of the last SGS launch (every launch takes the next one)
  unsigned long long* sgs_edge = nullptr;
  unsigned sgs_epoch = 0;
  int* blu_sync = nullptr;  // ticket / abort / per-strip progress of the BLU-SGS strip sweep
  // tagged last-row words of the BLU-SGS strips (level-0 strips x nx x 6) and
  // the epoch of the last launch that used them
  unsigned long long* blu_edge = nullptr;
  unsigned blu_epoch = 0;
  int* sticky = nullptr;    // set by a device wait that ran out of its bound
  double* hbuf = nullptr;   // pinned host scalars
  bool coarse_exact = false;
  bool coarse_inverse = false;   // exact coarse solve through X = A^-1 (guarded)
  // transposed (adjoint) operator hierarchy, FP64, allocated on first use
  bool adj_ready = false;
  swnmg::Level alv[13];
  void* acinv = nullptr;
  void* acaug = nullptr;
  int* acsing = nullptr;
  double* aband = nullptr;
  double* adj_A = nullptr;   // FP64 Jacobian at U* before transposition
  double* adj_cz = nullptr;      // per-edge z contributions (2 per edge)
  double* adj_cell = nullptr;    // per-cell scratch (n)
  // per-class kernel timing: event pairs resolved at synchronisation points
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<int> ev_class;     // class of pair k (events 2k, 2k+1)
  std::vector<double> ev_cells;  // cells processed inside pair k
  int ev_used = 0;
  double t_ms[SWNMG_T_COUNT] = {0};
  long long t_n[SWNMG_T_COUNT] = {0};
  double t_cells[SWNMG_T_COUNT] = {0};
  std::string err;
};
