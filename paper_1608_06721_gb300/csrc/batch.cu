// batch.cu -- Algorithm 1 for many independent 2D problems in lockstep.
//
// Every problem keeps the workspace of its own context (swnmg_create); the
// batch adds per-level tables of those buffers (BItem), block tables that
// deal each launch's blocks to the problems, SGS strip tickets, and
// per-problem masks.  The host runs the steps of Algorithm 1 once for the
// whole batch and decides each problem's stop tests exactly as swnmg_solve
// does for one problem; a problem that stops is masked out of every later
// launch.  Problems with different numbers of levels share the recursion of
// Algorithm 0: at level l, the problems whose coarsest level is l solve it
// while those with more levels smooth and descend.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.cuh"

using namespace swnmg;

namespace {

constexpr int MAXL = 13;
enum { D_CELLS = 0, D_EDGES = 1, D_SLOTS = 2, ND = 3 };
// mask slots (B flags each)
enum {
  M_ACT = 0,                 // Newton iteration still running
  M_CASC = 1,                // Step 1 sweeps still running on the current level
  M_SM = 2,                  // + l: running and level l is not the coarsest (smooth, descend)
  M_CO = M_SM + MAXL,        // + l: running and level l is the coarsest
  M_HI = M_CO + MAXL,        // + l: running and the problem has level l
  M_DOWN = M_HI + MAXL,      // + l: the problem has level l + 1
  M_HAS = M_DOWN + MAXL,     // + l: the problem has level l
  M_COUNT = M_HAS + MAXL
};

char g_berr[512] = "";

}  // namespace

struct swnmg_batch {
  int B = 0, maxNL = 0, minNL = 0, fp32 = 0, nsm = 0;
  swnmg_params prm;
  cudaStream_t user_st = nullptr, st = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::vector<swnmg_ctx*> ctx;
  std::vector<int> nl;
  bool coarse_inverse = true;
  // tables
  BItem* items = nullptr;            // [MAXL][B]
  std::vector<BItem> h_items;
  int* bstart = nullptr;             // [MAXL][ND][B + 1]
  std::vector<int> h_bstart;
  int2* tickets = nullptr;           // per level, concatenated
  std::vector<int> tick_off, tick_cnt, nslots, max_m, max_n, max_steps;
  int2* btickets = nullptr;          // BLU-SGS (problem, 2-row strip) tickets, per level, concatenated
  std::vector<int> btick_off, btick_cnt, nbslots;
  int* blu_sync = nullptr;           // ticket / abort / progress of the BLU-SGS strips
  int* mask = nullptr;               // [M_COUNT][B]
  int* h_mask = nullptr;             // pinned
  double* sums = nullptr;
  double* h_sums = nullptr;          // pinned
  int* sgs_sync = nullptr;
  int* bl_sync = nullptr;
  int* sticky = nullptr;
  int* h_sticky = nullptr;           // pinned
  // tuning
  int sgs_chunk[MAXL];
  int blusgs_blocks[MAXL];
  int blusgs_max = 0;
  // CUDA graph of the N_mg cycles
  bool use_graph = false;
  cudaGraphExec_t cyc_exec = nullptr;
  long long cyc_launches = 0;
  std::string err;
};

namespace {

swnmg_status bfail(swnmg_batch* b, swnmg_status s, const std::string& msg) {
  if (b) b->err = msg;
  snprintf(g_berr, sizeof g_berr, "%s", msg.c_str());
  return s;
}

#define BCUDA(bt, expr)                                                                   \
  do {                                                                                    \
    cudaError_t e_ = (expr);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return bfail(bt, e_ == cudaErrorMemoryAllocation ? SWNMG_ERR_OOM : SWNMG_ERR_CUDA,   \
                   std::string(#expr) + " -> " + cudaGetErrorString(e_));                 \
  } while (0)

#define BCHECK(bt) BCUDA(bt, cudaGetLastError())

inline int nblk128(long long n) { return (int)((n + 127) / 128); }

BLaunch bl(const swnmg_batch* b, int l, int dom, int slot) {
  const int* bs = b->bstart + ((size_t)l * ND + dom) * (b->B + 1);
  const int nb = b->h_bstart[((size_t)l * ND + dom) * (b->B + 1) + b->B];
  return BLaunch{b->items + (size_t)l * b->B, bs, nb, b->B, b->mask + (size_t)slot * b->B};
}

const BItem* tab(const swnmg_batch* b, int l) { return b->items + (size_t)l * b->B; }
const int* mk(const swnmg_batch* b, int slot) { return b->mask + (size_t)slot * b->B; }
int* hm(swnmg_batch* b, int slot) { return b->h_mask + (size_t)slot * b->B; }

bool any_mask(swnmg_batch* b, int slot) {
  const int* m = hm(b, slot);
  for (int p = 0; p < b->B; ++p)
    if (m[p]) return true;
  return false;
}

// largest diagonal count among the masked problems on level l
int steps_of(swnmg_batch* b, int l, int slot) {
  int s = 0;
  const int* m = hm(b, slot);
  for (int p = 0; p < b->B; ++p)
    if (m[p]) {
      const BItem& it = b->h_items[(size_t)l * b->B + p];
      s = std::max(s, it.L.nx + it.L.ny - 1);
    }
  return s;
}

void set_role_masks(swnmg_batch* b, const std::vector<int>& act) {
  for (int p = 0; p < b->B; ++p) {
    hm(b, M_ACT)[p] = act[p];
    for (int l = 0; l < MAXL; ++l) {
      hm(b, M_SM + l)[p] = act[p] && l < b->nl[p];
      hm(b, M_CO + l)[p] = act[p] && l == b->nl[p];
      hm(b, M_HI + l)[p] = act[p] && l <= b->nl[p];
    }
  }
}

swnmg_status upload_masks(swnmg_batch* b) {
  BCUDA(b, cudaMemcpyAsync(b->mask, b->h_mask, sizeof(int) * (size_t)M_COUNT * b->B, cudaMemcpyHostToDevice,
                           b->st));
  return SWNMG_OK;
}

swnmg_status upload_mask_slot(swnmg_batch* b, int slot) {
  BCUDA(b, cudaMemcpyAsync(b->mask + (size_t)slot * b->B, hm(b, slot), sizeof(int) * b->B,
                           cudaMemcpyHostToDevice, b->st));
  return SWNMG_OK;
}

swnmg_status check_sticky(swnmg_batch* b) {
  BCUDA(b, cudaMemcpyAsync(b->h_sticky, b->sticky, sizeof(int), cudaMemcpyDeviceToHost, b->st));
  BCUDA(b, cudaStreamSynchronize(b->st));
  if (*b->h_sticky) {
    cudaMemsetAsync(b->sticky, 0, sizeof(int), b->st);
    return bfail(b, SWNMG_ERR_TIMEOUT, "a wavefront sweep waited past its bound");
  }
  return SWNMG_OK;
}

// sum_i ||R_i||_1 on level l of every problem in mask slot, into out[p]
swnmg_status residual_sums(swnmg_batch* b, int l, int slot, std::vector<double>& out) {
  launch_b_residual(bl(b, l, D_EDGES, slot), bl(b, l, D_CELLS, slot), b->st);
  launch_b_sum(tab(b, l), mk(b, slot), b->B, b->max_n[l], b->sums, b->st);
  BCHECK(b);
  BCUDA(b, cudaMemcpyAsync(b->h_sums, b->sums, sizeof(double) * b->B, cudaMemcpyDeviceToHost, b->st));
  BCUDA(b, cudaStreamSynchronize(b->st));
  const int* m = hm(b, slot);
  for (int p = 0; p < b->B; ++p)
    if (m[p]) out[p] = b->h_sums[p];
  return SWNMG_OK;
}

// a half-sweep of every problem in mask slot: the strip-pipelined kernel,
// its grid capped at four warps per tuned BLU-SGS block
void blusgs(swnmg_batch* b, int l, int slot, int forward) {
  const int ns = steps_of(b, l, slot);
  if (ns == 0) return;
  launch_b_blusgs_strip(tab(b, l), b->btickets + b->btick_off[l], b->btick_cnt[l], b->nbslots[l], mk(b, slot),
                        b->B, forward, 4 * b->blusgs_blocks[l], b->blu_sync, b->sticky, b->st);
}

void sgs(swnmg_batch* b, int l, int slot, int forward) {
  launch_b_sgs_sweep(tab(b, l), b->tickets + b->tick_off[l], b->tick_cnt[l], b->nslots[l], mk(b, slot), forward,
                     b->fp32, b->sgs_chunk[l], b->sgs_sync, b->sticky, b->st);
}

void smooth(swnmg_batch* b, int l, int slot, int nsym) {
  for (int k = 0; k < nsym; ++k) {
    sgs(b, l, slot, 1);
    sgs(b, l, slot, 0);
  }
}

bool level_descends(const swnmg_batch* b, int l) {
  for (int p = 0; p < b->B; ++p)
    if (l < b->nl[p]) return true;
  return false;
}
bool level_is_coarsest(const swnmg_batch* b, int l) {
  for (int p = 0; p < b->B; ++p)
    if (l == b->nl[p]) return true;
  return false;
}

// Algorithm 0 from level l for every running problem.  The launch sequence
// depends on the problems' level counts only (running ones are selected by
// device masks), so it can be captured once and replayed.
void mg_cycle(swnmg_batch* b, int l) {
  if (level_is_coarsest(b, l)) {
    if (b->coarse_inverse) launch_b_coarse_apply(tab(b, l), mk(b, M_CO + l), b->B, b->max_m[l], b->fp32, b->st);
    else smooth(b, l, M_CO + l, b->prm.coarse_sweeps);
  }
  if (!level_descends(b, l)) return;
  smooth(b, l, M_SM + l, b->prm.nu1);
  launch_b_restrict(bl(b, l + 1, D_CELLS, M_SM + l), tab(b, l), b->fp32, b->st);
  launch_b_fill_x(bl(b, l + 1, D_CELLS, M_SM + l), b->fp32, b->st);
  const int gam = (l == 0) ? 1 : b->prm.gamma;
  for (int k = 0; k < gam; ++k) mg_cycle(b, l + 1);
  launch_b_prolong(bl(b, l, D_CELLS, M_SM + l), tab(b, l + 1), b->fp32, b->st);
  smooth(b, l, M_SM + l, b->prm.nu2);
}

void cycles(swnmg_batch* b) {
  for (int k = 0; k < b->prm.n_mg; ++k) mg_cycle(b, 0);
}

// eq. NewtonREG at U for every running problem: Jacobian, Galerkin
// hierarchy, block LU factors and the coarsest inverses
void assemble(swnmg_batch* b) {
  launch_b_jacobian(bl(b, 0, D_EDGES, M_ACT), bl(b, 0, D_CELLS, M_ACT), b->fp32, b->st);
  for (int l = 0; l < b->maxNL; ++l)
    launch_b_galerkin(bl(b, l + 1, D_CELLS, M_SM + l), tab(b, l), b->fp32, b->st);
  for (int l = 0; l <= b->maxNL; ++l) launch_b_lu_factor(bl(b, l, D_SLOTS, M_HI + l), b->fp32, b->st);
  if (b->coarse_inverse)
    for (int l = b->minNL; l <= b->maxNL; ++l)
      if (level_is_coarsest(b, l)) launch_b_coarse_inverse(tab(b, l), mk(b, M_CO + l), b->B, b->fp32, b->st);
}

swnmg_status run_cycles(swnmg_batch* b, bool first_step) {
  if (!b->use_graph) {
    cycles(b);
    BCHECK(b);
    return SWNMG_OK;
  }
  if (!b->cyc_exec) {
    if (first_step) {   // direct the first time (one-time launch set-up happens outside a capture)
      cycles(b);
      BCHECK(b);
      return SWNMG_OK;
    }
    cudaGraph_t g = nullptr;
    const long long l0 = launches_total();
    BCUDA(b, cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
    cycles(b);
    cudaError_t e = cudaStreamEndCapture(b->st, &g);
    if (e != cudaSuccess || !g) return bfail(b, SWNMG_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    b->cyc_launches = launches_total() - l0;
    e = cudaGraphInstantiate(&b->cyc_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      b->cyc_exec = nullptr;
      return bfail(b, SWNMG_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
  } else {
    count_launches(b->cyc_launches);
  }
  BCUDA(b, cudaGraphLaunch(b->cyc_exec, b->st));
  return SWNMG_OK;
}

void free_batch(swnmg_batch* b) {
  if (b->cyc_exec) cudaGraphExecDestroy(b->cyc_exec);
  if (b->items) cudaFree(b->items);
  if (b->bstart) cudaFree(b->bstart);
  if (b->tickets) cudaFree(b->tickets);
  if (b->btickets) cudaFree(b->btickets);
  if (b->blu_sync) cudaFree(b->blu_sync);
  if (b->mask) cudaFree(b->mask);
  if (b->sums) cudaFree(b->sums);
  if (b->sgs_sync) cudaFree(b->sgs_sync);
  if (b->bl_sync) cudaFree(b->bl_sync);
  if (b->sticky) cudaFree(b->sticky);
  if (b->h_mask) cudaFreeHost(b->h_mask);
  if (b->h_sums) cudaFreeHost(b->h_sums);
  if (b->h_sticky) cudaFreeHost(b->h_sticky);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->st) cudaStreamDestroy(b->st);
  for (auto* c : b->ctx)
    if (c) swnmg_destroy(c);
}

bool chunk_ok(int fp32, int c) { return fp32 ? (c == 4 || c == 8 || c == 16) : (c == 2 || c == 4 || c == 8); }

}  // namespace

// ============================== C ABI =========================================

SWNMG_API const char* swnmg_batch_last_error(const swnmg_batch* b) { return b ? b->err.c_str() : g_berr; }

SWNMG_API swnmg_status swnmg_batch_create(const swnmg_problem* probs, const int32_t* n_levels, int32_t B,
                                          const swnmg_params* prm, const double* const* z_dev, void* stream,
                                          swnmg_batch** out) {
  if (!probs || !n_levels || !prm || !z_dev || !out) return bfail(nullptr, SWNMG_ERR_ARG, "null pointer");
  *out = nullptr;
  if (B < 1 || B > BATCH_MAX) return bfail(nullptr, SWNMG_ERR_ARG, "batch size must be 1..256");
  if (prm->smoother != SWNMG_SMOOTH_LEX)
    return bfail(nullptr, SWNMG_ERR_ARG, "batches use the lexicographic block SGS smoother only");
  for (int p = 0; p < B; ++p) {
    if (probs[p].dim != 2) return bfail(nullptr, SWNMG_ERR_ARG, "batched problems must be 2D");
    if (n_levels[p] < 0 || n_levels[p] > 12) return bfail(nullptr, SWNMG_ERR_ARG, "bad n_levels");
    if (!z_dev[p]) return bfail(nullptr, SWNMG_ERR_ARG, "null bed pointer");
  }
  swnmg_batch* b = new swnmg_batch();
  b->B = B;
  b->prm = *prm;
  b->fp32 = prm->precision != SWNMG_PREC_FP64;   // MIXED_STEP1 runs as MIXED in a batch
  b->user_st = (cudaStream_t)stream;
  swnmg_status rc = SWNMG_OK;
  int dev = 0;
#define BTRY(expr)                                                                            \
  do {                                                                                        \
    cudaError_t e_ = (expr);                                                                  \
    if (e_ != cudaSuccess) {                                                                  \
      rc = bfail(b, e_ == cudaErrorMemoryAllocation ? SWNMG_ERR_OOM : SWNMG_ERR_CUDA,          \
                 std::string(#expr) + " -> " + cudaGetErrorString(e_));                       \
      goto fail_out;                                                                          \
    }                                                                                         \
  } while (0)
  BTRY(cudaGetDevice(&dev));
  BTRY(cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev));
  BTRY(cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking));
  BTRY(cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming));
  BTRY(cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming));
  b->ctx.assign(B, nullptr);
  b->nl.assign(B, 0);
  b->maxNL = 0;
  b->minNL = 99;
  for (int p = 0; p < B; ++p) {
    swnmg_params q = *prm;
    q.n_levels = n_levels[p];
    swnmg_status s = swnmg_create(&probs[p], &q, z_dev[p], stream, &b->ctx[p]);
    if (s != SWNMG_OK) {
      rc = bfail(b, s, "problem " + std::to_string(p) + ": " + swnmg_last_error(nullptr));
      goto fail_out;
    }
    swnmg_ctx* c = b->ctx[p];
    if (!c->coarse_inverse && c->coarse_exact) {
      rc = bfail(b, SWNMG_ERR_ARG, "problem " + std::to_string(p) +
                                       ": coarsest level above 128 cells; use more levels or coarse_sweeps > 0");
      goto fail_out;
    }
    b->nl[p] = n_levels[p];
    b->maxNL = std::max(b->maxNL, b->nl[p]);
    b->minNL = std::min(b->minNL, b->nl[p]);
  }
  b->coarse_inverse = b->ctx[0]->coarse_inverse;
  {
    // per-level tables
    b->h_items.assign((size_t)MAXL * B, BItem{});
    b->h_bstart.assign((size_t)MAXL * ND * (B + 1), 0);
    b->tick_off.assign(MAXL, 0);
    b->tick_cnt.assign(MAXL, 0);
    b->nslots.assign(MAXL, 0);
    b->btick_off.assign(MAXL, 0);
    b->btick_cnt.assign(MAXL, 0);
    b->nbslots.assign(MAXL, 0);
    b->max_m.assign(MAXL, 0);
    b->max_n.assign(MAXL, 0);
    std::vector<int2> tk, btk;
    for (int l = 0; l < MAXL; ++l) {
      int slot0 = 0, maxs = 0, bslot0 = 0, bmaxs = 0;
      for (int p = 0; p < B; ++p) {
        BItem& it = b->h_items[(size_t)l * B + p];
        memset(&it, 0, sizeof it);
        if (l > b->nl[p]) continue;
        swnmg_ctx* c = b->ctx[p];
        const Level& v = c->lv[l];
        it.L = ctx_dev_level(c, l);
        it.z = v.z;
        it.U = l > 0 ? v.U : nullptr;   // level 0: the caller's state, set per solve
        it.R = c->R;
        it.rn = c->rn;
        it.eb = c->eb;
        it.red = c->red;
        it.ghost = c->ghost;
        it.blk = v.blk;
        it.lu = v.lu;
        it.piv = v.piv;
        it.b = v.b;
        it.x = v.x;
        if (l == b->nl[p]) {
          it.cinv = c->cinv;
          it.caug = c->caug;
          it.csing = c->csing;
          b->max_m[l] = std::max(b->max_m[l], v.n * 3);
        }
        it.n_xe = (v.nx + 1) * v.ny;
        it.n_e = it.n_xe + v.nx * (v.ny + 1);
        it.strip0 = slot0;
        it.bstrip0 = bslot0;
        it.has = 1;
        const int ns = (v.ny + 31) / 32;
        slot0 += ns;
        bslot0 += (v.ny + 1) / 2;
        bmaxs = std::max(bmaxs, (v.ny + 1) / 2);
        maxs = std::max(maxs, ns);
        b->max_n[l] = std::max(b->max_n[l], v.n);
      }
      b->nslots[l] = slot0;
      b->nbslots[l] = bslot0;
      // block tables
      for (int d = 0; d < ND; ++d) {
        int* bs = &b->h_bstart[((size_t)l * ND + d) * (B + 1)];
        int acc = 0;
        for (int p = 0; p < B; ++p) {
          bs[p] = acc;
          const BItem& it = b->h_items[(size_t)l * B + p];
          if (!it.has) continue;
          const long long cnt = d == D_CELLS ? it.L.n : d == D_EDGES ? it.n_e : skew_slots(it.L.nx, it.L.ny);
          acc += nblk128(cnt);
        }
        bs[B] = acc;
      }
      // strip tickets: processing index first, then problem
      b->tick_off[l] = (int)tk.size();
      for (int q = 0; q < maxs; ++q)
        for (int p = 0; p < B; ++p) {
          const BItem& it = b->h_items[(size_t)l * B + p];
          if (it.has && q < (it.L.ny + 31) / 32) tk.push_back(make_int2(p, q));
        }
      b->tick_cnt[l] = (int)tk.size() - b->tick_off[l];
      // BLU-SGS strip tickets (2 rows): strip index first, then problem
      b->btick_off[l] = (int)btk.size();
      for (int q = 0; q < bmaxs; ++q)
        for (int p = 0; p < B; ++p) {
          const BItem& it = b->h_items[(size_t)l * B + p];
          if (it.has && q < (it.L.ny + 1) / 2) btk.push_back(make_int2(p, q));
        }
      b->btick_cnt[l] = (int)btk.size() - b->btick_off[l];
    }
    int maxslots = 0;
    for (int l = 0; l < MAXL; ++l) maxslots = std::max(maxslots, b->nslots[l]);
    BTRY(cudaMalloc((void**)&b->items, sizeof(BItem) * b->h_items.size()));
    BTRY(cudaMalloc((void**)&b->bstart, sizeof(int) * b->h_bstart.size()));
    BTRY(cudaMalloc((void**)&b->tickets, sizeof(int2) * std::max<size_t>(tk.size(), 1)));
    BTRY(cudaMalloc((void**)&b->btickets, sizeof(int2) * std::max<size_t>(btk.size(), 1)));
    int maxbslots = 0;
    for (int l = 0; l < MAXL; ++l) maxbslots = std::max(maxbslots, b->nbslots[l]);
    BTRY(cudaMalloc((void**)&b->blu_sync, sizeof(int) * (2 + maxbslots + 8)));
    BTRY(cudaMalloc((void**)&b->mask, sizeof(int) * (size_t)M_COUNT * B));
    BTRY(cudaMalloc((void**)&b->sums, sizeof(double) * B));
    BTRY(cudaMalloc((void**)&b->sgs_sync, sizeof(int) * (2 + maxslots + 8)));
    BTRY(cudaMalloc((void**)&b->bl_sync, sizeof(int) * 4));
    BTRY(cudaMalloc((void**)&b->sticky, sizeof(int)));
    BTRY(cudaMallocHost((void**)&b->h_mask, sizeof(int) * (size_t)M_COUNT * B));
    BTRY(cudaMallocHost((void**)&b->h_sums, sizeof(double) * B));
    BTRY(cudaMallocHost((void**)&b->h_sticky, sizeof(int)));
    BTRY(cudaMemcpy(b->items, b->h_items.data(), sizeof(BItem) * b->h_items.size(), cudaMemcpyHostToDevice));
    BTRY(cudaMemcpy(b->bstart, b->h_bstart.data(), sizeof(int) * b->h_bstart.size(), cudaMemcpyHostToDevice));
    if (!tk.empty())
      BTRY(cudaMemcpy(b->tickets, tk.data(), sizeof(int2) * tk.size(), cudaMemcpyHostToDevice));
    if (!btk.empty())
      BTRY(cudaMemcpy(b->btickets, btk.data(), sizeof(int2) * btk.size(), cudaMemcpyHostToDevice));
    BTRY(cudaMemset(b->sticky, 0, sizeof(int)));
    memset(b->h_mask, 0, sizeof(int) * (size_t)M_COUNT * B);
    for (int p = 0; p < B; ++p)
      for (int l = 0; l < MAXL; ++l) {
        b->h_mask[(size_t)(M_DOWN + l) * B + p] = l < b->nl[p];
        b->h_mask[(size_t)(M_HAS + l) * B + p] = l <= b->nl[p];
      }
    BTRY(cudaMemcpy(b->mask, b->h_mask, sizeof(int) * (size_t)M_COUNT * B, cudaMemcpyHostToDevice));
  }
  // default tuning: the deepest staging that fits, one BLU-SGS block per SM
  for (int l = 0; l < MAXL; ++l) b->sgs_chunk[l] = b->fp32 ? 16 : 8;
  b->blusgs_max = b_blusgs_max_blocks_per_sm() * b->nsm;
  if (b->blusgs_max < 1) {
    rc = bfail(b, SWNMG_ERR_CUDA, "BLU-SGS kernel cannot be resident");
    goto fail_out;
  }
  for (int l = 0; l < MAXL; ++l) b->blusgs_blocks[l] = b->nsm;
  BTRY(cudaDeviceSynchronize());
#undef BTRY
  *out = b;
  return SWNMG_OK;
fail_out:
  free_batch(b);
  delete b;
  return rc;
}

SWNMG_API swnmg_status swnmg_batch_destroy(swnmg_batch* b) {
  if (!b) return SWNMG_ERR_ARG;
  if (b->st) cudaStreamSynchronize(b->st);
  free_batch(b);
  delete b;
  return SWNMG_OK;
}

SWNMG_API swnmg_status swnmg_batch_set_graph(swnmg_batch* b, int32_t enable) {
  if (!b) return bfail(nullptr, SWNMG_ERR_ARG, "null batch");
  b->use_graph = enable != 0;
  return SWNMG_OK;
}

SWNMG_API swnmg_status swnmg_batch_set_tuning(swnmg_batch* b, const int32_t* chunk, int32_t blocks) {
  if (!b) return bfail(nullptr, SWNMG_ERR_ARG, "null batch");
  if (chunk)
    for (int l = 0; l < MAXL; ++l)
      if (!chunk_ok(b->fp32, chunk[l])) return bfail(b, SWNMG_ERR_ARG, "bad SGS chunk");
  if (blocks > b->blusgs_max) return bfail(b, SWNMG_ERR_ARG, "BLU-SGS grid above the co-resident limit");
  BCUDA(b, cudaStreamSynchronize(b->st));
  if (chunk)
    for (int l = 0; l < MAXL; ++l) b->sgs_chunk[l] = chunk[l];
  if (blocks > 0)
    for (int l = 0; l < MAXL; ++l) b->blusgs_blocks[l] = blocks;
  if (b->cyc_exec) {   // the graph holds the old launch shapes
    cudaGraphExecDestroy(b->cyc_exec);
    b->cyc_exec = nullptr;
  }
  return SWNMG_OK;
}

namespace {

swnmg_status set_level0_state(swnmg_batch* b, double* const* U) {
  for (int p = 0; p < b->B; ++p) b->h_items[p].U = U[p];
  BCUDA(b, cudaMemcpyAsync(b->items, b->h_items.data(), sizeof(BItem) * b->B, cudaMemcpyHostToDevice, b->st));
  return SWNMG_OK;
}

float time_ms(cudaEvent_t a, cudaEvent_t z) {
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, z);
  return ms;
}

}  // namespace

SWNMG_API swnmg_status swnmg_batch_tune(swnmg_batch* b, double* const* U, int32_t* chunk_out,
                                        int32_t* blocks_out) {
  if (!b || !U) return bfail(b, SWNMG_ERR_ARG, "null pointer");
  for (int p = 0; p < b->B; ++p)
    if (!U[p]) return bfail(b, SWNMG_ERR_ARG, "null state pointer");
  swnmg_status s;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  BCUDA(b, cudaEventCreate(&e0));
  BCUDA(b, cudaEventCreate(&e1));
  std::vector<double*> scratch(b->B, nullptr);
  std::vector<int> all(b->B, 1);
  set_role_masks(b, all);
  if ((s = upload_masks(b)) != SWNMG_OK) return s;
  // SGS staging depth per level (the sweep's cost does not depend on the
  // operator's values; x is workspace)
  const int cands32[3] = {4, 8, 16}, cands64[3] = {2, 4, 8};
  for (int l = 0; l <= b->maxNL; ++l) {
    if (b->tick_cnt[l] == 0) continue;
    float best = 1e30f;
    int pick = b->sgs_chunk[l];
    for (int k = 0; k < 3; ++k) {
      b->sgs_chunk[l] = b->fp32 ? cands32[k] : cands64[k];
      sgs(b, l, M_HI + l, 1);   // warm-up (first launch configures the kernel)
      cudaEventRecord(e0, b->st);
      for (int r = 0; r < 3; ++r) {
        sgs(b, l, M_HI + l, 1);
        sgs(b, l, M_HI + l, 0);
      }
      cudaEventRecord(e1, b->st);
      BCUDA(b, cudaEventSynchronize(e1));
      BCHECK(b);
      const float ms = time_ms(e0, e1);
      if (ms < best) { best = ms; pick = b->sgs_chunk[l]; }
    }
    b->sgs_chunk[l] = pick;
  }
  if ((s = check_sticky(b)) != SWNMG_OK) return s;
  // BLU-SGS grid per level, on copies of U averaged down the levels (the
  // Step 1 states of levels >= 1 are rebuilt by every solve)
  for (int p = 0; p < b->B; ++p) {
    const size_t bytes = sizeof(double) * 3 * (size_t)b->h_items[p].L.n;
    cudaError_t e = cudaMalloc((void**)&scratch[p], bytes);
    if (e == cudaSuccess) e = cudaMemcpyAsync(scratch[p], U[p], bytes, cudaMemcpyDeviceToDevice, b->st);
    if (e != cudaSuccess) {
      for (auto* q : scratch) if (q) cudaFree(q);
      return bfail(b, SWNMG_ERR_OOM, "tuning scratch");
    }
  }
  if ((s = set_level0_state(b, scratch.data())) != SWNMG_OK) return s;
  for (int l = 0; l < b->maxNL; ++l) launch_b_average(bl(b, l + 1, D_CELLS, M_DOWN + l), tab(b, l), b->st);
  for (int l = 0; l <= b->maxNL; ++l) {
    std::vector<int> cand;
    for (int m = b->nsm / 4; m <= b->blusgs_max; m *= 2) cand.push_back(m);
    float best = 1e30f;
    int pick = b->blusgs_blocks[l];
    for (int nb : cand) {
      b->blusgs_blocks[l] = nb;
      blusgs(b, l, M_HI + l, 1);   // warm-up
      cudaEventRecord(e0, b->st);
      blusgs(b, l, M_HI + l, 1);
      blusgs(b, l, M_HI + l, 0);
      cudaEventRecord(e1, b->st);
      cudaEventSynchronize(e1);
      const float ms = time_ms(e0, e1);
      if (ms < best) { best = ms; pick = nb; }
    }
    b->blusgs_blocks[l] = pick;
  }
  cudaError_t e = cudaStreamSynchronize(b->st);
  for (auto* q : scratch) if (q) cudaFree(q);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return bfail(b, SWNMG_ERR_CUDA, std::string("tuning: ") + cudaGetErrorString(e));
  BCHECK(b);
  if ((s = check_sticky(b)) != SWNMG_OK) return s;
  if (b->cyc_exec) {
    cudaGraphExecDestroy(b->cyc_exec);
    b->cyc_exec = nullptr;
  }
  if (chunk_out)
    for (int l = 0; l < MAXL; ++l) chunk_out[l] = b->sgs_chunk[l];
  if (blocks_out)
    for (int l = 0; l < MAXL; ++l) blocks_out[l] = b->blusgs_blocks[l];
  return SWNMG_OK;
}

SWNMG_API swnmg_status swnmg_batch_solve(swnmg_batch* b, double* const* U, swnmg_stats* stats) {
  if (!b || !U) return bfail(b, SWNMG_ERR_ARG, "null pointer");
  for (int p = 0; p < b->B; ++p)
    if (!U[p]) return bfail(b, SWNMG_ERR_ARG, "null state pointer");
  const int B = b->B;
  std::vector<swnmg_stats> local;
  if (!stats) {
    local.resize(B);
    stats = local.data();
  }
  for (int p = 0; p < B; ++p) memset(&stats[p], 0, sizeof(swnmg_stats));
  using clk = std::chrono::steady_clock;
  const auto t0 = clk::now();
  swnmg_status s;
  // work on the batch's own stream, ordered after the caller's
  BCUDA(b, cudaEventRecord(b->ev_in, b->user_st));
  BCUDA(b, cudaStreamWaitEvent(b->st, b->ev_in, 0));
  if ((s = set_level0_state(b, U)) != SWNMG_OK) return s;
  std::vector<int> act(B, 1);
  set_role_masks(b, act);
  if ((s = upload_masks(b)) != SWNMG_OK) return s;
  std::vector<double> res(B, 0.0);
  // Step 1: BLU-SGS from each problem's coarsest level to level 1 with
  // piecewise-constant prolongation (Algorithm 1)
  if (b->prm.init_mode == SWNMG_INIT_CASCADE && b->maxNL > 0) {
    // eps_p < 0: the paper's rule per problem, |eps_p| x sum_i ||R_i||_1 of
    // that problem's initial data
    std::vector<double> eps(B, b->prm.eps_p);
    if (b->prm.eps_p < 0.0) {
      if ((s = residual_sums(b, 0, M_HAS + 0, res)) != SWNMG_OK) return s;
      for (int p = 0; p < B; ++p) eps[p] = -b->prm.eps_p * res[p];
    }
    for (int l = 0; l < b->maxNL; ++l) launch_b_average(bl(b, l + 1, D_CELLS, M_DOWN + l), tab(b, l), b->st);
    BCHECK(b);
    for (int l = b->maxNL; l >= 1; --l) {
      std::vector<double> thr(B);
      for (int p = 0; p < B; ++p) thr[p] = eps[p] / (double)(1 << l);
      if ((s = residual_sums(b, l, M_HAS + l, res)) != SWNMG_OK) return s;
      std::vector<int> nsw(B, 0);
      int* casc = hm(b, M_CASC);
      for (int p = 0; p < B; ++p)
        casc[p] = (l <= b->nl[p]) && res[p] >= thr[p] && 0 < b->prm.max_blusgs && std::isfinite(res[p]);
      while (any_mask(b, M_CASC)) {
        if ((s = upload_mask_slot(b, M_CASC)) != SWNMG_OK) return s;
        blusgs(b, l, M_CASC, 1);
        blusgs(b, l, M_CASC, 0);
        BCHECK(b);
        for (int p = 0; p < B; ++p) nsw[p] += casc[p];
        if ((s = residual_sums(b, l, M_CASC, res)) != SWNMG_OK) return s;
        for (int p = 0; p < B; ++p)
          casc[p] = casc[p] && res[p] >= thr[p] && nsw[p] < b->prm.max_blusgs && std::isfinite(res[p]);
      }
      for (int p = 0; p < B; ++p)
        if (l <= b->nl[p] && l < 16) stats[p].blusgs_sweeps[l] = nsw[p];
      launch_b_inject(bl(b, l - 1, D_CELLS, M_HAS + l), tab(b, l), b->st);
      BCHECK(b);
    }
  }
  BCUDA(b, cudaStreamSynchronize(b->st));
  const auto t1 = clk::now();
  // Steps 2-3: Newton multigrid iteration of every problem
  if ((s = residual_sums(b, 0, M_HAS + 0, res)) != SWNMG_OK) return s;
  std::vector<double> best(B);
  std::vector<int> status(B), it(B, 0);
  for (int p = 0; p < B; ++p) {
    stats[p].init_res = res[p];
    best[p] = res[p];
    status[p] = std::isfinite(res[p]) ? SWNMG_ERR_NOT_CONVERGED : SWNMG_ERR_NONFINITE;
  }
  bool first = true;
  for (;;) {
    for (int p = 0; p < B; ++p) {
      act[p] = status[p] == SWNMG_ERR_NOT_CONVERGED && it[p] < b->prm.max_newton;
      if (act[p] && res[p] < b->prm.tol) {
        status[p] = SWNMG_OK;
        act[p] = 0;
      }
    }
    bool any = false;
    for (int p = 0; p < B; ++p) any = any || act[p];
    if (!any) break;
    set_role_masks(b, act);
    if ((s = upload_masks(b)) != SWNMG_OK) return s;
    blusgs(b, 0, M_ACT, 1);                                     // Step 2.1
    blusgs(b, 0, M_ACT, 0);
    BCHECK(b);
    assemble(b);                                                // eq. NewtonREG
    launch_b_neg_residual(bl(b, 0, D_CELLS, M_ACT), b->fp32, b->st);
    launch_b_fill_x(bl(b, 0, D_CELLS, M_ACT), b->fp32, b->st);
    BCHECK(b);
    if ((s = run_cycles(b, first)) != SWNMG_OK) return s;      // Step 2.2
    first = false;
    launch_b_newton_update(bl(b, 0, D_CELLS, M_ACT), b->prm.tau, b->prm.h_eps, b->fp32, b->st);   // Step 2.3
    BCHECK(b);
    if ((s = check_sticky(b)) != SWNMG_OK) return s;
    if ((s = residual_sums(b, 0, M_ACT, res)) != SWNMG_OK) return s;   // Step 3
    for (int p = 0; p < B; ++p) {
      if (!act[p]) continue;
      ++it[p];
      stats[p].n_vcycles += b->prm.n_mg;
      if (it[p] <= SWNMG_HIST) stats[p].res_hist[it[p] - 1] = res[p];
      if (!std::isfinite(res[p])) { status[p] = SWNMG_ERR_NONFINITE; continue; }
      if (res[p] < best[p]) best[p] = res[p];
      if (res[p] > 1e6 * best[p]) status[p] = SWNMG_ERR_DIVERGED;
    }
  }
  const auto t2 = clk::now();
  swnmg_status first_bad = SWNMG_OK;
  int bad_p = -1;
  for (int p = 0; p < B; ++p) {
    if (status[p] == SWNMG_ERR_NOT_CONVERGED && res[p] < b->prm.tol) status[p] = SWNMG_OK;
    stats[p].n_newton = it[p];
    stats[p].final_res = res[p];
    stats[p].status = status[p];
    stats[p].ms_step1 = std::chrono::duration<double, std::milli>(t1 - t0).count();
    stats[p].ms_newton = std::chrono::duration<double, std::milli>(t2 - t1).count();
    if (status[p] != SWNMG_OK && first_bad == SWNMG_OK) {
      first_bad = (swnmg_status)status[p];
      bad_p = p;
    }
  }
  BCUDA(b, cudaEventRecord(b->ev_out, b->st));
  BCUDA(b, cudaStreamWaitEvent(b->user_st, b->ev_out, 0));
  if (first_bad != SWNMG_OK)
    return bfail(b, first_bad, "problem " + std::to_string(bad_p) + " after " + std::to_string(it[bad_p]) +
                                   " Newton steps");
  return SWNMG_OK;
}
