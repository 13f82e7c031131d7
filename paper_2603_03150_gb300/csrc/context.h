// Host-side context of a solver (single LP or a batch of LPs) shared by the
// translation units of the C ABI.
#pragma once
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <future>
#include <string>
#include <vector>

#include "kernels.h"
#include "pdhg.h"
#include "spmv_tile.cuh"

namespace pdhg {
void set_error(const char* fmt, ...);
void clear_error();
}  // namespace pdhg

#define CK(call)                                                                    \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      pdhg::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,   \
                __LINE__);                                                          \
      return e_ == cudaErrorMemoryAllocation ? PDHG_OOM : PDHG_CUDA_ERROR;          \
    }                                                                               \
  } while (0)

#define CKS(expr)                          \
  do {                                     \
    pdhg_status s_ = (expr);               \
    if (s_ < 0) return s_;                 \
  } while (0)


namespace pdhg {

struct HostSched {
  std::vector<Tile> tiles;
  std::vector<SplitGroup> groups;
  int total_parts = 0;
  int tile_nnz = 0, max_rows = 0, e = 8;
  int64_t nwords = 0;             // window words of the whole-row tiles (e > 0)
  std::vector<int32_t> lp_tiles;  // [count + 1] first tile of each LP
};

// Tiles of whole rows (at most tile_capacity(kBlock, e) nonzeros and
// tile_max_rows(kBlock) rows, none of them empty), capacity-sized chunks of a
// longer row, or runs of empty rows.
// With lp_off (count + 1 row offsets) no tile crosses an LP boundary and each
// tile records its LP.
// cap > 0: at most cap nonzeros per tile (below the full capacity).
HostSched build_sched(const int32_t* rp, int nrows, int e, const int64_t* lp_off = nullptr,
                      int count = 1, int cap = 0);

struct DevSched {
  Tile* tiles = nullptr;
  SplitGroup* groups = nullptr;
  int32_t* counters = nullptr;
  double* slots = nullptr;
  uint32_t* wd = nullptr;
  SchedView view{};
};

// column-panel layout of one matrix (float32 single-LP iterations)
struct DevPanel {
  PanelTile* tiles = nullptr;
  PanelBlock* blocks = nullptr;
  float* val = nullptr;
  uint16_t* col = nullptr;
  uint32_t* wd = nullptr;
  int32_t* psrow = nullptr;
  float* partial = nullptr;
  PanelView view{};
  int64_t pseudo_rows = 0, nnz_padded = 0;
  bool on = false;  // the half-step over this matrix runs on the panels
};

}  // namespace pdhg

struct pdhg_ctx;
void pdhg_free_adjoint(pdhg_ctx* ctx);
// the active set fixed by pdhg_batch_polish no longer applies (new b, c)
void pdhg_adjoint_invalidate(pdhg_ctx* ctx);

using pdhg::DevPanel;
using pdhg::DevSched;
using pdhg::Launch;
using pdhg::PowerState;
using pdhg::Scalars;

struct pdhg_ctx {
  int m = 0, n = 0;
  int64_t nnz = 0, nnz_pad = 0;
  pdhg_options opt{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int nsm = 0;
  size_t smem_optin = 0;
  bool mixed = false;

  std::vector<void*> allocs;
  // matrices
  int32_t *a_rp = nullptr, *a_col = nullptr, *t_rp = nullptr, *t_col = nullptr;
  double *a_val_orig = nullptr, *t_val_orig = nullptr, *a_val64 = nullptr, *t_val64 = nullptr;
  float *a_val32 = nullptr, *t_val32 = nullptr;
  std::vector<int32_t> h_a_rp, h_t_rp;
  // [A, A^T][E = 16, 32]: the tuner's other whole-row schedules, built on a
  // host thread while the GPU runs the power iteration (declared after the
  // row pointers they read, so an early destruction joins them first)
  std::future<pdhg::HostSched> presched[2][2];
  // vectors
  double *b = nullptr, *c = nullptr, *b_t64 = nullptr, *c_t64 = nullptr, *D_r = nullptr,
         *D_c = nullptr;
  double *Dr_inv = nullptr, *Dc_inv = nullptr;  // 1 / D_r, 1 / D_c (the evaluation multiplies)
  float *b_t32 = nullptr, *c_t32 = nullptr;
  void *x = nullptr, *y = nullptr, *x_avg = nullptr, *y_avg = nullptr, *x_last = nullptr,
       *y_last = nullptr, *Ax = nullptr, *Ax_avg = nullptr, *Ax_last = nullptr;
  // adaptive step (options.step_rule 1): the accepted state before an attempt
  // (its x in adapt_xx)
  void *x_avg_prev = nullptr, *y_prev = nullptr, *y_avg_prev = nullptr, *Ax_prev = nullptr,
       *Ax_avg_prev = nullptr;
  void* adapt_xx = nullptr;  // the attempt's (x+_j, x_j), interleaved [2n]
  // the attempt's sums: per primal block, per split row of A~^T, per dual
  // block (pairs), per split row of A~ (pairs); one allocation
  double* adapt_sums = nullptr;
  Launch l_aprim{}, l_adual{};  // the adaptive half-steps' launches
  double *xs64 = nullptr, *ys64 = nullptr, *out_n1 = nullptr, *out_n2 = nullptr,
         *out_m1 = nullptr, *report = nullptr, *sums = nullptr;
  Scalars* sc = nullptr;
  PowerState* ps = nullptr;
  double* partials = nullptr;  // generic reduction scratch
  size_t partials_len = 0;
  double* split_q = nullptr;
  long long* log_k = nullptr;
  int32_t* log_flags = nullptr;
  double* log_kkt = nullptr;
  int log_cap = 4096;
  // batched solves: `count` independent LPs as one block-diagonal system
  int count = 1;
  bool batch = false;
  std::vector<int64_t> h_m_off, h_n_off;  // [count + 1] row / column offsets
  int32_t *lp_a_tiles = nullptr, *lp_t_tiles = nullptr;    // [count + 1] tile ranges
  int32_t *lp_a8_tiles = nullptr, *lp_t8_tiles = nullptr;  // same, float64 schedules
  double *rec_t = nullptr, *rec_a = nullptr;  // per-tile evaluation / report records
  int rec_tiles = 0;                          // tiles the record arrays hold
  int32_t* active = nullptr;                  // LPs not finished after the last evaluation
  int64_t *d_m_off = nullptr, *d_n_off = nullptr;  // [count + 1] row / column offsets (device)
  void* gsync = nullptr;                      // grid-barrier state of the persistent batched solve
  double* breport = nullptr;                  // [count][8] per-LP report
  void* adjoint = nullptr;                    // active-set polish / adjoint buffers
  // schedules and launch shapes
  DevSched sa, st;      // iteration schedules (autotuned nonzeros per thread)
  DevSched sa8, st8;    // float64 report / Algorithm 1 / power iteration
  DevPanel pa, pt;      // column panels of A~ (dual) and A~^T (primal), when chosen
  int32_t* panel_err = nullptr;  // 1 once a panel load's bounded wait ran out
  int panel_row_grid_a = 1, panel_row_grid_t = 1;
  Launch l_prim{}, l_dual{}, l_eval{}, l_a64{}, l_t64{};
  int restart_grid = 1;
  // graphs and polling
  cudaGraphExec_t chunk_exec[2] = {nullptr, nullptr};
  cudaEvent_t ev_done[2] = {nullptr, nullptr};
  // sampled iteration: before / between the two kernels / after the primal
  // half-step, then the same for the dual (CSR tiles: one kernel, nothing between)
  cudaEvent_t ev_k[2][6] = {};
  Scalars* h_sc[2] = {nullptr, nullptr};
  double timing_sum[4] = {0, 0, 0, 0};  // primal kernel 1, 2, dual kernel 1, 2
  long long timing_n = 0;
  // cached host data
  double omega0 = 1.0;
  int power_iters = 0;
  double report_h[8] = {0};
  long long launches = 0;  // kernels launched (graph replays count every node)
  bool report_valid = false;
  int last_status = PDHG_MAX_ITER;
};

namespace pdhg {

// With options.verbose: the wall time of each create stage on stderr (the
// stream is synchronised at every stage boundary, so it costs a little).
struct StageClock {
  pdhg_ctx* ctx;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now(), last = t0;
  void operator()(const char* name) {
    if (!ctx->opt.verbose) return;
    cudaStreamSynchronize(ctx->stream);
    const auto now = std::chrono::steady_clock::now();
    std::fprintf(stderr, "pdhg_create: %-24s %9.3f ms\n", name,
                 std::chrono::duration<double, std::milli>(now - last).count());
    last = now;
  }
};

template <typename T>
pdhg_status dalloc(pdhg_ctx* ctx, T** p, size_t count) {
  void* q = nullptr;
  const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) {
    pdhg::set_error("cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? PDHG_OOM : PDHG_CUDA_ERROR;
  }
  ctx->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return PDHG_OK;
}

pdhg_status copy_in(pdhg_ctx* ctx, void* dst, const void* src, size_t bytes);
pdhg_status copy_out(pdhg_ctx* ctx, void* dst, const void* src, size_t bytes);
// kind 0: one gathered vector in the iteration precision, 1: two, 2: one in float64
size_t smem_for(int kind, bool mixed, int max_rows, int e);
// copies the schedule to the device and computes its window words from the
// device row pointer rp of the same matrix
pdhg_status upload_sched(pdhg_ctx* ctx, const HostSched& h, DevSched* d, const int32_t* rp);
Launch make_launch(pdhg_ctx* ctx, int occ_kind, int e, size_t smem, int ntiles);
size_t elem(const pdhg_ctx* ctx);
// create stages shared by the single-LP and batched paths
pdhg_status setup_device(pdhg_ctx* ctx);
pdhg_status alloc_arrays(pdhg_ctx* ctx);
pdhg_status upload_lp(pdhg_ctx* ctx, const int32_t* col, const double* val, const double* b,
                      const double* c);
pdhg_status prepare_matrix(pdhg_ctx* ctx);
pdhg_status polling_resources(pdhg_ctx* ctx);
// column panels (panel.cu): the panel width and count for the rows of A~
// (on_a) or A~^T with tiles of at most `pscap` pseudo-rows, false where the
// panels do not apply (float64, batches, or dense partial sums above about
// twice the nonzeros); the device layout
bool panel_shape(const pdhg_ctx* ctx, bool on_a, int* P, int* npanels, int pscap = 256);
pdhg_status build_panel_layout(pdhg_ctx* ctx, bool on_a, DevPanel* out);
// batched solve from iteration k0 to max_iter in one cooperative launch
// (PDHG_TIMEOUT if a grid barrier's bounded wait ran out)
pdhg_status batch_persistent_solve(pdhg_ctx* ctx, long long k0, long long max_iter);

}  // namespace pdhg
