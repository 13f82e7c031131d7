// Host runtime of the single-LP solver behind the C ABI in include/pdhg.h:
// context set-up, the CSR tile scheduler and its autotuner, the chunked
// solve loop (CUDA-graph replay, status polled one chunk behind), and the
// getters.  All arithmetic of the method runs in the kernels.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "context.h"

// ---------------------------------------------------------------------------
// error reporting
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;

void pdhg::set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}
using pdhg::set_error;
#undef CK
#define CK(call)                                                                    \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      pdhg::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                      __LINE__);                                                    \
      return e_ == cudaErrorMemoryAllocation ? PDHG_OOM : PDHG_CUDA_ERROR;          \
    }                                                                               \
  } while (0)

void pdhg::clear_error() { g_last_error.clear(); }

extern "C" const char* pdhg_last_error(void) { return g_last_error.c_str(); }

namespace pdhg {

// ---------------------------------------------------------------------------
// tile schedule (host build + device copy)
// ---------------------------------------------------------------------------

// Tiles: runs of whole rows with at most tile_capacity(kBlock, e) nonzeros
// and at most tile_max_rows(kBlock) rows; a longer row becomes a split group
// of capacity-sized chunks.
HostSched build_sched(const int32_t* rp, int nrows, int e, const int64_t* lp_off, int count,
                      int cap) {
  HostSched h;
  // vector schedules (e < 0) use the tile capacity of e = 8; a smaller
  // capacity leaves the last thread windows of a full tile empty
  const int full = tile_capacity(kBlock, e > 0 ? e : 8);
  cap = (cap > 0 && cap < full) ? cap : full;
  h.tile_nnz = cap;
  h.max_rows = tile_max_rows(kBlock);
  h.e = e;
  int lp = 0;
  int lp_end = lp_off ? (int)lp_off[1] : nrows;
  int r = 0;
  h.lp_tiles.push_back(0);
  while (r < nrows) {
    while (lp_off && r >= lp_end && lp + 1 < count) {
      ++lp;
      lp_end = (int)lp_off[lp + 1];
      h.lp_tiles.push_back((int32_t)h.tiles.size());
    }
    const int64_t len = (int64_t)rp[r + 1] - rp[r];
    if (len > cap) {
      const int nparts = (int)((len + cap - 1) / cap);
      const int gid = (int)h.groups.size();
      h.groups.push_back(SplitGroup{r, nparts, h.total_parts, 0});
      for (int p = 0; p < nparts; ++p) {
        const int64_t b = rp[r] + (int64_t)p * cap;
        const int64_t en = std::min<int64_t>(b + cap, rp[r + 1]);
        h.tiles.push_back(Tile{r, r + 1, (int32_t)b, (int32_t)en, gid, p, lp, 0});
      }
      h.total_parts += nparts;
      ++r;
      continue;
    }
    const int start = r;
    if (len == 0) {  // a run of rows without nonzeros
      while (r < nrows && r < lp_end && r - start < h.max_rows && rp[r + 1] == rp[r]) ++r;
      h.tiles.push_back(Tile{start, r, rp[start], rp[start], -1, 0, lp, 0});
      continue;
    }
    int64_t nz = 0;
    while (r < nrows && r < lp_end && r - start < h.max_rows) {
      const int64_t l = (int64_t)rp[r + 1] - rp[r];
      if (l == 0 || l > cap || nz + l > cap) break;
      nz += l;
      ++r;
    }
    // whole rows: one window word per thread (segmented schedules)
    const int32_t word0 = e > 0 ? (int32_t)h.nwords : 0;
    if (e > 0) h.nwords += kBlock;
    h.tiles.push_back(Tile{start, r, rp[start], rp[r], -1, 0, lp, word0});
  }
  // LPs with no rows left (none with m >= 1) still get a range
  while ((int)h.lp_tiles.size() < count) h.lp_tiles.push_back((int32_t)h.tiles.size());
  h.lp_tiles.push_back((int32_t)h.tiles.size());
  return h;
}

}  // namespace pdhg


using namespace pdhg;

pdhg_status pdhg::copy_in(pdhg_ctx* ctx, void* dst, const void* src, size_t bytes) {
  if (bytes == 0) return PDHG_OK;
  CK(cudaMemcpyAsync(dst, src, bytes,
                     ctx->opt.io_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                     ctx->stream));
  return PDHG_OK;
}
pdhg_status pdhg::copy_out(pdhg_ctx* ctx, void* dst, const void* src, size_t bytes) {
  if (!dst || bytes == 0) return PDHG_OK;
  CK(cudaMemcpyAsync(dst, src, bytes,
                     ctx->opt.io_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     ctx->stream));
  return PDHG_OK;
}

// kind 0: one gathered vector in the iteration precision, 1: two, 2: one in float64
size_t pdhg::smem_for(int kind, bool mixed, int max_rows, int e) {
  if (kind == 0) return tile_smem(1, mixed, max_rows, e);
  if (kind == 1) return tile_smem(2, mixed, max_rows, e);
  return tile_smem(1, false, max_rows, e);
}

pdhg_status pdhg::upload_sched(pdhg_ctx* ctx, const HostSched& h, DevSched* d,
                               const int32_t* rp) {
  *d = DevSched{};
  if (h.nwords >= (int64_t)1 << 31) {
    set_error("tile schedule too large (%lld window words)", (long long)h.nwords);
    return PDHG_INVALID_ARG;
  }
  CKS(dalloc(ctx, &d->tiles, h.tiles.size()));
  CKS(dalloc(ctx, &d->groups, h.groups.size()));
  CKS(dalloc(ctx, &d->counters, h.groups.size()));
  CKS(dalloc(ctx, &d->slots, (size_t)h.total_parts * 2));
  // 32-bit words up to 16 nonzeros per thread, 64-bit words beyond
  CKS(dalloc(ctx, &d->wd, (size_t)h.nwords * (h.e > 16 ? 2 : 1) + 4));  // spare: L2 prefetches
  if (!h.tiles.empty())
    CK(cudaMemcpyAsync(d->tiles, h.tiles.data(), h.tiles.size() * sizeof(Tile),
                       cudaMemcpyHostToDevice, ctx->stream));
  if (!h.groups.empty())
    CK(cudaMemcpyAsync(d->groups, h.groups.data(), h.groups.size() * sizeof(SplitGroup),
                       cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemsetAsync(d->counters, 0, std::max<size_t>(h.groups.size(), 1) * sizeof(int32_t),
                     ctx->stream));
  if (h.nwords > 0) {
    launch_window_words(d->tiles, (int)h.tiles.size(), rp, h.e, d->wd, ctx->stream);
    ctx->launches += 1;
  }
  d->view.tiles = d->tiles;
  d->view.groups = d->groups;
  d->view.counters = d->counters;
  d->view.slots = d->slots;
  d->view.wd = d->wd;
  d->view.ntiles = (int32_t)h.tiles.size();
  d->view.tile_nnz = h.tile_nnz;
  d->view.max_rows = h.max_rows;
  d->view.ngroups = (int32_t)h.groups.size();
  d->view.e = h.e;
  // make the host vectors' lifetime irrelevant: copies are enqueued, wait here
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaGetLastError());
  return PDHG_OK;
}

// occupancy kinds of the iteration kernels (tile_occupancy numbering; the
// Halpern kernels from kOccHalpern on)
static constexpr int kOccHalpern = 100;
static int prim_kind(const pdhg_ctx* ctx) {
  return (ctx->opt.method == 1 ? kOccHalpern : 0) + (ctx->mixed ? 0 : 1);
}
static int dual_kind(const pdhg_ctx* ctx) {
  return (ctx->opt.method == 1 ? kOccHalpern : 0) + (ctx->mixed ? 2 : 3);
}

Launch pdhg::make_launch(pdhg_ctx* ctx, int occ_kind, int e, size_t smem, int ntiles) {
  const int occ = occ_kind >= kOccHalpern ? halpern_occupancy(occ_kind - kOccHalpern, e, smem)
                                          : tile_occupancy(occ_kind, e, smem);
  int grid = std::min(ntiles, ctx->nsm * occ);
  return Launch{std::max(grid, 1), smem};
}


// Float64 schedules (report, Algorithm 1, power iteration) and reduction
// scratch sized for any iteration schedule the tuner may pick.
static pdhg_status fixed_schedules(pdhg_ctx* ctx) {
  // rows that any candidate schedule could split: longer than the smallest
  // tile capacity the tuner may use (a forced options.tile_nnz below the
  // full capacity of 8 nonzeros per thread splits shorter rows too)
  const int cap_min = ctx->opt.tile_nnz > 0 ? std::min(ctx->opt.tile_nnz, tile_capacity(kBlock, 8))
                                            : tile_capacity(kBlock, 8);
  int64_t long_rows = 0;
  for (int which = 0; which < 2; ++which) {
    const bool on_a = which == 0;
    const std::vector<int32_t>& rp = on_a ? ctx->h_a_rp : ctx->h_t_rp;
    const int nrows = on_a ? ctx->m : ctx->n;
    HostSched h = build_sched(rp.data(), nrows, kFixedE);
    CKS(upload_sched(ctx, h, on_a ? &ctx->sa8 : &ctx->st8, on_a ? ctx->a_rp : ctx->t_rp));
    for (int r = 0; r < nrows; ++r) long_rows += (rp[r + 1] - rp[r]) > cap_min;
  }
  const bool mx = ctx->mixed;
  const SchedView &A8 = ctx->sa8.view, &T8 = ctx->st8.view;
  ctx->l_a64 = make_launch(ctx, 8, kFixedE, smem_for(2, mx, A8.max_rows, A8.e), A8.ntiles);
  ctx->l_t64 = make_launch(ctx, 8, kFixedE, smem_for(2, mx, T8.max_rows, T8.e), T8.ntiles);
  ctx->restart_grid = std::max(1, std::min(ctx->nsm * 8, (std::max(ctx->m, ctx->n) + 255) / 256));
  // grids never exceed SMs x 8 resident blocks of 256 threads
  const int64_t gmax = std::max<int64_t>({(int64_t)ctx->nsm * 8, ctx->l_a64.grid, ctx->l_t64.grid, 4096});
  ctx->partials_len = (size_t)(gmax + long_rows + 1) * kEvalQ;
  CKS(dalloc(ctx, &ctx->partials, ctx->partials_len));
  CKS(dalloc(ctx, &ctx->split_q, (size_t)(long_rows + 1) * kEvalQ));
  // the adaptive step's sums: one per primal block and split row of A~^T,
  // two per dual block and split row of A~, for any candidate schedule
  if (ctx->opt.step_rule == 1 && !ctx->batch)
    CKS(dalloc(ctx, &ctx->adapt_sums, 3 * (size_t)ctx->nsm * 8 + 2 * ((size_t)long_rows + 1)));
  return PDHG_OK;
}

// ---------------------------------------------------------------------------
template <typename T>
static IterBuffers<T> iter_buffers(pdhg_ctx* ctx) {
  IterBuffers<T> B{};
  B.a_rp = ctx->a_rp;
  B.a_col = ctx->a_col;
  B.t_rp = ctx->t_rp;
  B.t_col = ctx->t_col;
  if constexpr (sizeof(T) == 4) {
    B.a_val = (const T*)ctx->a_val32;
    B.t_val = (const T*)ctx->t_val32;
    B.c_t = (const T*)ctx->c_t32;
    B.b_t = (const T*)ctx->b_t32;
  } else {
    B.a_val = (const T*)ctx->a_val64;
    B.t_val = (const T*)ctx->t_val64;
    B.c_t = (const T*)ctx->c_t64;
    B.b_t = (const T*)ctx->b_t64;
  }
  B.a_sched = ctx->sa.view;
  B.t_sched = ctx->st.view;
  B.x = (T*)ctx->x;
  B.y = (T*)ctx->y;
  B.x_avg = (T*)ctx->x_avg;
  B.y_avg = (T*)ctx->y_avg;
  B.x_last = (T*)ctx->x_last;
  B.y_last = (T*)ctx->y_last;
  B.Ax = (T*)ctx->Ax;
  B.Ax_avg = (T*)ctx->Ax_avg;
  B.Ax_last = (T*)ctx->Ax_last;
  B.x_avg_prev = (T*)ctx->x_avg_prev;
  B.y_prev = (T*)ctx->y_prev;
  B.y_avg_prev = (T*)ctx->y_avg_prev;
  B.Ax_prev = (T*)ctx->Ax_prev;
  B.Ax_avg_prev = (T*)ctx->Ax_avg_prev;
  B.adapt_xx = (T*)ctx->adapt_xx;
  if (ctx->adapt_sums) {
    B.adapt_np = ctx->l_aprim.grid;
    B.adapt_pp = ctx->adapt_sums;
    B.adapt_sp = B.adapt_pp + ctx->l_aprim.grid;
    B.adapt_pd = B.adapt_sp + ctx->st.view.ngroups;
    B.adapt_sd = B.adapt_pd + 2 * (size_t)ctx->l_adual.grid;
  }
  B.rho = ctx->opt.reflection;
  B.c_t64 = ctx->c_t64;
  B.b_t64 = ctx->b_t64;
  B.D_r = ctx->D_r;
  B.D_c = ctx->D_c;
  B.Dr_inv = ctx->Dr_inv;
  B.Dc_inv = ctx->Dc_inv;
  B.sc = ctx->sc;
  B.partials = ctx->partials;
  B.split_q = ctx->split_q;
  B.log_k = ctx->log_k;
  B.log_flags = ctx->log_flags;
  B.log_kkt = ctx->log_kkt;
  B.m = ctx->m;
  B.n = ctx->n;
  return B;
}

// the iteration's half-steps for the configured method and layout (column
// panels: two kernels; CSR tiles: one fused kernel)
// `between` (optional): an event recorded between the half-step's kernels
// (right after the fused kernel of the CSR tiles)
template <typename T>
static void launch_prim_step(pdhg_ctx* ctx, const IterBuffers<T>& B, int i,
                             cudaEvent_t between = nullptr) {
  if constexpr (sizeof(T) == 4) {
    if (ctx->pt.on) {
      launch_panel_half(B, ctx->pt.view, false, ctx->opt.method, ctx->panel_row_grid_t, i,
                        ctx->stream, between);
      return;
    }
  }
  if (ctx->opt.method == 1)
    launch_hprimal<T>(B, ctx->l_prim, i, ctx->stream);
  else
    launch_primal<T>(B, ctx->l_prim, i, ctx->stream);
  if (between) cudaEventRecordWithFlags(between, ctx->stream, cudaEventRecordExternal);
}
template <typename T>
static void launch_dual_step(pdhg_ctx* ctx, const IterBuffers<T>& B, int i,
                             cudaEvent_t between = nullptr) {
  if constexpr (sizeof(T) == 4) {
    if (ctx->pa.on) {
      launch_panel_half(B, ctx->pa.view, true, ctx->opt.method, ctx->panel_row_grid_a, i,
                        ctx->stream, between);
      return;
    }
  }
  if (ctx->opt.method == 1)
    launch_hdual<T>(B, ctx->l_dual, i, ctx->stream);
  else
    launch_dual<T>(B, ctx->l_dual, i, ctx->stream);
  if (between) cudaEventRecordWithFlags(between, ctx->stream, cudaEventRecordExternal);
}
// the half-steps a solve runs: the adaptive step's own kernels (its dual
// half-step ends with the acceptance test of the attempt, then the undo of a rejected
// one), else the above
template <typename T>
static void launch_prim_half(pdhg_ctx* ctx, const IterBuffers<T>& B, int i,
                             cudaEvent_t between = nullptr) {
  if (ctx->opt.step_rule != 1) return launch_prim_step<T>(ctx, B, i, between);
  launch_adapt_primal<T>(B, ctx->l_aprim, i, ctx->stream);
  if (between) cudaEventRecordWithFlags(between, ctx->stream, cudaEventRecordExternal);
}
template <typename T>
static void launch_dual_half(pdhg_ctx* ctx, const IterBuffers<T>& B, int i,
                             cudaEvent_t between = nullptr) {
  if (ctx->opt.step_rule != 1) return launch_dual_step<T>(ctx, B, i, between);
  launch_adapt_dual<T>(B, ctx->l_adual, i, ctx->stream);
  if (between) cudaEventRecordWithFlags(between, ctx->stream, cudaEventRecordExternal);
  launch_adapt_revert<T>(B, ctx->restart_grid, ctx->stream);
}
static int prim_launches(const pdhg_ctx* ctx) { return ctx->pt.on ? 2 : 1; }
static int dual_launches(const pdhg_ctx* ctx) { return ctx->pa.on ? 2 : 1; }
// kernels of a chunk of `len` iterations: the half-steps, the evaluation, the
// float64 check (float32-mixed) and the restart
static long long chunk_launches(const pdhg_ctx* ctx, int len) {
  // adaptive step: the two half-steps and the undo of a rejected attempt
  const int per = ctx->opt.step_rule == 1 ? 3 : prim_launches(ctx) + dual_launches(ctx);
  return (long long)per * len + 2 + (ctx->mixed ? kFp64CheckLaunches : 0);
}

// what the float64 check of a float32-mixed candidate reads and writes
static Fp64Check fp64_check_args(pdhg_ctx* ctx) {
  Fp64Check C{};
  C.St = ctx->st8.view;
  C.Sa = ctx->sa8.view;
  C.t_val = ctx->t_val64;
  C.a_val = ctx->a_val64;
  C.xs = ctx->xs64;
  C.ys = ctx->ys64;
  C.Lt = ctx->l_t64;
  C.La = ctx->l_a64;
  C.gn = ctx->l_t64.grid + ctx->st8.view.ngroups;
  C.gm = ctx->l_a64.grid + ctx->sa8.view.ngroups;
  C.conv_grid = ctx->restart_grid;
  return C;
}

// `len` iterations followed by the evaluation and the restart.  With
// `timing`, events bracket the primal and dual kernels of iteration len/2.
template <typename T>
static void enqueue_chunk(pdhg_ctx* ctx, int len, cudaEvent_t* timing) {
  const IterBuffers<T> B = iter_buffers<T>(ctx);
  ctx->launches += chunk_launches(ctx, len);
  for (int i = 0; i < len; ++i) {
    const bool sample = timing && i == len / 2;
    if (sample) cudaEventRecordWithFlags(timing[0], ctx->stream, cudaEventRecordExternal);
    launch_prim_half<T>(ctx, B, i, sample ? timing[1] : nullptr);
    if (sample) {
      cudaEventRecordWithFlags(timing[2], ctx->stream, cudaEventRecordExternal);
      cudaEventRecordWithFlags(timing[3], ctx->stream, cudaEventRecordExternal);
    }
    launch_dual_half<T>(ctx, B, i, sample ? timing[4] : nullptr);
    if (sample) cudaEventRecordWithFlags(timing[5], ctx->stream, cudaEventRecordExternal);
  }
  launch_eval<T>(B, ctx->l_eval, len, ctx->stream);
  if constexpr (sizeof(T) == 4) launch_fp64_check<T>(B, fp64_check_args(ctx), ctx->stream);
  launch_restart<T>(B, ctx->restart_grid, ctx->stream);
}

static void enqueue_chunk_any(pdhg_ctx* ctx, int len, cudaEvent_t* timing) {
  if (ctx->mixed)
    enqueue_chunk<float>(ctx, len, timing);
  else
    enqueue_chunk<double>(ctx, len, timing);
}

// The adaptive step's launch of one half-step on schedule S (its dual
// gathers the pairs (x+, x): the shared memory of two vectors).
static void set_adaptive_launch(pdhg_ctx* ctx, bool on_a, const SchedView& S) {
  if (ctx->opt.step_rule != 1 || ctx->batch) return;
  const bool mx = ctx->mixed;
  const size_t sm = smem_for(on_a ? 1 : 0, mx, S.max_rows, S.e);
  const int occ = adaptive_occupancy((on_a ? 2 : 0) + (mx ? 0 : 1), S.e, sm);
  (on_a ? ctx->l_adual : ctx->l_aprim) = Launch{std::max(1, std::min(S.ntiles, ctx->nsm * occ)), sm};
}
static int half_launches(const pdhg_ctx* ctx, bool dual) {
  if (ctx->opt.step_rule == 1) return dual ? 2 : 1;
  return dual ? dual_launches(ctx) : prim_launches(ctx);
}

// Iteration schedules: every candidate is timed with the real fused primal
// (rows of A~^T) or dual (rows of A~) kernel on the initial state (with the
// adaptive step, its own half-steps: gathering two vectors changes which
// schedule wins); the state is zeroed again afterwards, and the step state
// the adaptive acceptance test changed is put back.  Candidates: the
// segmented kernel with 8, 16 or 32 nonzeros per thread (a vector kernel
// with -e lanes per row, e < 0, only when options.tile_nnz asks for it and
// all rows are short).  E = 8 is kept unless another choice is more than 5%
// faster, so timing noise does not flip the schedule from one context to the
// next.
template <typename T>
static pdhg_status time_iteration_kernel(pdhg_ctx* ctx, bool on_a, float* ms_out) {
  const IterBuffers<T> B = iter_buffers<T>(ctx);
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const int warm = 2, reps = 6;
  ctx->launches += (long long)(warm + reps) * half_launches(ctx, on_a);
  for (int it = 0; it < warm + reps; ++it) {
    if (it == warm) CK(cudaEventRecord(e0, ctx->stream));
    if (on_a)
      launch_dual_half<T>(ctx, B, 0);
    else
      launch_prim_half<T>(ctx, B, 0);
  }
  CK(cudaGetLastError());
  CK(cudaEventRecord(e1, ctx->stream));
  CK(cudaEventSynchronize(e1));
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms_out = ms / reps;
  return PDHG_OK;
}

// mean time of one whole iteration (primal then dual half-step) over 6,
// after 2 untimed
template <typename T>
static pdhg_status time_iterations(pdhg_ctx* ctx, float* ms_out) {
  const IterBuffers<T> B = iter_buffers<T>(ctx);
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const int warm = 2, reps = 6;
  ctx->launches += (long long)(warm + reps) * (prim_launches(ctx) + dual_launches(ctx));
  for (int it = 0; it < warm + reps; ++it) {
    if (it == warm) CK(cudaEventRecord(e0, ctx->stream));
    launch_prim_step<T>(ctx, B, 0);
    launch_dual_step<T>(ctx, B, 0);
  }
  CK(cudaGetLastError());
  CK(cudaEventRecord(e1, ctx->stream));
  CK(cudaEventSynchronize(e1));
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms_out = ms / reps;
  return PDHG_OK;
}

// mean nonzeros per row from which the tuner also tries 16 and 32 nonzeros
// per thread
constexpr int kLongWindowRows = 8;

static pdhg_status tune_schedules(pdhg_ctx* ctx) {
  const bool mx = ctx->mixed;
  Scalars sc0{};  // the adaptive acceptance test moves the step state while candidates run
  CK(cudaMemcpyAsync(&sc0, ctx->sc, sizeof(sc0), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  for (int which = 0; which < 2; ++which) {
    const bool on_a = which == 0;
    const std::vector<int32_t>& rp = on_a ? ctx->h_a_rp : ctx->h_t_rp;
    const int nrows = on_a ? ctx->m : ctx->n;
    int64_t longest = 0;
    for (int r = 0; r < nrows; ++r) longest = std::max<int64_t>(longest, rp[r + 1] - rp[r]);
    std::vector<std::pair<int, int>> cands;  // (variant, tile capacity; 0 = full)
    const int tn = ctx->opt.tile_nnz;
    if (tn < 0)  // forced vector variant (only where rows are short)
      cands.push_back({longest <= 256 ? (tn <= -8 ? -8 : -4) : 8, 0});
    else if (tn > 0)
      cands.push_back({tn <= 2044 ? 8 : (tn <= 4092 ? 16 : 32), tn});
    else if (ctx->opt.autotune && (int64_t)rp[nrows] >= (int64_t)kLongWindowRows * nrows) {
      // the vector variants were slower than E = 8 on every measured matrix
      // since the window words; they stay available through tile_nnz < 0.
      // E = 16 and 32 are tried only where rows average kLongWindowRows
      // nonzeros or more: on shorter rows E = 8 won every measurement
      cands = {{8, 0}, {16, 0}, {32, 0}};
    } else {
      cands = {{8, 0}};
    }
    DevSched best{};
    float best_ms = 1e30f;
    for (const auto& cand : cands) {
      const int e = cand.first;
      DevSched d;
      if (e == kFixedE && cand.second == 0) {
        d = on_a ? ctx->sa8 : ctx->st8;
      } else {
        std::future<HostSched>& pre = ctx->presched[which][e == 16 ? 0 : 1];
        HostSched h = (cand.second == 0 && (e == 16 || e == 32) && pre.valid())
                          ? pre.get()
                          : build_sched(rp.data(), nrows, e, nullptr, 1, cand.second);
        CKS(upload_sched(ctx, h, &d, on_a ? ctx->a_rp : ctx->t_rp));
      }
      (on_a ? ctx->sa : ctx->st) = d;
      if (on_a)
        ctx->l_dual = make_launch(ctx, dual_kind(ctx), d.view.e,
                                  smem_for(0, mx, d.view.max_rows, d.view.e), d.view.ntiles);
      else
        ctx->l_prim = make_launch(ctx, prim_kind(ctx), d.view.e,
                                  smem_for(0, mx, d.view.max_rows, d.view.e), d.view.ntiles);
      set_adaptive_launch(ctx, on_a, d.view);
      float ms = 0.f;
      if (cands.size() > 1) {
        if (mx)
          CKS(time_iteration_kernel<float>(ctx, on_a, &ms));
        else
          CKS(time_iteration_kernel<double>(ctx, on_a, &ms));
      }
      const float bias = (e == 8) ? 0.95f : 1.0f;
      if (ctx->opt.verbose)
        std::fprintf(stderr, "pdhg_create: tune %s variant %3d cap %5d: %8.4f ms\n",
                     on_a ? "A  " : "A^T", e, d.view.tile_nnz, ms);
      if (ms * bias < best_ms) {
        best_ms = ms * bias;
        best = d;
      }
    }
    (on_a ? ctx->sa : ctx->st) = best;
    if (on_a)
      ctx->l_dual = make_launch(ctx, dual_kind(ctx), best.view.e,
                                smem_for(0, mx, best.view.max_rows, best.view.e), best.view.ntiles);
    else
      ctx->l_prim = make_launch(ctx, prim_kind(ctx), best.view.e,
                                smem_for(0, mx, best.view.max_rows, best.view.e), best.view.ntiles);
    set_adaptive_launch(ctx, on_a, best.view);

    // column panels where they apply: forced (spmv_layout 2), or candidates
    // timed below against the CSR tiles picked above (autotune on, tile_nnz 0,
    // and at least 2^20 nonzeros: below that the gathered vectors live in L1/L2
    // anyway and building the panels costs more create time than it saves)
    const int lay = ctx->opt.spmv_layout;
    int pw = 0, np = 0;
    const bool auto_panels = lay == 0 && ctx->opt.autotune && ctx->opt.tile_nnz == 0 &&
                             ctx->opt.step_rule == 0 && ctx->nnz >= (int64_t(1) << 20);
    if ((lay == 2 || auto_panels) && panel_shape(ctx, on_a, &pw, &np)) {
      DevPanel& dp = on_a ? ctx->pa : ctx->pt;
      CKS(build_panel_layout(ctx, on_a, &dp));
      const int rows = on_a ? ctx->m : ctx->n;
      (on_a ? ctx->panel_row_grid_a : ctx->panel_row_grid_t) =
          panel_row_grid(rows, dp.view.npanels, ctx->nsm);
    }
  }
  // With panel candidates: whole iterations (both half-steps in turn, as the
  // solve runs them, so each matrix streams from where the other left the
  // L2) for every CSR / panel combination; the fastest is kept.
  if (ctx->opt.spmv_layout == 0 && (ctx->pa.on || ctx->pt.on)) {
    const bool ca = ctx->pa.on, ct = ctx->pt.on;
    float best = 1e30f;
    int best_combo = 0;
    for (int combo = 0; combo < 4; ++combo) {
      const bool ua = combo & 1, ut = (combo >> 1) & 1;
      if ((ua && !ca) || (ut && !ct)) continue;
      ctx->pa.on = ua;
      ctx->pt.on = ut;
      float ms = 0.f;
      CKS(time_iterations<float>(ctx, &ms));
      if (ctx->opt.verbose)
        std::fprintf(stderr, "pdhg_create: tune iteration A %s, A^T %s: %8.4f ms\n",
                     ua ? "panels" : "CSR   ", ut ? "panels" : "CSR   ", ms);
      if (ms < best) {
        best = ms;
        best_combo = combo;
      }
    }
    ctx->pa.on = (best_combo & 1) != 0;
    ctx->pt.on = ((best_combo >> 1) & 1) != 0;
  }
  const SchedView &A = ctx->sa.view, &T = ctx->st.view;
  ctx->l_prim = make_launch(ctx, prim_kind(ctx), T.e, smem_for(0, mx, T.max_rows, T.e), T.ntiles);
  ctx->l_dual = make_launch(ctx, dual_kind(ctx), A.e, smem_for(0, mx, A.max_rows, A.e), A.ntiles);
  {
    const size_t sm = smem_for(1, mx, T.max_rows, T.e);
    const int occ = tile_occupancy(mx ? 4 : 5, T.e, sm);
    // the eval kernel also walks the m rows elementwise: at least enough blocks for that
    int grid = std::max(T.ntiles, (ctx->m + kBlock - 1) / kBlock);
    grid = std::max(1, std::min(grid, ctx->nsm * occ));
    ctx->l_eval = Launch{grid, sm};
  }
  // the tuning launches moved the iterate: back to x = 0, y = 0
  const size_t es = elem(ctx);
  for (void* p : {ctx->x, ctx->x_avg, ctx->x_last})
    CK(cudaMemsetAsync(p, 0, es * ctx->n, ctx->stream));
  for (void* p : {ctx->y, ctx->y_avg, ctx->y_last, ctx->Ax, ctx->Ax_avg, ctx->Ax_last})
    CK(cudaMemsetAsync(p, 0, es * ctx->m, ctx->stream));
  CK(cudaMemcpyAsync(ctx->sc, &sc0, sizeof(sc0), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return PDHG_OK;
}

static pdhg_status build_graphs(pdhg_ctx* ctx) {
  const int F = ctx->opt.eval_freq;
  for (int g = 0; g < 2; ++g) {
    if (ctx->chunk_exec[g]) continue;
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    const long long before = ctx->launches;
    enqueue_chunk_any(ctx, F, ctx->opt.kernel_timing ? ctx->ev_k[g] : nullptr);
    ctx->launches = before;  // captured, not launched
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
    if (e != cudaSuccess) {
      set_error("graph capture failed: %s", cudaGetErrorString(e));
      return PDHG_CUDA_ERROR;
    }
    CK(cudaGraphInstantiate(&ctx->chunk_exec[g], graph, 0));
    cudaGraphDestroy(graph);
  }
  return PDHG_OK;
}

size_t pdhg::elem(const pdhg_ctx* ctx) { return ctx->mixed ? sizeof(float) : sizeof(double); }

// ---------------------------------------------------------------------------
// create
// ---------------------------------------------------------------------------
extern "C" void pdhg_default_options(pdhg_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = PDHG_FP64;
  o->eval_freq = 64;
  o->ruiz_iters = 10;
  o->pock_chambolle = 1;
  o->eta_safety = 0.95;
  o->power_max_iter = 200;
  o->power_rel_tol = 1e-10;
  o->beta_sufficient = 0.2;
  o->beta_necessary = 0.8;
  o->beta_artificial = 0.36;
  o->theta = 0.5;
  o->io_on_device = 0;
  o->stream = nullptr;
  o->use_graphs = 1;
  o->autotune = 1;
  o->tile_nnz = 0;
  o->kernel_timing = 0;
  o->verbose = 0;
  o->method = 0;
  o->reflection = 1.0;
  o->spmv_layout = 0;
  o->panel_width = 0;
  o->fp32_screen = 1.0;
  o->omega_rule = 0;
  o->pid_kp = 0.99;
  o->pid_ki = 0.01;
  o->pid_kd = 0.0;
  o->persistent = 0;
  o->wait_limit_ms = 1000;
  o->wait_test = 0;
}

// device attributes, stream, kernel shared-memory limits
pdhg_status pdhg::setup_device(pdhg_ctx* ctx) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, dev));
  int optin = 0;
  CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  ctx->smem_optin = (size_t)optin;
  if (ctx->opt.stream) {
    ctx->stream = (cudaStream_t)ctx->opt.stream;
  } else {
    CK(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
    ctx->own_stream = true;
  }
  CK(configure_tile_kernels(ctx->smem_optin));
  CK(configure_halpern_kernels(ctx->smem_optin));
  CK(configure_adaptive_kernels(ctx->smem_optin));
  CK(configure_panel_kernels(ctx->smem_optin));
  CK(configure_setup_kernels(ctx->smem_optin));

  return PDHG_OK;
}

// every device array of the context (sizes m, n, nnz and count set)
pdhg_status pdhg::alloc_arrays(pdhg_ctx* ctx) {
  const int m = ctx->m, n = ctx->n;
  ctx->nnz_pad = (ctx->nnz + 7) / 4 * 4 + 4;
  const int64_t np = ctx->nnz_pad;
  CKS(dalloc(ctx, &ctx->a_rp, (size_t)m + 1));
  CKS(dalloc(ctx, &ctx->t_rp, (size_t)n + 1));
  CKS(dalloc(ctx, &ctx->a_col, np));
  CKS(dalloc(ctx, &ctx->t_col, np));
  CKS(dalloc(ctx, &ctx->a_val_orig, np));
  CKS(dalloc(ctx, &ctx->t_val_orig, np));
  CKS(dalloc(ctx, &ctx->a_val64, np));
  CKS(dalloc(ctx, &ctx->t_val64, np));
  if (ctx->mixed) {
    CKS(dalloc(ctx, &ctx->a_val32, np));
    CKS(dalloc(ctx, &ctx->t_val32, np));
    CKS(dalloc(ctx, &ctx->b_t32, m));
    CKS(dalloc(ctx, &ctx->c_t32, n));
  }
  CKS(dalloc(ctx, &ctx->b, m));
  CKS(dalloc(ctx, &ctx->c, n));
  CKS(dalloc(ctx, &ctx->b_t64, m));
  CKS(dalloc(ctx, &ctx->c_t64, n));
  CKS(dalloc(ctx, &ctx->D_r, m));
  CKS(dalloc(ctx, &ctx->D_c, n));
  CKS(dalloc(ctx, &ctx->Dr_inv, m));
  CKS(dalloc(ctx, &ctx->Dc_inv, n));
  const size_t es = elem(ctx);
  void** vecs_n[] = {&ctx->x, &ctx->x_avg, &ctx->x_last};
  void** vecs_m[] = {&ctx->y, &ctx->y_avg, &ctx->y_last, &ctx->Ax, &ctx->Ax_avg, &ctx->Ax_last};
  for (void** p : vecs_n) CKS(dalloc(ctx, (char**)p, es * n));
  for (void** p : vecs_m) CKS(dalloc(ctx, (char**)p, es * m));
  if (ctx->opt.step_rule == 1 && !ctx->batch) {
    CKS(dalloc(ctx, (char**)&ctx->x_avg_prev, es * n));
    CKS(dalloc(ctx, (char**)&ctx->adapt_xx, es * 2 * (size_t)n));
    CK(cudaMemsetAsync(ctx->adapt_xx, 0, es * 2 * (size_t)n, ctx->stream));
    for (void** p : {&ctx->y_prev, &ctx->y_avg_prev, &ctx->Ax_prev, &ctx->Ax_avg_prev})
      CKS(dalloc(ctx, (char**)p, es * m));
  }
  CKS(dalloc(ctx, &ctx->xs64, n));
  CKS(dalloc(ctx, &ctx->ys64, m));
  CKS(dalloc(ctx, &ctx->out_n1, n));
  CKS(dalloc(ctx, &ctx->out_n2, n));
  CKS(dalloc(ctx, &ctx->out_m1, m));
  CKS(dalloc(ctx, &ctx->report, 8));
  CKS(dalloc(ctx, &ctx->sums, 8));
  CKS(dalloc(ctx, &ctx->sc, (size_t)ctx->count));
  CKS(dalloc(ctx, &ctx->ps, (size_t)ctx->count));
  CKS(dalloc(ctx, &ctx->log_k, ctx->log_cap));
  CKS(dalloc(ctx, &ctx->log_flags, ctx->log_cap));
  CKS(dalloc(ctx, &ctx->log_kkt, 3 * (size_t)ctx->log_cap));

  return PDHG_OK;
}

// A (row pointer from ctx->h_a_rp), b, c onto the device
pdhg_status pdhg::upload_lp(pdhg_ctx* ctx, const int32_t* col, const double* val, const double* b,
                            const double* c) {
  const int m = ctx->m, n = ctx->n;
  const int64_t nnz = ctx->nnz, np = ctx->nnz_pad;
  CK(cudaMemsetAsync(ctx->a_col, 0, sizeof(int32_t) * np, ctx->stream));
  CK(cudaMemsetAsync(ctx->t_col, 0, sizeof(int32_t) * np, ctx->stream));
  CK(cudaMemsetAsync(ctx->a_val_orig, 0, sizeof(double) * np, ctx->stream));
  CK(cudaMemsetAsync(ctx->t_val_orig, 0, sizeof(double) * np, ctx->stream));
  CK(cudaMemsetAsync(ctx->a_val64, 0, sizeof(double) * np, ctx->stream));
  CK(cudaMemsetAsync(ctx->t_val64, 0, sizeof(double) * np, ctx->stream));
  if (ctx->mixed) {
    CK(cudaMemsetAsync(ctx->a_val32, 0, sizeof(float) * np, ctx->stream));
    CK(cudaMemsetAsync(ctx->t_val32, 0, sizeof(float) * np, ctx->stream));
  }
  CK(cudaMemcpyAsync(ctx->a_rp, ctx->h_a_rp.data(), sizeof(int32_t) * (m + 1),
                     cudaMemcpyHostToDevice, ctx->stream));
  CKS(copy_in(ctx, ctx->a_col, col, sizeof(int32_t) * nnz));
  CKS(copy_in(ctx, ctx->a_val_orig, val, sizeof(double) * nnz));
  CKS(copy_in(ctx, ctx->b, b, sizeof(double) * m));
  CKS(copy_in(ctx, ctx->c, c, sizeof(double) * n));

  return PDHG_OK;
}

// validation, a1 transpose, a2 scaling, scaled copies, zero iterate
pdhg_status pdhg::prepare_matrix(pdhg_ctx* ctx) {
  const int m = ctx->m, n = ctx->n;
  const int64_t nnz = ctx->nnz, np = ctx->nnz_pad;
  const size_t es = elem(ctx);
  void** vecs_n[] = {&ctx->x, &ctx->x_avg, &ctx->x_last};
  void** vecs_m[] = {&ctx->y, &ctx->y_avg, &ctx->y_last, &ctx->Ax, &ctx->Ax_avg, &ctx->Ax_last};
  int32_t* flags = nullptr;
  int32_t *cnt = nullptr, *tmp = nullptr;
  StageClock sub{ctx};  // verbose: the parts of this stage
  CKS(dalloc(ctx, &flags, 1));
  CKS(dalloc(ctx, &cnt, (size_t)n + 1));
  CKS(dalloc(ctx, &tmp, (size_t)n / 1024 + 8));
  // validation on device
  CK(cudaMemsetAsync(flags, 0, sizeof(int32_t), ctx->stream));
  launch_validate(m, n, ctx->a_rp, ctx->a_col, ctx->a_val_orig, ctx->b, ctx->c, flags, ctx->stream);
  ctx->launches += 1;
  int32_t hflags = 0;
  CK(cudaMemcpyAsync(&hflags, flags, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (hflags) {
    set_error("invalid LP data (flags 0x%x: 1 column out of range, 2 columns not strictly "
              "increasing in a row, 4 non-finite A, 8 non-finite b, 16 non-finite c)",
              hflags);
    return PDHG_INVALID_ARG;
  }
  sub("  validation");

  // a1: stable transpose A -> A^T (original values)
  CK(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (n + 1), ctx->stream));
  launch_col_hist(nnz, ctx->a_col, cnt, ctx->stream);
  launch_scan(cnt, ctx->t_rp, n, tmp, ctx->stream);
  CK(cudaMemcpyAsync(cnt, ctx->t_rp, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, ctx->stream));
  launch_scatter(m, ctx->a_rp, ctx->a_col, ctx->a_val_orig, cnt, ctx->t_col, ctx->t_val_orig,
                 ctx->stream);
  ctx->launches += 1 + (n > 0 ? 3 : 0) + 1;  // histogram, scan, scatter
  ctx->h_t_rp.resize((size_t)n + 1);
  CK(cudaMemcpyAsync(ctx->h_t_rp.data(), ctx->t_rp, sizeof(int32_t) * (n + 1),
                     cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  {
    std::vector<int32_t> longs;
    for (int j = 0; j < n; ++j)
      if (ctx->h_t_rp[j + 1] - ctx->h_t_rp[j] > 32) longs.push_back(j);
    int32_t* d_ids = nullptr;
    int32_t* tk = nullptr;
    double* tv = nullptr;
    if (!longs.empty()) {
      CKS(dalloc(ctx, &d_ids, longs.size()));
      CKS(dalloc(ctx, &tk, np));
      CKS(dalloc(ctx, &tv, np));
      CK(cudaMemcpyAsync(d_ids, longs.data(), sizeof(int32_t) * longs.size(),
                         cudaMemcpyHostToDevice, ctx->stream));
    }
    launch_segsort(n, ctx->t_rp, ctx->t_col, ctx->t_val_orig, d_ids, (int)longs.size(), tk, tv,
                   ctx->stream);
    ctx->launches += longs.empty() ? 1 : 2;
    CK(cudaStreamSynchronize(ctx->stream));
  }
  CK(cudaGetLastError());
  sub("  transpose");

  // a2: Ruiz (infinity norm) then Pock-Chambolle (alpha = 1)
  RowStatPlan plan_a, plan_t;
  {
    constexpr int kLongRow = 1024;
    auto make_plan = [&](const std::vector<int32_t>& rp, int nrows, RowStatPlan* pl) -> pdhg_status {
      const double mean = nrows > 0 ? (double)rp[nrows] / nrows : 0.0;
      pl->lanes = mean <= 6 ? 4 : mean <= 12 ? 8 : mean <= 24 ? 16 : 32;
      pl->long_len = kLongRow;
      std::vector<int32_t> ids;
      for (int i = 0; i < nrows; ++i)
        if (rp[i + 1] - rp[i] > kLongRow) ids.push_back(i);
      pl->nlong = (int)ids.size();
      if (!ids.empty()) {
        int32_t* d = nullptr;
        CKS(dalloc(ctx, &d, ids.size()));
        CK(cudaMemcpyAsync(d, ids.data(), sizeof(int32_t) * ids.size(), cudaMemcpyHostToDevice,
                           ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));  // ids is a local vector
        pl->long_ids = d;
      }
      return PDHG_OK;
    };
    CKS(make_plan(ctx->h_a_rp, m, &plan_a));
    CKS(make_plan(ctx->h_t_rp, n, &plan_t));
  }
  sub("  row-length plans");
  double *r = ctx->out_m1, *s = ctx->out_n1;
  launch_fill(ctx->D_r, 1.0, m, ctx->stream);
  launch_fill(ctx->D_c, 1.0, n, ctx->stream);
  const int rounds = ctx->opt.ruiz_iters + (ctx->opt.pock_chambolle ? 1 : 0);
  for (int it = 0; it < rounds; ++it) {
    const int mode = it < ctx->opt.ruiz_iters ? 0 : 1;
    launch_row_stat(m, ctx->a_rp, ctx->a_col, ctx->a_val_orig, ctx->D_r, ctx->D_c, mode, r,
                    plan_a, ctx->stream);
    launch_row_stat(n, ctx->t_rp, ctx->t_col, ctx->t_val_orig, ctx->D_c, ctx->D_r, mode, s,
                    plan_t, ctx->stream);
    launch_div(ctx->D_r, r, m, ctx->stream);
    launch_div(ctx->D_c, s, n, ctx->stream);
  }
  sub("  scaling rounds");
  launch_scale_vals(m, ctx->a_rp, ctx->a_col, ctx->a_val_orig, ctx->D_r, ctx->D_c, 0,
                    ctx->a_val64, ctx->a_val32, ctx->stream);
  launch_scale_vals(n, ctx->t_rp, ctx->t_col, ctx->t_val_orig, ctx->D_r, ctx->D_c, 1,
                    ctx->t_val64, ctx->t_val32, ctx->stream);
  launch_scale_vec(m, ctx->D_r, ctx->b, ctx->b_t64, ctx->b_t32, ctx->stream);
  launch_scale_vec(n, ctx->D_c, ctx->c, ctx->c_t64, ctx->c_t32, ctx->stream);
  launch_recip(ctx->D_r, ctx->Dr_inv, m, ctx->stream);
  launch_recip(ctx->D_c, ctx->Dc_inv, n, ctx->stream);
  ctx->launches += 2;
  ctx->launches += 2 + 4LL * rounds + 4 +
                   (long long)rounds * ((plan_a.nlong > 0) + (plan_t.nlong > 0));
  CK(cudaGetLastError());

  // zero state (also what the autotuner multiplies)
  for (void** p : vecs_n) CK(cudaMemsetAsync(*p, 0, es * n, ctx->stream));
  for (void** p : vecs_m) CK(cudaMemsetAsync(*p, 0, es * m, ctx->stream));

  return PDHG_OK;
}

static pdhg_status create_impl(pdhg_ctx* ctx, const int32_t* row_ptr, const int32_t* col,
                               const double* val, const double* b, const double* c) {
  const int m = ctx->m, n = ctx->n;
  StageClock stage{ctx};
  CKS(setup_device(ctx));
  stage("device set-up");
  // row pointer on the host (scheduler) and its checks
  ctx->h_a_rp.resize((size_t)m + 1);
  if (ctx->opt.io_on_device) {
    CK(cudaMemcpyAsync(ctx->h_a_rp.data(), row_ptr, sizeof(int32_t) * (m + 1),
                       cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  } else {
    std::memcpy(ctx->h_a_rp.data(), row_ptr, sizeof(int32_t) * (m + 1));
  }
  if (ctx->h_a_rp[0] != 0) {
    set_error("row_ptr[0] must be 0");
    return PDHG_INVALID_ARG;
  }
  for (int i = 0; i < m; ++i)
    if (ctx->h_a_rp[i + 1] < ctx->h_a_rp[i]) {
      set_error("row_ptr decreases at row %d", i);
      return PDHG_INVALID_ARG;
    }
  ctx->nnz = ctx->h_a_rp[m];
  if (ctx->nnz > kMaxNnz) {
    set_error("nnz = %lld exceeds the limit %lld of the int32 tile indexing",
              (long long)ctx->nnz, (long long)kMaxNnz);
    return PDHG_INVALID_ARG;
  }

  stage("row pointer checks");
  CKS(alloc_arrays(ctx));
  stage("allocation");
  CKS(upload_lp(ctx, col, val, b, c));
  stage("upload");
  CKS(prepare_matrix(ctx));
  stage("validate/transpose/scale");

  // float64 schedules (the iteration schedules are tuned once the scalars exist)
  CKS(fixed_schedules(ctx));
  stage("float64 schedules");

  // the tuner's E = 16 and E = 32 schedules are host work: build them on a
  // host thread while the GPU runs the power iteration
  if (ctx->opt.autotune && ctx->opt.tile_nnz == 0) {
    for (int which = 0; which < 2; ++which)
      for (int q = 0; q < 2; ++q) {
        const int32_t* rp = which == 0 ? ctx->h_a_rp.data() : ctx->h_t_rp.data();
        const int nrows = which == 0 ? m : n;
        if ((int64_t)rp[nrows] < (int64_t)kLongWindowRows * nrows) continue;  // not tried
        const int e = q == 0 ? 16 : 32;
        ctx->presched[which][q] = std::async(std::launch::async, [rp, nrows, e] {
          return build_sched(rp, nrows, e, nullptr, 1, 0);
        });
      }
  }

  // a3: power iteration on A~^T A~ (float64)
  {
    double *v = ctx->xs64, *u = ctx->ys64, *w = ctx->out_n2;
    launch_pow_init(n, v, ctx->ps, ctx->opt.power_max_iter, ctx->opt.power_rel_tol, ctx->stream);
    ctx->launches += 1;
    // grids from the power kernels' own occupancy (the float64 report
    // kernel's, which l_a64 / l_t64 follow, holds more registers)
    const Launch la{std::max(1, std::min(ctx->sa8.view.ntiles, ctx->nsm * pow_occupancy(false, ctx->l_a64.smem))),
                    ctx->l_a64.smem};
    const Launch lt{std::max(1, std::min(ctx->st8.view.ntiles, ctx->nsm * pow_occupancy(true, ctx->l_t64.smem))),
                    ctx->l_t64.smem};
    for (int it = 0; it < ctx->opt.power_max_iter; ++it) {
      launch_pow_Av(ctx->sa8.view, ctx->a_rp, ctx->a_col, ctx->a_val64, v, u, ctx->ps, la,
                    ctx->stream);
      launch_pow_ATu(ctx->st8.view, ctx->t_rp, ctx->t_col, ctx->t_val64, u, v, w, ctx->partials,
                     ctx->ps, lt, ctx->stream);
      launch_pow_norm(n, w, v, ctx->ps, ctx->stream);
      ctx->launches += 3;
      if ((it & 15) == 15) {
        PowerState hp;
        CK(cudaMemcpyAsync(&hp, ctx->ps, sizeof(hp), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        if (hp.stopped) break;
      }
    }
    CK(cudaGetLastError());
  }
  stage("power iteration");

  // norms, omega_0, tau, sigma, first restart point
  {
    Scalars h{};
    h.eval_freq = ctx->opt.eval_freq;
    h.beta_suff = ctx->opt.beta_sufficient;
    h.beta_nec = ctx->opt.beta_necessary;
    h.beta_art = ctx->opt.beta_artificial;
    h.theta = ctx->opt.theta;
    h.omega_rule = ctx->opt.omega_rule;
    h.pid_kp = ctx->opt.pid_kp;
    h.pid_ki = ctx->opt.pid_ki;
    h.pid_kd = ctx->opt.pid_kd;
    h.step_rule = ctx->opt.step_rule;
    h.avg_w = 1.0;
    h.avg_first = 1;
    h.log_cap = ctx->log_cap;
    h.status = PDHG_MAX_ITER;
    CK(cudaMemcpyAsync(ctx->sc, &h, sizeof(h), cudaMemcpyHostToDevice, ctx->stream));
    const int g = 256;
    const double* srcs[5] = {ctx->b, ctx->c, ctx->b_t64, ctx->c_t64, ctx->c_t64};
    const int64_t lens[5] = {m, n, m, n, n};
    const int modes[5] = {1, 1, 1, 1, 2};
    for (int q = 0; q < 5; ++q) {
      launch_dot_partials(lens[q], srcs[q], nullptr, modes[q], ctx->partials, g, ctx->stream);
      launch_sum_final(ctx->partials, g, ctx->sums + q, ctx->stream);
    }
    launch_init_scalars(ctx->sc, ctx->sums, ctx->ps, ctx->opt.eta_safety, ctx->stream);
    ctx->launches += 11;
    Scalars hs;
    PowerState hp;
    CK(cudaMemcpyAsync(&hs, ctx->sc, sizeof(hs), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(&hp, ctx->ps, sizeof(hp), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->omega0 = hs.omega;
    ctx->power_iters = hp.k;
  }

  stage("scalars");
  CKS(tune_schedules(ctx));
  stage("schedule tuning");
  CKS(polling_resources(ctx));
  stage("polling resources");
  return PDHG_OK;
}

// events and pinned status copies of the chunked solve loop
pdhg_status pdhg::polling_resources(pdhg_ctx* ctx) {
  for (int g = 0; g < 2; ++g) {
    CK(cudaEventCreateWithFlags(&ctx->ev_done[g], cudaEventDisableTiming));
    CK(cudaMallocHost((void**)&ctx->h_sc[g], sizeof(Scalars)));
    for (int e = 0; e < 6; ++e) CK(cudaEventCreate(&ctx->ev_k[g][e]));
  }
  CK(cudaGetLastError());
  return PDHG_OK;
}

extern "C" pdhg_status pdhg_create(pdhg_ctx** out, int32_t m, int32_t n, const int32_t* row_ptr,
                                   const int32_t* col, const double* val, const double* b,
                                   const double* c, const pdhg_options* opt) {
  g_last_error.clear();
  if (!out) {
    set_error("out is NULL");
    return PDHG_INVALID_ARG;
  }
  *out = nullptr;
  if (m < 1 || n < 1 || !row_ptr || !b || !c) {
    set_error("need m >= 1, n >= 1 and non-NULL row_ptr, b, c");
    return PDHG_INVALID_ARG;
  }
  pdhg_ctx* ctx = new (std::nothrow) pdhg_ctx();
  if (!ctx) {
    set_error("out of host memory");
    return PDHG_OOM;
  }
  if (opt)
    ctx->opt = *opt;
  else
    pdhg_default_options(&ctx->opt);
  if (ctx->opt.eval_freq < 1 || ctx->opt.ruiz_iters < 0 || ctx->opt.power_max_iter < 0 ||
      (ctx->opt.precision != PDHG_FP64 && ctx->opt.precision != PDHG_FP32_MIXED) ||
      ctx->opt.tile_nnz < -8 || ctx->opt.tile_nnz > 8192 ||
      (ctx->opt.method != 0 && ctx->opt.method != 1) ||
      !(ctx->opt.reflection >= 0.0 && ctx->opt.reflection <= 1.0) ||
      ctx->opt.spmv_layout < 0 || ctx->opt.spmv_layout > 2 || ctx->opt.panel_width < 0 ||
      !(ctx->opt.fp32_screen >= 1.0 && ctx->opt.fp32_screen <= 1e6) ||
      (ctx->opt.omega_rule != 0 && ctx->opt.omega_rule != 1) ||
      !std::isfinite(ctx->opt.pid_kp) || !std::isfinite(ctx->opt.pid_ki) ||
      !std::isfinite(ctx->opt.pid_kd) || ctx->opt.wait_limit_ms < 1 ||
      (ctx->opt.wait_test != 0 && ctx->opt.wait_test != 1) ||
      (ctx->opt.step_rule != 0 && ctx->opt.step_rule != 1) ||
      (ctx->opt.step_rule == 1 && (ctx->opt.method != 0 || ctx->opt.spmv_layout == 2))) {
    set_error("invalid options (eval_freq >= 1, ruiz_iters >= 0, precision 0/1, "
              "-8 <= tile_nnz <= 8192, method 0/1, 0 <= reflection <= 1, spmv_layout 0..2, "
              "panel_width >= 0, 1 <= fp32_screen <= 1e6, omega_rule 0/1, finite PID gains, "
              "wait_limit_ms >= 1, wait_test 0/1, step_rule 0/1 (1: method 0, not spmv_layout 2))");
    delete ctx;
    return PDHG_INVALID_ARG;
  }
  ctx->m = m;
  ctx->n = n;
  ctx->mixed = ctx->opt.precision == PDHG_FP32_MIXED;
  pdhg_status st = PDHG_OK;
  if ((col == nullptr || val == nullptr) && row_ptr) {
    // an all-zero A is legal only with nnz = 0; checked after row_ptr is read
  }
  st = create_impl(ctx, row_ptr, col, val, b, c);
  if (st < 0) {
    const std::string msg = g_last_error;
    pdhg_destroy(ctx);
    g_last_error = msg;
    return st;
  }
  *out = ctx;
  return PDHG_OK;
}

extern "C" void pdhg_destroy(pdhg_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (int g = 0; g < 2; ++g) {
    if (ctx->chunk_exec[g]) cudaGraphExecDestroy(ctx->chunk_exec[g]);
    if (ctx->ev_done[g]) cudaEventDestroy(ctx->ev_done[g]);
    if (ctx->h_sc[g]) cudaFreeHost(ctx->h_sc[g]);
    for (int e = 0; e < 6; ++e)
      if (ctx->ev_k[g][e]) cudaEventDestroy(ctx->ev_k[g][e]);
  }
  pdhg_free_adjoint(ctx);
  for (void* p : ctx->allocs) cudaFree(p);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

// ---------------------------------------------------------------------------
// solve
// ---------------------------------------------------------------------------
extern "C" pdhg_status pdhg_solve(pdhg_ctx* ctx, double eps_rel, int64_t max_iter) {
  g_last_error.clear();
  if (!ctx) {
    set_error("ctx is NULL");
    return PDHG_INVALID_ARG;
  }  if (ctx->batch) {
    set_error("this entry point takes a single-LP context; use the pdhg_batch_* calls");
    return PDHG_INVALID_ARG;
  }

  if (!(eps_rel >= 0.0) || max_iter < 0) {
    set_error("need eps_rel >= 0 and max_iter >= 0");
    return PDHG_INVALID_ARG;
  }
  ctx->report_valid = false;
  Scalars hs;
  CK(cudaMemcpyAsync(&hs, ctx->sc, sizeof(hs), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  long long k = hs.k;
  if (k >= max_iter) {
    ctx->last_status = PDHG_MAX_ITER;
    return PDHG_MAX_ITER;
  }
  hs.eps = eps_rel;
  hs.max_iter = max_iter;
  hs.done = 0;
  hs.status = PDHG_MAX_ITER;
  hs.restart_pending = 0;
  hs.ticket = 0;
  hs.fp64_check = ctx->mixed ? 1 : 0;
  hs.screen = ctx->opt.fp32_screen;
  hs.verify = 0;
  hs.checks = 0;
  hs.rejects = 0;
  CK(cudaMemcpyAsync(ctx->sc, &hs, sizeof(hs), cudaMemcpyHostToDevice, ctx->stream));
  if (ctx->opt.use_graphs) CKS(build_graphs(ctx));
  for (double& v : ctx->timing_sum) v = 0.0;
  ctx->timing_n = 0;

  // Chunks are issued one ahead: after issuing chunk j the host waits for
  // chunk j-1's status copy, so the GPU always has queued work.  A chunk
  // issued after the device finished runs as no-op kernels.
  const long long F = ctx->opt.eval_freq;
  int slot = 0;
  bool pending[2] = {false, false}, sampled[2] = {false, false}, stop = false;
  long long expect_k[2] = {0, 0};
  auto drain = [&](int sl) -> pdhg_status {
    CK(cudaEventSynchronize(ctx->ev_done[sl]));
    pending[sl] = false;
    const Scalars* h = ctx->h_sc[sl];
    if (sampled[sl] && h->k == expect_k[sl]) {
      float t[4] = {0.f, 0.f, 0.f, 0.f};
      CK(cudaEventElapsedTime(&t[0], ctx->ev_k[sl][0], ctx->ev_k[sl][1]));
      CK(cudaEventElapsedTime(&t[1], ctx->ev_k[sl][1], ctx->ev_k[sl][2]));
      CK(cudaEventElapsedTime(&t[2], ctx->ev_k[sl][3], ctx->ev_k[sl][4]));
      CK(cudaEventElapsedTime(&t[3], ctx->ev_k[sl][4], ctx->ev_k[sl][5]));
      for (int q = 0; q < 4; ++q) ctx->timing_sum[q] += t[q];
      ctx->timing_n += 1;
    }
    sampled[sl] = false;
    if (h->done) stop = true;
    return PDHG_OK;
  };
  while (k < max_iter && !stop) {
    const long long next = std::min<long long>((k / F + 1) * F, max_iter);
    const int len = (int)(next - k);
    if (len == F && ctx->opt.use_graphs) {
      CK(cudaGraphLaunch(ctx->chunk_exec[slot], ctx->stream));
      ctx->launches += chunk_launches(ctx, (int)F);
      sampled[slot] = ctx->opt.kernel_timing != 0;
    } else {
      enqueue_chunk_any(ctx, len, nullptr);
      CK(cudaGetLastError());
      sampled[slot] = false;
    }
    CK(cudaMemcpyAsync(ctx->h_sc[slot], ctx->sc, sizeof(Scalars), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaEventRecord(ctx->ev_done[slot], ctx->stream));
    pending[slot] = true;
    expect_k[slot] = next;
    k = next;
    const int other = slot ^ 1;
    if (pending[other]) CKS(drain(other));
    slot = other;
  }
  for (int i = 0; i < 2; ++i) {
    const int sl = slot ^ 1 ^ i;  // the older pending chunk first
    if (pending[sl]) CKS(drain(sl));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaGetLastError());
  CK(cudaMemcpy(&hs, ctx->sc, sizeof(hs), cudaMemcpyDeviceToHost));
  ctx->last_status = hs.done ? hs.status : PDHG_MAX_ITER;
  if (!hs.done && hs.k >= max_iter) ctx->last_status = PDHG_MAX_ITER;
  if (ctx->panel_err) {
    int32_t perr = 0;
    CK(cudaMemcpy(&perr, ctx->panel_err, sizeof(perr), cudaMemcpyDeviceToHost));
    if (perr) {
      CK(cudaMemset(ctx->panel_err, 0, sizeof(int32_t)));
      set_error("a column-panel load waited longer than options.wait_limit_ms for its bulk "
                "copy; the iterate is not meaningful");
      ctx->last_status = PDHG_TIMEOUT;
    }
  }
  return (pdhg_status)ctx->last_status;
}

// ---------------------------------------------------------------------------
// report of the returned iterate (float64, original model)
// ---------------------------------------------------------------------------
static pdhg_status returned_iterate64(pdhg_ctx* ctx, const double** xs, const double** ys) {
  Scalars hs;
  CK(cudaMemcpyAsync(&hs, ctx->sc, sizeof(hs), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  const bool avg = hs.done && hs.status == PDHG_OK && hs.chosen_avg;
  void* xsrc = avg ? ctx->x_avg : ctx->x;
  void* ysrc = avg ? ctx->y_avg : ctx->y;
  if (ctx->mixed) {
    launch_convert_f2d((const float*)xsrc, ctx->xs64, ctx->n, ctx->stream);
    launch_convert_f2d((const float*)ysrc, ctx->ys64, ctx->m, ctx->stream);
    ctx->launches += 2;
    *xs = ctx->xs64;
    *ys = ctx->ys64;
  } else {
    *xs = (const double*)xsrc;
    *ys = (const double*)ysrc;
  }
  return PDHG_OK;
}

static pdhg_status compute_report(pdhg_ctx* ctx) {
  const double *xs, *ys;
  CKS(returned_iterate64(ctx, &xs, &ys));
  double* pn = ctx->partials;
  const int gn = ctx->l_t64.grid + ctx->st8.view.ngroups;
  double* pm = ctx->partials + 4 * (size_t)(gn + 1);
  const int gm = ctx->l_a64.grid + ctx->sa8.view.ngroups;
  launch_report_n(ctx->st8.view, ctx->t_rp, ctx->t_col, ctx->t_val64, xs, ys, ctx->c_t64, ctx->D_c,
                  ctx->out_n1, ctx->out_n2, pn, ctx->l_t64, ctx->stream);
  launch_report_m(ctx->sa8.view, ctx->a_rp, ctx->a_col, ctx->a_val64, xs, ys, ctx->b_t64, ctx->D_r,
                  ctx->out_m1, pm, ctx->l_a64, ctx->stream);
  launch_report_final(pn, gn, pm, gm, ctx->report, ctx->stream);
  ctx->launches += 3;
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(ctx->report_h, ctx->report, 8 * sizeof(double), cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->report_valid = true;
  return PDHG_OK;
}

extern "C" pdhg_status pdhg_get(pdhg_ctx* ctx, double* x, double* y, double* z, double* r_P,
                                double* r_D, double* gap) {
  g_last_error.clear();
  if (!ctx) {
    set_error("ctx is NULL");
    return PDHG_INVALID_ARG;
  }  if (ctx->batch) {
    set_error("this entry point takes a single-LP context; use the pdhg_batch_* calls");
    return PDHG_INVALID_ARG;
  }

  CKS(compute_report(ctx));
  CKS(copy_out(ctx, x, ctx->out_n1, sizeof(double) * ctx->n));
  CKS(copy_out(ctx, z, ctx->out_n2, sizeof(double) * ctx->n));
  CKS(copy_out(ctx, y, ctx->out_m1, sizeof(double) * ctx->m));
  CK(cudaStreamSynchronize(ctx->stream));
  if (r_P) *r_P = ctx->report_h[0];
  if (r_D) *r_D = ctx->report_h[1];
  if (gap) *gap = ctx->report_h[2];
  return PDHG_OK;
}

extern "C" pdhg_status pdhg_get_info(pdhg_ctx* ctx, int64_t* iters, int64_t* restarts,
                                     double* max_violation, int32_t* chosen_average,
                                     int32_t* last_status) {
  g_last_error.clear();
  if (!ctx) {
    set_error("ctx is NULL");
    return PDHG_INVALID_ARG;
  }
  Scalars hs;
  CK(cudaMemcpyAsync(&hs, ctx->sc, sizeof(hs), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (iters) *iters = hs.k;
  if (restarts) *restarts = hs.restarts;
  if (chosen_average) *chosen_average = (hs.done && hs.status == PDHG_OK) ? hs.chosen_avg : 0;
  if (last_status) *last_status = ctx->last_status;
  if (max_violation) {
    if (!ctx->report_valid) CKS(compute_report(ctx));
    *max_violation = ctx->report_h[3];
  }
  return PDHG_OK;
}

extern "C" pdhg_status pdhg_warmstart_point(pdhg_ctx* ctx, double mu_min, double delta_max,
                                            double alpha_min, int32_t unscaled, double* x_ws,
                                            double* y_ws, double* z_ws, double* mu_target) {
  g_last_error.clear();
  if (!ctx) {
    set_error("ctx is NULL");
    return PDHG_INVALID_ARG;
  }  if (ctx->batch) {
    set_error("this entry point takes a single-LP context; use the pdhg_batch_* calls");
    return PDHG_INVALID_ARG;
  }

  if (!(mu_min > 0.0) || !(delta_max >= 0.0) || !(alpha_min > 0.0)) {
    set_error("need mu_min > 0, delta_max >= 0, alpha_min > 0");
    return PDHG_INVALID_ARG;
  }
  const double *xs, *ys;
  CKS(returned_iterate64(ctx, &xs, &ys));
  double* zs = ctx->out_n2;
  double* mu = ctx->report + 7;
  launch_ws_z(ctx->st8.view, ctx->t_rp, ctx->t_col, ctx->t_val64, xs, ys, ctx->c_t64, zs,
              ctx->partials, ctx->l_t64, ctx->stream);
  launch_ws_mu(ctx->partials, ctx->l_t64.grid + ctx->st8.view.ngroups, ctx->n, mu_min, mu,
               ctx->stream);
  // outputs land in out_n1 (x'), out_m1 (y), and z' overwrites z~ in place
  launch_ws_apply(ctx->n, ctx->m, xs, zs, ys, mu, delta_max, alpha_min, unscaled, ctx->D_r,
                  ctx->D_c, ctx->out_n1, ctx->out_m1, zs, ctx->stream);
  ctx->launches += 3;
  CK(cudaGetLastError());
  CKS(copy_out(ctx, x_ws, ctx->out_n1, sizeof(double) * ctx->n));
  CKS(copy_out(ctx, y_ws, ctx->out_m1, sizeof(double) * ctx->m));
  CKS(copy_out(ctx, z_ws, zs, sizeof(double) * ctx->n));
  double hmu = 0;
  CK(cudaMemcpyAsync(&hmu, mu, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (mu_target) *mu_target = hmu;
  ctx->report_valid = false;  // report buffers were reused
  return PDHG_OK;
}

extern "C" pdhg_status pdhg_get_scaling(pdhg_ctx* ctx, double* D_r, double* D_c,
                                        double* sigma_max, double* eta, double* omega0,
                                        int32_t* power_iters) {
  g_last_error.clear();
  if (!ctx) {
    set_error("ctx is NULL");
    return PDHG_INVALID_ARG;
  }
  CKS(copy_out(ctx, D_r, ctx->D_r, sizeof(double) * ctx->m));
  CKS(copy_out(ctx, D_c, ctx->D_c, sizeof(double) * ctx->n));
  PowerState hp;
  Scalars hs;
  CK(cudaMemcpyAsync(&hp, ctx->ps, sizeof(hp), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(&hs, ctx->sc, sizeof(hs), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (sigma_max) *sigma_max = std::sqrt(std::max(hp.lam, 0.0));
  if (eta) *eta = hs.eta;
  if (omega0) *omega0 = ctx->omega0;
  if (power_iters) *power_iters = hp.k;
  return PDHG_OK;
}

extern "C" pdhg_status pdhg_get_transpose(pdhg_ctx* ctx, int32_t* row_ptr_t, int32_t* col_t,
                                          double* val_t) {
  g_last_error.clear();
  if (!ctx) {
    set_error("ctx is NULL");
    return PDHG_INVALID_ARG;
  }
  CKS(copy_out(ctx, row_ptr_t, ctx->t_rp, sizeof(int32_t) * ((size_t)ctx->n + 1)));
  CKS(copy_out(ctx, col_t, ctx->t_col, sizeof(int32_t) * ctx->nnz));
  CKS(copy_out(ctx, val_t, ctx->t_val_orig, sizeof(double) * ctx->nnz));
  CK(cudaStreamSynchronize(ctx->stream));
  return PDHG_OK;
}

// float64 host/device buffer <-> iterate buffer in the iteration precision
static pdhg_status state_out(pdhg_ctx* ctx, double* dst, const void* src, int len) {
  if (!dst) return PDHG_OK;
  if (ctx->mixed) {
    double* tmp = len == ctx->n ? ctx->xs64 : ctx->ys64;
    launch_convert_f2d((const float*)src, tmp, len, ctx->stream);
    return copy_out(ctx, dst, tmp, sizeof(double) * len);
  }
  return copy_out(ctx, dst, src, sizeof(double) * len);
}
static pdhg_status state_in(pdhg_ctx* ctx, void* dst, const double* src, int len) {
  if (!src) return PDHG_OK;
  if (ctx->mixed) {
    double* tmp = len == ctx->n ? ctx->xs64 : ctx->ys64;
    CKS(copy_in(ctx, tmp, src, sizeof(double) * len));
    launch_convert_d2f(tmp, (float*)dst, len, ctx->stream);
    CK(cudaStreamSynchronize(ctx->stream));
    return PDHG_OK;
  }
  return copy_in(ctx, dst, src, sizeof(double) * len);
}

extern "C" pdhg_status pdhg_get_state(pdhg_ctx* ctx, double* x, double* y, double* x_avg,
                                      double* y_avg, double* x_last, double* y_last,
                                      double* scalars) {
  g_last_error.clear();
  if (!ctx) {
    set_error("ctx is NULL");
    return PDHG_INVALID_ARG;
  }  if (ctx->batch) {
    set_error("this entry point takes a single-LP context; use the pdhg_batch_* calls");
    return PDHG_INVALID_ARG;
  }

  const int n = ctx->n, m = ctx->m;
  CKS(state_out(ctx, x, ctx->x, n));
  CK(cudaStreamSynchronize(ctx->stream));
  CKS(state_out(ctx, x_avg, ctx->x_avg, n));
  CK(cudaStreamSynchronize(ctx->stream));
  CKS(state_out(ctx, x_last, ctx->x_last, n));
  CK(cudaStreamSynchronize(ctx->stream));
  CKS(state_out(ctx, y, ctx->y, m));
  CK(cudaStreamSynchronize(ctx->stream));
  CKS(state_out(ctx, y_avg, ctx->y_avg, m));
  CK(cudaStreamSynchronize(ctx->stream));
  CKS(state_out(ctx, y_last, ctx->y_last, m));
  Scalars hs;
  CK(cudaMemcpyAsync(&hs, ctx->sc, sizeof(hs), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (scalars) {
    scalars[0] = hs.omega;
    scalars[1] = (double)hs.k;
    scalars[2] = (double)hs.t;
    scalars[3] = (double)hs.restarts;
    scalars[4] = hs.kkt_last;
    scalars[5] = hs.kkt_prev;
    scalars[6] = hs.eta;
    scalars[7] = 0.0;
  }
  return PDHG_OK;
}

extern "C" pdhg_status pdhg_set_state(pdhg_ctx* ctx, const double* x, const double* y,
                                      const double* x_avg, const double* y_avg,
                                      const double* x_last, const double* y_last,
                                      const double* scalars) {
  g_last_error.clear();
  if (!ctx || !x || !y || !x_avg || !y_avg || !x_last || !y_last || !scalars) {
    set_error("pdhg_set_state needs every argument");
    return PDHG_INVALID_ARG;
  }  if (ctx->batch) {
    set_error("this entry point takes a single-LP context; use the pdhg_batch_* calls");
    return PDHG_INVALID_ARG;
  }

  const int n = ctx->n, m = ctx->m;
  CKS(state_in(ctx, ctx->x, x, n));
  CKS(state_in(ctx, ctx->x_avg, x_avg, n));
  CKS(state_in(ctx, ctx->x_last, x_last, n));
  CKS(state_in(ctx, ctx->y, y, m));
  CKS(state_in(ctx, ctx->y_avg, y_avg, m));
  CKS(state_in(ctx, ctx->y_last, y_last, m));
  // caches A~x, A~x_avg and A~x_last in the iteration precision
  for (auto pr : {std::make_pair(ctx->x, ctx->Ax), std::make_pair(ctx->x_avg, ctx->Ax_avg),
                  std::make_pair(ctx->x_last, ctx->Ax_last)}) {
    if (ctx->mixed)
      launch_spmv<float>(ctx->sa.view, ctx->a_rp, ctx->a_col, ctx->a_val32,
                         (const float*)pr.first, (float*)pr.second, ctx->l_dual, ctx->stream);
    else
      launch_spmv<double>(ctx->sa.view, ctx->a_rp, ctx->a_col, ctx->a_val64,
                          (const double*)pr.first, (double*)pr.second, ctx->l_dual, ctx->stream);
  }
  ctx->launches += 3;
  Scalars hs;
  CK(cudaMemcpyAsync(&hs, ctx->sc, sizeof(hs), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  hs.omega = scalars[0];
  hs.k = (long long)scalars[1];
  hs.t = (long long)scalars[2];
  hs.restarts = (long long)scalars[3];
  hs.kkt_last = scalars[4];
  hs.kkt_prev = scalars[5];
  hs.tau = hs.eta / hs.omega;
  hs.sigma = hs.eta * hs.omega;
  hs.done = 0;
  hs.restart_pending = 0;
  hs.ticket = 0;
  CK(cudaMemcpyAsync(ctx->sc, &hs, sizeof(hs), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaGetLastError());
  ctx->report_valid = false;
  return PDHG_OK;
}

extern "C" pdhg_status pdhg_get_caches(pdhg_ctx* ctx, double* Ax, double* Ax_avg,
                                       double* Ax_last) {
  g_last_error.clear();
  if (!ctx || ctx->batch) {
    set_error("pdhg_get_caches needs a single-LP context");
    return PDHG_INVALID_ARG;
  }
  const int m = ctx->m;
  CKS(state_out(ctx, Ax, ctx->Ax, m));
  CKS(state_out(ctx, Ax_avg, ctx->Ax_avg, m));
  CKS(state_out(ctx, Ax_last, ctx->Ax_last, m));
  CK(cudaStreamSynchronize(ctx->stream));
  return PDHG_OK;
}

extern "C" pdhg_status pdhg_set_caches(pdhg_ctx* ctx, const double* Ax, const double* Ax_avg,
                                       const double* Ax_last) {
  g_last_error.clear();
  if (!ctx || ctx->batch) {
    set_error("pdhg_set_caches needs a single-LP context");
    return PDHG_INVALID_ARG;
  }
  const int m = ctx->m;
  CKS(state_in(ctx, ctx->Ax, Ax, m));
  CKS(state_in(ctx, ctx->Ax_avg, Ax_avg, m));
  CKS(state_in(ctx, ctx->Ax_last, Ax_last, m));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->report_valid = false;
  return PDHG_OK;
}

extern "C" pdhg_status pdhg_get_log(pdhg_ctx* ctx, int32_t cap, int32_t* count, int64_t* k,
                                    int32_t* flags, double* kkt) {
  g_last_error.clear();
  if (!ctx || cap < 0) {
    set_error("ctx is NULL or cap < 0");
    return PDHG_INVALID_ARG;
  }
  Scalars hs;
  CK(cudaMemcpyAsync(&hs, ctx->sc, sizeof(hs), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  const int cnt = std::min(cap, hs.log_count);
  if (count) *count = hs.log_count;
  if (cnt > 0) {
    if (k) CK(cudaMemcpy(k, ctx->log_k, sizeof(int64_t) * cnt, cudaMemcpyDeviceToHost));
    if (flags) CK(cudaMemcpy(flags, ctx->log_flags, sizeof(int32_t) * cnt, cudaMemcpyDeviceToHost));
    if (kkt) CK(cudaMemcpy(kkt, ctx->log_kkt, sizeof(double) * 3 * cnt, cudaMemcpyDeviceToHost));
  }
  return PDHG_OK;
}

extern "C" pdhg_status pdhg_get_kernel_timing(pdhg_ctx* ctx, double* primal_ms, double* dual_ms,
                                              int64_t* samples) {
  g_last_error.clear();
  if (!ctx) {
    set_error("ctx is NULL");
    return PDHG_INVALID_ARG;
  }
  const double nn = ctx->timing_n > 0 ? (double)ctx->timing_n : 1.0;
  if (primal_ms) *primal_ms = (ctx->timing_sum[0] + ctx->timing_sum[1]) / nn;
  if (dual_ms) *dual_ms = (ctx->timing_sum[2] + ctx->timing_sum[3]) / nn;
  if (samples) *samples = ctx->timing_n;
  return PDHG_OK;
}

extern "C" pdhg_status pdhg_get_kernel_timing_parts(pdhg_ctx* ctx, double* ms, int64_t* samples) {
  if (!ctx) {
    set_error("ctx is NULL");
    return PDHG_INVALID_ARG;
  }
  const double nn = ctx->timing_n > 0 ? (double)ctx->timing_n : 1.0;
  if (ms)
    for (int q = 0; q < 4; ++q) ms[q] = ctx->timing_sum[q] / nn;
  if (samples) *samples = ctx->timing_n;
  return PDHG_OK;
}

// Mean duration of back-to-back launches of each half-step on the context's
// current state (the solver state is saved first and restored after).
template <typename T>
static pdhg_status time_kernels_impl(pdhg_ctx* ctx, int reps, double* ms) {
  const IterBuffers<T> B = iter_buffers<T>(ctx);
  const size_t es = sizeof(T), n = (size_t)ctx->n, m = (size_t)ctx->m;
  // what a half-step writes: x, x_avg (n side); y, y_avg, Ax, Ax_avg (m side)
  void* nvec[2] = {ctx->x, ctx->x_avg};
  void* mvec[4] = {ctx->y, ctx->y_avg, ctx->Ax, ctx->Ax_avg};
  char* save = nullptr;
  const size_t bytes = es * (2 * n + 4 * m) + sizeof(Scalars);
  CK(cudaMalloc(&save, bytes));
  struct Free {
    char* p;
    ~Free() { cudaFree(p); }
  } guard{save};
  auto snapshot = [&](bool restore) -> pdhg_status {
    size_t off = 0;
    for (void* v : nvec) {
      CK(restore ? cudaMemcpyAsync(v, save + off, es * n, cudaMemcpyDeviceToDevice, ctx->stream)
                 : cudaMemcpyAsync(save + off, v, es * n, cudaMemcpyDeviceToDevice, ctx->stream));
      off += es * n;
    }
    for (void* v : mvec) {
      CK(restore ? cudaMemcpyAsync(v, save + off, es * m, cudaMemcpyDeviceToDevice, ctx->stream)
                 : cudaMemcpyAsync(save + off, v, es * m, cudaMemcpyDeviceToDevice, ctx->stream));
      off += es * m;
    }
    CK(restore ? cudaMemcpyAsync(ctx->sc, save + off, sizeof(Scalars), cudaMemcpyDeviceToDevice,
                                 ctx->stream)
               : cudaMemcpyAsync(save + off, ctx->sc, sizeof(Scalars), cudaMemcpyDeviceToDevice,
                                 ctx->stream));
    return PDHG_OK;
  };
  CKS(snapshot(false));
  // the kernels do nothing once a solve has finished: run them as mid-solve
  Scalars hs;
  CK(cudaMemcpyAsync(&hs, ctx->sc, sizeof(hs), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  hs.done = 0;
  hs.verify = 0;
  CK(cudaMemcpyAsync(ctx->sc, &hs, sizeof(hs), cudaMemcpyHostToDevice, ctx->stream));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  // which: 0 primal half-step, 1 dual, 2 iteration, 3 primal panel SpMV, 4 dual panel SpMV
  // (the half-steps the solve runs: with the adaptive step, its own kernels)
  auto run = [&](int which) {
    switch (which) {
      case 0: launch_prim_half<T>(ctx, B, 0); break;
      case 1: launch_dual_half<T>(ctx, B, 0); break;
      case 2:
        launch_prim_half<T>(ctx, B, 0);
        launch_dual_half<T>(ctx, B, 0);
        break;
      case 3:
        if constexpr (sizeof(T) == 4) launch_panel_spmv_only(B, ctx->pt.view, false, ctx->opt.method, ctx->stream);
        break;
      default:
        if constexpr (sizeof(T) == 4) launch_panel_spmv_only(B, ctx->pa.view, true, ctx->opt.method, ctx->stream);
        break;
    }
  };
  const int warm = 3;
  pdhg_status st = PDHG_OK;
  for (int which = 0; which < 5 && st == PDHG_OK; ++which) {
    ms[which] = 0.0;
    if ((which == 3 && !(ctx->mixed && ctx->pt.on)) || (which == 4 && !(ctx->mixed && ctx->pa.on)))
      continue;
    const bool ad = ctx->opt.step_rule == 1;
    const long long np = ad ? 1 : prim_launches(ctx), nd = ad ? 2 : dual_launches(ctx);
    const long long per = which == 0 ? np : which == 1 ? nd : which == 2 ? np + nd : 1;
    ctx->launches += per * (warm + reps);
    for (int it = 0; it < warm + reps; ++it) {
      if (it == warm) cudaEventRecord(e0, ctx->stream);
      run(which);
    }
    cudaEventRecord(e1, ctx->stream);
    cudaError_t e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
      set_error("kernel timing: %s", cudaGetErrorString(e));
      st = PDHG_CUDA_ERROR;
      break;
    }
    ms[which] = (double)t / reps;
    // the next measurement starts from the same state, again as mid-solve
    if (snapshot(true) != PDHG_OK ||
        cudaMemcpyAsync(ctx->sc, &hs, sizeof(hs), cudaMemcpyHostToDevice, ctx->stream) !=
            cudaSuccess)
      st = PDHG_CUDA_ERROR;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CKS(st);
  CKS(snapshot(true));
  CK(cudaStreamSynchronize(ctx->stream));
  return PDHG_OK;
}

extern "C" pdhg_status pdhg_time_kernels(pdhg_ctx* ctx, int32_t reps, double* ms) {
  g_last_error.clear();
  if (!ctx || ctx->batch || reps < 1 || !ms) {
    set_error("need a single-LP context, reps >= 1 and ms[5]");
    return PDHG_INVALID_ARG;
  }
  return ctx->mixed ? time_kernels_impl<float>(ctx, reps, ms) : time_kernels_impl<double>(ctx, reps, ms);
}

extern "C" pdhg_status pdhg_get_schedule(pdhg_ctx* ctx, int32_t* a_tile_nnz, int32_t* a_block,
                                         int32_t* a_tiles, int32_t* at_tile_nnz,
                                         int32_t* at_block, int32_t* at_tiles,
                                         int32_t* a_variant, int32_t* at_variant) {
  g_last_error.clear();
  if (!ctx) {
    set_error("ctx is NULL");
    return PDHG_INVALID_ARG;
  }
  if (a_tile_nnz) *a_tile_nnz = ctx->sa.view.tile_nnz;
  if (a_block) *a_block = kBlock;
  if (a_tiles) *a_tiles = ctx->sa.view.ntiles;
  if (at_tile_nnz) *at_tile_nnz = ctx->st.view.tile_nnz;
  if (at_block) *at_block = kBlock;
  if (at_tiles) *at_tiles = ctx->st.view.ntiles;
  if (a_variant) *a_variant = ctx->sa.view.e;
  if (at_variant) *at_variant = ctx->st.view.e;
  return PDHG_OK;
}

extern "C" pdhg_status pdhg_get_pid_state(pdhg_ctx* ctx, double* integral, double* prev_error) {
  g_last_error.clear();
  if (!ctx || ctx->batch) {
    set_error("need a single-LP context");
    return PDHG_INVALID_ARG;
  }
  Scalars hs;
  CK(cudaMemcpyAsync(&hs, ctx->sc, sizeof(hs), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (integral) *integral = hs.pid_integral;
  if (prev_error) *prev_error = hs.pid_prev;
  return PDHG_OK;
}

extern "C" pdhg_status pdhg_set_pid_state(pdhg_ctx* ctx, double integral, double prev_error) {
  g_last_error.clear();
  if (!ctx || ctx->batch || !std::isfinite(integral) || !std::isfinite(prev_error)) {
    set_error("need a single-LP context and finite values");
    return PDHG_INVALID_ARG;
  }
  Scalars hs;
  CK(cudaMemcpyAsync(&hs, ctx->sc, sizeof(hs), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  hs.pid_integral = integral;
  hs.pid_prev = prev_error;
  CK(cudaMemcpyAsync(ctx->sc, &hs, sizeof(hs), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return PDHG_OK;
}

extern "C" pdhg_status pdhg_get_step_state(pdhg_ctx* ctx, double* eta, double* eta_sum,
                                           int64_t* rejects) {
  g_last_error.clear();
  if (!ctx || ctx->batch) {
    set_error("need a single-LP context");
    return PDHG_INVALID_ARG;
  }
  Scalars hs;
  CK(cudaMemcpyAsync(&hs, ctx->sc, sizeof(hs), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (eta) *eta = hs.eta;
  if (eta_sum) *eta_sum = hs.eta_sum;
  if (rejects) *rejects = hs.step_rejects;
  return PDHG_OK;
}

extern "C" pdhg_status pdhg_set_step_state(pdhg_ctx* ctx, double eta, double eta_sum) {
  g_last_error.clear();
  if (!ctx || ctx->batch || !(eta > 0.0) || !std::isfinite(eta) || !(eta_sum >= 0.0) ||
      !std::isfinite(eta_sum)) {
    set_error("need a single-LP context, eta > 0 and eta_sum >= 0, both finite");
    return PDHG_INVALID_ARG;
  }
  Scalars hs;
  CK(cudaMemcpyAsync(&hs, ctx->sc, sizeof(hs), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  hs.eta = eta;
  hs.eta_sum = eta_sum;
  hs.tau = eta / hs.omega;
  hs.sigma = eta * hs.omega;
  hs.avg_w = eta / (eta_sum + eta);
  hs.avg_first = eta_sum == 0.0 ? 1 : 0;
  CK(cudaMemcpyAsync(ctx->sc, &hs, sizeof(hs), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return PDHG_OK;
}

extern "C" pdhg_status pdhg_get_fp64_checks(pdhg_ctx* ctx, int64_t* checks, int64_t* rejects) {
  g_last_error.clear();
  if (!ctx) {
    set_error("ctx is NULL");
    return PDHG_INVALID_ARG;
  }
  std::vector<Scalars> hs((size_t)ctx->count);
  CK(cudaMemcpyAsync(hs.data(), ctx->sc, sizeof(Scalars) * hs.size(), cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  long long c = 0, r = 0;
  for (const Scalars& s : hs) {
    c += s.checks;
    r += s.rejects;
  }
  if (checks) *checks = c;
  if (rejects) *rejects = r;
  return PDHG_OK;
}

extern "C" pdhg_status pdhg_get_layout(pdhg_ctx* ctx, int64_t* panels, int64_t* panel_width,
                                       int64_t* pseudo_rows, int64_t* tiles) {
  if (!ctx) {
    set_error("ctx is NULL");
    return PDHG_INVALID_ARG;
  }
  const DevPanel* d[2] = {&ctx->pa, &ctx->pt};
  for (int k = 0; k < 2; ++k) {
    const bool on = d[k]->on;
    if (panels) panels[k] = on ? d[k]->view.npanels : 0;
    if (panel_width) panel_width[k] = on ? d[k]->view.P : 0;
    if (pseudo_rows) pseudo_rows[k] = on ? d[k]->pseudo_rows : 0;
    if (tiles) tiles[k] = on ? d[k]->view.ntiles : 0;
  }
  return PDHG_OK;
}

extern "C" pdhg_status pdhg_gather_floor(pdhg_ctx* ctx, int32_t on_a, int32_t reps, double* ms) {
  g_last_error.clear();
  if (!ctx || !ms || reps < 1) {
    set_error("need ctx, ms and reps >= 1");
    return PDHG_INVALID_ARG;
  }
  if (ctx->batch) {
    set_error("this entry point takes a single-LP context");
    return PDHG_INVALID_ARG;
  }
  const int32_t* col = on_a ? ctx->a_col : ctx->t_col;
  const void* val = ctx->mixed ? (const void*)(on_a ? ctx->a_val32 : ctx->t_val32)
                               : (const void*)(on_a ? ctx->a_val64 : ctx->t_val64);
  const void* v = on_a ? ctx->x : ctx->y;  // the gathered vector of that half-step
  const int grid = ctx->nsm * 8;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  for (int it = 0; it < reps + 2; ++it) {
    if (it == 2) CK(cudaEventRecord(e0, ctx->stream));
    if (ctx->mixed)
      launch_gather_floor<float>(col, (const float*)val, (const float*)v, ctx->nnz,
                                 (float*)ctx->out_m1, grid, ctx->stream);
    else
      launch_gather_floor<double>(col, (const double*)val, (const double*)v, ctx->nnz,
                                  (double*)ctx->out_m1, grid, ctx->stream);
  }
  ctx->launches += reps + 2;
  CK(cudaGetLastError());
  CK(cudaEventRecord(e1, ctx->stream));
  CK(cudaEventSynchronize(e1));
  float t = 0.f;
  CK(cudaEventElapsedTime(&t, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = (double)t / reps;
  return PDHG_OK;
}

extern "C" pdhg_status pdhg_get_launch_count(pdhg_ctx* ctx, int64_t* launches) {
  g_last_error.clear();
  if (!ctx || !launches) {
    set_error("ctx or launches is NULL");
    return PDHG_INVALID_ARG;
  }
  *launches = ctx->launches;
  return PDHG_OK;
}
