// Differentiation through the converged batch solution by the active-set
// fixed point of the projected primal step.
//
// At a PDHG fixed point x = max(0, x - tau (c - A^T y)) the positive
// entries B satisfy A_B x_B = b and x_j = 0 off B, so (with B fixed) x_B is
// the least-squares solution of A_B x_B = b and does not move with c.  From an
// approximate iterate (possibly the running average) B is predicted by
// complementarity in the scaled model: B = {j : x~_j > z~_j}, z~ =
// max(0, c~ - A~^T y~).  For a loss L(x):
//   dL/db = A_B (A_B^T A_B)^{-1} g_B,  g = dL/dx,   dL/dc = 0.
// The polish solves A_B x_B = b (consistent, so any row weighting gives the
// same x_B) in the scaled model, which is better conditioned: CG on
// A~_B^T A~_B x~_B = A~_B^T b~ warm-started at the PDHG iterate.  The adjoint
// is the min-norm Jacobian A_B (A_B^T A_B)^{-1}, which a row weighting would
// change off range(A_B), so its CG runs on the original A:
// A_B^T A_B w = g_B, dL/db = A_B w.  Products use the tile SpMV kernels
// (float64).
#include <cmath>
#include <cstring>

#include "context.h"

namespace pdhg {

struct CgState {
  double rr, rr0, pq, alpha, beta, tol2;
  int32_t iters, max_iter, done, pad;
};

// mask of B = {j : x~_j > z~_j} and its size per LP (z~ through the tiles)
template <int BLOCK>
struct MaskEpi {
  const double *x_s, *c_t;
  const Scalars* sc;
  double *mask, *rec, *red;
  double cnt, unused;
  __device__ __forceinline__ bool begin_tile(const Tile&) {
    cnt = 0.0;
    return true;
  }
  __device__ __forceinline__ void row(int j, const double (&s)[1], int) {
    const bool in = x_s[j] > fmax(0.0, c_t[j] - s[0]);
    mask[j] = in ? 1.0 : 0.0;
    cnt += in ? 1.0 : 0.0;
  }
  __device__ __forceinline__ void end_tile(const Tile&, int t) {
    const double v[1] = {cnt};
    double o[1];
    block_sum<BLOCK, 1>(v, o, red);
    if (threadIdx.x == 0) rec[t] = o[0];
  }
};

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_adj_mask(SchedView S, const int32_t* rp, const int32_t* col,
                                                   const double* val, const double* x_s,
                                                   const double* y_s, const double* c_t,
                                                   const Scalars* sc, double* mask, double* rec) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[BLOCK / 32];
  MaskEpi<BLOCK> epi{x_s, c_t, sc, mask, rec, red, 0.0, 0.0};
  Gather<double, 1> g{{y_s}};
  run_tiles<double, 1, BLOCK, kFixedE>(S, rp, col, val, g, epi, smem);
}

// u = A~ p  (p is zero off B); LPs whose CG is done are skipped
struct CgAvEpi {
  double* u;
  const CgState* cg;
  __device__ __forceinline__ bool begin_tile(const Tile& tl) { return !cg[tl.lp].done; }
  __device__ __forceinline__ void row(int i, const double (&s)[1], int) { u[i] = s[0]; }
};

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_cg_Av(SchedView S, const int32_t* rp, const int32_t* col,
                                                const double* val, const double* p, double* u,
                                                const CgState* cg) {
  extern __shared__ __align__(16) unsigned char smem[];
  CgAvEpi epi{u, cg};
  Gather<double, 1> g{{p}};
  run_tiles<double, 1, BLOCK, kFixedE>(S, rp, col, val, g, epi, smem);
}

// q = mask * (A~^T u); records p^T q per tile; the last block sets alpha
template <int BLOCK>
struct CgATuEpi {
  const double *mask, *p;
  double *q, *rec, *red;
  const CgState* cg;
  double pq;
  __device__ __forceinline__ bool begin_tile(const Tile& tl) {
    if (cg[tl.lp].done) return false;
    pq = 0.0;
    return true;
  }
  __device__ __forceinline__ void row(int j, const double (&s)[1], int) {
    const double v = mask[j] * s[0];
    q[j] = v;
    pq += p[j] * v;
  }
  __device__ __forceinline__ void end_tile(const Tile&, int t) {
    const double v[1] = {pq};
    double o[1];
    block_sum<BLOCK, 1>(v, o, red);
    if (threadIdx.x == 0) rec[t] = o[0];
  }
};

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_cg_ATu(SchedView S, const int32_t* rp, const int32_t* col,
                                                 const double* val, const double* u,
                                                 const double* mask, const double* p, double* q,
                                                 double* rec, CgState* cg, const int32_t* lp_tiles,
                                                 int count, int32_t* ticket, int set_alpha) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[BLOCK / 32];
  __shared__ int is_last;
  CgATuEpi<BLOCK> epi{mask, p, q, rec, red, cg, 0.0};
  Gather<double, 1> g{{u}};
  run_tiles<double, 1, BLOCK, kFixedE>(S, rp, col, val, g, epi, smem);
  if (!set_alpha) return;
  if (threadIdx.x == 0) {
    __threadfence();
    is_last = (atomicAdd(ticket, 1) == (int)gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  for (int l = threadIdx.x; l < count; l += BLOCK) {
    CgState& c = cg[l];
    if (c.done) continue;
    double s = 0.0;
#pragma unroll 4  // independent record loads in flight together
    for (int t = lp_tiles[l]; t < lp_tiles[l + 1]; ++t) s += __ldcg(rec + t);
    c.pq = s;
    c.alpha = s > 0.0 ? c.rr / s : 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) *ticket = 0;
}

// w += alpha p; r -= alpha q; rr per tile; the last block sets beta / done
__global__ void k_cg_update(SchedView S, double* w, double* r, const double* p, const double* q,
                            double* rec, CgState* cg, const int32_t* lp_tiles, int count,
                            int32_t* ticket, int32_t* active) {
  __shared__ double red[8];
  __shared__ int is_last, nact;
  for (int t = blockIdx.x; t < S.ntiles; t += gridDim.x) {
    const Tile tl = S.tiles[t];
    const CgState& c = cg[tl.lp];
    if (c.done) continue;
    double acc = 0.0;
    if (tl.split < 0 || tl.part == 0) {
      const double a = c.alpha;
      for (int j = tl.row_begin + threadIdx.x; j < tl.row_end; j += blockDim.x) {
        w[j] += a * p[j];
        const double rn = r[j] - a * q[j];
        r[j] = rn;
        acc += rn * rn;
      }
    }
    const double v[1] = {acc};
    double o[1];
    block_sum<256, 1>(v, o, red);
    if (threadIdx.x == 0) rec[t] = o[0];
  }
  if (threadIdx.x == 0) {
    __threadfence();
    is_last = (atomicAdd(ticket, 1) == (int)gridDim.x - 1);
    nact = 0;
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  int mine = 0;
  for (int l = threadIdx.x; l < count; l += blockDim.x) {
    CgState& c = cg[l];
    if (c.done) continue;
    double s = 0.0;
#pragma unroll 4  // independent record loads in flight together
    for (int t = lp_tiles[l]; t < lp_tiles[l + 1]; ++t) s += __ldcg(rec + t);
    c.beta = c.rr > 0.0 ? s / c.rr : 0.0;
    c.rr = s;
    c.iters += 1;
    if (s <= c.tol2 * c.rr0 || c.iters >= c.max_iter || !(c.pq > 0.0)) c.done = 1;
    if (!c.done) ++mine;
  }
  atomicAdd(&nact, mine);
  __syncthreads();
  if (threadIdx.x == 0) {
    *active = nact;
    *ticket = 0;
  }
}

__global__ void k_cg_p(SchedView S, double* p, const double* r, const CgState* cg) {
  for (int t = blockIdx.x; t < S.ntiles; t += gridDim.x) {
    const Tile tl = S.tiles[t];
    const CgState& c = cg[tl.lp];
    if (c.done || (tl.split >= 0 && tl.part != 0)) continue;
    const double b = c.beta;
    for (int j = tl.row_begin + threadIdx.x; j < tl.row_end; j += blockDim.x) p[j] = r[j] + b * p[j];
  }
}

// CG start: r = rhs - q (q = M w0), p = r, rr = r^T r, rr0 = rhs^T rhs
__global__ void k_cg_start(SchedView S, const double* rhs, const double* q, double* r, double* p,
                           double* rec2) {
  __shared__ double red[2 * 8];
  for (int t = blockIdx.x; t < S.ntiles; t += gridDim.x) {
    const Tile tl = S.tiles[t];
    double a = 0.0, b = 0.0;
    if (tl.split < 0 || tl.part == 0) {
      for (int j = tl.row_begin + threadIdx.x; j < tl.row_end; j += blockDim.x) {
        const double rj = rhs[j] - q[j];
        r[j] = rj;
        p[j] = rj;
        a += rj * rj;
        b += rhs[j] * rhs[j];
      }
    }
    const double v[2] = {a, b};
    double o[2];
    block_sum<256, 2>(v, o, red);
    if (threadIdx.x == 0) {
      rec2[2 * (size_t)t] = o[0];
      rec2[2 * (size_t)t + 1] = o[1];
    }
  }
}

__global__ void k_cg_start_final(const double* rec2, const int32_t* lp_tiles, int count,
                                 CgState* cg, double tol, int max_iter) {
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < count; l += gridDim.x * blockDim.x) {
    double a = 0.0, b = 0.0;
#pragma unroll 4  // independent record loads in flight together
    for (int t = lp_tiles[l]; t < lp_tiles[l + 1]; ++t) {
      a += rec2[2 * (size_t)t];
      b += rec2[2 * (size_t)t + 1];
    }
    CgState& c = cg[l];
    c.rr = a;
    c.rr0 = b;
    c.tol2 = tol * tol;
    c.iters = 0;
    c.max_iter = max_iter;
    c.alpha = c.beta = c.pq = 0.0;
    c.done = (a <= c.tol2 * b || max_iter <= 0) ? 1 : 0;
  }
}

// elementwise helpers over the rows of a schedule (one pass per tile)
// mode 0: out = mask * a            1: out = mask * D * a
//      2: out = D * a (no mask)     3: out = 0        4: out = a
__global__ void k_adj_vec(SchedView S, int mode, const double* mask, const double* D,
                          const double* a, double* out) {
  for (int t = blockIdx.x; t < S.ntiles; t += gridDim.x) {
    const Tile tl = S.tiles[t];
    if (tl.split >= 0 && tl.part != 0) continue;
    for (int j = tl.row_begin + threadIdx.x; j < tl.row_end; j += blockDim.x) {
      double v;
      if (mode == 0) v = mask[j] * a[j];
      else if (mode == 1) v = mask[j] * D[j] * a[j];
      else if (mode == 2) v = D[j] * a[j];
      else if (mode == 4) v = a[j];
      else v = 0.0;
      out[j] = v;
    }
  }
}

// plain u = A~ v on every LP (no CG masking)
struct PlainEpi {
  double* u;
  __device__ __forceinline__ void row(int i, const double (&s)[1], int) { u[i] = s[0]; }
};
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_adj_spmv(SchedView S, const int32_t* rp, const int32_t* col,
                                                   const double* val, const double* v, double* u) {
  extern __shared__ __align__(16) unsigned char smem[];
  PlainEpi epi{u};
  Gather<double, 1> g{{v}};
  run_tiles<double, 1, BLOCK, kFixedE>(S, rp, col, val, g, epi, smem);
}

static cudaError_t set_dyn_adj(const void* f, size_t max_smem) {
  cudaFuncAttributes a;
  cudaError_t r = cudaFuncGetAttributes(&a, f);
  if (r == cudaSuccess)
    r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(max_smem - a.sharedSizeBytes));
  return r;
}

}  // namespace pdhg

using namespace pdhg;

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct AdjointData {
  double *mask = nullptr, *w = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *rhs = nullptr,
         *u = nullptr, *rec = nullptr, *xpol = nullptr;
  CgState* cg = nullptr;
  bool polished = false;
};

static AdjointData* adj_of(pdhg_ctx* ctx) { return static_cast<AdjointData*>(ctx->adjoint); }

void pdhg_adjoint_invalidate(pdhg_ctx* ctx) {
  if (ctx->adjoint) adj_of(ctx)->polished = false;
}

void pdhg_free_adjoint(pdhg_ctx* ctx) {
  delete adj_of(ctx);
  ctx->adjoint = nullptr;
}

static pdhg_status adj_alloc(pdhg_ctx* ctx) {
  if (ctx->adjoint) return PDHG_OK;
  AdjointData* d = new (std::nothrow) AdjointData();
  if (!d) {
    set_error("out of host memory");
    return PDHG_OOM;
  }
  ctx->adjoint = d;
  const size_t n = ctx->n, m = ctx->m;
  CKS(dalloc(ctx, &d->mask, n));
  CKS(dalloc(ctx, &d->w, n));
  CKS(dalloc(ctx, &d->r, n));
  CKS(dalloc(ctx, &d->p, n));
  CKS(dalloc(ctx, &d->q, n));
  CKS(dalloc(ctx, &d->rhs, n));
  CKS(dalloc(ctx, &d->xpol, n));
  CKS(dalloc(ctx, &d->u, m));
  CKS(dalloc(ctx, &d->rec, 2 * (size_t)std::max(ctx->st8.view.ntiles, 1) + 2));
  CKS(dalloc(ctx, &d->cg, (size_t)ctx->count));
  for (const void* f : {(const void*)k_adj_mask<kBlock>, (const void*)k_cg_Av<kBlock>,
                        (const void*)k_cg_ATu<kBlock>, (const void*)k_adj_spmv<kBlock>}) {
    CK(set_dyn_adj(f, ctx->smem_optin));
  }
  return PDHG_OK;
}

// CG on (M_B^T M_B) w = rhs per LP for the matrix with values aval (rows of
// A) and tval (rows of A^T), starting from the w already in d->w (zero off
// B); p, r, q, u are scratch.  Per-LP iterations into `iters`.
static pdhg_status run_cg(pdhg_ctx* ctx, AdjointData* d, double tol, int max_iter,
                          std::vector<int32_t>* iters, const double* aval, const double* tval) {
  const SchedView &A = ctx->sa8.view, &T = ctx->st8.view;
  const int count = ctx->count;
  int32_t* ticket = ctx->active + 2;
  int32_t* active = ctx->active + 3;
  const int eg = ctx->restart_grid;
  // q = M w0 with every LP active
  CK(cudaMemsetAsync(d->cg, 0, sizeof(CgState) * count, ctx->stream));
  k_cg_Av<kBlock><<<ctx->l_a64.grid, kBlock, ctx->l_a64.smem, ctx->stream>>>(
      A, ctx->a_rp, ctx->a_col, aval, d->w, d->u, d->cg);
  k_cg_ATu<kBlock><<<ctx->l_t64.grid, kBlock, ctx->l_t64.smem, ctx->stream>>>(
      T, ctx->t_rp, ctx->t_col, tval, d->u, d->mask, d->w, d->q, d->rec, d->cg,
      ctx->lp_t8_tiles, count, ticket, 0);
  k_cg_start<<<eg, 256, 0, ctx->stream>>>(T, d->rhs, d->q, d->r, d->p, d->rec);
  k_cg_start_final<<<(count + 255) / 256, 256, 0, ctx->stream>>>(d->rec, ctx->lp_t8_tiles, count,
                                                                  d->cg, tol, max_iter);
  ctx->launches += 5;
  int32_t* h_act = reinterpret_cast<int32_t*>(ctx->h_sc[0]);
  for (int it = 0; it < max_iter; ++it) {
    k_cg_Av<kBlock><<<ctx->l_a64.grid, kBlock, ctx->l_a64.smem, ctx->stream>>>(
        A, ctx->a_rp, ctx->a_col, aval, d->p, d->u, d->cg);
    k_cg_ATu<kBlock><<<ctx->l_t64.grid, kBlock, ctx->l_t64.smem, ctx->stream>>>(
        T, ctx->t_rp, ctx->t_col, tval, d->u, d->mask, d->p, d->q, d->rec, d->cg,
        ctx->lp_t8_tiles, count, ticket, 1);
    k_cg_update<<<eg, 256, 0, ctx->stream>>>(T, d->w, d->r, d->p, d->q, d->rec, d->cg,
                                             ctx->lp_t8_tiles, count, ticket, active);
    k_cg_p<<<eg, 256, 0, ctx->stream>>>(T, d->p, d->r, d->cg);
    ctx->launches += 4;
    if ((it & 15) == 15 || it == max_iter - 1) {
      CK(cudaMemcpyAsync(h_act, active, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      if (*h_act == 0) break;
    }
  }
  CK(cudaGetLastError());
  if (iters) {
    std::vector<CgState> hc(count);
    CK(cudaMemcpyAsync(hc.data(), d->cg, sizeof(CgState) * count, cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    iters->resize(count);
    for (int l = 0; l < count; ++l) (*iters)[l] = hc[l].iters;
  }
  return PDHG_OK;
}

pdhg_status batch_returned64_adj(pdhg_ctx* ctx);  // batch.cu

extern "C" pdhg_status pdhg_batch_polish(pdhg_ctx* ctx, double cg_tol, int32_t cg_max_iter,
                                         double* x, int32_t* lp_active, int32_t* lp_cg_iters) {
  clear_error();
  if (!ctx || !ctx->batch) {
    set_error("pdhg_batch_polish needs a context from pdhg_batch_create");
    return PDHG_INVALID_ARG;
  }
  if (!(cg_tol > 0.0) || cg_max_iter < 0) {
    set_error("need cg_tol > 0 and cg_max_iter >= 0");
    return PDHG_INVALID_ARG;
  }
  CKS(adj_alloc(ctx));
  AdjointData* d = adj_of(ctx);
  const SchedView& T = ctx->st8.view;
  const SchedView& A = ctx->sa8.view;
  const int count = ctx->count, eg = ctx->restart_grid;
  CKS(batch_returned64_adj(ctx));  // x~, y~ of the returned iterates in xs64, ys64
  // B from the projected primal step at the returned iterate
  k_adj_mask<kBlock><<<ctx->l_t64.grid, kBlock, ctx->l_t64.smem, ctx->stream>>>(
      T, ctx->t_rp, ctx->t_col, ctx->t_val64, ctx->xs64, ctx->ys64, ctx->c_t64, ctx->sc, d->mask,
      d->rec);
  // rhs = mask * A~^T b~; w0 = mask * x~
  k_adj_spmv<kBlock><<<ctx->l_t64.grid, kBlock, ctx->l_t64.smem, ctx->stream>>>(
      T, ctx->t_rp, ctx->t_col, ctx->t_val64, ctx->b_t64, d->q);
  k_adj_vec<<<eg, 256, 0, ctx->stream>>>(T, 0, d->mask, nullptr, d->q, d->rhs);
  k_adj_vec<<<eg, 256, 0, ctx->stream>>>(T, 0, d->mask, nullptr, ctx->xs64, d->w);
  ctx->launches += 4;
  std::vector<double> cnt((size_t)std::max(T.ntiles, 1));
  std::vector<int32_t> lpt((size_t)count + 1);
  CK(cudaMemcpyAsync(cnt.data(), d->rec, sizeof(double) * T.ntiles, cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaMemcpyAsync(lpt.data(), ctx->lp_t8_tiles, sizeof(int32_t) * (count + 1),
                     cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (lp_active)
    for (int l = 0; l < count; ++l) {
      double s = 0.0;
      for (int t = lpt[l]; t < lpt[l + 1]; ++t) s += cnt[t];
      lp_active[l] = (int32_t)s;
    }
  std::vector<int32_t> iters;
  CKS(run_cg(ctx, d, cg_tol, cg_max_iter, &iters, ctx->a_val64, ctx->t_val64));
  if (lp_cg_iters)
    for (int l = 0; l < count; ++l) lp_cg_iters[l] = iters[l];
  // x = D_c x~ (zero off B)
  k_adj_vec<<<eg, 256, 0, ctx->stream>>>(T, 2, nullptr, ctx->D_c, d->w, d->xpol);
  ctx->launches += 1;
  CK(cudaGetLastError());
  (void)A;
  d->polished = true;
  CKS(copy_out(ctx, x, d->xpol, sizeof(double) * ctx->n));
  CK(cudaStreamSynchronize(ctx->stream));
  return PDHG_OK;
}

extern "C" pdhg_status pdhg_batch_adjoint(pdhg_ctx* ctx, const double* grad_x, double* grad_b,
                                          double* grad_c, double cg_tol, int32_t cg_max_iter,
                                          int32_t* lp_cg_iters) {
  clear_error();
  if (!ctx || !ctx->batch || !grad_x) {
    set_error("pdhg_batch_adjoint needs a batch context and grad_x");
    return PDHG_INVALID_ARG;
  }
  AdjointData* d = adj_of(ctx);
  if (!d || !d->polished) {
    set_error("call pdhg_batch_polish first (it fixes the active set)");
    return PDHG_INVALID_ARG;
  }
  if (!(cg_tol > 0.0) || cg_max_iter < 0) {
    set_error("need cg_tol > 0 and cg_max_iter >= 0");
    return PDHG_INVALID_ARG;
  }
  const SchedView &T = ctx->st8.view, &A = ctx->sa8.view;
  const int eg = ctx->restart_grid;
  // rhs = mask * g; w0 = 0  (original A)
  CKS(copy_in(ctx, d->q, grad_x, sizeof(double) * ctx->n));
  k_adj_vec<<<eg, 256, 0, ctx->stream>>>(T, 0, d->mask, nullptr, d->q, d->rhs);
  k_adj_vec<<<eg, 256, 0, ctx->stream>>>(T, 3, nullptr, nullptr, nullptr, d->w);
  ctx->launches += 2;
  std::vector<int32_t> iters;
  CKS(run_cg(ctx, d, cg_tol, cg_max_iter, &iters, ctx->a_val_orig, ctx->t_val_orig));
  if (lp_cg_iters)
    for (int l = 0; l < ctx->count; ++l) lp_cg_iters[l] = iters[l];
  // dL/db = A_B w  (w is zero off B)
  k_adj_spmv<kBlock><<<ctx->l_a64.grid, kBlock, ctx->l_a64.smem, ctx->stream>>>(
      A, ctx->a_rp, ctx->a_col, ctx->a_val_orig, d->w, d->u);
  k_adj_vec<<<eg, 256, 0, ctx->stream>>>(A, 4, nullptr, nullptr, d->u, ctx->out_m1);
  ctx->launches += 2;
  CK(cudaGetLastError());
  CKS(copy_out(ctx, grad_b, ctx->out_m1, sizeof(double) * ctx->m));
  if (grad_c) {
    if (ctx->opt.io_on_device)
      CK(cudaMemsetAsync(grad_c, 0, sizeof(double) * ctx->n, ctx->stream));
    else
      std::memset(grad_c, 0, sizeof(double) * ctx->n);
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return PDHG_OK;
}
