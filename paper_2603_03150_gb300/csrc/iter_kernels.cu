// PDHG iteration kernels: primal half-step (A~^T y + projection), dual
// half-step (A~ x + extrapolated dual step), the fused evaluation with the
// on-device restart / termination rule, restart-apply, the float64 report of
// an iterate, and Algorithm 1 (centered start point, Section 3.1).
#include <math.h>

#include "dispatch.cuh"
#include "epilogues.cuh"
#include "eval_rule.cuh"
#include "kernels.h"
#include "spmv_tile.cuh"

namespace pdhg {

// ---------------------------------------------------------------------------
// K1: x+ = max(0, x - tau (c~ - A~^T y)), running average of x.
// ---------------------------------------------------------------------------

template <typename T, int BLOCK, int E>
__global__ void __launch_bounds__(BLOCK) k_primal(IterBuffers<T> B, int i) {
  pdl_enter();
  if (B.sc->done) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const long long tt = B.sc->t + i;  // iterations since restart before this one
  PrimalEpi<T> epi{B.x, B.c_t, B.x_avg, (T)B.sc->tau, (T)(1.0 / (double)(tt + 1)), tt == 0};
  Gather<T, 1> g{{B.y}};
  run_sched<T, 1, BLOCK, E>(B.t_sched, B.t_rp, B.t_col, B.t_val, g, epi, smem);
}

// ---------------------------------------------------------------------------
// K2: h = A~ x+;  y+ = y + sigma (b~ - 2h + A~x)   (= b~ - A~(2x+ - x));
// caches A~x+ and the running averages of y and A~x.
// ---------------------------------------------------------------------------

template <typename T, int BLOCK, int E>
__global__ void __launch_bounds__(BLOCK) k_dual(IterBuffers<T> B, int i) {
  pdl_enter();
  if (B.sc->done) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const long long tt = B.sc->t + i;
  DualEpi<T> epi{B.y,   B.b_t, B.Ax, B.y_avg, B.Ax_avg, (T)B.sc->sigma, (T)(1.0 / (double)(tt + 1)),
                 tt == 0};
  Gather<T, 1> g{{B.x}};
  run_sched<T, 1, BLOCK, E>(B.a_sched, B.a_rp, B.a_col, B.a_val, g, epi, smem);
}

// ---------------------------------------------------------------------------
// Evaluation: one pass over A~^T with y and y_avg gathered together, plus an
// elementwise pass over the m rows, reduced in float64 for both candidates
// (current iterate and running average).  The last block to finish applies
// the termination test and the restart rule on device.
// ---------------------------------------------------------------------------
template <typename T>
struct EvalEpi {
  const T *x, *x_avg, *x_last;
  const double *c_t, *Dc_inv;
  double* split_q;
  double q[2][Q_N];
  __device__ __forceinline__ void contrib(int j, const T (&s)[2], double (&o)[2][Q_N]) const {
    const double cj = c_t[j], dci = Dc_inv[j];
    const double xl = (double)x_last[j];
    const double xs[2] = {(double)x[j], (double)x_avg[j]};
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const double rd = fmin(0.0, cj - (double)s[c]);
      const double ru = rd * dci;
      const double dx = xs[c] - xl;
      o[c][Q_S2] = rd * rd;
      o[c][Q_U2] = ru * ru;
      o[c][Q_S3] = cj * xs[c];
      o[c][Q_D1] = dx * dx;
    }
  }
  __device__ __forceinline__ void row(int j, const T (&s)[2], int group) {
    double o[2][Q_N];
    contrib(j, s, o);
    if (group < 0) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        q[c][Q_S2] += o[c][Q_S2];
        q[c][Q_U2] += o[c][Q_U2];
        q[c][Q_S3] += o[c][Q_S3];
        q[c][Q_D1] += o[c][Q_D1];
      }
    } else {  // a split row: its own record, added in group order at the end
      double* rec = split_q + (size_t)group * kEvalQ;
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int k = 0; k < Q_N; ++k) rec[c * Q_N + k] = 0.0;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        rec[c * Q_N + Q_S2] = o[c][Q_S2];
        rec[c * Q_N + Q_U2] = o[c][Q_U2];
        rec[c * Q_N + Q_S3] = o[c][Q_S3];
        rec[c * Q_N + Q_D1] = o[c][Q_D1];
      }
    }
  }
};

// Float32-mixed evaluations ask for 4 resident blocks per SM (64 registers,
// no spill; 3 at the 76 it takes otherwise): the kernel is bound by the
// float64 pipe at low occupancy, so more warps keep that pipe busier.  The
// float64 variants would spill under that bound and keep the default.
template <typename T, int BLOCK, int E>
__global__ void __launch_bounds__(BLOCK, sizeof(T) == 4 ? 4 : 1) k_eval(IterBuffers<T> B, int chunk) {
  if (B.sc->done) return;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[kEvalQ * (BLOCK / 32)];
  __shared__ double tot[kEvalQ];
  __shared__ int is_last;
  EvalEpi<T> epi{B.x, B.x_avg, B.x_last, B.c_t64, B.Dc_inv, B.split_q, {}};
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int k = 0; k < Q_N; ++k) epi.q[c][k] = 0.0;
  Gather<T, 2> g{{B.y, B.y_avg}};
  run_sched<T, 2, BLOCK, E>(B.t_sched, B.t_rp, B.t_col, B.t_val, g, epi, smem);
  // m side: primal residual, dual objective, distance to the last restart point
  for (int i = blockIdx.x * BLOCK + threadIdx.x; i < B.m; i += gridDim.x * BLOCK) {
    const double bi = B.b_t64[i], dri = B.Dr_inv[i], yl = (double)B.y_last[i];
    const double axs[2] = {(double)B.Ax[i], (double)B.Ax_avg[i]};
    const double ys[2] = {(double)B.y[i], (double)B.y_avg[i]};
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const double rp = bi - axs[c];
      const double ru = rp * dri;
      const double dy = ys[c] - yl;
      epi.q[c][Q_S1] += rp * rp;
      epi.q[c][Q_U1] += ru * ru;
      epi.q[c][Q_S4] += bi * ys[c];
      epi.q[c][Q_D2] += dy * dy;
    }
  }
  double mine[kEvalQ];
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int k = 0; k < Q_N; ++k) mine[c * Q_N + k] = epi.q[c][k];
  // the block's record (16 sums), then the ticket: the barrier that ends
  // block_sum_scatter orders its writers' stores before thread 0's fence
  block_sum_scatter<BLOCK, kEvalQ>(mine, red, B.partials + (size_t)blockIdx.x * kEvalQ);
  if (threadIdx.x == 0) {
    __threadfence();
    is_last = (atomicAdd(&B.sc->ticket, 1) == (int)gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  parts_sum<BLOCK, kEvalQ>(B.partials, (int)gridDim.x, B.split_q, B.t_sched.ngroups, tot, red);
  if (threadIdx.x == 0) {
    B.sc->ticket = 0;
    apply_eval_rule(*B.sc, tot, chunk, B.log_k, B.log_flags, B.log_kkt);
  }
}

// Restart: the candidate becomes the iterate and the new last restart point
// (with its product A~x, the Halpern method's anchor term).
template <typename T>
__global__ void k_restart(IterBuffers<T> B) {
  if (!B.sc->restart_pending) return;
  const bool avg = B.sc->restart_to_avg != 0;
  const int stride = gridDim.x * blockDim.x;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < B.n; j += stride) {
    if (avg) {
      const T v = B.x_avg[j];
      B.x[j] = v;
      B.x_last[j] = v;
    } else {
      B.x_last[j] = B.x[j];
    }
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B.m; i += stride) {
    if (avg) {
      const T v = B.y_avg[i];
      const T h = B.Ax_avg[i];
      B.y[i] = v;
      B.y_last[i] = v;
      B.Ax[i] = h;
      B.Ax_last[i] = h;
    } else {
      B.y_last[i] = B.y[i];
      B.Ax_last[i] = B.Ax[i];
    }
  }
}

template <typename T>
void launch_primal(const IterBuffers<T>& B, const Launch& L, int i, cudaStream_t s) {
  PDHG_DISPATCH_E(B.t_sched.e, launch_pdl(k_primal<T, kBlock, E_>, L.grid, kBlock, L.smem, s, B, i));
}
template <typename T>
void launch_dual(const IterBuffers<T>& B, const Launch& L, int i, cudaStream_t s) {
  PDHG_DISPATCH_E(B.a_sched.e, launch_pdl(k_dual<T, kBlock, E_>, L.grid, kBlock, L.smem, s, B, i));
}
template <typename T>
void launch_eval(const IterBuffers<T>& B, const Launch& L, int chunk, cudaStream_t s) {
  PDHG_DISPATCH_E(B.t_sched.e, k_eval<T, kBlock, E_><<<L.grid, kBlock, L.smem, s>>>(B, chunk));
}
template <typename T>
void launch_restart(const IterBuffers<T>& B, int grid, cudaStream_t s) {
  k_restart<T><<<grid, 256, 0, s>>>(B);
}

// ---------------------------------------------------------------------------
// Plain SpMV out = M v (autotuner probe).
// ---------------------------------------------------------------------------
template <typename T>
struct StoreEpi {
  T* out;
  __device__ __forceinline__ void row(int r, const T (&s)[1], int) { out[r] = s[0]; }
};

template <typename T, int BLOCK, int E>
__global__ void __launch_bounds__(BLOCK) k_spmv(SchedView S, const int32_t* rp, const int32_t* col,
                                               const T* val, const T* v, T* out) {
  extern __shared__ __align__(16) unsigned char smem[];
  StoreEpi<T> epi{out};
  Gather<T, 1> g{{v}};
  run_sched<T, 1, BLOCK, E>(S, rp, col, val, g, epi, smem);
}

template <typename T>
void launch_spmv(const SchedView& S, const int32_t* rp, const int32_t* col, const T* val,
                 const T* v, T* out, const Launch& L, cudaStream_t s) {
  PDHG_DISPATCH_E(S.e, k_spmv<T, kBlock, E_><<<L.grid, kBlock, L.smem, s>>>(S, rp, col, val, v, out));
}

// ---------------------------------------------------------------------------
// float64 report of an iterate on the original model.
// ---------------------------------------------------------------------------
struct ReportNEpi {
  const double *x_s, *c_t, *D_c;
  double *x_out, *z_out;
  double u2, s3, xz, inf_rd;
  double* split_q;  // per split group: 4 values
  __device__ __forceinline__ void row(int j, const double (&s)[1], int group) {
    const double d = c_t[j] - s[0];
    const double zs = fmax(0.0, d), rd = fmin(0.0, d) / D_c[j];
    const double xs = x_s[j];
    if (x_out) x_out[j] = D_c[j] * xs;
    if (z_out) z_out[j] = zs / D_c[j];
    if (group < 0) {
      u2 += rd * rd;
      s3 += c_t[j] * xs;
      xz += xs * zs;
      inf_rd = fmax(inf_rd, fabs(rd));
    } else {
      double* r = split_q + 4 * (size_t)group;
      r[0] = rd * rd;
      r[1] = c_t[j] * xs;
      r[2] = xs * zs;
      r[3] = fabs(rd);
    }
  }
};

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_report_n(SchedView S, const int32_t* rp, const int32_t* col,
                                                   const double* val, const double* x_s,
                                                   const double* y_s, const double* c_t,
                                                   const double* D_c, double* x_out, double* z_out,
                                                   double* partials, const Scalars* gate) {
  if (gate && !gate->verify) return;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[4 * (BLOCK / 32)];
  double* split_q = partials + 4 * (size_t)gridDim.x;
  ReportNEpi epi{x_s, c_t, D_c, x_out, z_out, 0.0, 0.0, 0.0, 0.0, split_q};
  Gather<double, 1> g{{y_s}};
  run_tiles<double, 1, BLOCK, kFixedE>(S, rp, col, val, g, epi, smem);
  // infinity norm through a max-reduction, sums through block_sum
  const double v[3] = {epi.u2, epi.s3, epi.xz};
  double o[3];
  block_sum<BLOCK, 3>(v, o, red);
  double mx = epi.inf_rd;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < BLOCK / 32; ++w) mx = fmax(mx, red[w]);
    partials[4 * (size_t)blockIdx.x + 0] = o[0];
    partials[4 * (size_t)blockIdx.x + 1] = o[1];
    partials[4 * (size_t)blockIdx.x + 2] = o[2];
    partials[4 * (size_t)blockIdx.x + 3] = mx;
  }
}

struct ReportMEpi {
  const double *y_s, *b_t, *D_r;
  double* y_out;
  double u1, s4, inf_rp;
  double* split_q;
  __device__ __forceinline__ void row(int i, const double (&s)[1], int group) {
    const double rp = (b_t[i] - s[0]) / D_r[i];
    if (y_out) y_out[i] = D_r[i] * y_s[i];
    if (group < 0) {
      u1 += rp * rp;
      s4 += b_t[i] * y_s[i];
      inf_rp = fmax(inf_rp, fabs(rp));
    } else {
      double* r = split_q + 4 * (size_t)group;
      r[0] = rp * rp;
      r[1] = b_t[i] * y_s[i];
      r[2] = 0.0;
      r[3] = fabs(rp);
    }
  }
};

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_report_m(SchedView S, const int32_t* rp, const int32_t* col,
                                                   const double* val, const double* x_s,
                                                   const double* y_s, const double* b_t,
                                                   const double* D_r, double* y_out,
                                                   double* partials, const Scalars* gate) {
  if (gate && !gate->verify) return;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[4 * (BLOCK / 32)];
  double* split_q = partials + 4 * (size_t)gridDim.x;
  ReportMEpi epi{y_s, b_t, D_r, y_out, 0.0, 0.0, 0.0, split_q};
  Gather<double, 1> g{{x_s}};
  run_tiles<double, 1, BLOCK, kFixedE>(S, rp, col, val, g, epi, smem);
  const double v[2] = {epi.u1, epi.s4};
  double o[2];
  block_sum<BLOCK, 2>(v, o, red);
  double mx = epi.inf_rp;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < BLOCK / 32; ++w) mx = fmax(mx, red[w]);
    partials[4 * (size_t)blockIdx.x + 0] = o[0];
    partials[4 * (size_t)blockIdx.x + 1] = o[1];
    partials[4 * (size_t)blockIdx.x + 2] = 0.0;
    partials[4 * (size_t)blockIdx.x + 3] = mx;
  }
}

// pn/pm hold [grid][4] block partials followed by [groups][4] split records;
// gn/gm count all of those records.
__global__ void k_report_final(const double* pn, int gn, const double* pm, int gm, double* out) {
  if (threadIdx.x != 0) return;
  double u2 = 0, s3 = 0, xz = 0, ird = 0, u1 = 0, s4 = 0, irp = 0;
  for (int b = 0; b < gn; ++b) {
    u2 += pn[4 * b];
    s3 += pn[4 * b + 1];
    xz += pn[4 * b + 2];
    ird = fmax(ird, pn[4 * b + 3]);
  }
  for (int b = 0; b < gm; ++b) {
    u1 += pm[4 * b];
    s4 += pm[4 * b + 1];
    irp = fmax(irp, pm[4 * b + 3]);
  }
  out[0] = sqrt(u1);
  out[1] = sqrt(u2);
  out[2] = fabs(s3 - s4);
  out[3] = fmax(fmax(irp, ird), xz / (1.0 + fabs(s3)));
  out[4] = s3;
  out[5] = s4;
  out[6] = xz;
  out[7] = 0.0;
}

void launch_report_n(const SchedView& S, const int32_t* rp, const int32_t* col, const double* val,
                     const double* x_s, const double* y_s, const double* c_t, const double* D_c,
                     double* x_out, double* z_out, double* partials, const Launch& L,
                     cudaStream_t s) {
  k_report_n<kBlock><<<L.grid, kBlock, L.smem, s>>>(S, rp, col, val, x_s, y_s, c_t, D_c, x_out,
                                                    z_out, partials, nullptr);
}
void launch_report_m(const SchedView& S, const int32_t* rp, const int32_t* col, const double* val,
                     const double* x_s, const double* y_s, const double* b_t, const double* D_r,
                     double* y_out, double* partials, const Launch& L, cudaStream_t s) {
  k_report_m<kBlock><<<L.grid, kBlock, L.smem, s>>>(S, rp, col, val, x_s, y_s, b_t, D_r, y_out,
                                                    partials, nullptr);
}
void launch_report_final(const double* pn, int gn, const double* pm, int gm, double* out,
                         cudaStream_t s) {
  k_report_final<<<1, 32, 0, s>>>(pn, gn, pm, gm, out);
}

// ---------------------------------------------------------------------------
// Float64 check of a float32-mixed candidate that passed the screen (every
// kernel returns at once unless a check is pending): the candidate in
// float64, the report sums of its products recomputed from the float64
// scaled matrices, then the Section 2 test at eps in one thread.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_fp64_prep(IterBuffers<T> B, double* xs, double* ys) {
  const Scalars* sc = B.sc;
  if (!sc->verify) return;
  const bool avg = sc->verify_avg != 0;
  const T* x = avg ? B.x_avg : B.x;
  const T* y = avg ? B.y_avg : B.y;
  const int stride = gridDim.x * blockDim.x;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < B.n; j += stride) xs[j] = (double)x[j];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B.m; i += stride) ys[i] = (double)y[i];
}

__global__ void k_fp64_final(Scalars* sc, const double* pn, int gn, const double* pm, int gm,
                             long long* log_k, int32_t* log_flags, double* log_kkt) {
  if (threadIdx.x != 0 || !sc->verify) return;
  double u2 = 0, s3 = 0, u1 = 0, s4 = 0;
  for (int b = 0; b < gn; ++b) {
    u2 += pn[4 * b];
    s3 += pn[4 * b + 1];
  }
  for (int b = 0; b < gm; ++b) {
    u1 += pm[4 * b];
    s4 += pm[4 * b + 1];
  }
  eval_fp64_check(*sc, u1, u2, s3, s4, log_k, log_flags, log_kkt);
}

template <typename T>
void launch_fp64_check(const IterBuffers<T>& B, const Fp64Check& C, cudaStream_t s) {
  k_fp64_prep<T><<<C.conv_grid, 256, 0, s>>>(B, C.xs, C.ys);
  double* pn = B.partials;
  double* pm = B.partials + 4 * (size_t)(C.gn + 1);
  k_report_n<kBlock><<<C.Lt.grid, kBlock, C.Lt.smem, s>>>(C.St, B.t_rp, B.t_col, C.t_val, C.xs, C.ys,
                                                          B.c_t64, B.D_c, nullptr, nullptr, pn,
                                                          B.sc);
  k_report_m<kBlock><<<C.La.grid, kBlock, C.La.smem, s>>>(C.Sa, B.a_rp, B.a_col, C.a_val, C.xs, C.ys,
                                                          B.b_t64, B.D_r, nullptr, pm, B.sc);
  k_fp64_final<<<1, 32, 0, s>>>(B.sc, pn, C.gn, pm, C.gm, B.log_k, B.log_flags, B.log_kkt);
}
template void launch_fp64_check<float>(const IterBuffers<float>&, const Fp64Check&, cudaStream_t);

// ---------------------------------------------------------------------------
// Algorithm 1 (Section 3.1): the centered start point (target mu, then the per-entry update).
// ---------------------------------------------------------------------------
struct WsEpi {
  const double *x_s, *c_t;
  double* z_s;
  double xz;
  double* split_q;
  __device__ __forceinline__ void row(int j, const double (&s)[1], int group) {
    const double z = fmax(0.0, c_t[j] - s[0]);
    z_s[j] = z;
    if (group < 0)
      xz += x_s[j] * z;
    else
      split_q[group] = x_s[j] * z;
  }
};

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_ws_z(SchedView S, const int32_t* rp, const int32_t* col,
                                               const double* val, const double* x_s,
                                               const double* y_s, const double* c_t, double* z_s,
                                               double* partials) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[BLOCK / 32];
  WsEpi epi{x_s, c_t, z_s, 0.0, partials + gridDim.x};
  Gather<double, 1> g{{y_s}};
  run_tiles<double, 1, BLOCK, kFixedE>(S, rp, col, val, g, epi, smem);
  const double v[1] = {epi.xz};
  double o[1];
  block_sum<BLOCK, 1>(v, o, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = o[0];
}

__global__ void k_ws_mu(const double* partials, int g, int n, double mu_min, double* mu) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < g; ++b) s += partials[b];
  *mu = fmax(s / (double)n, mu_min);
}

__device__ __forceinline__ double ws_move(double target, double v, double delta) {
  return fmin(fmax(target, v - delta), v + delta);
}

__global__ void k_ws_apply(int n, int m, const double* x_s, const double* z_s, const double* y_s,
                           const double* mu_p, double delta, double alpha, int unscaled,
                           const double* D_r, const double* D_c, double* x_out, double* y_out,
                           double* z_out) {
  const double mu = *mu_p;
  const int stride = gridDim.x * blockDim.x;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
    double xp = fmax(x_s[j], alpha), zp = fmax(z_s[j], alpha);
    if (xp < zp) {
      xp = ws_move(mu / zp, xp, delta);
      zp = ws_move(mu / xp, zp, delta);
    } else {
      zp = ws_move(mu / xp, zp, delta);
      xp = ws_move(mu / zp, xp, delta);
    }
    if (unscaled) {
      xp = D_c[j] * xp;
      zp = zp / D_c[j];
    }
    if (x_out) x_out[j] = xp;
    if (z_out) z_out[j] = zp;
  }
  if (y_out)
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride)
      y_out[i] = unscaled ? D_r[i] * y_s[i] : y_s[i];
}

void launch_ws_z(const SchedView& S, const int32_t* rp, const int32_t* col, const double* val,
                 const double* x_s, const double* y_s, const double* c_t, double* z_s,
                 double* partials, const Launch& L, cudaStream_t s) {
  k_ws_z<kBlock><<<L.grid, kBlock, L.smem, s>>>(S, rp, col, val, x_s, y_s, c_t, z_s, partials);
}
void launch_ws_mu(const double* partials, int g, int n, double mu_min, double* mu, cudaStream_t s) {
  k_ws_mu<<<1, 32, 0, s>>>(partials, g, n, mu_min, mu);
}
void launch_ws_apply(int n, int m, const double* x_s, const double* z_s, const double* y_s,
                     const double* mu, double delta_max, double alpha_min, int unscaled,
                     const double* D_r, const double* D_c, double* x_out, double* y_out,
                     double* z_out, cudaStream_t s) {
  const int grid = (int)((((n > m) ? n : m) + 255) / 256);
  k_ws_apply<<<grid < 1 ? 1 : grid, 256, 0, s>>>(n, m, x_s, z_s, y_s, mu, delta_max, alpha_min,
                                                 unscaled, D_r, D_c, x_out, y_out, z_out);
}

// ---------------------------------------------------------------------------
__global__ void k_d2f(const double* src, float* dst, int64_t len) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}
__global__ void k_f2d(const float* src, double* dst, int64_t len) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (double)src[i];
}
static int grid_for(int64_t len) {
  int64_t g = (len + 255) / 256;
  if (g > 4096) g = 4096;
  return g < 1 ? 1 : (int)g;
}
void launch_convert_d2f(const double* src, float* dst, int64_t len, cudaStream_t s) {
  k_d2f<<<grid_for(len), 256, 0, s>>>(src, dst, len);
}
void launch_convert_f2d(const float* src, double* dst, int64_t len, cudaStream_t s) {
  k_f2d<<<grid_for(len), 256, 0, s>>>(src, dst, len);
}

// explicit instantiations
#define PDHG_INST(T)                                                                        \
  template void launch_primal<T>(const IterBuffers<T>&, const Launch&, int, cudaStream_t); \
  template void launch_dual<T>(const IterBuffers<T>&, const Launch&, int, cudaStream_t);   \
  template void launch_eval<T>(const IterBuffers<T>&, const Launch&, int, cudaStream_t);   \
  template void launch_restart<T>(const IterBuffers<T>&, int, cudaStream_t);               \
  template void launch_spmv<T>(const SchedView&, const int32_t*, const int32_t*, const T*,  \
                               const T*, T*, const Launch&, cudaStream_t);
PDHG_INST(float)
PDHG_INST(double)
#undef PDHG_INST

// shared memory of the tile kernels (NV vectors, precision, rows per tile,
// schedule variant: e < 0 is the vector kernel)
size_t tile_smem(int nv, bool f32, int max_rows, int e) {
  if (e < 0) {
    if (nv == 1)
      return f32 ? tile_vec_smem_bytes<float, 1, kBlock>(max_rows)
                 : tile_vec_smem_bytes<double, 1, kBlock>(max_rows);
    return f32 ? tile_vec_smem_bytes<float, 2, kBlock>(max_rows)
               : tile_vec_smem_bytes<double, 2, kBlock>(max_rows);
  }
  if (nv == 1) return f32 ? tile_smem_bytes<float, 1, kBlock>(max_rows)
                          : tile_smem_bytes<double, 1, kBlock>(max_rows);
  return f32 ? tile_smem_bytes<float, 2, kBlock>(max_rows) : tile_smem_bytes<double, 2, kBlock>(max_rows);
}


template <int E>
static const void* tile_kernel(int which) {
  switch (which) {
    case 0: return (const void*)k_primal<float, kBlock, E>;
    case 1: return (const void*)k_primal<double, kBlock, E>;
    case 2: return (const void*)k_dual<float, kBlock, E>;
    case 3: return (const void*)k_dual<double, kBlock, E>;
    case 4: return (const void*)k_eval<float, kBlock, E>;
    case 5: return (const void*)k_eval<double, kBlock, E>;
    case 6: return (const void*)k_spmv<float, kBlock, E>;
    case 7: return (const void*)k_spmv<double, kBlock, E>;
    default: return nullptr;
  }
}
static const void* fixed_kernel(int which) {
  switch (which) {
    case 0: return (const void*)k_report_n<kBlock>;
    case 1: return (const void*)k_report_m<kBlock>;
    case 2: return (const void*)k_ws_z<kBlock>;
    default: return nullptr;
  }
}

// raise the dynamic shared-memory limit of every tile kernel
cudaError_t configure_tile_kernels(size_t max_smem) {
  cudaError_t e = cudaSuccess;
  for (int w = 0; w < 8; ++w)
    for (const void* f : {tile_kernel<8>(w), tile_kernel<16>(w), tile_kernel<32>(w),
                          tile_kernel<-4>(w), tile_kernel<-8>(w)}) {
      cudaError_t r = set_max_dyn_smem(f, max_smem);
      if (r != cudaSuccess) e = r;
    }
  for (int w = 0; w < 3; ++w) {
    cudaError_t r = set_max_dyn_smem(fixed_kernel(w), max_smem);
    if (r != cudaSuccess) e = r;
  }
  return e;
}

// blocks per SM of a tile kernel (which: 0/1 primal f32/f64, 2/3 dual,
// 4/5 eval, 6/7 spmv; 8: the float64 report kernels) at a dynamic smem size
int tile_occupancy(int which, int e, size_t smem) {
  const void* f = nullptr;
  if (which >= 8)
    f = fixed_kernel(0);
  else if (e == 32)
    f = tile_kernel<32>(which);
  else if (e == -4)
    f = tile_kernel<-4>(which);
  else if (e == -8)
    f = tile_kernel<-8>(which);
  else if (e == 16)
    f = tile_kernel<16>(which);
  else
    f = tile_kernel<8>(which);
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, kBlock, smem);
  return nb < 1 ? 1 : nb;
}

}  // namespace pdhg
