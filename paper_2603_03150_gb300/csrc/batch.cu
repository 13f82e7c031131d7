// Batched restarted PDHG: `count` independent LPs stacked as one
// block-diagonal system and iterated together, each with its own step sizes,
// primal weight, restart state and status (converged LPs are masked).
//
// Tiles never cross an LP boundary and carry their LP index, so the tuned
// tile SpMV serves the batch unchanged: epilogues read the tile's LP scalars,
// a finished LP's tiles are skipped, and every reduction is written as one
// record per tile and summed per LP in tile order (deterministic).  Scaling
// of the stacked matrix equals per-LP scaling (rows and columns of different
// blocks never meet); power iteration, norms, the termination test and the
// restart rule are per LP.
#include <cmath>
#include <cstring>

#include "context.h"
#include "dispatch.cuh"
#include "eval_rule.cuh"

namespace pdhg {

constexpr int kRecP = 2;  // power-iteration record: v.w, |w|^2
constexpr int kRecR = 4;  // report record

// One tile's record (the block's sums of NQ float64 quantities, written by
// threads 0..NQ-1): block_sum_scatter's reduce-scatter order.  Every lane
// adding all NQ quantities at each shuffle step, on GB300's slow float64
// pipe, had bounded the per-tile records.
template <int BLOCK, int NQ>
__device__ __forceinline__ void tile_record(double (&v)[NQ], double* red, double* out) {
  block_sum_scatter<BLOCK, NQ>(v, red, out);
}

template <typename T>
struct BatchBuffers {
  IterBuffers<T> it;  // it.sc: per-LP scalars [count]
  double* rec_t;      // [A^T tiles][kEvalQ]
  double* rec_a;      // [A tiles][kEvalQ]
  const int32_t* lp_t_tiles;
  const int32_t* lp_a_tiles;
  int32_t* ctl;  // [0] LPs not finished, [1] last-block ticket
  int32_t count;
};

// ---------------------------------------------------------------------------
// iteration kernels
// ---------------------------------------------------------------------------
template <typename T>
struct BPrimalEpi {
  T* __restrict__ x;
  const T* __restrict__ c;
  T* __restrict__ x_avg;
  const Scalars* sc;
  int i;
  T tau, w;
  bool first;
  __device__ __forceinline__ bool begin_tile(const Tile& tl) {
    const Scalars& s = sc[tl.lp];
    if (s.done) return false;
    const long long tt = s.t + i;
    tau = (T)s.tau;
    w = (T)(1.0 / (double)(tt + 1));
    first = tt == 0;
    return true;
  }
  __device__ __forceinline__ void row(int j, const T (&s)[1], int) {
    const T xn = fmax(T(0), x[j] - tau * (c[j] - s[0]));
    x[j] = xn;
    x_avg[j] = first ? xn : x_avg[j] + (xn - x_avg[j]) * w;
  }
};

template <typename T>
struct BDualEpi {
  T* __restrict__ y;
  const T* __restrict__ b;
  T* __restrict__ Ax;
  T* __restrict__ y_avg;
  T* __restrict__ Ax_avg;
  const Scalars* sc;
  int i;
  T sigma, w;
  bool first;
  __device__ __forceinline__ bool begin_tile(const Tile& tl) {
    const Scalars& s = sc[tl.lp];
    if (s.done) return false;
    const long long tt = s.t + i;
    sigma = (T)s.sigma;
    w = (T)(1.0 / (double)(tt + 1));
    first = tt == 0;
    return true;
  }
  __device__ __forceinline__ void row(int r, const T (&s)[1], int) {
    const T h = s[0];
    const T yn = y[r] + sigma * (b[r] - (h + h) + Ax[r]);
    Ax[r] = h;
    y[r] = yn;
    y_avg[r] = first ? yn : y_avg[r] + (yn - y_avg[r]) * w;
    Ax_avg[r] = first ? h : Ax_avg[r] + (h - Ax_avg[r]) * w;
  }
};

// Kernel bodies are device functions: the per-half-step kernels below run
// one each, the persistent kernel (k_bpersist) runs them all in turn.
template <typename T, int BLOCK, int E>
__device__ __forceinline__ void bprimal_body(const BatchBuffers<T>& B, int i, unsigned char* smem) {
  BPrimalEpi<T> epi{B.it.x, B.it.c_t, B.it.x_avg, B.it.sc, i, T(0), T(0), false};
  Gather<T, 1> g{{B.it.y}};
  run_sched<T, 1, BLOCK, E>(B.it.t_sched, B.it.t_rp, B.it.t_col, B.it.t_val, g, epi, smem);
}

template <typename T, int BLOCK, int E>
__device__ __forceinline__ void bdual_body(const BatchBuffers<T>& B, int i, unsigned char* smem) {
  BDualEpi<T> epi{B.it.y, B.it.b_t, B.it.Ax, B.it.y_avg, B.it.Ax_avg, B.it.sc, i, T(0), T(0), false};
  Gather<T, 1> g{{B.it.x}};
  run_sched<T, 1, BLOCK, E>(B.it.a_sched, B.it.a_rp, B.it.a_col, B.it.a_val, g, epi, smem);
}

template <typename T, int BLOCK, int E>
__global__ void __launch_bounds__(BLOCK) k_bprimal(BatchBuffers<T> B, int i) {
  extern __shared__ __align__(16) unsigned char smem[];
  bprimal_body<T, BLOCK, E>(B, i, smem);
}

template <typename T, int BLOCK, int E>
__global__ void __launch_bounds__(BLOCK) k_bdual(BatchBuffers<T> B, int i) {
  extern __shared__ __align__(16) unsigned char smem[];
  bdual_body<T, BLOCK, E>(B, i, smem);
}

// ---------------------------------------------------------------------------
// evaluation: per-tile records, per-LP termination test and restart rule
// ---------------------------------------------------------------------------
template <typename T, int BLOCK>
struct BEvalEpi {
  const T *x, *x_avg, *x_last;
  const double *c_t, *Dc_inv;
  const Scalars* sc;
  double* rec;
  double* red;
  double q[2][Q_N];
  __device__ __forceinline__ bool begin_tile(const Tile& tl) {
    if (sc[tl.lp].done) return false;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int k = 0; k < Q_N; ++k) q[c][k] = 0.0;
    return true;
  }
  __device__ __forceinline__ void row(int j, const T (&s)[2], int) {
    const double cj = c_t[j], dci = Dc_inv[j];
    const double xl = (double)x_last[j];
    const double xs[2] = {(double)x[j], (double)x_avg[j]};
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const double rd = fmin(0.0, cj - (double)s[c]);
      const double ru = rd * dci;
      const double dx = xs[c] - xl;
      q[c][Q_S2] += rd * rd;
      q[c][Q_U2] += ru * ru;
      q[c][Q_S3] += cj * xs[c];
      q[c][Q_D1] += dx * dx;
    }
  }
  __device__ __forceinline__ void end_tile(const Tile&, int t) {
    double mine[kEvalQ];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int k = 0; k < Q_N; ++k) mine[c * Q_N + k] = q[c][k];
    tile_record<BLOCK, kEvalQ>(mine, red, rec + (size_t)t * kEvalQ);
  }
};

template <typename T, int BLOCK, int E>
__device__ __forceinline__ void beval_body(const BatchBuffers<T>& B, int chunk, unsigned char* smem) {
  __shared__ double red[kEvalQ * (BLOCK / 32)];
  __shared__ int is_last, active;
  const IterBuffers<T>& I = B.it;
  BEvalEpi<T, BLOCK> epi{I.x, I.x_avg, I.x_last, I.c_t64, I.Dc_inv, I.sc, B.rec_t, red, {}};
  Gather<T, 2> g{{I.y, I.y_avg}};
  run_sched<T, 2, BLOCK, E>(I.t_sched, I.t_rp, I.t_col, I.t_val, g, epi, smem);
  // m side over the row ranges of A's tiles (no products needed)
  for (int t = blockIdx.x; t < I.a_sched.ntiles; t += gridDim.x) {
    const Tile tl = I.a_sched.tiles[t];
    if (I.sc[tl.lp].done) continue;
    double q[kEvalQ];
#pragma unroll
    for (int k = 0; k < kEvalQ; ++k) q[k] = 0.0;
    if (tl.split < 0 || tl.part == 0) {
      for (int i = tl.row_begin + threadIdx.x; i < tl.row_end; i += BLOCK) {
        const double bi = I.b_t64[i], dri = I.Dr_inv[i], yl = (double)I.y_last[i];
        const double axs[2] = {(double)I.Ax[i], (double)I.Ax_avg[i]};
        const double ys[2] = {(double)I.y[i], (double)I.y_avg[i]};
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const double rp = bi - axs[c], ru = rp * dri, dy = ys[c] - yl;
          q[c * Q_N + Q_S1] += rp * rp;
          q[c * Q_N + Q_U1] += ru * ru;
          q[c * Q_N + Q_S4] += bi * ys[c];
          q[c * Q_N + Q_D2] += dy * dy;
        }
      }
    }
    tile_record<BLOCK, kEvalQ>(q, red, B.rec_a + (size_t)t * kEvalQ);
  }
  if (threadIdx.x == 0) {
    __threadfence();
    is_last = (atomicAdd(B.ctl + 1, 1) == (int)gridDim.x - 1);
    active = 0;
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  int mine = 0;
  for (int l = threadIdx.x; l < B.count; l += BLOCK) {
    Scalars& sc = I.sc[l];
    if (sc.done) continue;
    double tot[kEvalQ];
#pragma unroll
    for (int k = 0; k < kEvalQ; ++k) tot[k] = 0.0;
#pragma unroll 4  // independent record loads in flight together
    for (int t = B.lp_t_tiles[l]; t < B.lp_t_tiles[l + 1]; ++t)
#pragma unroll
      for (int k = 0; k < kEvalQ; ++k) tot[k] += __ldcg(B.rec_t + (size_t)t * kEvalQ + k);
#pragma unroll 4  // independent record loads in flight together
    for (int t = B.lp_a_tiles[l]; t < B.lp_a_tiles[l + 1]; ++t)
#pragma unroll
      for (int k = 0; k < kEvalQ; ++k) tot[k] += __ldcg(B.rec_a + (size_t)t * kEvalQ + k);
    apply_eval_rule(sc, tot, chunk, nullptr, nullptr, nullptr);
    if (!sc.done) ++mine;
  }
  atomicAdd(&active, mine);
  __syncthreads();
  if (threadIdx.x == 0) {
    B.ctl[0] = active;
    B.ctl[1] = 0;
  }
}

template <typename T, int BLOCK, int E>
__global__ void __launch_bounds__(BLOCK) k_beval(BatchBuffers<T> B, int chunk) {
  extern __shared__ __align__(16) unsigned char smem[];
  beval_body<T, BLOCK, E>(B, chunk, smem);
}

// restart of the LPs whose rule fired: candidate -> iterate and last point
template <typename T>
__device__ __forceinline__ void brestart_body(const BatchBuffers<T>& B) {
  const IterBuffers<T>& I = B.it;
  for (int t = blockIdx.x; t < I.t_sched.ntiles; t += gridDim.x) {
    const Tile tl = I.t_sched.tiles[t];
    const Scalars& s = I.sc[tl.lp];
    if (!s.restart_pending || (tl.split >= 0 && tl.part != 0)) continue;
    const bool avg = s.restart_to_avg != 0;
    for (int j = tl.row_begin + threadIdx.x; j < tl.row_end; j += blockDim.x) {
      if (avg) {
        const T v = I.x_avg[j];
        I.x[j] = v;
        I.x_last[j] = v;
      } else {
        I.x_last[j] = I.x[j];
      }
    }
  }
  for (int t = blockIdx.x; t < I.a_sched.ntiles; t += gridDim.x) {
    const Tile tl = I.a_sched.tiles[t];
    const Scalars& s = I.sc[tl.lp];
    if (!s.restart_pending || (tl.split >= 0 && tl.part != 0)) continue;
    const bool avg = s.restart_to_avg != 0;
    for (int i = tl.row_begin + threadIdx.x; i < tl.row_end; i += blockDim.x) {
      if (avg) {
        const T v = I.y_avg[i];
        I.y[i] = v;
        I.y_last[i] = v;
        I.Ax[i] = I.Ax_avg[i];
      } else {
        I.y_last[i] = I.y[i];
      }
    }
  }
}

template <typename T>
__global__ void k_brestart(BatchBuffers<T> B) {
  brestart_body<T>(B);
}

// ---------------------------------------------------------------------------
// per-LP power iteration on A~^T A~ (float64, fixed-E schedules)
// ---------------------------------------------------------------------------
struct BPowAvEpi {
  double* u;
  const PowerState* ps;
  __device__ __forceinline__ bool begin_tile(const Tile& tl) { return !ps[tl.lp].stopped; }
  __device__ __forceinline__ void row(int r, const double (&s)[1], int) { u[r] = s[0]; }
};

template <int BLOCK>
struct BPowATuEpi {
  const double* v;
  double* w;
  const PowerState* ps;
  double* rec;
  double* red;
  double lam, nw2;
  __device__ __forceinline__ bool begin_tile(const Tile& tl) {
    if (ps[tl.lp].stopped) return false;
    lam = 0.0;
    nw2 = 0.0;
    return true;
  }
  __device__ __forceinline__ void row(int j, const double (&s)[1], int) {
    w[j] = s[0];
    lam += v[j] * s[0];
    nw2 += s[0] * s[0];
  }
  __device__ __forceinline__ void end_tile(const Tile&, int t) {
    double mine[kRecP] = {lam, nw2};
    tile_record<BLOCK, kRecP>(mine, red, rec + (size_t)t * kRecP);
  }
};

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_bpow_Av(SchedView S, const int32_t* rp, const int32_t* col,
                                                  const double* val, const double* v, double* u,
                                                  const PowerState* ps) {
  extern __shared__ __align__(16) unsigned char smem[];
  BPowAvEpi epi{u, ps};
  Gather<double, 1> g{{v}};
  run_tiles<double, 1, BLOCK, kFixedE>(S, rp, col, val, g, epi, smem);
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_bpow_ATu(SchedView S, const int32_t* rp, const int32_t* col,
                                                   const double* val, const double* u,
                                                   const double* v, double* w, double* rec,
                                                   PowerState* ps, const int32_t* lp_tiles,
                                                   int count, int32_t* ticket) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[kRecP * (BLOCK / 32)];
  __shared__ int is_last;
  BPowATuEpi<BLOCK> epi{v, w, ps, rec, red, 0.0, 0.0};
  Gather<double, 1> g{{u}};
  run_tiles<double, 1, BLOCK, kFixedE>(S, rp, col, val, g, epi, smem);
  if (threadIdx.x == 0) {
    __threadfence();
    is_last = (atomicAdd(ticket, 1) == (int)gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  for (int l = threadIdx.x; l < count; l += BLOCK) {
    PowerState& p = ps[l];
    if (p.stopped) continue;
    double lam = 0.0, nw2 = 0.0;
#pragma unroll 4  // independent record loads in flight together
    for (int t = lp_tiles[l]; t < lp_tiles[l + 1]; ++t) {
      lam += __ldcg(rec + (size_t)t * kRecP);
      nw2 += __ldcg(rec + (size_t)t * kRecP + 1);
    }
    p.k += 1;
    p.lam = lam;
    const double nw = sqrt(nw2);
    if (nw == 0.0) {
      p.stopped = 1;
      p.inv_norm = 0.0;
      continue;
    }
    p.inv_norm = 1.0 / nw;
    if (p.k > 1 && fabs(lam - p.lam_prev) <= p.rel_tol * lam) p.stopped = 1;
    p.lam_prev = lam;
    if (p.k >= p.max_iter) p.stopped = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) *ticket = 0;
}

// v <- w / |w| per LP (rows of A^T's tiles); with init = 1: v = 1/sqrt(n_l)
__global__ void k_bpow_norm(SchedView S, const double* w, double* v, const PowerState* ps,
                            const int64_t* n_off, int init) {
  for (int t = blockIdx.x; t < S.ntiles; t += gridDim.x) {
    const Tile tl = S.tiles[t];
    if (tl.split >= 0 && tl.part != 0) continue;
    double s;
    if (init) {
      s = 1.0 / sqrt((double)(n_off[tl.lp + 1] - n_off[tl.lp]));
    } else {
      if (ps[tl.lp].stopped) continue;
      s = ps[tl.lp].inv_norm;
    }
    for (int j = tl.row_begin + threadIdx.x; j < tl.row_end; j += blockDim.x)
      v[j] = init ? s : w[j] * s;
  }
}

__global__ void k_bpow_init(PowerState* ps, int count, int max_iter, double rel_tol) {
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < count; l += gridDim.x * blockDim.x) {
    PowerState& p = ps[l];
    p.lam = p.lam_prev = p.inv_norm = 0.0;
    p.k = 0;
    p.max_iter = max_iter;
    p.stopped = max_iter <= 0 ? 1 : 0;
    p.ticket = 0;
    p.rel_tol = rel_tol;
  }
}

// per-LP norms and the scalar set-up (one block per LP)
template <int BLOCK>
__global__ void k_binit(Scalars* sc, const PowerState* ps, const int64_t* m_off,
                        const int64_t* n_off, const double* b, const double* c,
                        const double* b_t, const double* c_t, double eta_safety) {
  __shared__ double red[5 * (BLOCK / 32)];
  const int l = blockIdx.x;
  double v[5] = {0, 0, 0, 0, 0};
  for (int64_t i = m_off[l] + threadIdx.x; i < m_off[l + 1]; i += BLOCK) {
    v[0] += b[i] * b[i];
    v[2] += b_t[i] * b_t[i];
  }
  for (int64_t j = n_off[l] + threadIdx.x; j < n_off[l + 1]; j += BLOCK) {
    v[1] += c[j] * c[j];
    v[3] += c_t[j] * c_t[j];
    const double mc = fmin(0.0, c_t[j]);
    v[4] += mc * mc;
  }
  double o[5];
  block_sum<BLOCK, 5>(v, o, red);
  if (threadIdx.x != 0) return;
  Scalars& s = sc[l];
  const double smax = sqrt(fmax(ps[l].lam, 0.0));
  s.eta = smax > 0.0 ? eta_safety / smax : 1.0;
  const double nb = sqrt(o[2]), nc = sqrt(o[3]);
  s.omega = (nb > 0.0 && nc > 0.0) ? nc / nb : 1.0;
  s.tau = s.eta / s.omega;
  s.sigma = s.eta * s.omega;
  s.norm_b = sqrt(o[0]);
  s.norm_c = sqrt(o[1]);
  const double w2 = s.omega * s.omega;
  s.kkt_last = sqrt(w2 * o[2] + o[4] / w2);
  s.kkt_prev = s.kkt_last;
}

// ---------------------------------------------------------------------------
// float64 report and Algorithm 1 per LP
// ---------------------------------------------------------------------------
// the returned iterate of each LP (average if that passed the test) in float64
// checking = true: only the LPs with a pending float64 check, their screened
// candidate
template <typename T>
__device__ __forceinline__ void bchoose_body(const SchedView& Sn, const SchedView& Sm,
                                             const Scalars* sc, const T* x, const T* x_avg,
                                             const T* y, const T* y_avg, double* xs, double* ys,
                                             bool checking) {
  for (int t = blockIdx.x; t < Sn.ntiles; t += gridDim.x) {
    const Tile tl = Sn.tiles[t];
    if (tl.split >= 0 && tl.part != 0) continue;
    const Scalars& s = sc[tl.lp];
    if (checking && !s.verify) continue;
    const bool avg = checking ? s.verify_avg != 0 : (s.done && s.status == 0 && s.chosen_avg);
    for (int j = tl.row_begin + threadIdx.x; j < tl.row_end; j += blockDim.x)
      xs[j] = (double)(avg ? x_avg[j] : x[j]);
  }
  for (int t = blockIdx.x; t < Sm.ntiles; t += gridDim.x) {
    const Tile tl = Sm.tiles[t];
    if (tl.split >= 0 && tl.part != 0) continue;
    const Scalars& s = sc[tl.lp];
    if (checking && !s.verify) continue;
    const bool avg = checking ? s.verify_avg != 0 : (s.done && s.status == 0 && s.chosen_avg);
    for (int i = tl.row_begin + threadIdx.x; i < tl.row_end; i += blockDim.x)
      ys[i] = (double)(avg ? y_avg[i] : y[i]);
  }
}

template <typename T>
__global__ void k_bchoose(SchedView Sn, SchedView Sm, const Scalars* sc, const T* x, const T* x_avg,
                          const T* y, const T* y_avg, double* xs, double* ys, bool checking) {
  bchoose_body<T>(Sn, Sm, sc, x, x_avg, y, y_avg, xs, ys, checking);
}

// gate (optional): only the tiles of LPs with a pending float64 check
template <int BLOCK>
struct BRepNEpi {
  const double *x_s, *c_t, *D_c;
  double *x_out, *z_out, *rec, *red;
  const Scalars* gate;
  double u2, s3, xz, inf;
  __device__ __forceinline__ bool begin_tile(const Tile& tl) {
    u2 = s3 = xz = inf = 0.0;
    return !gate || gate[tl.lp].verify;
  }
  __device__ __forceinline__ void row(int j, const double (&s)[1], int) {
    const double d = c_t[j] - s[0];
    const double zs = fmax(0.0, d), rd = fmin(0.0, d) / D_c[j];
    if (x_out) x_out[j] = D_c[j] * x_s[j];
    if (z_out) z_out[j] = zs / D_c[j];
    u2 += rd * rd;
    s3 += c_t[j] * x_s[j];
    xz += x_s[j] * zs;
    inf = fmax(inf, fabs(rd));
  }
  __device__ __forceinline__ void end_tile(const Tile&, int t) {
    const double v[3] = {u2, s3, xz};
    double o[3];
    block_sum<BLOCK, 3>(v, o, red);
    double mx = inf;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, off));
    __shared__ double wmx[BLOCK / 32];
    if ((threadIdx.x & 31) == 0) wmx[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < BLOCK / 32; ++w) mx = fmax(mx, wmx[w]);
      rec[(size_t)t * kRecR + 0] = o[0];
      rec[(size_t)t * kRecR + 1] = o[1];
      rec[(size_t)t * kRecR + 2] = o[2];
      rec[(size_t)t * kRecR + 3] = mx;
    }
    __syncthreads();
  }
};

template <int BLOCK>
struct BRepMEpi {
  const double *y_s, *b_t, *D_r;
  double *y_out, *rec, *red;
  const Scalars* gate;
  double u1, s4, inf;
  __device__ __forceinline__ bool begin_tile(const Tile& tl) {
    u1 = s4 = inf = 0.0;
    return !gate || gate[tl.lp].verify;
  }
  __device__ __forceinline__ void row(int i, const double (&s)[1], int) {
    const double rp = (b_t[i] - s[0]) / D_r[i];
    if (y_out) y_out[i] = D_r[i] * y_s[i];
    u1 += rp * rp;
    s4 += b_t[i] * y_s[i];
    inf = fmax(inf, fabs(rp));
  }
  __device__ __forceinline__ void end_tile(const Tile&, int t) {
    const double v[2] = {u1, s4};
    double o[2];
    block_sum<BLOCK, 2>(v, o, red);
    double mx = inf;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, off));
    __shared__ double wmx[BLOCK / 32];
    if ((threadIdx.x & 31) == 0) wmx[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < BLOCK / 32; ++w) mx = fmax(mx, wmx[w]);
      rec[(size_t)t * kRecR + 0] = o[0];
      rec[(size_t)t * kRecR + 1] = o[1];
      rec[(size_t)t * kRecR + 2] = 0.0;
      rec[(size_t)t * kRecR + 3] = mx;
    }
    __syncthreads();
  }
};

template <int BLOCK>
__device__ __forceinline__ void brep_n_body(const SchedView& S, const int32_t* rp, const int32_t* col,
                                            const double* val, const double* x_s, const double* y_s,
                                            const double* c_t, const double* D_c, double* x_out,
                                            double* z_out, double* rec, const Scalars* gate,
                                            unsigned char* smem) {
  __shared__ double red[3 * (BLOCK / 32)];
  BRepNEpi<BLOCK> epi{x_s, c_t, D_c, x_out, z_out, rec, red, gate, 0, 0, 0, 0};
  Gather<double, 1> g{{y_s}};
  run_tiles<double, 1, BLOCK, kFixedE>(S, rp, col, val, g, epi, smem);
}

template <int BLOCK>
__device__ __forceinline__ void brep_m_body(const SchedView& S, const int32_t* rp, const int32_t* col,
                                            const double* val, const double* x_s, const double* y_s,
                                            const double* b_t, const double* D_r, double* y_out,
                                            double* rec, const Scalars* gate, unsigned char* smem) {
  __shared__ double red[2 * (BLOCK / 32)];
  BRepMEpi<BLOCK> epi{y_s, b_t, D_r, y_out, rec, red, gate, 0, 0, 0};
  Gather<double, 1> g{{x_s}};
  run_tiles<double, 1, BLOCK, kFixedE>(S, rp, col, val, g, epi, smem);
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_brep_n(SchedView S, const int32_t* rp, const int32_t* col,
                                                 const double* val, const double* x_s,
                                                 const double* y_s, const double* c_t,
                                                 const double* D_c, double* x_out, double* z_out,
                                                 double* rec, const Scalars* gate) {
  extern __shared__ __align__(16) unsigned char smem[];
  brep_n_body<BLOCK>(S, rp, col, val, x_s, y_s, c_t, D_c, x_out, z_out, rec, gate, smem);
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_brep_m(SchedView S, const int32_t* rp, const int32_t* col,
                                                 const double* val, const double* x_s,
                                                 const double* y_s, const double* b_t,
                                                 const double* D_r, double* y_out, double* rec,
                                                 const Scalars* gate) {
  extern __shared__ __align__(16) unsigned char smem[];
  brep_m_body<BLOCK>(S, rp, col, val, x_s, y_s, b_t, D_r, y_out, rec, gate, smem);
}

// out[l][8] = {r_P, r_D, gap, max violation, c^T x, b^T y, x^T z, 0}
__global__ void k_brep_final(const double* rec_n, const int32_t* lp_n, const double* rec_m,
                             const int32_t* lp_m, int count, double* out) {
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < count; l += gridDim.x * blockDim.x) {
    double u2 = 0, s3 = 0, xz = 0, ird = 0, u1 = 0, s4 = 0, irp = 0;
    for (int t = lp_n[l]; t < lp_n[l + 1]; ++t) {
      u2 += rec_n[(size_t)t * kRecR];
      s3 += rec_n[(size_t)t * kRecR + 1];
      xz += rec_n[(size_t)t * kRecR + 2];
      ird = fmax(ird, rec_n[(size_t)t * kRecR + 3]);
    }
    for (int t = lp_m[l]; t < lp_m[l + 1]; ++t) {
      u1 += rec_m[(size_t)t * kRecR];
      s4 += rec_m[(size_t)t * kRecR + 1];
      irp = fmax(irp, rec_m[(size_t)t * kRecR + 3]);
    }
    double* o = out + (size_t)l * 8;
    o[0] = sqrt(u1);
    o[1] = sqrt(u2);
    o[2] = fabs(s3 - s4);
    o[3] = fmax(fmax(irp, ird), xz / (1.0 + fabs(s3)));
    o[4] = s3;
    o[5] = s4;
    o[6] = xz;
    o[7] = 0.0;
  }
}

// Float64 check of each LP whose screen passed: the Section 2 test at eps on
// its report records; an LP that passes is finished (one fewer active LP)
__device__ __forceinline__ void bfp64_final_body(const double* rec_n, const int32_t* lp_n,
                                                 const double* rec_m, const int32_t* lp_m, int count,
                                                 Scalars* sc, int32_t* ctl) {
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < count; l += gridDim.x * blockDim.x) {
    Scalars& s = sc[l];
    if (!s.verify) continue;
    double u2 = 0, s3 = 0, u1 = 0, s4 = 0;
    for (int t = lp_n[l]; t < lp_n[l + 1]; ++t) {
      u2 += rec_n[(size_t)t * kRecR];
      s3 += rec_n[(size_t)t * kRecR + 1];
    }
    for (int t = lp_m[l]; t < lp_m[l + 1]; ++t) {
      u1 += rec_m[(size_t)t * kRecR];
      s4 += rec_m[(size_t)t * kRecR + 1];
    }
    eval_fp64_check(s, u1, u2, s3, s4, nullptr, nullptr, nullptr);
    if (s.done) atomicSub(ctl, 1);
  }
}

__global__ void k_bfp64_final(const double* rec_n, const int32_t* lp_n, const double* rec_m,
                              const int32_t* lp_m, int count, Scalars* sc, int32_t* ctl) {
  bfp64_final_body(rec_n, lp_n, rec_m, lp_m, count, sc, ctl);
}

// Algorithm 1 per LP: z~ = max(0, c~ - A~^T y~) and x~^T z~ per tile
template <int BLOCK>
struct BWsEpi {
  const double *x_s, *c_t;
  double *z_s, *rec, *red;
  double xz;
  __device__ __forceinline__ bool begin_tile(const Tile&) {
    xz = 0.0;
    return true;
  }
  __device__ __forceinline__ void row(int j, const double (&s)[1], int) {
    const double z = fmax(0.0, c_t[j] - s[0]);
    z_s[j] = z;
    xz += x_s[j] * z;
  }
  __device__ __forceinline__ void end_tile(const Tile&, int t) {
    const double v[1] = {xz};
    double o[1];
    block_sum<BLOCK, 1>(v, o, red);
    if (threadIdx.x == 0) rec[t] = o[0];
  }
};

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_bws_z(SchedView S, const int32_t* rp, const int32_t* col,
                                                const double* val, const double* x_s,
                                                const double* y_s, const double* c_t, double* z_s,
                                                double* rec) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[BLOCK / 32];
  BWsEpi<BLOCK> epi{x_s, c_t, z_s, rec, red, 0.0};
  Gather<double, 1> g{{y_s}};
  run_tiles<double, 1, BLOCK, kFixedE>(S, rp, col, val, g, epi, smem);
}

__global__ void k_bws_mu(const double* rec, const int32_t* lp_tiles, const int64_t* n_off,
                         int count, double mu_min, double* mu) {
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < count; l += gridDim.x * blockDim.x) {
    double s = 0.0;
#pragma unroll 4  // independent record loads in flight together
    for (int t = lp_tiles[l]; t < lp_tiles[l + 1]; ++t) s += rec[t];
    mu[l] = fmax(s / (double)(n_off[l + 1] - n_off[l]), mu_min);
  }
}

__device__ __forceinline__ double bws_move(double target, double v, double delta) {
  return fmin(fmax(target, v - delta), v + delta);
}

__global__ void k_bws_apply(SchedView Sn, SchedView Sm, const double* x_s, const double* z_s,
                            const double* y_s, const double* mu, double delta, double alpha,
                            int unscaled, const double* D_r, const double* D_c, double* x_out,
                            double* y_out, double* z_out) {
  for (int t = blockIdx.x; t < Sn.ntiles; t += gridDim.x) {
    const Tile tl = Sn.tiles[t];
    if (tl.split >= 0 && tl.part != 0) continue;
    const double m_t = mu[tl.lp];
    for (int j = tl.row_begin + threadIdx.x; j < tl.row_end; j += blockDim.x) {
      double xp = fmax(x_s[j], alpha), zp = fmax(z_s[j], alpha);
      if (xp < zp) {
        xp = bws_move(m_t / zp, xp, delta);
        zp = bws_move(m_t / xp, zp, delta);
      } else {
        zp = bws_move(m_t / xp, zp, delta);
        xp = bws_move(m_t / zp, xp, delta);
      }
      if (unscaled) {
        xp = D_c[j] * xp;
        zp = zp / D_c[j];
      }
      x_out[j] = xp;
      z_out[j] = zp;
    }
  }
  for (int t = blockIdx.x; t < Sm.ntiles; t += gridDim.x) {
    const Tile tl = Sm.tiles[t];
    if (tl.split >= 0 && tl.part != 0) continue;
    for (int i = tl.row_begin + threadIdx.x; i < tl.row_end; i += blockDim.x)
      y_out[i] = unscaled ? D_r[i] * y_s[i] : y_s[i];
  }
}

// local column indices -> global (block per LP), with range and order checks
__global__ void k_bglobalize(const int64_t* nnz_off, const int64_t* n_off, int32_t* col,
                             int32_t* flags) {
  const int l = blockIdx.x;
  const int64_t n_l = n_off[l + 1] - n_off[l];
  int f = 0;
  for (int64_t k = nnz_off[l] + threadIdx.x; k < nnz_off[l + 1]; k += blockDim.x) {
    const int c = col[k];
    if (c < 0 || c >= n_l) f |= 1;
  }
  if (f) atomicOr(flags, f);
  __syncthreads();
  for (int64_t k = nnz_off[l] + threadIdx.x; k < nnz_off[l + 1]; k += blockDim.x)
    col[k] = (int32_t)(col[k] + n_off[l]);
}

// ---------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------

template <int E>
static cudaError_t configure_batch_e(size_t mx) {
  cudaError_t e = cudaSuccess;
  for (const void* f :
       {(const void*)k_bprimal<float, kBlock, E>, (const void*)k_bprimal<double, kBlock, E>,
        (const void*)k_bdual<float, kBlock, E>, (const void*)k_bdual<double, kBlock, E>,
        (const void*)k_beval<float, kBlock, E>, (const void*)k_beval<double, kBlock, E>}) {
    cudaError_t r = set_max_dyn_smem(f, mx);
    if (r != cudaSuccess) e = r;
  }
  return e;
}

struct PersistArgs;
template <typename T>
__global__ void __launch_bounds__(kBlock, 1) k_bpersist(BatchBuffers<T> B, PersistArgs P);

static cudaError_t configure_batch_kernels(size_t mx) {
  cudaError_t e = configure_batch_e<8>(mx);
  if (e == cudaSuccess) e = configure_batch_e<32>(mx);
  if (e == cudaSuccess) e = configure_batch_e<16>(mx);
  if (e == cudaSuccess) e = configure_batch_e<-4>(mx);
  if (e == cudaSuccess) e = configure_batch_e<-8>(mx);
  for (const void* f : {(const void*)k_bpow_Av<kBlock>, (const void*)k_bpow_ATu<kBlock>,
                        (const void*)k_brep_n<kBlock>, (const void*)k_brep_m<kBlock>,
                        (const void*)k_bws_z<kBlock>, (const void*)k_bpersist<float>,
                        (const void*)k_bpersist<double>}) {
    cudaError_t r = set_max_dyn_smem(f, mx);
    if (r != cudaSuccess) e = r;
  }
  return e;
}

template <typename T>
static BatchBuffers<T> batch_buffers(pdhg_ctx* ctx) {
  BatchBuffers<T> B{};
  IterBuffers<T>& I = B.it;
  I.a_rp = ctx->a_rp;
  I.a_col = ctx->a_col;
  I.t_rp = ctx->t_rp;
  I.t_col = ctx->t_col;
  if constexpr (sizeof(T) == 4) {
    I.a_val = (const T*)ctx->a_val32;
    I.t_val = (const T*)ctx->t_val32;
    I.c_t = (const T*)ctx->c_t32;
    I.b_t = (const T*)ctx->b_t32;
  } else {
    I.a_val = (const T*)ctx->a_val64;
    I.t_val = (const T*)ctx->t_val64;
    I.c_t = (const T*)ctx->c_t64;
    I.b_t = (const T*)ctx->b_t64;
  }
  I.a_sched = ctx->sa.view;
  I.t_sched = ctx->st.view;
  I.x = (T*)ctx->x;
  I.y = (T*)ctx->y;
  I.x_avg = (T*)ctx->x_avg;
  I.y_avg = (T*)ctx->y_avg;
  I.x_last = (T*)ctx->x_last;
  I.y_last = (T*)ctx->y_last;
  I.Ax = (T*)ctx->Ax;
  I.Ax_avg = (T*)ctx->Ax_avg;
  I.Ax_last = (T*)ctx->Ax_last;
  I.c_t64 = ctx->c_t64;
  I.b_t64 = ctx->b_t64;
  I.D_r = ctx->D_r;
  I.D_c = ctx->D_c;
  I.Dr_inv = ctx->Dr_inv;
  I.Dc_inv = ctx->Dc_inv;
  I.sc = ctx->sc;
  I.m = ctx->m;
  I.n = ctx->n;
  B.rec_t = ctx->rec_t;
  B.rec_a = ctx->rec_a;
  B.lp_t_tiles = ctx->lp_t_tiles;
  B.lp_a_tiles = ctx->lp_a_tiles;
  B.ctl = ctx->active;
  B.count = ctx->count;
  return B;
}

template <typename T>
static void enqueue_bchunk(pdhg_ctx* ctx, int len) {
  const BatchBuffers<T> B = batch_buffers<T>(ctx);
  ctx->launches += 2LL * len + 2;
  for (int i = 0; i < len; ++i) {
    PDHG_DISPATCH_E(B.it.t_sched.e,
                     (k_bprimal<T, kBlock, E_><<<ctx->l_prim.grid, kBlock, ctx->l_prim.smem,
                                                  ctx->stream>>>(B, i)));
    PDHG_DISPATCH_E(B.it.a_sched.e,
                     (k_bdual<T, kBlock, E_><<<ctx->l_dual.grid, kBlock, ctx->l_dual.smem,
                                                ctx->stream>>>(B, i)));
  }
  PDHG_DISPATCH_E(B.it.t_sched.e,
                   (k_beval<T, kBlock, E_><<<ctx->l_eval.grid, kBlock, ctx->l_eval.smem,
                                              ctx->stream>>>(B, len)));
  if constexpr (sizeof(T) == 4) {
    // float64 check of the LPs whose screen passed
    k_bchoose<T><<<ctx->restart_grid, 256, 0, ctx->stream>>>(
        ctx->st8.view, ctx->sa8.view, ctx->sc, B.it.x, B.it.x_avg, B.it.y, B.it.y_avg, ctx->xs64,
        ctx->ys64, true);
    k_brep_n<kBlock><<<ctx->l_t64.grid, kBlock, ctx->l_t64.smem, ctx->stream>>>(
        ctx->st8.view, ctx->t_rp, ctx->t_col, ctx->t_val64, ctx->xs64, ctx->ys64, ctx->c_t64,
        ctx->D_c, nullptr, nullptr, ctx->rec_t, ctx->sc);
    k_brep_m<kBlock><<<ctx->l_a64.grid, kBlock, ctx->l_a64.smem, ctx->stream>>>(
        ctx->sa8.view, ctx->a_rp, ctx->a_col, ctx->a_val64, ctx->xs64, ctx->ys64, ctx->b_t64,
        ctx->D_r, nullptr, ctx->rec_a, ctx->sc);
    k_bfp64_final<<<(ctx->count + 255) / 256, 256, 0, ctx->stream>>>(
        ctx->rec_t, ctx->lp_t8_tiles, ctx->rec_a, ctx->lp_a8_tiles, ctx->count, ctx->sc,
        ctx->active);
    ctx->launches += kFp64CheckLaunches;
  }
  k_brestart<T><<<ctx->restart_grid, 256, 0, ctx->stream>>>(B);
}

void enqueue_batch_chunk(pdhg_ctx* ctx, int len) {
  if (ctx->mixed)
    enqueue_bchunk<float>(ctx, len);
  else
    enqueue_bchunk<double>(ctx, len);
}

// ---------------------------------------------------------------------------
// Persistent batched solve: one cooperative launch runs every chunk (the
// half-steps, the evaluation, the float64 check and the restart) with a
// grid-wide barrier between phases.  Each barrier's wait is bounded: past the
// limit the block records a timeout and every block returns at its next
// barrier, so the host reads PDHG_TIMEOUT instead of waiting on a hang.
// ---------------------------------------------------------------------------
struct GridSync {
  unsigned int count, gen;
  int err;    // 1: a barrier's wait ran past its limit
  int extra;  // arrivals a barrier waits for beyond the grid: 0 (1 tests the bounded wait)
};

struct PersistArgs {
  GridSync* gs;
  unsigned long long limit_ns;
  long long k0, max_iter;
  int eval_freq;
  // the float64 check of screened float32-mixed candidates
  SchedView st8, sa8;
  const double *t_val64, *a_val64;
  double *xs64, *ys64;
  const int32_t *lp_t8, *lp_a8;
};

// false in every thread of the block once any block's wait ran past limit_ns
__device__ __forceinline__ bool grid_barrier(GridSync* g, unsigned long long limit_ns) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = &g->gen;
    volatile int* verr = &g->err;
    const unsigned int gen0 = *vgen;  // read before arriving: only the last arrival moves it
    const unsigned int want = gridDim.x + (unsigned int)g->extra;
    __threadfence();
    int res = 1;
    if (atomicAdd(&g->count, 1u) == want - 1u) {
      atomicExch(&g->count, 0u);
      __threadfence();
      atomicAdd(&g->gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (*vgen == gen0) {
        if (*verr != 0) {
          res = 0;
          break;
        }
        if (global_ns() - t0 > limit_ns) {
          atomicExch(&g->err, 1);
          res = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    ok = res && *verr == 0;
  }
  __syncthreads();
  return ok != 0;
}

template <typename T>
__global__ void __launch_bounds__(kBlock, 1) k_bpersist(BatchBuffers<T> B, PersistArgs P) {
  extern __shared__ __align__(16) unsigned char smem[];
  const IterBuffers<T>& I = B.it;
  const long long F = P.eval_freq;
  long long k = P.k0;
  while (k < P.max_iter) {
    const long long next = min((k / F + 1) * F, P.max_iter);
    const int len = (int)(next - k);
    for (int i = 0; i < len; ++i) {
      bprimal_body<T, kBlock, kFixedE>(B, i, smem);
      if (!grid_barrier(P.gs, P.limit_ns)) return;
      bdual_body<T, kBlock, kFixedE>(B, i, smem);
      if (!grid_barrier(P.gs, P.limit_ns)) return;
    }
    beval_body<T, kBlock, kFixedE>(B, len, smem);
    if (!grid_barrier(P.gs, P.limit_ns)) return;
    if constexpr (sizeof(T) == 4) {
      bchoose_body<T>(P.st8, P.sa8, I.sc, I.x, I.x_avg, I.y, I.y_avg, P.xs64, P.ys64, true);
      if (!grid_barrier(P.gs, P.limit_ns)) return;
      brep_n_body<kBlock>(P.st8, I.t_rp, I.t_col, P.t_val64, P.xs64, P.ys64, I.c_t64, I.D_c,
                          nullptr, nullptr, B.rec_t, I.sc, smem);
      brep_m_body<kBlock>(P.sa8, I.a_rp, I.a_col, P.a_val64, P.xs64, P.ys64, I.b_t64, I.D_r,
                          nullptr, B.rec_a, I.sc, smem);
      if (!grid_barrier(P.gs, P.limit_ns)) return;
      bfp64_final_body(B.rec_t, P.lp_t8, B.rec_a, P.lp_a8, B.count, I.sc, B.ctl);
      if (!grid_barrier(P.gs, P.limit_ns)) return;
    }
    brestart_body<T>(B);
    if (!grid_barrier(P.gs, P.limit_ns)) return;
    k = next;
    if (*reinterpret_cast<volatile int32_t*>(B.ctl) == 0) break;  // every LP has finished
  }
}

// shared memory of the persistent kernel: its iteration and evaluation phases
// on the fixed E = 8 schedules (one or two gathered vectors in the iteration
// precision) and the float64 report passes
static size_t persist_smem(const pdhg_ctx* ctx) {
  const SchedView &A = ctx->sa8.view, &T = ctx->st8.view;
  const bool mx = ctx->mixed;
  return std::max({smem_for(0, mx, A.max_rows, A.e), smem_for(0, mx, T.max_rows, T.e),
                   smem_for(1, mx, T.max_rows, T.e), ctx->l_t64.smem, ctx->l_a64.smem});
}

// the whole solve from iteration k0 to max_iter in one cooperative launch
template <typename T>
static pdhg_status persistent_solve(pdhg_ctx* ctx, long long k0, long long max_iter) {
  const GridSync g{0u, 0u, 0, ctx->opt.wait_test ? 1 : 0};
  CK(cudaMemcpyAsync(ctx->gsync, &g, sizeof(g), cudaMemcpyHostToDevice, ctx->stream));
  // every phase on the fixed E = 8 schedules (the per-LP tile ranges with them)
  BatchBuffers<T> B = batch_buffers<T>(ctx);
  B.it.a_sched = ctx->sa8.view;
  B.it.t_sched = ctx->st8.view;
  B.lp_a_tiles = ctx->lp_a8_tiles;
  B.lp_t_tiles = ctx->lp_t8_tiles;
  PersistArgs P{};
  P.gs = static_cast<GridSync*>(ctx->gsync);
  P.limit_ns = (unsigned long long)ctx->opt.wait_limit_ms * 1000000ull;
  P.k0 = k0;
  P.max_iter = max_iter;
  P.eval_freq = ctx->opt.eval_freq;
  P.st8 = ctx->st8.view;
  P.sa8 = ctx->sa8.view;
  P.t_val64 = ctx->t_val64;
  P.a_val64 = ctx->a_val64;
  P.xs64 = ctx->xs64;
  P.ys64 = ctx->ys64;
  P.lp_t8 = ctx->lp_t8_tiles;
  P.lp_a8 = ctx->lp_a8_tiles;
  const size_t smem = persist_smem(ctx);
  const void* f = reinterpret_cast<const void*>(k_bpersist<T>);
  int per_sm = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bpersist<T>, kBlock, smem));
  if (per_sm < 1) {
    set_error("persistent batched solve: the kernel does not fit on an SM (%zu bytes of shared memory)",
              smem);
    return PDHG_CUDA_ERROR;
  }
  const int grid = per_sm * ctx->nsm;
  void* args[] = {&B, &P};
  CK(cudaLaunchCooperativeKernel(f, grid, kBlock, args, smem, ctx->stream));
  ctx->launches += 1;
  GridSync out{};
  CK(cudaMemcpyAsync(&out, ctx->gsync, sizeof(out), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaGetLastError());
  if (out.err) {
    set_error("persistent batched solve: a grid barrier waited longer than %d ms; the iterates "
              "are not meaningful",
              ctx->opt.wait_limit_ms);
    return PDHG_TIMEOUT;
  }
  return PDHG_OK;
}

pdhg_status batch_persistent_solve(pdhg_ctx* ctx, long long k0, long long max_iter) {
  return ctx->mixed ? persistent_solve<float>(ctx, k0, max_iter)
                    : persistent_solve<double>(ctx, k0, max_iter);
}

}  // namespace pdhg

using namespace pdhg;

// ---------------------------------------------------------------------------
// host API
// ---------------------------------------------------------------------------
static pdhg_status batch_schedules(pdhg_ctx* ctx, int32_t** lp_a, int32_t** lp_t, DevSched* sa,
                                   DevSched* st, int e) {
  HostSched ha = build_sched(ctx->h_a_rp.data(), ctx->m, e, ctx->h_m_off.data(), ctx->count);
  HostSched ht = build_sched(ctx->h_t_rp.data(), ctx->n, e, ctx->h_n_off.data(), ctx->count);
  CKS(upload_sched(ctx, ha, sa, ctx->a_rp));
  CKS(upload_sched(ctx, ht, st, ctx->t_rp));
  CKS(dalloc(ctx, lp_a, (size_t)ctx->count + 1));
  CKS(dalloc(ctx, lp_t, (size_t)ctx->count + 1));
  CK(cudaMemcpyAsync(*lp_a, ha.lp_tiles.data(), sizeof(int32_t) * (ctx->count + 1),
                     cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(*lp_t, ht.lp_tiles.data(), sizeof(int32_t) * (ctx->count + 1),
                     cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return PDHG_OK;
}

// Time the real batched primal (rows of A~^T) or dual (rows of A~) kernel.
template <typename T>
static pdhg_status time_batch_kernel(pdhg_ctx* ctx, bool on_a, float* ms_out) {
  const BatchBuffers<T> B = batch_buffers<T>(ctx);
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const int warm = 3, reps = 10;
  ctx->launches += warm + reps;
  for (int it = 0; it < warm + reps; ++it) {
    if (it == warm) CK(cudaEventRecord(e0, ctx->stream));
    if (on_a) {
      PDHG_DISPATCH_E(B.it.a_sched.e,
                       (k_bdual<T, kBlock, E_><<<ctx->l_dual.grid, kBlock, ctx->l_dual.smem,
                                                  ctx->stream>>>(B, 0)));
    } else {
      PDHG_DISPATCH_E(B.it.t_sched.e,
                       (k_bprimal<T, kBlock, E_><<<ctx->l_prim.grid, kBlock, ctx->l_prim.smem,
                                                    ctx->stream>>>(B, 0)));
    }
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

// LP-aligned iteration schedules picked by timing the candidates with the
// real batched kernels on the initial state (zeroed again afterwards); E = 8
// is kept unless another choice is more than 5% faster.
static pdhg_status tune_batch_schedules(pdhg_ctx* ctx) {
  const int count = ctx->count;
  const bool mx = ctx->mixed;
  for (int which = 0; which < 2; ++which) {
    const bool on_a = which == 0;
    const std::vector<int32_t>& rp = on_a ? ctx->h_a_rp : ctx->h_t_rp;
    const int nrows = on_a ? ctx->m : ctx->n;
    const int64_t* off = on_a ? ctx->h_m_off.data() : ctx->h_n_off.data();
    std::vector<int> cands = {kFixedE};
    if (ctx->opt.autotune) cands = {8, 16, 32};  // vector variants: never faster (measured)
    DevSched best = on_a ? ctx->sa8 : ctx->st8;
    int32_t* best_lp = on_a ? ctx->lp_a8_tiles : ctx->lp_t8_tiles;
    float best_ms = 1e30f;
    for (int e : cands) {
      DevSched d;
      int32_t* lpt = nullptr;
      if (e == kFixedE) {
        d = on_a ? ctx->sa8 : ctx->st8;
        lpt = on_a ? ctx->lp_a8_tiles : ctx->lp_t8_tiles;
      } else {
        HostSched h = build_sched(rp.data(), nrows, e, off, count);
        CKS(upload_sched(ctx, h, &d, on_a ? ctx->a_rp : ctx->t_rp));
        CKS(dalloc(ctx, &lpt, (size_t)count + 1));
        CK(cudaMemcpyAsync(lpt, h.lp_tiles.data(), sizeof(int32_t) * (count + 1),
                           cudaMemcpyHostToDevice, ctx->stream));
      }
      (on_a ? ctx->sa : ctx->st) = d;
      if (on_a)
        ctx->l_dual = make_launch(ctx, mx ? 2 : 3, d.view.e,
                                  smem_for(0, mx, d.view.max_rows, d.view.e), d.view.ntiles);
      else
        ctx->l_prim = make_launch(ctx, mx ? 0 : 1, d.view.e,
                                  smem_for(0, mx, d.view.max_rows, d.view.e), d.view.ntiles);
      float ms = 0.f;
      if (cands.size() > 1) {
        if (mx)
          CKS(time_batch_kernel<float>(ctx, on_a, &ms));
        else
          CKS(time_batch_kernel<double>(ctx, on_a, &ms));
      }
      const float bias = (e == 8) ? 0.95f : 1.0f;
      if (ctx->opt.verbose)
        std::fprintf(stderr, "pdhg_create: tune %s variant %3d: %8.4f ms\n",
                     on_a ? "A  " : "A^T", e, ms);
      if (ms * bias < best_ms) {
        best_ms = ms * bias;
        best = d;
        best_lp = lpt;
      }
    }
    (on_a ? ctx->sa : ctx->st) = best;
    (on_a ? ctx->lp_a_tiles : ctx->lp_t_tiles) = best_lp;
  }
  const SchedView &A = ctx->sa.view, &T = ctx->st.view;
  ctx->l_prim = make_launch(ctx, mx ? 0 : 1, T.e, smem_for(0, mx, T.max_rows, T.e), T.ntiles);
  ctx->l_dual = make_launch(ctx, mx ? 2 : 3, A.e, smem_for(0, mx, A.max_rows, A.e), A.ntiles);
  ctx->l_eval = make_launch(ctx, mx ? 4 : 5, T.e, smem_for(1, mx, T.max_rows, T.e),
                            std::max(T.ntiles, A.ntiles));
  if (std::max(A.ntiles, T.ntiles) > ctx->rec_tiles) {
    ctx->rec_tiles = std::max(A.ntiles, T.ntiles);
    CKS(dalloc(ctx, &ctx->rec_t, (size_t)ctx->rec_tiles * kEvalQ));
    CKS(dalloc(ctx, &ctx->rec_a, (size_t)ctx->rec_tiles * kEvalQ));
  }
  const size_t es = elem(ctx);
  for (void* p : {ctx->x, ctx->x_avg, ctx->x_last})
    CK(cudaMemsetAsync(p, 0, es * ctx->n, ctx->stream));
  for (void* p : {ctx->y, ctx->y_avg, ctx->y_last, ctx->Ax, ctx->Ax_avg, ctx->Ax_last})
    CK(cudaMemsetAsync(p, 0, es * ctx->m, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return PDHG_OK;
}

// every LP's scalar state as before its first iteration (the step sizes and
// weights are set by k_binit from the power iteration and the scaled b, c)
static pdhg_status batch_fresh_scalars(pdhg_ctx* ctx) {
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
  h.log_cap = 0;
  h.status = PDHG_MAX_ITER;
  std::vector<Scalars> hv(ctx->count, h);
  CK(cudaMemcpyAsync(ctx->sc, hv.data(), sizeof(Scalars) * ctx->count, cudaMemcpyHostToDevice,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return PDHG_OK;
}

__global__ void k_bfinite(int64_t len, const double* __restrict__ v, int32_t* flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(v[i])) atomicOr(flag, 1);
}

static pdhg_status batch_create_impl(pdhg_ctx* ctx, const int32_t* m, const int32_t* n,
                                     const int32_t* row_ptr, const int32_t* col,
                                     const double* val, const double* b, const double* c) {
  const int count = ctx->count;
  StageClock stage{ctx};
  CKS(setup_device(ctx));
  CK(configure_batch_kernels(ctx->smem_optin));
  stage("device set-up");
  // offsets and the stacked row pointer on the host
  ctx->h_m_off.assign(count + 1, 0);
  ctx->h_n_off.assign(count + 1, 0);
  for (int l = 0; l < count; ++l) {
    ctx->h_m_off[l + 1] = ctx->h_m_off[l] + m[l];
    ctx->h_n_off[l + 1] = ctx->h_n_off[l] + n[l];
  }
  if (ctx->h_m_off[count] >= (1LL << 31) || ctx->h_n_off[count] >= (1LL << 31)) {
    set_error("batch too large: total rows and columns must fit in int32");
    return PDHG_INVALID_ARG;
  }
  ctx->m = (int)ctx->h_m_off[count];
  ctx->n = (int)ctx->h_n_off[count];
  const size_t nrp = (size_t)ctx->m + count;  // concatenated local row pointers
  std::vector<int32_t> lrp(nrp);
  if (ctx->opt.io_on_device) {
    CK(cudaMemcpyAsync(lrp.data(), row_ptr, sizeof(int32_t) * nrp, cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  } else {
    std::memcpy(lrp.data(), row_ptr, sizeof(int32_t) * nrp);
  }
  std::vector<int64_t> nnz_off(count + 1, 0);
  ctx->h_a_rp.assign((size_t)ctx->m + 1, 0);
  for (int l = 0; l < count; ++l) {
    const int32_t* r = lrp.data() + ctx->h_m_off[l] + l;
    if (r[0] != 0) {
      set_error("LP %d: row_ptr[0] must be 0", l);
      return PDHG_INVALID_ARG;
    }
    for (int i = 0; i < m[l]; ++i) {
      if (r[i + 1] < r[i]) {
        set_error("LP %d: row_ptr decreases at row %d", l, i);
        return PDHG_INVALID_ARG;
      }
      const int64_t g = nnz_off[l] + r[i + 1];
      if (g > kMaxNnz) {
        set_error("batch too large: total nonzeros above %lld (int32 tile indexing)",
                  (long long)kMaxNnz);
        return PDHG_INVALID_ARG;
      }
      ctx->h_a_rp[ctx->h_m_off[l] + i + 1] = (int32_t)g;
    }
    nnz_off[l + 1] = nnz_off[l] + r[m[l]];
  }
  ctx->nnz = nnz_off[count];
  CKS(alloc_arrays(ctx));
  CKS(upload_lp(ctx, col, val, b, c));
  // local -> global column indices
  int64_t *d_nnz_off = nullptr, *d_m_off = nullptr, *d_n_off = nullptr;
  int32_t* flags = nullptr;
  CKS(dalloc(ctx, &d_nnz_off, count + 1));
  CKS(dalloc(ctx, &d_m_off, count + 1));
  CKS(dalloc(ctx, &d_n_off, count + 1));
  ctx->d_m_off = d_m_off;
  ctx->d_n_off = d_n_off;
  CKS(dalloc(ctx, &flags, 1));
  CK(cudaMemcpyAsync(d_nnz_off, nnz_off.data(), sizeof(int64_t) * (count + 1),
                     cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(d_m_off, ctx->h_m_off.data(), sizeof(int64_t) * (count + 1),
                     cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(d_n_off, ctx->h_n_off.data(), sizeof(int64_t) * (count + 1),
                     cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemsetAsync(flags, 0, sizeof(int32_t), ctx->stream));
  k_bglobalize<<<count, 256, 0, ctx->stream>>>(d_nnz_off, d_n_off, ctx->a_col, flags);
  ctx->launches += 1;
  int32_t hflags = 0;
  CK(cudaMemcpyAsync(&hflags, flags, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (hflags) {
    set_error("invalid batch: a column index is outside its LP's [0, n)");
    return PDHG_INVALID_ARG;
  }
  stage("checks/allocation/upload");
  CKS(prepare_matrix(ctx));
  stage("validate/transpose/scale");

  // LP-aligned float64 schedules (set-up, report, adjoint); the iteration
  // schedules start as the same and are tuned once the scalars exist
  CKS(batch_schedules(ctx, &ctx->lp_a8_tiles, &ctx->lp_t8_tiles, &ctx->sa8, &ctx->st8, kFixedE));
  ctx->sa = ctx->sa8;
  ctx->st = ctx->st8;
  ctx->lp_a_tiles = ctx->lp_a8_tiles;
  ctx->lp_t_tiles = ctx->lp_t8_tiles;
  const bool mx = ctx->mixed;
  const SchedView &A = ctx->sa.view, &T = ctx->st.view;
  const SchedView &A8 = ctx->sa8.view, &T8 = ctx->st8.view;
  ctx->l_prim = make_launch(ctx, mx ? 0 : 1, T.e, smem_for(0, mx, T.max_rows, T.e), T.ntiles);
  ctx->l_dual = make_launch(ctx, mx ? 2 : 3, A.e, smem_for(0, mx, A.max_rows, A.e), A.ntiles);
  ctx->l_eval = make_launch(ctx, mx ? 4 : 5, T.e, smem_for(1, mx, T.max_rows, T.e),
                            std::max(T.ntiles, A.ntiles));
  ctx->l_a64 = make_launch(ctx, 8, kFixedE, smem_for(2, mx, A8.max_rows, A8.e), A8.ntiles);
  ctx->l_t64 = make_launch(ctx, 8, kFixedE, smem_for(2, mx, T8.max_rows, T8.e), T8.ntiles);
  ctx->restart_grid = std::max(1, std::min(ctx->nsm * 8, std::max(A.ntiles, T.ntiles)));
  // per-tile records; tune_batch_schedules grows them for the tuned schedules
  ctx->rec_tiles = std::max({A.ntiles, T.ntiles, A8.ntiles, T8.ntiles, 1});
  CKS(dalloc(ctx, &ctx->rec_t, (size_t)ctx->rec_tiles * kEvalQ));
  CKS(dalloc(ctx, &ctx->rec_a, (size_t)ctx->rec_tiles * kEvalQ));
  CKS(dalloc(ctx, &ctx->active, 5));
  {
    int32_t* g = nullptr;  // the persistent solve's grid-barrier state (4 words)
    CKS(dalloc(ctx, &g, 4));
    ctx->gsync = g;
  }  // [4]: pdhg_batch_set_rhs's finiteness flag
  CKS(dalloc(ctx, &ctx->breport, (size_t)count * 8));
  CK(cudaMemsetAsync(ctx->active, 0, 4 * sizeof(int32_t), ctx->stream));

  // per-LP scalar state
  CKS(batch_fresh_scalars(ctx));
  // a3 per LP: power iteration
  {
    double *v = ctx->xs64, *u = ctx->ys64, *w = ctx->out_n2;
    int32_t* ticket = ctx->active + 2;
    k_bpow_init<<<(count + 255) / 256, 256, 0, ctx->stream>>>(ctx->ps, count,
                                                               ctx->opt.power_max_iter,
                                                               ctx->opt.power_rel_tol);
    k_bpow_norm<<<ctx->restart_grid, 256, 0, ctx->stream>>>(T8, w, v, ctx->ps, d_n_off, 1);
    ctx->launches += 2;
    std::vector<PowerState> hp(count);
    for (int it = 0; it < ctx->opt.power_max_iter; ++it) {
      k_bpow_Av<kBlock><<<ctx->l_a64.grid, kBlock, ctx->l_a64.smem, ctx->stream>>>(
          A8, ctx->a_rp, ctx->a_col, ctx->a_val64, v, u, ctx->ps);
      k_bpow_ATu<kBlock><<<ctx->l_t64.grid, kBlock, ctx->l_t64.smem, ctx->stream>>>(
          T8, ctx->t_rp, ctx->t_col, ctx->t_val64, u, v, w, ctx->rec_t, ctx->ps, ctx->lp_t8_tiles,
          count, ticket);
      k_bpow_norm<<<ctx->restart_grid, 256, 0, ctx->stream>>>(T8, w, v, ctx->ps, d_n_off, 0);
      ctx->launches += 3;
      if ((it & 15) == 15) {
        CK(cudaMemcpyAsync(hp.data(), ctx->ps, sizeof(PowerState) * count, cudaMemcpyDeviceToHost,
                           ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        bool all = true;
        for (const PowerState& p : hp) all = all && p.stopped;
        if (all) break;
      }
    }
    CK(cudaGetLastError());
  }
  stage("power iteration");
  k_binit<kBlock><<<count, kBlock, 0, ctx->stream>>>(ctx->sc, ctx->ps, d_m_off, d_n_off, ctx->b,
                                                     ctx->c, ctx->b_t64, ctx->c_t64,
                                                     ctx->opt.eta_safety);
  ctx->launches += 1;
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(ctx->stream));
  stage("scalars");
  CKS(tune_batch_schedules(ctx));
  stage("schedule tuning");
  CKS(polling_resources(ctx));
  return PDHG_OK;
}

extern "C" pdhg_status pdhg_batch_create(pdhg_ctx** out, int32_t count, const int32_t* m,
                                         const int32_t* n, const int32_t* row_ptr,
                                         const int32_t* col, const double* val, const double* b,
                                         const double* c, const pdhg_options* opt) {
  clear_error();
  if (!out) {
    set_error("out is NULL");
    return PDHG_INVALID_ARG;
  }
  *out = nullptr;
  if (count < 1 || !m || !n || !row_ptr || !b || !c) {
    set_error("need count >= 1 and non-NULL m, n, row_ptr, b, c");
    return PDHG_INVALID_ARG;
  }
  for (int l = 0; l < count; ++l)
    if (m[l] < 1 || n[l] < 1) {
      set_error("LP %d: need m >= 1 and n >= 1", l);
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
  if (ctx->opt.eval_freq < 1 ||
      (ctx->opt.precision != PDHG_FP64 && ctx->opt.precision != PDHG_FP32_MIXED) ||
      ctx->opt.method != 0 || !(ctx->opt.fp32_screen >= 1.0 && ctx->opt.fp32_screen <= 1e6) ||
      (ctx->opt.omega_rule != 0 && ctx->opt.omega_rule != 1) ||
      (ctx->opt.persistent != 0 && ctx->opt.persistent != 1) || ctx->opt.wait_limit_ms < 1 ||
      (ctx->opt.wait_test != 0 && ctx->opt.wait_test != 1) || ctx->opt.step_rule != 0) {
    set_error("invalid options (eval_freq >= 1, precision 0/1, 1 <= fp32_screen <= 1e6, "
              "omega_rule 0/1, persistent 0/1, wait_limit_ms >= 1, wait_test 0/1, "
              "method 0: batched solves use the averaged iteration, step_rule 0: the "
              "constant step)");
    delete ctx;
    return PDHG_INVALID_ARG;
  }
  ctx->count = count;
  ctx->batch = true;
  ctx->mixed = ctx->opt.precision == PDHG_FP32_MIXED;
  ctx->log_cap = 1;
  pdhg_status st = batch_create_impl(ctx, m, n, row_ptr, col, val, b, c);
  if (st < 0) {
    const std::string msg = pdhg_last_error();
    pdhg_destroy(ctx);
    set_error("%s", msg.c_str());
    return st;
  }
  *out = ctx;
  return PDHG_OK;
}

static pdhg_status build_batch_graphs(pdhg_ctx* ctx) {
  for (int g = 0; g < 2; ++g) {
    if (ctx->chunk_exec[g]) continue;
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    const long long before = ctx->launches;
    enqueue_batch_chunk(ctx, ctx->opt.eval_freq);
    ctx->launches = before;
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

extern "C" pdhg_status pdhg_batch_set_rhs(pdhg_ctx* ctx, const double* b, const double* c) {
  clear_error();
  if (!ctx || !ctx->batch || !b || !c) {
    set_error("pdhg_batch_set_rhs needs a context from pdhg_batch_create and non-NULL b, c");
    return PDHG_INVALID_ARG;
  }
  const int m = ctx->m, n = ctx->n;
  CKS(copy_in(ctx, ctx->b, b, sizeof(double) * m));
  CKS(copy_in(ctx, ctx->c, c, sizeof(double) * n));
  int32_t* flag = ctx->active + 4;
  CK(cudaMemsetAsync(flag, 0, sizeof(int32_t), ctx->stream));
  k_bfinite<<<std::max(1, std::min(ctx->nsm * 4, (m + 255) / 256)), 256, 0, ctx->stream>>>(m, ctx->b, flag);
  k_bfinite<<<std::max(1, std::min(ctx->nsm * 4, (n + 255) / 256)), 256, 0, ctx->stream>>>(n, ctx->c, flag);
  int32_t hflag = 0;
  CK(cudaMemcpyAsync(&hflag, flag, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->launches += 2;
  if (hflag) {
    set_error("b and c must be finite");
    return PDHG_INVALID_ARG;
  }
  // scaled right-hand sides (the scaling depends on A only)
  launch_scale_vec(m, ctx->D_r, ctx->b, ctx->b_t64, ctx->b_t32, ctx->stream);
  launch_scale_vec(n, ctx->D_c, ctx->c, ctx->c_t64, ctx->c_t32, ctx->stream);
  // every LP back to x = 0, y = 0 with fresh restart state
  const size_t es = elem(ctx);
  for (void* v : {ctx->x, ctx->x_avg, ctx->x_last}) CK(cudaMemsetAsync(v, 0, es * n, ctx->stream));
  for (void* v : {ctx->y, ctx->y_avg, ctx->y_last, ctx->Ax, ctx->Ax_avg, ctx->Ax_last})
    CK(cudaMemsetAsync(v, 0, es * m, ctx->stream));
  CKS(batch_fresh_scalars(ctx));
  k_binit<kBlock><<<ctx->count, kBlock, 0, ctx->stream>>>(ctx->sc, ctx->ps, ctx->d_m_off,
                                                          ctx->d_n_off, ctx->b, ctx->c, ctx->b_t64,
                                                          ctx->c_t64, ctx->opt.eta_safety);
  ctx->launches += 3;
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(ctx->stream));
  pdhg_adjoint_invalidate(ctx);
  ctx->report_valid = false;
  ctx->last_status = PDHG_MAX_ITER;
  return PDHG_OK;
}

extern "C" pdhg_status pdhg_batch_solve(pdhg_ctx* ctx, double eps_rel, int64_t max_iter,
                                        int32_t* lp_status) {
  clear_error();
  if (!ctx || !ctx->batch) {
    set_error("pdhg_batch_solve needs a context from pdhg_batch_create");
    return PDHG_INVALID_ARG;
  }
  if (!(eps_rel >= 0.0) || max_iter < 0) {
    set_error("need eps_rel >= 0 and max_iter >= 0");
    return PDHG_INVALID_ARG;
  }
  const int count = ctx->count;
  std::vector<Scalars> hs(count);
  CK(cudaMemcpyAsync(hs.data(), ctx->sc, sizeof(Scalars) * count, cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  long long k = hs[0].k;
  for (const Scalars& s : hs) k = std::max(k, s.k);
  for (Scalars& s : hs) {
    // an LP restarts from where it stopped; all advance in lockstep from k
    s.eps = eps_rel;
    s.max_iter = max_iter;
    s.done = 0;
    s.status = PDHG_MAX_ITER;
    s.restart_pending = 0;
    s.k = k;
    s.fp64_check = ctx->mixed ? 1 : 0;
    s.screen = ctx->opt.fp32_screen;
    s.verify = 0;
    s.checks = 0;
    s.rejects = 0;
  }
  CK(cudaMemcpyAsync(ctx->sc, hs.data(), sizeof(Scalars) * count, cudaMemcpyHostToDevice,
                     ctx->stream));
  CK(cudaMemsetAsync(ctx->active, 0, 4 * sizeof(int32_t), ctx->stream));
  if (ctx->opt.persistent) {
    // the active count the kernel polls starts at every LP
    const int32_t all = count;
    CK(cudaMemcpyAsync(ctx->active, &all, sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
    const pdhg_status ps = batch_persistent_solve(ctx, k, max_iter);
    if (ps != PDHG_OK) {
      ctx->last_status = ps;
      ctx->report_valid = false;
      if (lp_status)
        for (int l = 0; l < count; ++l) lp_status[l] = ps;
      return ps;
    }
    k = max_iter;  // the kernel ran to the end (or until every LP finished)
  }
  if (!ctx->opt.persistent && ctx->opt.use_graphs) CKS(build_batch_graphs(ctx));
  const long long F = ctx->opt.eval_freq;
  // pinned status words (the context's pinned status buffers are large enough)
  int32_t* h_ctl[2] = {reinterpret_cast<int32_t*>(ctx->h_sc[0]),
                       reinterpret_cast<int32_t*>(ctx->h_sc[1])};
  int slot = 0;
  bool pending[2] = {false, false}, stop = false;
  auto drain = [&](int sl) -> pdhg_status {
    CK(cudaEventSynchronize(ctx->ev_done[sl]));
    pending[sl] = false;
    if (h_ctl[sl][0] == 0) stop = true;
    return PDHG_OK;
  };
  while (k < max_iter && !stop) {
    const long long next = std::min<long long>((k / F + 1) * F, max_iter);
    const int len = (int)(next - k);
    if (len == F && ctx->opt.use_graphs) {
      CK(cudaGraphLaunch(ctx->chunk_exec[slot], ctx->stream));
      ctx->launches += 2 * F + 2 + (ctx->mixed ? kFp64CheckLaunches : 0);
    } else {
      enqueue_batch_chunk(ctx, len);
      CK(cudaGetLastError());
    }
    CK(cudaMemcpyAsync(h_ctl[slot], ctx->active, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaEventRecord(ctx->ev_done[slot], ctx->stream));
    pending[slot] = true;
    k = next;
    const int other = slot ^ 1;
    if (pending[other]) CKS(drain(other));
    slot = other;
  }
  for (int i = 0; i < 2; ++i) {
    const int sl = slot ^ 1 ^ i;
    if (pending[sl]) CKS(drain(sl));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaGetLastError());
  CK(cudaMemcpy(hs.data(), ctx->sc, sizeof(Scalars) * count, cudaMemcpyDeviceToHost));
  int worst = PDHG_OK;
  for (int l = 0; l < count; ++l) {
    const int s = hs[l].done ? hs[l].status : PDHG_MAX_ITER;
    if (lp_status) lp_status[l] = s;
    worst = std::max(worst, s);
  }
  ctx->last_status = worst;
  ctx->report_valid = false;
  return (pdhg_status)worst;
}

static pdhg_status batch_returned64(pdhg_ctx* ctx) {
  if (ctx->mixed)
    k_bchoose<float><<<ctx->restart_grid, 256, 0, ctx->stream>>>(
        ctx->st.view, ctx->sa.view, ctx->sc, (const float*)ctx->x, (const float*)ctx->x_avg,
        (const float*)ctx->y, (const float*)ctx->y_avg, ctx->xs64, ctx->ys64, false);
  else
    k_bchoose<double><<<ctx->restart_grid, 256, 0, ctx->stream>>>(
        ctx->st.view, ctx->sa.view, ctx->sc, (const double*)ctx->x, (const double*)ctx->x_avg,
        (const double*)ctx->y, (const double*)ctx->y_avg, ctx->xs64, ctx->ys64, false);
  ctx->launches += 1;
  CK(cudaGetLastError());
  return PDHG_OK;
}

pdhg_status batch_returned64_adj(pdhg_ctx* ctx) { return batch_returned64(ctx); }

extern "C" pdhg_status pdhg_batch_get(pdhg_ctx* ctx, double* x, double* y, double* z,
                                      double* lp_r_P, double* lp_r_D, double* lp_gap,
                                      double* lp_max_violation, int64_t* lp_iters) {
  clear_error();
  if (!ctx || !ctx->batch) {
    set_error("pdhg_batch_get needs a context from pdhg_batch_create");
    return PDHG_INVALID_ARG;
  }
  const int count = ctx->count;
  CKS(batch_returned64(ctx));
  k_brep_n<kBlock><<<ctx->l_t64.grid, kBlock, ctx->l_t64.smem, ctx->stream>>>(
      ctx->st8.view, ctx->t_rp, ctx->t_col, ctx->t_val64, ctx->xs64, ctx->ys64, ctx->c_t64,
      ctx->D_c, ctx->out_n1, ctx->out_n2, ctx->rec_t, nullptr);
  k_brep_m<kBlock><<<ctx->l_a64.grid, kBlock, ctx->l_a64.smem, ctx->stream>>>(
      ctx->sa8.view, ctx->a_rp, ctx->a_col, ctx->a_val64, ctx->xs64, ctx->ys64, ctx->b_t64,
      ctx->D_r, ctx->out_m1, ctx->rec_a, nullptr);
  k_brep_final<<<(count + 255) / 256, 256, 0, ctx->stream>>>(ctx->rec_t, ctx->lp_t8_tiles,
                                                             ctx->rec_a, ctx->lp_a8_tiles, count,
                                                             ctx->breport);
  ctx->launches += 3;
  CK(cudaGetLastError());
  CKS(copy_out(ctx, x, ctx->out_n1, sizeof(double) * ctx->n));
  CKS(copy_out(ctx, z, ctx->out_n2, sizeof(double) * ctx->n));
  CKS(copy_out(ctx, y, ctx->out_m1, sizeof(double) * ctx->m));
  std::vector<double> rep((size_t)count * 8);
  std::vector<Scalars> hs(count);
  CK(cudaMemcpyAsync(rep.data(), ctx->breport, sizeof(double) * 8 * count, cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaMemcpyAsync(hs.data(), ctx->sc, sizeof(Scalars) * count, cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  for (int l = 0; l < count; ++l) {
    if (lp_r_P) lp_r_P[l] = rep[8 * l + 0];
    if (lp_r_D) lp_r_D[l] = rep[8 * l + 1];
    if (lp_gap) lp_gap[l] = rep[8 * l + 2];
    if (lp_max_violation) lp_max_violation[l] = rep[8 * l + 3];
    if (lp_iters) lp_iters[l] = hs[l].k;
  }
  return PDHG_OK;
}

extern "C" pdhg_status pdhg_batch_warmstart_point(pdhg_ctx* ctx, double mu_min, double delta_max,
                                                  double alpha_min, int32_t unscaled,
                                                  double* x_ws, double* y_ws, double* z_ws,
                                                  double* lp_mu) {
  clear_error();
  if (!ctx || !ctx->batch) {
    set_error("pdhg_batch_warmstart_point needs a context from pdhg_batch_create");
    return PDHG_INVALID_ARG;
  }
  if (!(mu_min > 0.0) || !(delta_max >= 0.0) || !(alpha_min > 0.0)) {
    set_error("need mu_min > 0, delta_max >= 0, alpha_min > 0");
    return PDHG_INVALID_ARG;
  }
  const int count = ctx->count;
  CKS(batch_returned64(ctx));
  int64_t* d_n_off = nullptr;
  double* mu = nullptr;
  CKS(dalloc(ctx, &d_n_off, count + 1));
  CKS(dalloc(ctx, &mu, count));
  CK(cudaMemcpyAsync(d_n_off, ctx->h_n_off.data(), sizeof(int64_t) * (count + 1),
                     cudaMemcpyHostToDevice, ctx->stream));
  double* zs = ctx->out_n2;
  k_bws_z<kBlock><<<ctx->l_t64.grid, kBlock, ctx->l_t64.smem, ctx->stream>>>(
      ctx->st8.view, ctx->t_rp, ctx->t_col, ctx->t_val64, ctx->xs64, ctx->ys64, ctx->c_t64, zs,
      ctx->rec_t);
  k_bws_mu<<<(count + 255) / 256, 256, 0, ctx->stream>>>(ctx->rec_t, ctx->lp_t8_tiles, d_n_off,
                                                         count, mu_min, mu);
  k_bws_apply<<<ctx->restart_grid, 256, 0, ctx->stream>>>(
      ctx->st8.view, ctx->sa8.view, ctx->xs64, zs, ctx->ys64, mu, delta_max, alpha_min, unscaled,
      ctx->D_r, ctx->D_c, ctx->out_n1, ctx->out_m1, zs);
  ctx->launches += 3;
  CK(cudaGetLastError());
  CKS(copy_out(ctx, x_ws, ctx->out_n1, sizeof(double) * ctx->n));
  CKS(copy_out(ctx, y_ws, ctx->out_m1, sizeof(double) * ctx->m));
  CKS(copy_out(ctx, z_ws, zs, sizeof(double) * ctx->n));
  if (lp_mu) CK(cudaMemcpyAsync(lp_mu, mu, sizeof(double) * count, cudaMemcpyDeviceToHost,
                                ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return PDHG_OK;
}
