// Set-up kernels: CSR validation, stable transpose, diagonal scaling (Ruiz and
// Pock-Chambolle statistics), scaled copies, reductions and power iteration.
#include <algorithm>
#include <math.h>

#include "dispatch.cuh"
#include "kernels.h"
#include "spmv_tile.cuh"

namespace pdhg {

static int grid_cap(int64_t work, int per_block = 256, int cap = 8192) {
  int64_t g = (work + per_block - 1) / per_block;
  if (g > cap) g = cap;
  return g < 1 ? 1 : (int)g;
}

// ---------------------------------------------------------------------------
// validation: flags |= 1 column out of range, 2 columns not strictly
// increasing in a row, 4 non-finite value, 8 non-finite b, 16 non-finite c
// ---------------------------------------------------------------------------
__global__ void k_validate(int m, int n, const int32_t* rp, const int32_t* col, const double* val,
                           const double* b, const double* c, int32_t* flags) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  int f = 0;
  for (int i = warp; i < m; i += nw) {
    const int s = rp[i], e = rp[i + 1];
    for (int k = s + lane; k < e; k += 32) {
      const int cj = col[k];
      if (cj < 0 || cj >= n) f |= 1;
      if (k > s && col[k - 1] >= cj) f |= 2;
      if (!isfinite(val[k])) f |= 4;
    }
  }
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
  for (int i = tid; i < m; i += nt)
    if (!isfinite(b[i])) f |= 8;
  for (int j = tid; j < n; j += nt)
    if (!isfinite(c[j])) f |= 16;
  if (f) atomicOr(flags, f);
}

void launch_validate(int m, int n, const int32_t* rp, const int32_t* col, const double* val,
                     const double* b, const double* c, int32_t* flags, cudaStream_t s) {
  k_validate<<<grid_cap((int64_t)m * 32), 256, 0, s>>>(m, n, rp, col, val, b, c, flags);
}

// ---------------------------------------------------------------------------
// transpose: column histogram, exclusive scan, scatter, per-column sort
// ---------------------------------------------------------------------------
__global__ void k_col_hist(int64_t nnz, const int32_t* col, int32_t* cnt) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
       k += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(cnt + col[k], 1);
}
void launch_col_hist(int64_t nnz, const int32_t* col, int32_t* cnt, cudaStream_t s) {
  k_col_hist<<<grid_cap(nnz), 256, 0, s>>>(nnz, col, cnt);
}

constexpr int kScanT = 256, kScanPer = 4, kScanTile = kScanT * kScanPer;

__device__ __forceinline__ int warp_incl_scan(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// exclusive scan of one 1024-element tile; tile total -> tops[blockIdx]
__global__ void k_scan_tile(const int32_t* in, int32_t* out, int len, int32_t* tops) {
  __shared__ int wsum[kScanT / 32];
  const int base = blockIdx.x * kScanTile + threadIdx.x * kScanPer;
  int v[kScanPer], s = 0;
#pragma unroll
  for (int e = 0; e < kScanPer; ++e) {
    v[e] = (base + e < len) ? in[base + e] : 0;
    s += v[e];
  }
  const int incl = warp_incl_scan(s);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  if (w == 0) {
    int x = (lane < kScanT / 32) ? wsum[lane] : 0;
    x = warp_incl_scan(x);
    if (lane < kScanT / 32) wsum[lane] = x;
  }
  __syncthreads();
  int run = incl - s + (w > 0 ? wsum[w - 1] : 0);
#pragma unroll
  for (int e = 0; e < kScanPer; ++e) {
    if (base + e < len) out[base + e] = run;
    run += v[e];
  }
  if (threadIdx.x == kScanT - 1) tops[blockIdx.x] = run;
}

// exclusive scan of the tile totals in one block (sequential over chunks)
__global__ void k_scan_tops(int32_t* tops, int ntiles, int32_t* total_out) {
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < ntiles; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const int v = (i < ntiles) ? tops[i] : 0;
    // block-wide inclusive scan of blockDim.x (= 1024) values
    __shared__ int ws[32];
    const int incl = warp_incl_scan(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 31) ws[w] = incl;
    __syncthreads();
    if (w == 0) {
      int x = ws[lane];
      x = warp_incl_scan(x);
      ws[lane] = x;
    }
    __syncthreads();
    const int excl = incl - v + (w > 0 ? ws[w - 1] : 0) + carry;
    if (i < ntiles) tops[i] = excl;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total_out = carry;
}

__global__ void k_scan_add(int32_t* out, int len, const int32_t* tops) {
  const int i = blockIdx.x * kScanTile + threadIdx.x;
  const int add = tops[blockIdx.x];
#pragma unroll
  for (int e = 0; e < kScanPer; ++e) {
    const int k = i + e * kScanT;
    if (k < len) out[k] += add;
  }
}

void launch_scan(const int32_t* cnt, int32_t* out, int len, int32_t* tmp, cudaStream_t s) {
  const int ntiles = (len + kScanTile - 1) / kScanTile;
  if (ntiles == 0) {
    cudaMemsetAsync(out, 0, sizeof(int32_t), s);
    return;
  }
  k_scan_tile<<<ntiles, kScanT, 0, s>>>(cnt, out, len, tmp);
  k_scan_tops<<<1, 1024, 0, s>>>(tmp, ntiles, out + len);
  k_scan_add<<<ntiles, kScanT, 0, s>>>(out, len, tmp);
}

__global__ void k_scatter(int m, const int32_t* rp, const int32_t* col, const double* val,
                          int32_t* cursor, int32_t* col_t, double* val_t) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int i = warp; i < m; i += nw)
    for (int k = rp[i] + lane; k < rp[i + 1]; k += 32) {
      const int pos = atomicAdd(cursor + col[k], 1);
      col_t[pos] = i;
      val_t[pos] = val[k];
    }
}
void launch_scatter(int m, const int32_t* rp, const int32_t* col, const double* val,
                    int32_t* cursor, int32_t* col_t, double* val_t, cudaStream_t s) {
  k_scatter<<<grid_cap((int64_t)m * 32), 256, 0, s>>>(m, rp, col, val, cursor, col_t, val_t);
}

// segments of <= 32 entries: one thread, insertion sort in place
__global__ void k_segsort_small(int nseg, const int32_t* seg, int32_t* keys, double* vals) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nseg; j += gridDim.x * blockDim.x) {
    const int s = seg[j], e = seg[j + 1];
    if (e - s > 32 || e - s < 2) continue;
    for (int a = s + 1; a < e; ++a) {
      const int kk = keys[a];
      const double vv = vals[a];
      int b = a - 1;
      while (b >= s && keys[b] > kk) {
        keys[b + 1] = keys[b];
        vals[b + 1] = vals[b];
        --b;
      }
      keys[b + 1] = kk;
      vals[b + 1] = vv;
    }
  }
}

constexpr int kBitonicMax = 2048;

// longer segments: one block each; bitonic sort in shared memory up to 2048
// entries, else rank by counting (keys within a segment are distinct rows)
__global__ void __launch_bounds__(1024) k_segsort_long(const int32_t* seg, int32_t* keys, double* vals,
                                                       const int32_t* ids, int32_t* tmp_k,
                                                       double* tmp_v) {
  __shared__ int sk[kBitonicMax];
  __shared__ double sv[kBitonicMax];
  const int j = ids[blockIdx.x];
  const int s = seg[j], e = seg[j + 1], len = e - s;
  if (len <= kBitonicMax) {
    int p2 = 1;
    while (p2 < len) p2 <<= 1;
    for (int i = threadIdx.x; i < p2; i += blockDim.x) {
      sk[i] = (i < len) ? keys[s + i] : 0x7fffffff;
      sv[i] = (i < len) ? vals[s + i] : 0.0;
    }
    __syncthreads();
    for (int size = 2; size <= p2; size <<= 1)
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int i = threadIdx.x; i < p2; i += blockDim.x) {
          const int pr = i ^ stride;
          if (pr > i) {
            const bool up = (i & size) == 0;
            if ((sk[i] > sk[pr]) == up) {
              const int tk = sk[i];
              sk[i] = sk[pr];
              sk[pr] = tk;
              const double tv = sv[i];
              sv[i] = sv[pr];
              sv[pr] = tv;
            }
          }
        }
        __syncthreads();
      }
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
      keys[s + i] = sk[i];
      vals[s + i] = sv[i];
    }
    return;
  }
  for (int a = threadIdx.x; a < len; a += blockDim.x) {
    const int ka = keys[s + a];
    int rank = 0;
    for (int b = 0; b < len; ++b) rank += (keys[s + b] < ka) ? 1 : 0;
    tmp_k[s + rank] = ka;
    tmp_v[s + rank] = vals[s + a];
  }
  __syncthreads();
  for (int a = threadIdx.x; a < len; a += blockDim.x) {
    keys[s + a] = tmp_k[s + a];
    vals[s + a] = tmp_v[s + a];
  }
}

void launch_segsort(int nseg, const int32_t* seg_ptr, int32_t* keys, double* vals,
                    const int32_t* long_ids, int n_long, int32_t* tmp_k, double* tmp_v,
                    cudaStream_t s) {
  k_segsort_small<<<grid_cap(nseg), 256, 0, s>>>(nseg, seg_ptr, keys, vals);
  if (n_long > 0) k_segsort_long<<<n_long, 1024, 0, s>>>(seg_ptr, keys, vals, long_ids, tmp_k, tmp_v);
}

// ---------------------------------------------------------------------------
// scaling statistics of D_self M D_other and scaled copies
// ---------------------------------------------------------------------------
// Row statistic sqrt(d_self[i] * max_j |M_ij| d_other[j]) (mode 0) or
// sqrt(d_self[i] * sum_j |M_ij| d_other[j]) (mode 1); zero -> 1.  G lanes per
// row (G sized to the mean row length, every lane of a warp takes part in the
// shuffles); rows longer than long_len are left to k_row_stat_long.
template <int G>
__global__ void k_row_stat(int nrows, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                           const double* __restrict__ val, const double* __restrict__ d_self,
                           const double* __restrict__ d_other, int mode, int long_len,
                           double* __restrict__ out) {
  // mode 0 (Ruiz): the maximum of |a| d over non-negative doubles, taken on
  // their bit patterns (ordered like the values) with 64-bit integer max, so
  // only the product and the row's square root use the slow float64 pipe;
  // mode 1 (Pock-Chambolle): the float64 sum
  constexpr int RPW = 32 / G;  // rows per warp and pass
  const int lane = threadIdx.x & 31, gw = lane / G, gl = lane & (G - 1);
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int base = warp * RPW; base < nrows; base += nw * RPW) {
    const int i = base + gw;
    double acc = 0.0;
    long long mx = 0;
    bool mine = false;
    if (i < nrows) {
      const int b = rp[i], e = rp[i + 1];
      if (e - b <= long_len) {
        mine = true;
        if (mode) {
          for (int k = b + gl; k < e; k += G) acc += fabs(val[k]) * d_other[col[k]];
        } else {
          for (int k = b + gl; k < e; k += G)
            mx = max(mx, __double_as_longlong(fabs(val[k]) * d_other[col[k]]));
        }
      }
    }
    if (mode) {
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o, G);
    } else {
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) mx = max(mx, __shfl_down_sync(0xffffffffu, mx, o, G));
      acc = __longlong_as_double(mx);
    }
    if (mine && gl == 0) {
      const double r = sqrt(d_self[i] * acc);
      out[i] = (r == 0.0) ? 1.0 : r;
    }
  }
}

// the same statistic for the rows listed in ids, one block of 256 per row
__global__ void k_row_stat_long(const int32_t* __restrict__ ids, const int32_t* __restrict__ rp,
                                const int32_t* __restrict__ col, const double* __restrict__ val,
                                const double* __restrict__ d_self,
                                const double* __restrict__ d_other, int mode,
                                double* __restrict__ out) {
  __shared__ double red[8];
  const int i = ids[blockIdx.x];
  double acc = 0.0;
  long long mx = 0;
  if (mode) {
    for (int k = rp[i] + threadIdx.x; k < rp[i + 1]; k += blockDim.x)
      acc += fabs(val[k]) * d_other[col[k]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  } else {
    for (int k = rp[i] + threadIdx.x; k < rp[i + 1]; k += blockDim.x)
      mx = max(mx, __double_as_longlong(fabs(val[k]) * d_other[col[k]]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_down_sync(0xffffffffu, mx, o));
    acc = __longlong_as_double(mx);
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = red[0];
    for (int w = 1; w < 8; ++w) v = mode ? v + red[w] : fmax(v, red[w]);
    const double r = sqrt(d_self[i] * v);
    out[i] = (r == 0.0) ? 1.0 : r;
  }
}

void launch_row_stat(int nrows, const int32_t* rp, const int32_t* col, const double* val,
                     const double* d_self, const double* d_other, int mode, double* out,
                     const RowStatPlan& plan, cudaStream_t s) {
  const int g = grid_cap((int64_t)nrows * plan.lanes);
#define PDHG_ROW_STAT(G) \
  k_row_stat<G><<<g, 256, 0, s>>>(nrows, rp, col, val, d_self, d_other, mode, plan.long_len, out)
  switch (plan.lanes) {
    case 4: PDHG_ROW_STAT(4); break;
    case 8: PDHG_ROW_STAT(8); break;
    case 16: PDHG_ROW_STAT(16); break;
    default: PDHG_ROW_STAT(32); break;
  }
#undef PDHG_ROW_STAT
  if (plan.nlong > 0)
    k_row_stat_long<<<plan.nlong, 256, 0, s>>>(plan.long_ids, rp, col, val, d_self, d_other, mode,
                                              out);
}

__global__ void k_fill(double* d, double v, int64_t len) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x)
    d[i] = v;
}
void launch_fill(double* d, double v, int64_t len, cudaStream_t s) {
  k_fill<<<grid_cap(len), 256, 0, s>>>(d, v, len);
}

__global__ void k_div(double* d, const double* r, int len) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < len; i += gridDim.x * blockDim.x)
    d[i] = d[i] / r[i];
}
void launch_div(double* d, const double* r, int len, cudaStream_t s) {
  k_div<<<grid_cap(len), 256, 0, s>>>(d, r, len);
}

// A~_ij = (D_r[i] A_ij) D_c[j], evaluated in that order for A and for A^T so
// both stored copies hold identical values.  For A^T rows are columns of A.
__global__ void k_scale_vals(int nrows, const int32_t* rp, const int32_t* col, const double* val,
                             const double* d_row, const double* d_col, int transposed,
                             double* out64, float* out32) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int i = warp; i < nrows; i += nw)
    for (int k = rp[i] + lane; k < rp[i + 1]; k += 32) {
      const double dr = transposed ? d_row[col[k]] : d_row[i];
      const double dc = transposed ? d_col[i] : d_col[col[k]];
      const double v = (dr * val[k]) * dc;
      out64[k] = v;
      if (out32) out32[k] = (float)v;
    }
}
void launch_scale_vals(int nrows, const int32_t* rp, const int32_t* col, const double* val,
                       const double* D_r, const double* D_c, int transposed, double* out64,
                       float* out32, cudaStream_t s) {
  k_scale_vals<<<grid_cap((int64_t)nrows * 32), 256, 0, s>>>(nrows, rp, col, val, D_r, D_c,
                                                            transposed, out64, out32);
}

__global__ void k_scale_vec(int len, const double* d, const double* v, double* out64, float* out32) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < len; i += gridDim.x * blockDim.x) {
    const double o = d[i] * v[i];
    out64[i] = o;
    if (out32) out32[i] = (float)o;
  }
}
void launch_scale_vec(int len, const double* d, const double* v, double* out64, float* out32,
                      cudaStream_t s) {
  k_scale_vec<<<grid_cap(len), 256, 0, s>>>(len, d, v, out64, out32);
}

// mode 0: sum a*b; 1: sum a^2; 2: sum min(0,a)^2
__global__ void k_dot_partials(int64_t len, const double* a, const double* b, int mode,
                               double* partials) {
  __shared__ double red[8];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double x = a[i];
    acc += mode == 0 ? x * b[i] : (mode == 1 ? x * x : fmin(0.0, x) * fmin(0.0, x));
  }
  const double v[1] = {acc};
  double o[1];
  block_sum<256, 1>(v, o, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = o[0];
}
void launch_dot_partials(int64_t len, const double* a, const double* b, int mode, double* partials,
                         int grid, cudaStream_t s) {
  k_dot_partials<<<grid, 256, 0, s>>>(len, a, b, mode, partials);
}

__global__ void k_sum_final(const double* partials, int g, double* out) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int i = 0; i < g; ++i) s += partials[i];
  *out = s;
}
void launch_sum_final(const double* partials, int g, double* out, cudaStream_t s) {
  k_sum_final<<<1, 32, 0, s>>>(partials, g, out);
}

// ---------------------------------------------------------------------------
// power iteration on A~^T A~ (float64).  Its three kernels are launched with
// programmatic dependent launch and wait on entry, so each launch is set up
// while the previous kernel drains.
// ---------------------------------------------------------------------------
__global__ void k_pow_init(int n, double* v, PowerState* ps, int max_iter, double rel_tol) {
  const double v0 = 1.0 / sqrt((double)n);
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) v[j] = v0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ps->lam = 0.0;
    ps->lam_prev = 0.0;
    ps->inv_norm = 0.0;
    ps->k = 0;
    ps->max_iter = max_iter;
    ps->stopped = (max_iter <= 0 || n == 0) ? 1 : 0;
    ps->ticket = 0;
    ps->rel_tol = rel_tol;
  }
}
void launch_pow_init(int n, double* v, PowerState* ps, int max_iter, double rel_tol,
                     cudaStream_t s) {
  k_pow_init<<<grid_cap(n), 256, 0, s>>>(n, v, ps, max_iter, rel_tol);
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_pow_Av(SchedView S, const int32_t* rp, const int32_t* col,
                                                 const double* val, const double* v, double* u,
                                                 const PowerState* ps) {
  pdl_enter();
  if (ps->stopped) return;
  extern __shared__ __align__(16) unsigned char smem[];
  struct E {
    double* u;
    __device__ void row(int r, const double (&s)[1], int) { u[r] = s[0]; }
  } epi{u};
  Gather<double, 1> g{{v}};
  run_tiles<double, 1, BLOCK, kFixedE>(S, rp, col, val, g, epi, smem);
}

struct PowEpi {
  const double* v;
  double* w;
  double lam, nw2;
  double* split_q;
  __device__ __forceinline__ void row(int j, const double (&s)[1], int group) {
    w[j] = s[0];
    if (group < 0) {
      lam += v[j] * s[0];
      nw2 += s[0] * s[0];
    } else {
      split_q[2 * group] = v[j] * s[0];
      split_q[2 * group + 1] = s[0] * s[0];
    }
  }
};

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_pow_ATu(SchedView S, const int32_t* rp, const int32_t* col,
                                                  const double* val, const double* u,
                                                  const double* v, double* w, double* partials,
                                                  PowerState* ps, int ngroups) {
  pdl_enter();
  if (ps->stopped) return;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[2 * (BLOCK / 32)];
  __shared__ int is_last;
  double* split_q = partials + 2 * (size_t)gridDim.x;
  PowEpi epi{v, w, 0.0, 0.0, split_q};
  Gather<double, 1> g{{u}};
  run_tiles<double, 1, BLOCK, kFixedE>(S, rp, col, val, g, epi, smem);
  const double vv[2] = {epi.lam, epi.nw2};
  double o[2];
  block_sum<BLOCK, 2>(vv, o, red);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = o[0];
    partials[2 * blockIdx.x + 1] = o[1];
    __threadfence();
    is_last = (atomicAdd(&ps->ticket, 1) == (int)gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  __shared__ double tot[2];
  parts_sum<BLOCK, 2>(partials, (int)gridDim.x + ngroups, nullptr, 0, tot, red);
  if (threadIdx.x != 0) return;
  const double lam = tot[0], nw2 = tot[1];
  ps->ticket = 0;
  ps->k += 1;
  ps->lam = lam;
  const double nw = sqrt(nw2);
  if (nw == 0.0) {
    ps->stopped = 1;
    ps->inv_norm = 0.0;
    return;
  }
  ps->inv_norm = 1.0 / nw;
  if (ps->k > 1 && fabs(lam - ps->lam_prev) <= ps->rel_tol * lam) ps->stopped = 1;
  ps->lam_prev = lam;
  if (ps->k >= ps->max_iter) ps->stopped = 1;
}

__global__ void k_pow_norm(int n, const double* w, double* v, const PowerState* ps) {
  pdl_enter();
  const double s = ps->inv_norm;
  if (s == 0.0) return;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) v[j] = w[j] * s;
}

void launch_pow_Av(const SchedView& S, const int32_t* rp, const int32_t* col, const double* val,
                   const double* v, double* u, PowerState* ps, const Launch& L, cudaStream_t s) {
  launch_pdl(k_pow_Av<kBlock>, L.grid, kBlock, L.smem, s, S, rp, col, val, v, u, (const PowerState*)ps);
}
void launch_pow_ATu(const SchedView& S, const int32_t* rp, const int32_t* col, const double* val,
                    const double* u, const double* v, double* w, double* partials,
                    PowerState* ps, const Launch& L, cudaStream_t s) {
  launch_pdl(k_pow_ATu<kBlock>, L.grid, kBlock, L.smem, s, S, rp, col, val, u, v, w, partials, ps,
             (int)S.ngroups);
}
int pow_occupancy(bool at, size_t smem) {
  const void* f = at ? (const void*)k_pow_ATu<kBlock> : (const void*)k_pow_Av<kBlock>;
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, kBlock, smem);
  return nb < 1 ? 1 : nb;
}
void launch_pow_norm(int n, const double* w, double* v, PowerState* ps, cudaStream_t s) {
  launch_pdl(k_pow_norm, grid_cap(n), 256, 0, s, n, w, v, (const PowerState*)ps);
}

// sums: |b|^2, |c|^2, |b~|^2, |c~|^2, |min(0, c~)|^2
__global__ void k_init_scalars(Scalars* sc, const double* sums, const PowerState* ps,
                               double eta_safety) {
  if (threadIdx.x != 0) return;
  const double smax = sqrt(fmax(ps->lam, 0.0));
  sc->eta = smax > 0.0 ? eta_safety / smax : 1.0;
  const double nb = sqrt(sums[2]), nc = sqrt(sums[3]);
  sc->omega = (nb > 0.0 && nc > 0.0) ? nc / nb : 1.0;
  sc->tau = sc->eta / sc->omega;
  sc->sigma = sc->eta * sc->omega;
  sc->norm_b = sqrt(sums[0]);
  sc->norm_c = sqrt(sums[1]);
  const double w2 = sc->omega * sc->omega;
  sc->kkt_last = sqrt(w2 * sums[2] + sums[4] / w2);
  sc->kkt_prev = sc->kkt_last;
}
__global__ void k_recip(const double* __restrict__ in, double* out, int64_t len) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = 1.0 / in[i];
}
void launch_recip(const double* in, double* out, int64_t len, cudaStream_t s) {
  const int64_t g = std::min<int64_t>(std::max<int64_t>((len + 255) / 256, 1), 4096);
  k_recip<<<(int)g, 256, 0, s>>>(in, out, len);
}

void launch_init_scalars(Scalars* sc, const double* sums, const PowerState* ps, double eta_safety,
                         cudaStream_t s) {
  k_init_scalars<<<1, 32, 0, s>>>(sc, sums, ps, eta_safety);
}

// shared memory limit for the power-iteration tile kernels
cudaError_t configure_setup_kernels(size_t max_smem) {
  cudaError_t e = cudaSuccess;
  for (const void* f : {(const void*)k_pow_Av<kBlock>, (const void*)k_pow_ATu<kBlock>}) {
    cudaFuncAttributes a;
    cudaError_t r = cudaFuncGetAttributes(&a, f);
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(max_smem - a.sharedSizeBytes));
    if (r != cudaSuccess) e = r;
  }
  return e;
}

// ---------------------------------------------------------------------------
// window words of a segmented schedule: one thread per (whole-row tile,
// thread window); the row of the window's first nonzero by binary search over
// the tile's rows, then the row ends inside the window
// ---------------------------------------------------------------------------
template <int E>
__global__ void k_window_words(const Tile* __restrict__ tiles, int ntiles,
                               const int32_t* __restrict__ rp,
                               typename WindowWord<E>::type* __restrict__ wd) {
  constexpr int e = E;
  const int64_t total = (int64_t)ntiles * kBlock;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(idx / kBlock), th = (int)(idx % kBlock);
    const Tile tl = tiles[t];
    if (tl.split >= 0 || tl.nz_begin == tl.nz_end) continue;
    const int w0 = (tl.nz_begin & ~3) + th * e;
    const int k0 = max(w0, tl.nz_begin), k1 = min(w0 + e, tl.nz_end);
    typename WindowWord<E>::type word = 0;
    if (k0 < k1) {
      int lo = tl.row_begin, hi = tl.row_end;  // rp[lo] <= k0 < rp[hi]
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (rp[mid] <= k0) lo = mid; else hi = mid;
      }
      uint64_t mask = 0;
      int r = lo, next_end = rp[lo + 1];
      for (int k = k0; k < k1; ++k)
        if (k + 1 == next_end) {
          mask |= 1ull << (k - w0);
          if (++r < tl.row_end) next_end = rp[r + 1];
        }
      word = window_word<E>(lo - tl.row_begin, rp[lo] < k0, mask);
    }
    wd[tl.word0 + th] = word;
  }
}

void launch_window_words(const Tile* tiles, int ntiles, const int32_t* rp, int e, uint32_t* wd,
                         cudaStream_t s) {
  if (ntiles <= 0) return;
  const int g = grid_cap((int64_t)ntiles * kBlock);
  if (e == 32)
    k_window_words<32><<<g, 256, 0, s>>>(tiles, ntiles, rp, reinterpret_cast<uint64_t*>(wd));
  else if (e == 16)
    k_window_words<16><<<g, 256, 0, s>>>(tiles, ntiles, rp, wd);
  else
    k_window_words<8><<<g, 256, 0, s>>>(tiles, ntiles, rp, wd);
}

}  // namespace pdhg
