// PDLP's adaptive step (options.step_rule 1) fused into the two half-steps.
//
// An attempt with step eta (tau = eta / omega, sigma = eta omega) is the
// usual PDHG step from the accepted state z = (x, y) to z+ = (x+, y+).  With
// dx = x+ - x and dy = y+ - y the attempt is accepted when
//   eta <= eta_max = (omega ||dx||^2 + ||dy||^2 / omega) / (2 |dy^T A~ dx|),
// the next attempt's step is min((1 - (j+1)^-0.3) eta_max, (1 + (j+1)^-0.6) eta)
// with j the attempts so far including this one, and a rejected attempt
// leaves z and the running averages as they were.  The averages weight each
// accepted iterate by its step.
//
// K1 (rows of A~^T): the primal epilogue writes x+, the new average, the
//   pair (x+_j, x_j) into an interleaved vector (the accepted x is kept
//   there) and the saved x_avg, and sums dx_j^2.
// K2 (rows of A~): the pairs are gathered with one load per nonzero and
//   dx_j = x+_j - x_j formed as in K1, so one pass over A~ gives h = A~x+
//   and A~dx; the epilogue saves y, y_avg, A~x, A~x_avg,
//   writes the dual step, and sums dy_i^2 and dy_i (A~dx)_i.  The last block
//   adds every block's sums in block order and applies the rule above.
// K3: when the attempt was rejected, the saved state is copied back (x from
//   the pairs).
//
// A thread accumulates its rows in the iteration precision (in float32-mixed
// contexts the float64 pipe would bound the epilogue); blocks' sums are
// float64.  A row split across tiles is finished by whichever chunk arrives
// last, so its terms go to a record of its own, added in group order: the
// sums do not depend on the order in which blocks finish.
#include "dispatch.cuh"
#include "kernels.h"
#include "spmv_tile.cuh"

namespace pdhg {

template <typename T>
struct AdaptPrimalEpi {
  T* __restrict__ x;
  const T* __restrict__ c;
  T* __restrict__ x_avg;
  T* __restrict__ x_avg_prev;
  T* __restrict__ xx;  // (x+_j, x_j) at 2j, 2j + 1
  double* __restrict__ split_rec;  // one per split group of A~^T
  T tau, w;
  bool first;
  T acc;  // this thread's sum of dx_j^2 over rows finished in one tile
  __device__ __forceinline__ void row(int j, const T (&s)[1], int group) {
    const T xo = x[j], xa = x_avg[j];
    const T xn = fmax(T(0), xo - tau * (c[j] - s[0]));
    const T d = xn - xo;
    x_avg_prev[j] = xa;
    x[j] = xn;
    x_avg[j] = first ? xn : xa + (xn - xa) * w;
    if constexpr (sizeof(T) == 4)
      reinterpret_cast<float2*>(xx)[j] = make_float2(xn, xo);
    else
      reinterpret_cast<double2*>(xx)[j] = make_double2(xn, xo);
    if (group < 0)
      acc = fmadd(d, d, acc);
    else
      split_rec[group] = (double)d * (double)d;
  }
};

// x+_j and dx_j = x+_j - x_j (the same rounding as K1's) from one load of the pair
template <typename T>
struct GatherMove {
  GatherPair<T> pair;
  __device__ __forceinline__ void load(int c, T (&o)[2]) const {
    pair.load(c, o);
    o[1] = o[0] - o[1];
  }
};

template <typename T>
struct AdaptDualEpi {
  T* __restrict__ y;
  const T* __restrict__ b;
  T* __restrict__ Ax;
  T* __restrict__ y_avg;
  T* __restrict__ Ax_avg;
  T* __restrict__ y_prev;
  T* __restrict__ y_avg_prev;
  T* __restrict__ Ax_prev;
  T* __restrict__ Ax_avg_prev;
  double* __restrict__ split_rec;  // two per split group of A~
  T sigma, w;
  bool first;
  T dy2, cross;  // this thread's sums of dy_i^2 and dy_i (A~dx)_i
  // s[0] = (A~x+)_i, s[1] = (A~dx)_i
  __device__ __forceinline__ void row(int i, const T (&s)[2], int group) {
    const T yo = y[i], ax = Ax[i], ya = y_avg[i], axa = Ax_avg[i];
    const T h = s[0];
    const T yn = yo + sigma * (b[i] - (h + h) + ax);
    const T d = yn - yo;
    y_prev[i] = yo;
    y_avg_prev[i] = ya;
    Ax_prev[i] = ax;
    Ax_avg_prev[i] = axa;
    Ax[i] = h;
    y[i] = yn;
    y_avg[i] = first ? yn : ya + (yn - ya) * w;
    Ax_avg[i] = first ? h : axa + (h - axa) * w;
    if (group < 0) {
      dy2 = fmadd(d, d, dy2);
      cross = fmadd(d, s[1], cross);
    } else {
      split_rec[2 * group] = (double)d * (double)d;
      split_rec[2 * group + 1] = (double)d * (double)s[1];
    }
  }
};

template <typename T, int BLOCK, int E>
__global__ void __launch_bounds__(BLOCK) k_aprimal(IterBuffers<T> B, int i) {
  pdl_enter();
  if (B.sc->done) return;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[BLOCK / 32];
  __shared__ double out[1];
  AdaptPrimalEpi<T> epi{B.x,          B.c_t,          B.x_avg,               B.x_avg_prev, B.adapt_xx,
                        B.adapt_sp,   (T)B.sc->tau,   (T)B.sc->avg_w,        B.sc->avg_first != 0,
                        T(0)};
  Gather<T, 1> g{{B.y}};
  run_sched<T, 1, BLOCK, E>(B.t_sched, B.t_rp, B.t_col, B.t_val, g, epi, smem);
  double mine[1] = {(double)epi.acc};
  block_sum<BLOCK, 1>(mine, out, red);
  if (threadIdx.x == 0) B.adapt_pp[blockIdx.x] = out[0];
}

template <typename T, int BLOCK, int E>
__global__ void __launch_bounds__(BLOCK) k_adual(IterBuffers<T> B, int i) {
  pdl_enter();
  if (B.sc->done) return;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[2 * (BLOCK / 32)];
  __shared__ double out[2];
  __shared__ double tot[3];
  __shared__ int is_last;
  AdaptDualEpi<T> epi{B.y,
                      B.b_t,
                      B.Ax,
                      B.y_avg,
                      B.Ax_avg,
                      B.y_prev,
                      B.y_avg_prev,
                      B.Ax_prev,
                      B.Ax_avg_prev,
                      B.adapt_sd,
                      (T)B.sc->sigma,
                      (T)B.sc->avg_w,
                      B.sc->avg_first != 0,
                      T(0),
                      T(0)};
  GatherMove<T> g{{B.adapt_xx}};
  run_sched<T, 2, BLOCK, E>(B.a_sched, B.a_rp, B.a_col, B.a_val, g, epi, smem);
  double mine[2] = {(double)epi.dy2, (double)epi.cross};
  block_sum<BLOCK, 2>(mine, out, red);
  if (threadIdx.x == 0) {
    B.adapt_pd[2 * blockIdx.x] = out[0];
    B.adapt_pd[2 * blockIdx.x + 1] = out[1];
    __threadfence();
    is_last = atomicAdd(&B.sc->ticket, 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  // ||dx||^2 from the primal kernel's blocks and split rows (that kernel has
  // completed: pdl_enter waited for it), then this kernel's two sums
  parts_sum<BLOCK, 1>(B.adapt_pp, B.adapt_np, B.adapt_sp, B.t_sched.ngroups, tot, red);
  parts_sum<BLOCK, 2>(B.adapt_pd, (int)gridDim.x, B.adapt_sd, B.a_sched.ngroups, tot + 1, red);
  if (threadIdx.x != 0) return;
  Scalars& sc = *B.sc;
  sc.ticket = 0;
  const double eta = sc.eta, om = sc.omega;
  const double inter = fabs(tot[2]);
  const double num = om * tot[0] + tot[1] / om;
  const double inf = __longlong_as_double(0x7ff0000000000000LL);
  const double eta_max = inter > 0.0 ? num / (2.0 * inter) : inf;
  const double j1 = (double)(sc.k + i + 1) + 1.0;
  const double nxt = fmin((1.0 - pow(j1, -0.3)) * eta_max, (1.0 + pow(j1, -0.6)) * eta);
  const bool acc = eta <= eta_max;
  sc.accept = acc ? 1 : 0;
  if (acc)
    sc.eta_sum += eta;
  else
    sc.step_rejects += 1;
  sc.eta = nxt;
  sc.tau = nxt / om;
  sc.sigma = nxt * om;
  sc.avg_w = nxt / (sc.eta_sum + nxt);
  sc.avg_first = sc.eta_sum == 0.0 ? 1 : 0;
}

template <typename T>
__global__ void k_adapt_revert(IterBuffers<T> B) {
  if (B.sc->done || B.sc->accept) return;
  const int n = B.n, m = B.m, len = max(n, m);
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < len; j += gridDim.x * blockDim.x) {
    if (j < n) {
      B.x[j] = B.adapt_xx[2 * (size_t)j + 1];
      B.x_avg[j] = B.x_avg_prev[j];
    }
    if (j < m) {
      B.y[j] = B.y_prev[j];
      B.y_avg[j] = B.y_avg_prev[j];
      B.Ax[j] = B.Ax_prev[j];
      B.Ax_avg[j] = B.Ax_avg_prev[j];
    }
  }
}

template <typename T>
void launch_adapt_primal(const IterBuffers<T>& B, const Launch& L, int i, cudaStream_t s) {
  PDHG_DISPATCH_E(B.t_sched.e, launch_pdl(k_aprimal<T, kBlock, E_>, L.grid, kBlock, L.smem, s, B, i));
}
template <typename T>
void launch_adapt_dual(const IterBuffers<T>& B, const Launch& L, int i, cudaStream_t s) {
  PDHG_DISPATCH_E(B.a_sched.e, launch_pdl(k_adual<T, kBlock, E_>, L.grid, kBlock, L.smem, s, B, i));
}
template <typename T>
void launch_adapt_revert(const IterBuffers<T>& B, int grid, cudaStream_t s) {
  k_adapt_revert<T><<<grid, 256, 0, s>>>(B);
}

#define PDHG_INST(T)                                                                           \
  template void launch_adapt_primal<T>(const IterBuffers<T>&, const Launch&, int, cudaStream_t); \
  template void launch_adapt_dual<T>(const IterBuffers<T>&, const Launch&, int, cudaStream_t);   \
  template void launch_adapt_revert<T>(const IterBuffers<T>&, int, cudaStream_t);
PDHG_INST(float)
PDHG_INST(double)
#undef PDHG_INST

template <int E>
static const void* adaptive_kernel(int which) {
  switch (which) {
    case 0: return (const void*)k_aprimal<float, kBlock, E>;
    case 1: return (const void*)k_aprimal<double, kBlock, E>;
    case 2: return (const void*)k_adual<float, kBlock, E>;
    case 3: return (const void*)k_adual<double, kBlock, E>;
    default: return nullptr;
  }
}

cudaError_t configure_adaptive_kernels(size_t max_smem) {
  cudaError_t e = cudaSuccess;
  for (int w = 0; w < 4; ++w)
    for (const void* f : {adaptive_kernel<8>(w), adaptive_kernel<16>(w), adaptive_kernel<32>(w),
                          adaptive_kernel<-4>(w), adaptive_kernel<-8>(w)}) {
      cudaError_t r = set_max_dyn_smem(f, max_smem);
      if (r != cudaSuccess) e = r;
    }
  return e;
}

int adaptive_occupancy(int which, int e, size_t smem) {
  const void* f = nullptr;
  PDHG_DISPATCH_E(e, f = adaptive_kernel<E_>(which));
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, kBlock, smem);
  return nb < 1 ? 1 : nb;
}

}  // namespace pdhg
