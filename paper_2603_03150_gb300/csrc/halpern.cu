// Reflected Halpern iteration (optional method 1): the primal and dual
// half-steps with the Halpern combination fused into their epilogues.
//
// With T one PDHG step, z = (x, y), the anchor z0 = (x_last, y_last) (the
// last restart point) and t the iterations since it:
//   (x^, y^) = T(x, y):  x^ = max(0, x - tau (c~ - A~^T y)),
//                        y^ = y + sigma (b~ - A~(2 x^ - x)),
//   z <- lam ((1 + rho) T(z) - rho z) + (1 - lam) z0,   lam = (t+1)/(t+2).
// K1 (rows of A~^T): x^ into x_avg, the new x in place.
// K2 (rows of A~): h = A~x^ (x^ gathered), A~(2x^ - x) = 2h - A~x from the
// cache of A~x; y^ into y_avg, h into Ax_avg, the new y in place and the
// cache A~x <- lam((1+rho) h - rho A~x) + (1-lam) A~x0 by linearity.
// The evaluation then sees (x, y) and T(z) = (x^, y^) as its two candidates.
#include "dispatch.cuh"
#include "epilogues.cuh"
#include "kernels.h"
#include "spmv_tile.cuh"

namespace pdhg {


template <typename T, int BLOCK, int E>
__global__ void __launch_bounds__(BLOCK) k_hprimal(IterBuffers<T> B, int i) {
  pdl_enter();
  if (B.sc->done) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const long long tt = B.sc->t + i;  // iterations since restart before this one
  const double lam = (double)(tt + 1) / (double)(tt + 2);
  HalpernPrimalEpi<T> epi{B.x, B.x_avg, B.c_t, B.x_last, (T)B.sc->tau, (T)lam, (T)B.rho};
  Gather<T, 1> g{{B.y}};
  run_sched<T, 1, BLOCK, E>(B.t_sched, B.t_rp, B.t_col, B.t_val, g, epi, smem);
}


template <typename T, int BLOCK, int E>
__global__ void __launch_bounds__(BLOCK) k_hdual(IterBuffers<T> B, int i) {
  pdl_enter();
  if (B.sc->done) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const long long tt = B.sc->t + i;
  const double lam = (double)(tt + 1) / (double)(tt + 2);
  HalpernDualEpi<T> epi{B.y,      B.b_t,       B.Ax,    B.y_avg,           B.Ax_avg,
                        B.y_last, B.Ax_last,   (T)B.sc->sigma, (T)lam,     (T)B.rho};
  Gather<T, 1> g{{B.x_avg}};  // x^ of this iteration
  run_sched<T, 1, BLOCK, E>(B.a_sched, B.a_rp, B.a_col, B.a_val, g, epi, smem);
}

template <typename T>
void launch_hprimal(const IterBuffers<T>& B, const Launch& L, int i, cudaStream_t s) {
  PDHG_DISPATCH_E(B.t_sched.e, launch_pdl(k_hprimal<T, kBlock, E_>, L.grid, kBlock, L.smem, s, B, i));
}
template <typename T>
void launch_hdual(const IterBuffers<T>& B, const Launch& L, int i, cudaStream_t s) {
  PDHG_DISPATCH_E(B.a_sched.e, launch_pdl(k_hdual<T, kBlock, E_>, L.grid, kBlock, L.smem, s, B, i));
}
template void launch_hprimal<float>(const IterBuffers<float>&, const Launch&, int, cudaStream_t);
template void launch_hprimal<double>(const IterBuffers<double>&, const Launch&, int, cudaStream_t);
template void launch_hdual<float>(const IterBuffers<float>&, const Launch&, int, cudaStream_t);
template void launch_hdual<double>(const IterBuffers<double>&, const Launch&, int, cudaStream_t);

template <int E>
static const void* halpern_kernel(int which) {
  switch (which) {
    case 0: return (const void*)k_hprimal<float, kBlock, E>;
    case 1: return (const void*)k_hprimal<double, kBlock, E>;
    case 2: return (const void*)k_hdual<float, kBlock, E>;
    case 3: return (const void*)k_hdual<double, kBlock, E>;
    default: return nullptr;
  }
}

cudaError_t configure_halpern_kernels(size_t max_smem) {
  cudaError_t e = cudaSuccess;
  for (int w = 0; w < 4; ++w)
    for (const void* f : {halpern_kernel<8>(w), halpern_kernel<16>(w), halpern_kernel<32>(w),
                          halpern_kernel<-4>(w), halpern_kernel<-8>(w)}) {
      cudaError_t r = set_max_dyn_smem(f, max_smem);
      if (r != cudaSuccess) e = r;
    }
  return e;
}

int halpern_occupancy(int which, int e, size_t smem) {
  const void* f = nullptr;
  PDHG_DISPATCH_E(e, f = halpern_kernel<E_>(which));
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, kBlock, smem);
  return nb < 1 ? 1 : nb;
}

}  // namespace pdhg
