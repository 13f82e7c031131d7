// Algorithm 1 (Section 3.1) centered start point on caller-provided device
// vectors with no device allocation (pdhg_centered_point_noalloc in
// include/pdhg.h).
//
// Some callers cannot call cudaMalloc: an interior-point solver that owns a
// fixed device memory pool and must not grow it, or a host thread that must
// not take the device allocator's locks.  For them the scratch this
// computation needs -- one partial sum of x^T z per block and mu_target --
// lives in a file-scope __device__ array that every GPU which loads this
// library holds until the process exits.
#include <mutex>

#include "common.cuh"
#include "pdhg.h"

namespace pdhg {
void set_error(const char* fmt, ...);
}

namespace {

constexpr int kNaThreads = 256;
constexpr int kNaPerBlock = 2048;   // entries of x^T z reduced by one block
constexpr int kNaMaxBlocks = 4096;  // partial-sum slots
constexpr long long kNaMaxN = (long long)kNaPerBlock * kNaMaxBlocks;  // 8,388,608

// [0, kNaMaxBlocks): per-block partial sums of x^T z; [kNaMaxBlocks]: mu_target.
// Every call writes each slot it reads before reading it, so nothing has to
// be cleared between calls.  32 KB per device.
static __device__ __align__(256) double g_na_scratch[kNaMaxBlocks + 2];

__global__ void k_na_partial(int n, const double* __restrict__ x, const double* __restrict__ z,
                             double* scratch) {
  __shared__ double red[kNaThreads / 32];
  const int base = blockIdx.x * kNaPerBlock;
  const int end = min(n, base + kNaPerBlock);
  double acc = 0.0;
  for (int i = base + threadIdx.x; i < end; i += kNaThreads) acc += x[i] * z[i];
  const double v[1] = {acc};
  double o[1];
  pdhg::block_sum<kNaThreads, 1>(v, o, red);
  if (threadIdx.x == 0) scratch[blockIdx.x] = o[0];
}

__global__ void k_na_mu(int nblocks, int n, double mu_min, double* scratch, double* mu_out) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += scratch[b];
  const double mu = fmax(s / (double)n, mu_min);
  scratch[kNaMaxBlocks] = mu;
  if (mu_out) *mu_out = mu;
}

__device__ __forceinline__ double na_move(double target, double v, double delta) {
  return fmin(fmax(target, v - delta), v + delta);
}

// Algorithm 1's per-entry update (Section 3.1)
__global__ void k_na_apply(int n, const double* __restrict__ x, const double* __restrict__ z,
                           const double* scratch, double delta, double alpha,
                           double* __restrict__ x_out, double* __restrict__ z_out) {
  const double mu = scratch[kNaMaxBlocks];
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    double xp = fmax(x[j], alpha), zp = fmax(z[j], alpha);
    if (xp < zp) {
      xp = na_move(mu / zp, xp, delta);
      zp = na_move(mu / xp, zp, delta);
    } else {
      zp = na_move(mu / xp, zp, delta);
      xp = na_move(mu / zp, xp, delta);
    }
    x_out[j] = xp;
    z_out[j] = zp;
  }
}

// Device address of g_na_scratch, looked up once per device (in the device's
// primary context; a cudaDeviceReset would leave it stale, and the header
// rules that out).
std::mutex g_na_mutex;
constexpr int kNaMaxDevices = 256;
double* g_na_ptr[kNaMaxDevices] = {};

}  // namespace

extern "C" pdhg_status pdhg_centered_point_noalloc(int32_t n, const double* x, const double* z,
                                                   double mu_min, double delta_max,
                                                   double alpha_min, double* x_out, double* z_out,
                                                   double* mu_target, void* stream) {
  if (n < 1 || (long long)n > kNaMaxN) {
    pdhg::set_error("pdhg_centered_point_noalloc: n = %d outside [1, %lld] (the static scratch "
                    "holds %d partial sums of %d entries each)",
                    n, kNaMaxN, kNaMaxBlocks, kNaPerBlock);
    return PDHG_INVALID_ARG;
  }
  if (!x || !z || !x_out || !z_out) {
    pdhg::set_error("pdhg_centered_point_noalloc: x, z, x_out and z_out must be device pointers");
    return PDHG_INVALID_ARG;
  }
  if (!(mu_min > 0.0) || !(delta_max >= 0.0) || !(alpha_min > 0.0)) {
    pdhg::set_error("pdhg_centered_point_noalloc: need mu_min > 0, delta_max >= 0, alpha_min > 0");
    return PDHG_INVALID_ARG;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) {
    pdhg::set_error("pdhg_centered_point_noalloc: cudaGetDevice failed: %s", cudaGetErrorString(e));
    return PDHG_CUDA_ERROR;
  }
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
      // set-up on the first call on this device (the current device)
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_na_scratch);
      if (e != cudaSuccess || !p) {
        pdhg::set_error("pdhg_centered_point_noalloc: cudaGetSymbolAddress failed: %s",
                        cudaGetErrorString(e));
        return PDHG_CUDA_ERROR;
      }
      g_na_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_na_ptr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nblocks = (int)((n + kNaPerBlock - 1) / kNaPerBlock);
  k_na_partial<<<nblocks, kNaThreads, 0, s>>>(n, x, z, scratch);
  k_na_mu<<<1, 32, 0, s>>>(nblocks, n, mu_min, scratch, mu_target);
  int grid = (n + 255) / 256;
  if (grid > 4096) grid = 4096;
  k_na_apply<<<grid, 256, 0, s>>>(n, x, z, scratch, delta_max, alpha_min, x_out, z_out);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    pdhg::set_error("pdhg_centered_point_noalloc: launch failed: %s", cudaGetErrorString(e));
    return PDHG_CUDA_ERROR;
  }
  return PDHG_OK;
}
