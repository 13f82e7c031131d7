// Launch helpers shared by the translation units that launch tile kernels.
#pragma once
#include <cuda_runtime.h>

// SpMV variant of a schedule -> template instantiation: segmented with
// E = 8, 16, 32 nonzeros per thread, or vector with 4 / 8 lanes per row
// (E_ = -4, -8).
#define PDHG_DISPATCH_E(e, ...)                 \
  switch (e) {                                  \
    case -4: {                                  \
      constexpr int E_ = -4;                    \
      __VA_ARGS__;                              \
    } break;                                    \
    case -8: {                                  \
      constexpr int E_ = -8;                    \
      __VA_ARGS__;                              \
    } break;                                    \
    case 32: {                                  \
      constexpr int E_ = 32;                    \
      __VA_ARGS__;                              \
    } break;                                    \
    case 16: {                                  \
      constexpr int E_ = 16;                    \
      __VA_ARGS__;                              \
    } break;                                    \
    default: {                                  \
      constexpr int E_ = 8;                     \
      __VA_ARGS__;                              \
    } break;                                    \
  }

namespace pdhg {

// Launch with programmatic stream serialization (the kernel must start with
// pdl_enter(): it may begin while the previous kernel on the stream drains).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), int grid, int block, size_t smem,
                              cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// raises a kernel's dynamic shared-memory limit to what the device allows
// next to its static shared memory
inline cudaError_t set_max_dyn_smem(const void* f, size_t max_smem) {
  cudaFuncAttributes a;
  cudaError_t r = cudaFuncGetAttributes(&a, f);
  if (r == cudaSuccess)
    r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(max_smem - a.sharedSizeBytes));
  return r;
}

}  // namespace pdhg
