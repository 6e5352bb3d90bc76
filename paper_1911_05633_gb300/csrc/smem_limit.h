// Dynamic shared-memory opt-in shared by every plan of the process.
#pragma once

#include <cuda_runtime.h>

namespace gw {

// Raise (never lower) a kernel's dynamic shared-memory limit on the current device.
// The attribute belongs to the function, not to a plan: lowering it for a small plan
// would make the launches of a larger plan that is still alive fail.
template <typename F>
inline cudaError_t raise_smem_limit(F* func, size_t bytes) {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, func);
  if (e != cudaSuccess) return e;
  if ((size_t)a.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
  return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace gw
