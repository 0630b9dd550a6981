// Per-device kernel attributes.  cudaFuncSetAttribute applies to the device
// that is current when it is called, so the opt-in dynamic shared memory of a
// kernel is set once per (kernel, device) pair, under a lock, and its return
// code is passed on.
#pragma once
#include <cuda_runtime.h>

#include <mutex>
#include <set>
#include <utility>

namespace dmrg {

inline cudaError_t ensure_smem_attr(const void* func, int bytes) {
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  if (done.count({func, dev})) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done.insert({func, dev});
  return e;
}

}  // namespace dmrg
