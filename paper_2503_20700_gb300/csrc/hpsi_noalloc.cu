// Static device scratch of the allocation-free fused H_eff psi entry point
// (dmrg_hpsi_contract_noalloc).  The task lists and partial tiles of one call
// live in a file-scope __device__ array; its address is looked up once per
// device with cudaGetSymbolAddress and cached.  No device memory is
// allocated or freed on this path.
#include <cuda_runtime.h>

#include <mutex>

#include "hpsi_noalloc.hpp"

namespace dmrg {

namespace {
__device__ __align__(256) unsigned char g_hpsi_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};
}  // namespace

cudaError_t noalloc_scratch(int device, void** addr) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[device]) {
    int prev = 0;
    cudaError_t e = cudaGetDevice(&prev);
    if (e != cudaSuccess) return e;
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return e;
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_hpsi_scratch);
    cudaError_t e2 = cudaSetDevice(prev);
    if (e != cudaSuccess) return e;
    if (e2 != cudaSuccess) return e2;
    g_addr[device] = p;
  }
  *addr = g_addr[device];
  return cudaSuccess;
}

}  // namespace dmrg
