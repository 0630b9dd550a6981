// Static device scratch of the allocation-free fused H_eff psi entry point.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>

namespace dmrg {

// Capacity of the static scratch: block, item, task and reduction lists and
// the partial tiles of one call (about one thousand 64 x 64 float64 partial
// tiles).
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;

// Device address of the static scratch on `device`, looked up once (with that
// device current) and cached; later calls only read the cache.
cudaError_t noalloc_scratch(int device, void** addr);

}  // namespace dmrg
