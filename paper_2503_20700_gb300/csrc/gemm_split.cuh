// Split-precision grouped GEMM: C += sum_s alpha_s op(A_s) op(B_s) with the
// float64 operands split into two TF32 parts, x = hi + lo, and the product
// evaluated as hi*hi + hi*lo + lo*hi (3xTF32) with FP32 accumulation inside
// one segment and a float64 accumulator across segments.
//
// This file holds the warp-level (mma.sync m16n8k8) implementation, used for
// small sector blocks and as the baseline of the tcgen05 kernel in
// gemm_tc.cu, which takes the large tiles.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <functional>
#include <vector>

#include "backend.hpp"

namespace dmrg {

struct SplitTile {
  int group, r0, c0, pad;
};

using UploadFn = std::function<char*(const std::vector<std::pair<const void*, size_t>>&, std::vector<size_t>&)>;

void gemm_split_launch(const std::vector<GemmGroup>& groups, const std::vector<GemmSeg>& segs,
                       Precision prec, cudaStream_t st, const UploadFn& upload);

}  // namespace dmrg
