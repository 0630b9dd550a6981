// tcgen05 (5th-generation tensor core) fused H_eff psi contraction,
// 3xTF32 split precision (Sec. II.B two-site effective Hamiltonian):
//
//   sigma(a', b') += sum_i alpha_i op(A_i) P_i op(B_i)^T
//
// Operands are split once into TF32 hi/lo planes (float32 storage,
// row-major, row length padded to a multiple of 32 with zeros): the operator
// blocks once per bond (they are constant during Davidson), the psi blocks
// once per product (transposed, so that both products are K-major).  One CTA
// owns a 128 x N (N <= 256) tile of a sigma block and a chunk of its items;
// per item and per 64-wide chunk j of psi's columns
//   stage 1:  X' = op(A)(tile rows, :) P(:, j)           (TMEM, 128 x 64)
//   X = alpha X'  ->  hi/lo TF32 planes in shared memory
//   stage 2:  S += X op(B)(tile cols, j)^T               (TMEM, 128 x N)
// with 16-byte cp.async copies in three slots: the MMAs of a k-block are
// issued once its copies land, then the copies two blocks ahead refill the
// slot whose MMAs precede them.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <functional>
#include <vector>

#include "hpsi_fused.cuh"

namespace dmrg {

// hi/lo TF32 planes of a matrix; rows = output index of the product, columns
// = contraction index; ld = padded row length (multiple of 32 floats)
struct TcMat {
  const float* hi = nullptr;
  const float* lo = nullptr;
  int ld = 0;
};

struct TcItem {
  TcMat A;             // op(A): m' x ka; A.hi == nullptr: identity (ka == m')
  TcMat Pt;            // P^T: kb x ka
  const double* P;     // P (ka x kb, float64, row length ldp) for identity-A items
  int ldp;
  TcMat B;             // op(B): n' x kb; B.hi == nullptr: identity (kb == n')
  int ka, kb;
  double alpha;
};

// dst (rows x ldd, float32 hi/lo) = split(op(src)) with op(src)(r, c) =
// trans ? src[c*ld + r] : src[r*ld + c] for c < cols, zero for cols <= c < ldd
struct SplitJob {
  const double* src;
  int rows, cols, ld, trans;
  float* hi;
  float* lo;
  int ldd;
};

constexpr int kTcTileM = 128, kTcTileN = 256;

struct TcPlan {
  std::vector<SplitJob> op_jobs;   // operator blocks (run once per plan)
  std::vector<SplitJob> psi_jobs;  // psi blocks (run before every product)
  std::vector<TcItem> items;
  std::vector<HpsiTask> tasks;     // (block, r0, c0, items, partial offset)
  std::vector<HpsiReduce> reds;    // one per tile: its chunks' partial tiles into sigma
  size_t scratch = 0;              // 8-byte words of partial tiles (kTcTileM x kTcTileN float pairs per task)
  size_t pool_bytes = 0;           // split planes
};

// Split planes, items and tasks for the fused contraction of `blocks`/`items`
// (device pointers inside).  alloc(bytes) returns the device memory of the
// split planes; the caller owns it.
void hpsi_tc_prepare(const std::vector<HpsiBlock>& blocks, const std::vector<HpsiItem>& items,
                     const std::function<void*(size_t)>& alloc, TcPlan& plan);

// Runs the split jobs (device list of n jobs).
void split_launch(const SplitJob* jobs, int n, cudaStream_t st);

// The fused kernel and the reduction of item chunks (device lists).  err: a
// device int set to 1 when a bounded wait ran out (the CTA then skips the
// rest of its work).
void hpsi_tc_launch(const HpsiBlock* blocks, const TcItem* items, const HpsiTask* tasks, int ntasks,
                    const HpsiReduce* reds, int nreds, double* scratch, int* err, cudaStream_t st);

}  // namespace dmrg
