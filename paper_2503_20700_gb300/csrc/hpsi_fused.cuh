// Fused H_eff psi contraction (Sec. II.B two-site effective Hamiltonian):
//
//   sigma(a', b') += sum_i alpha_i op(A_i) P_i op(B_i)^T
//
// with A_i a left-block operator sector block (m_a' x m_a, or the identity),
// P_i the psi block (m_a x m_b) and B_i a right-block operator sector block
// (m_b' x m_b, or the identity).  One CTA owns one 64 x 64 tile of one sigma
// block and a chunk of its items; for every item and every 64-wide column
// chunk of psi it forms X = alpha A P(:, chunk) on chip and accumulates
// X B(:, chunk)^T, so the intermediate never reaches HBM.  Chunks of items of
// the same tile are reduced by a second kernel in a fixed order
// (deterministic, no atomics).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "backend.hpp"

namespace dmrg {

struct HpsiItem {
  const double* A;  // nullptr: identity (m_a == m_a')
  const double* P;
  const double* B;  // nullptr: identity (m_b == m_b')
  int lda, ldp, ldb;
  int transA, transB;  // A: 0 -> stored m_a' x m_a; 1 -> stored m_a x m_a'
                       // B: 0 -> stored m_b' x m_b (used transposed); 1 -> stored m_b x m_b'
  int ka, kb;          // m_a, m_b
  double alpha;
};

struct HpsiBlock {
  double* C;
  int m, n, ldc;
  int item_begin, item_count;
};

struct HpsiTask {
  int block, r0, c0;
  int it_begin, it_count;
  long long part;  // offset (elements) of this task's partial tile in scratch, or -1: add into C
};

struct HpsiReduce {
  int block, r0, c0, nparts;
  long long part0;  // first partial; the others follow at +tile_m*tile_n each
};

// sigma tile owned by one CTA of the kernel used for `prec`: 64 x 64 (FP64 and
// SPLIT_TF32 on mma.sync; the tcgen05 contraction plans its own 128 x 256
// tiles in hpsi_tc_prepare).
void hpsi_tile(Precision prec, int* tile_m, int* tile_n);

// Builds the task list (tiles x item chunks) for the given blocks; returns the
// scratch size (elements) the partial tiles need.  The item chunk length is
// chosen so that one launch has several waves of CTAs on 152 SMs.
size_t hpsi_plan_tasks(const std::vector<HpsiBlock>& blocks, Precision prec, std::vector<HpsiTask>& tasks,
                       std::vector<HpsiReduce>& reds);

// Launches the fused kernel and the reduction (device pointers in the lists).
// prec: FP64 or SPLIT_TF32 (err is unused by these kernels).
void hpsi_launch(const HpsiBlock* blocks, const HpsiItem* items, const HpsiTask* tasks, int ntasks,
                 const HpsiReduce* reds, int nreds, double* scratch, Precision prec, int* err,
                 cudaStream_t st);


}  // namespace dmrg
