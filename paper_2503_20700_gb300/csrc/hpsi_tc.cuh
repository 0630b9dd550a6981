// tcgen05 (5th-generation tensor core) fused H_eff psi contraction,
// 3xTF32 split precision (Sec. II.B two-site effective Hamiltonian):
//
//   sigma(a', b') += sum_i alpha_i op(A_i) P_i op(B_i)^T
//
// Operands are split into TF32 hi/lo planes once: the operator blocks once
// per bond (they are constant during Davidson), the psi blocks before every
// product (transposed, so that both products are K-major).  Identity factors
// become explicit identity planes, so every item has the same three operands.
//
// Plane layout in the pool (1 KB units, 256 floats each).  A matrix of R rows
// and K columns has G = ceil(R/8) row groups and ceil(K/32) k-blocks; unit
// 2 (kb G + g) holds the hi plane and unit 2 (kb G + g) + 1 the lo plane of
// rows [8g, 8g+8) x columns [32kb, 32kb+32), each as eight 8-row x 16-byte
// core matrices (k-core c at byte 128 c, row r at byte 16 r within it), the
// canonical no-swizzle K-major layout of the tensor core.  Half a unit holds
// one k-block of 16, so a TMA box of 128 floats by 2 R/8 units brings an R-row
// tile of a k-block of 16 (hi and lo planes interleaved by row group).  Rows
// and columns beyond the matrix are zero inside a plane; a box that runs past
// a plane reads other planes' finite values, which only reach unstored output
// rows and columns or meet zero padding.
//
// The persistent kernel runs in clusters of 2 or 4 CTAs.  A task is a
// 128 x N (N <= 256) tile of a sigma block and a chunk of its items; the CTAs
// of a cluster take tasks of the same block and chunk together (lockstep over
// the same items), and CTAs whose tiles share their rows form a group that
// shares stage 1.  Per item and per super-chunk of 256 columns of psi:
//   stage 1:  X' = op(A)(tile rows, :) P(:, super-chunk)   (TMEM, 128 x 256)
//             by one CTA of the group (super-chunks dealt round-robin)
//   X = alpha X' per 16-column piece -> hi/lo TF32 planes, written into the
//             shared memory of every CTA of the group
//   stage 2:  S += X op(B)(tile cols, piece)^T             (TMEM, 128 x N)
//             by every CTA for its own columns
// Warp roles: one producer warp issues the TMA copies into a ring of stages,
// one warp issues the MMAs, four warps convert X' and drain S into the task's
// partial tile of float pairs.  Every wait is bounded.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <functional>
#include <string>
#include <vector>

#include "hpsi_fused.cuh"

namespace dmrg {

// split plane pair of a matrix in the pool: first unit and row groups
struct TcMat {
  int unit = 0;
  int groups = 0;
};

struct TcItem {
  TcMat A;   // op(A): m' x ka
  TcMat Pt;  // P^T: kb x ka
  TcMat B;   // op(B): n' x kb
  int ka, kb;
  double alpha;
};

// Split of one matrix into its plane pair: op(src)(r, c) =
// trans ? src[c*ld + r] : src[r*ld + c] for r < rows, c < cols (src ==
// nullptr: the identity), zero elsewhere in the plane.
struct SplitJob {
  const double* src;
  int rows, cols, ld, trans;
  int unit;  // first unit of the plane pair
};

constexpr int kTcTileM = 128, kTcTileN = 256;
constexpr int kTcCluster = 2;     // CTAs per cluster of the persistent launch (default schedule)
constexpr int kTcClusterMax = 4;  // largest cluster a schedule may use
constexpr int kTcUnitFloats = 256;  // one 1 KB unit
constexpr int kTcDrainTerms = 1024;  // default FP32 accumulation length (terms) between drains

// One entry of a CTA's list: the task, and the CTA's group within the
// cluster for it (cluster ranks [grp0, grp0 + grpn), the CTAs whose tiles
// have the same rows).  A ghost entry (a cluster slot without a tile) names a
// task of its cluster slot, walks its items and computes nothing.
struct TcSlot {
  int task;
  int grp0, grpn;
  int ghost;
};

// Schedule of a planned contraction: the column width of the sigma tiles
// (multiple of 16, at most kTcTileN; stage-1 sharing is per group of tiles
// with the same rows), the number of tasks per CTA that the item chunks aim
// at (finer chunks: better balance, more partial tiles), and the order in
// which cluster tasks are placed on the clusters (0: longest first onto the
// least-loaded cluster; 1: sigma block by sigma block, the cluster tasks of
// one block and item chunk dealt round-robin, so that the CTAs running at
// the same time share their operands in L2), and the CTAs per cluster (the
// column tiles of one row tile are grouped that many at a time and share
// stage 1).
struct TcShape {
  int tile_n = kTcTileN;
  int chunks_per_cta = 4;
  int order = 0;
  int cluster = kTcCluster;
  bool operator==(const TcShape& o) const {
    return tile_n == o.tile_n && chunks_per_cta == o.chunks_per_cta && order == o.order &&
           cluster == o.cluster;
  }
};
// The shapes an autotuner tries, the default first.
std::vector<TcShape> tc_shape_candidates();

struct TcPlan {
  TcShape shape;                   // of tasks, reds and the CTA lists
  std::vector<SplitJob> op_jobs;   // operator blocks and identities (run once per plan)
  std::vector<SplitJob> psi_jobs;  // psi blocks (run before every product)
  std::vector<TcItem> items;
  std::vector<HpsiTask> tasks;     // (block, r0, c0, items, partial offset)
  std::vector<HpsiReduce> reds;    // one per tile: its chunks' partial tiles into sigma
  std::vector<int> cta_off;        // entries of CTA c: cta_task[cta_off[c] .. cta_off[c+1])
  std::vector<TcSlot> cta_task;    // the CTAs of a cluster have lists of equal length, entry k of
                                   // each belonging to the same block and item chunk
  size_t scratch = 0;              // 8-byte words of partial tiles (kTcTileM x kTcTileN float pairs per task)
  double cost = 0.0;               // modelled tensor work of the launch (busiest cluster)
  size_t units = 0;                // pool size in 1 KB units
  size_t pool_bytes = 0;
};

// Split planes, items, tasks and the per-CTA task lists of the fused
// contraction of `blocks`/`items` (device pointers inside).  alloc(bytes)
// returns the device memory of the pool; the caller owns it.  ncta: CTAs of
// the persistent launch, rounded down to whole clusters (0: 152).
void hpsi_tc_prepare(const std::vector<HpsiBlock>& blocks, const std::vector<HpsiItem>& items,
                     const std::function<void*(size_t)>& alloc, TcPlan& plan, int ncta = 0,
                     const TcShape& shape = TcShape());
// The two phases of hpsi_tc_prepare: the operands (split jobs, pool, item
// descriptors), which do not depend on the schedule, and the schedule
// (tasks, reductions, CTA lists and scratch size) for a shape; a plan can be
// rescheduled for another shape without touching its operands.
void hpsi_tc_operands(const std::vector<HpsiBlock>& blocks, const std::vector<HpsiItem>& items,
                      const std::function<void*(size_t)>& alloc, TcPlan& plan);
void hpsi_tc_schedule(const std::vector<HpsiBlock>& blocks, TcPlan& plan, const TcShape& shape, int ncta = 0);
// Key of the sector histogram of a contraction (block shapes in 64-row and
// 64-column steps with their item counts on a log scale, and the CTA count):
// contractions with equal keys share an autotuned shape.
uint64_t tc_histogram_key(const std::vector<HpsiBlock>& blocks, int ncta);

// Device-side lists and the pool of one planned contraction.
struct TcLaunch {
  const HpsiBlock* blocks = nullptr;
  const TcItem* items = nullptr;
  const HpsiTask* tasks = nullptr;
  const int* cta_off = nullptr;
  const TcSlot* cta_task = nullptr;
  int ncta = 0;  // a multiple of cluster
  const HpsiReduce* reds = nullptr;
  int nreds = 0;
  double* scratch = nullptr;
  const void* pool = nullptr;
  size_t units = 0;
  // FP32 accumulation length of S between drains into the float-pair partial
  // tile: once the items since the last drain reach this many terms of psi's
  // column index (sum of kb), after the item (0: after every item)
  int drain_terms = kTcDrainTerms;
  int tile_n = kTcTileN;  // column width of the tiles the plan was scheduled for
  int cluster = kTcCluster;  // CTAs per cluster the plan was scheduled for
};

// Runs the split jobs (device list of n jobs) into the pool.
void split_launch(const SplitJob* jobs, int n, float* pool, cudaStream_t st);

// The persistent contraction and the reduction of item chunks.  err: a
// device int set to 1 when a bounded wait ran out (the CTA then stops);
// wait_ns bounds every wait (0: a wait not complete at its first probe
// gives up).
void hpsi_tc_launch(const TcLaunch& L, int* err, unsigned long long wait_ns, cudaStream_t st);

// CTAs of the persistent launch that the device runs at once (whole clusters
// of `cluster` CTAs, one CTA per SM); 0 without a device.
int hpsi_tc_max_ctas(int cluster = kTcCluster);

// Host-side check of a plan against its own ranges (debug_bounds): every
// TMA box of every item inside the pool's units or its zero-filled tail,
// every task's items and partial tile inside their lists, the CTA lists a
// permutation of the tasks plus ghosts, in clusters of equal-length lists
// whose entries agree on block and items, with consistent groups.  Returns an empty string or the first violation.
std::string tc_plan_check(const TcPlan& plan, const std::vector<HpsiBlock>& blocks);

}  // namespace dmrg
