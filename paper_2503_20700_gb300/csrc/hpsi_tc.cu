// tcgen05 fused H_eff psi contraction (see hpsi_tc.cuh), persistent and
// warp-specialised, with operand tiles brought in by TMA, in clusters of
// two or four CTAs (a launch parameter of the schedule).
//
// Per item of a task (a 128 x N, N <= 256, sigma tile) and per super-chunk
// of up to 256 columns of psi (columns [c, c+256) of P):
//   stage 1:  X' = op(A)(tile rows, :) P(:, c..c+256)          (TMEM, 128 x 256)
// then per 32-column piece p of the super-chunk:
//   X = alpha X'(:, p)  ->  TF32 hi/lo planes in shared memory (converters)
//   stage 2:  S += X op(B)(tile cols, p)^T                      (TMEM, 128 x N)
// Stage 1 uses N = 256 (one A panel fetch per 256 columns of psi) and stage 2
// the full tile width, so the MMAs are as wide as the tile allows.
//
// The CTAs of a cluster walk the same items; CTAs whose tiles have the same
// rows (a group) need the same X, so stage 1 of the super-chunks is dealt
// round-robin over the group (up to the cluster size), and the CTA that
// computes a super-chunk writes its pieces into its own X buffer and, by one
// bulk copy each, into those of the other CTAs of the group (distributed
// shared memory), completing their piece barriers.  Each CTA's MMA issuer
// signals the end of its reads of a piece buffer to every CTA of the cluster
// (multicast commit), so a buffer is rewritten once the whole cluster has read
// it.  A ghost entry (a cluster slot without a tile) only keeps that count.
//
// Shared memory (bytes): two X piece buffers (each hi | lo, 128 x 32, 16 KB
// per plane, 1 KB between 8-row groups) and three 48 KB stages, each holding
// the TMA tiles of one k-block of 16:
//   stage 1: A (128 rows: 16 KB) | P^T (256 rows: 32 KB)
//   stage 2: B (256 rows, the tile's columns: 32 KB)
// A TMA tile of a k-block of 16 takes half of each 1 KB pool unit: row group
// g holds its hi core matrices at 1024 g and its lo ones at 1024 g + 512,
// k-cores 128 B apart.  TMEM: S in columns [0, 256), X' in [256, 512).
//
// Warps: 0 producer (one lane issues cp.async.bulk.tensor into the stages;
// full/empty mbarriers), 1 MMA issuer (one lane; owns the TMEM allocation),
// 2..5 converters (TMEM lanes 32 (w % 4) .. +31: X' pieces -> alpha X' as
// TF32 hi/lo planes, double-buffered, and the drains of S into the task's
// partial tile of float pairs).  The MMA issuer runs stage 1 of this CTA's
// next super-chunk before stage 2 of the last piece of its current one, so
// the tensor pipe runs it while that piece is converted.  S is drained once
// the items accumulated in FP32 since the last drain reach drain_terms terms
// of psi's column index (sum of kb; 0: after every item) and at the end of
// every task.  Every wait gives up after the launch's wait bound (2 s of wall
// clock by default): the CTA then sets the error flag and the abort flag of
// every CTA of the cluster, waits (bounded by 2 s) for its copies and MMAs in
// flight, frees TMEM and leaves with the cluster.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>
#include <stdexcept>
#include <string>

#include "hpsi_tc.cuh"
#include "kattr.hpp"

namespace dmrg {

namespace {

constexpr int TM = kTcTileM, TNMAX = kTcTileN;
constexpr int W1 = 256;               // stage-1 super-chunk width (columns of psi)
constexpr int PW = 32;                // piece width (X planes, stage-2 K per piece)
constexpr uint32_t LBO = 128;         // between K-adjacent core matrices
constexpr uint32_t SBO_OP = 1024;     // between 8-row groups of a TMA tile (hi and lo interleaved)
constexpr uint32_t LO_OP = 512;       // lo plane of a row group in a TMA tile
constexpr uint32_t SBO_X = 1024;      // between 8-row groups of a 32-wide X plane
constexpr int NSTAGE = 3;
constexpr int STAGE = 49152;
constexpr int XBUF = 32768, XLO = 16384;  // X piece buffer (hi | lo)
constexpr int OFF_X = 0, OFF_STAGE = 2 * XBUF;
constexpr int SMEM_USED = OFF_STAGE + NSTAGE * STAGE;  // 208 KB
constexpr int SMEM_BYTES = SMEM_USED + 1024;            // slack for 1 KB alignment of the base
constexpr int A_BYTES = 16384, P_BYTES = 32768, B_BYTES = 32768;
constexpr uint32_t TCOL_S = 0, TCOL_X = 256;
constexpr int NTHREADS = 192;
constexpr unsigned long long kWaitNs = 2000000000ull;
constexpr unsigned long long kDrainCopiesNs = 100000ull;  // in-flight peer copies land within this

// barriers
enum { B_FULL = 0, B_EMPTY = B_FULL + NSTAGE, B_XPF = B_EMPTY + NSTAGE, B_XPE, B_XF, B_XE = B_XF + 2,
       B_XA = B_XE + 2, B_SF = B_XA + 2, B_SE, B_DONE, B_COUNT };

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t desc(uint32_t saddr, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((LBO >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of this architecture; no swizzle
  return d;
}
// kind::tf32, FP32 accumulator, both operands K-major
__device__ __forceinline__ uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ uint32_t tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// one arrival on the barrier at the same offset in every CTA of the cluster,
// once the MMAs issued so far by this thread have completed
__device__ __forceinline__ void commit_all(uint64_t* bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"(mask)
      : "memory");
}
__device__ __forceinline__ void arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void arrive_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// cluster shared address of this CTA's shared address `saddr` in CTA `rank`
__device__ __forceinline__ uint32_t map_to(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}
// copy of `bytes` of this CTA's shared memory into a peer's (cluster
// addresses dst and its barrier), by the bulk copy engine; the peer's barrier
// receives the bytes as transaction count
__device__ __forceinline__ void copy_to_peer(uint32_t dst, uint32_t src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "r"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// TMA copy of the box at (x floats, y units) of `map` into shared memory
__device__ __forceinline__ void tma_load(uint32_t dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// a probe of the phase with the given parity; CL: acquire at cluster scope
// (the phase may have been completed by arrivals from other CTAs)
template <bool CL>
__device__ __forceinline__ bool test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  if (CL)
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.test_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
  else
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
  return done != 0;
}
// a probe that may suspend the thread for up to ~1 us while the phase is
// incomplete (frees the issue slot for the warps that share the scheduler)
template <bool CL>
__device__ __forceinline__ bool try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  if (CL)
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity), "r"(1000u)
        : "memory");
  else
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity), "r"(1000u)
        : "memory");
  return done != 0;
}
// bounded wait on the phase with the given parity; false after wait_ns of
// wall clock (0: after the first probe), or at once when a role of this CTA
// or of another CTA of the cluster has aborted (abort != 0)
template <bool CL = false>
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, volatile int* abort,
                                         unsigned long long wait_ns) {
  if (test_wait<CL>(bar, parity)) return true;
  if (wait_ns == 0) return false;
  const unsigned long long t0 = global_ns();
  for (;;) {
    if (try_wait<CL>(bar, parity)) return true;
    if (*abort) return false;
    if (global_ns() - t0 > wait_ns) return false;
  }
}
// the same, with one outcome for the whole warp (the converter warps issue
// .sync.aligned TMEM loads right after their waits)
template <bool CL = false>
__device__ __forceinline__ bool wait_bar_warp(uint64_t* bar, uint32_t parity, volatile int* abort,
                                              unsigned long long wait_ns) {
  const bool ok = wait_bar<CL>(bar, parity, abort, wait_ns);
  return __all_sync(0xffffffffu, ok);
}
// byte offset of element (r, k) (k multiple of 4) in a 32-wide X plane
__device__ __forceinline__ uint32_t x_off(int r, int k) {
  return (uint32_t)(r >> 3) * SBO_X + (uint32_t)(k >> 2) * LBO + (uint32_t)(r & 7) * 16;
}

// The piece sequence of one CTA: its list entries in order, their items, the
// super-chunks of 256 columns of psi of every item and their 32-column pieces.
// Every CTA of a cluster walks the same sequence (its entries name tasks of
// the same items).
struct Walk {
  const HpsiBlock* blocks;
  const TcItem* items;
  const HpsiTask* tasks;
  const TcSlot* list;
  int t, t_end;
  int rank;  // of this CTA in the cluster
  TcSlot sl;
  HpsiTask tk;
  int N;    // MMA width of the tile (multiple of 16)
  int ii;   // item (global index)
  int k;    // item position within the task
  int jc;   // first column of the super-chunk
  int p;    // piece within the super-chunk
  int sct;  // super-chunk within the task
  int acc;          // sum of kb over the items since the last drain, this one included
  int drain_terms;  // drain once acc reaches it
  int tile_n;       // column width of the plan's tiles (multiple of 16, <= TNMAX)
  TcItem it;
  bool valid;
};
__device__ __forceinline__ void walk_task(Walk& w) {
  w.sl = w.list[w.t];
  w.tk = w.tasks[w.sl.task];
  const HpsiBlock bk = w.blocks[w.tk.block];
  const int nvalid = min(w.tile_n, bk.n - w.tk.c0);
  w.N = (nvalid + 15) & ~15;
  w.ii = w.tk.it_begin;
  w.k = 0;
  w.jc = 0;
  w.p = 0;
  w.sct = 0;
  w.it = w.items[w.ii];
  w.acc = w.it.kb;
}
__device__ __forceinline__ void walk_start(Walk& w, const HpsiBlock* blocks, const TcItem* items,
                                           const HpsiTask* tasks, const TcSlot* list, int t0, int t1,
                                           int drain_terms, int tile_n, int rank) {
  w.drain_terms = drain_terms;
  w.tile_n = tile_n;
  w.blocks = blocks;
  w.items = items;
  w.tasks = tasks;
  w.list = list;
  w.rank = rank;
  w.t = t0;
  w.t_end = t1;
  w.valid = t0 < t1;
  if (w.valid) walk_task(w);
}
__device__ __forceinline__ bool ghost(const Walk& w) { return w.sl.ghost != 0; }
// stage 1 of the current super-chunk is this CTA's (dealt round-robin over the group)
__device__ __forceinline__ bool owned(const Walk& w) {
  return !w.sl.ghost && w.sct % w.sl.grpn == w.rank - w.sl.grp0;
}
__device__ __forceinline__ int sc_width(const Walk& w) { return min(W1, w.it.kb - w.jc); }
__device__ __forceinline__ int sc_pieces(const Walk& w) { return (sc_width(w) + PW - 1) / PW; }
__device__ __forceinline__ bool last_piece(const Walk& w) { return w.p + 1 >= sc_pieces(w); }
__device__ __forceinline__ bool last_piece_of_item(const Walk& w) {
  return last_piece(w) && w.jc + W1 >= w.it.kb;
}
__device__ __forceinline__ bool drain_point(const Walk& w) {
  return last_piece_of_item(w) && (w.acc >= w.drain_terms || w.k + 1 == w.tk.it_count);
}
// to the next item (after its last piece)
__device__ __forceinline__ void walk_next_item(Walk& w, bool drained) {
  w.jc = 0;
  w.p = 0;
  ++w.ii;
  ++w.k;
  if (w.k < w.tk.it_count) {
    w.it = w.items[w.ii];
    w.acc = drained ? w.it.kb : w.acc + w.it.kb;
    return;
  }
  if (++w.t >= w.t_end) {
    w.valid = false;
    return;
  }
  walk_task(w);
}
// to the next piece
__device__ __forceinline__ void walk_next(Walk& w) {
  const bool drained = drain_point(w);  // only true at an item's last piece
  if (!last_piece(w)) {
    ++w.p;
    return;
  }
  w.p = 0;
  ++w.sct;
  w.jc += W1;
  if (w.jc < w.it.kb) return;
  walk_next_item(w, drained);
}
// to the start of the next super-chunk (from any of its pieces)
__device__ __forceinline__ void walk_next_sc(Walk& w) {
  w.p = sc_pieces(w) - 1;
  walk_next(w);
}
// to the start of the next super-chunk whose stage 1 is this CTA's
__device__ __forceinline__ void walk_next_owned(Walk& w) {
  do walk_next_sc(w);
  while (w.valid && !owned(w));
}
__device__ __forceinline__ void walk_first_owned(Walk& w) {
  if (w.valid && !owned(w)) walk_next_owned(w);
}
__device__ __forceinline__ int s1_blocks(const Walk& w) { return (w.it.ka + 15) >> 4; }
__device__ __forceinline__ int s2_kblocks(const Walk& w) { return min(2, (w.it.kb - w.jc - PW * w.p + 15) >> 4); }
__device__ __forceinline__ bool same_sc(const Walk& a, const Walk& b) { return a.t == b.t && a.sct == b.sct; }

// The issue order of stage 1, shared by the producer and the MMA issuer.
// s1w is this CTA's next super-chunk to compute, `done` of its k-blocks
// issued; `held` tells that X' holds a computed super-chunk whose last piece
// s2w has not reached.  Before the piece at s2w:
//  - nothing while X' is held;
//  - the rest of stage 1 of s1w when its pieces start now, or when s2w is the
//    last piece of this CTA's super-chunk and s1w comes right after it;
//  - while s2w walks a super-chunk of the group's other CTA (or a ghost
//    entry), a share of stage 1 of s1w proportional to the pieces walked, so
//    that the tensor pipe interleaves it with those pieces.
struct S1Order {
  Walk w;
  int done;
  bool held;
  int ht, hsct;  // the held super-chunk
};
__device__ __forceinline__ void s1_order_start(S1Order& o, const Walk& s2w) {
  o.w = s2w;
  walk_first_owned(o.w);
  o.done = 0;
  o.held = false;
}
// k-blocks of stage 1 of o.w to issue before the piece at s2w
__device__ __forceinline__ int s1_now(S1Order& o, const Walk& s2w) {
  if (o.held && o.ht == s2w.t && o.hsct == s2w.sct && last_piece(s2w)) o.held = false;
  if (o.held || !o.w.valid) return 0;
  const int nb = s1_blocks(o.w);
  if (same_sc(o.w, s2w)) return nb - o.done;
  if (owned(s2w)) {
    if (!last_piece(s2w)) return 0;
    Walk n = s2w;
    walk_next_sc(n);
    return (n.valid && same_sc(n, o.w)) ? nb - o.done : 0;
  }
  const int np = sc_pieces(s2w);
  return max(0, (nb * (s2w.p + 1) + np - 1) / np - o.done);
}
// after k-blocks [done, done + k) were issued
__device__ __forceinline__ void s1_issued(S1Order& o, const Walk& s2w, int k) {
  o.done += k;
  if (o.done < s1_blocks(o.w)) return;
  o.held = true;
  o.ht = o.w.t;
  o.hsct = o.w.sct;
  if (same_sc(o.w, s2w) && last_piece(s2w)) o.held = false;
  walk_next_owned(o.w);
  o.done = 0;
}

__global__ void __launch_bounds__(NTHREADS, 1)
    hpsi_tc_kernel(const __grid_constant__ CUtensorMap map32, const __grid_constant__ CUtensorMap map64,
                   const HpsiBlock* __restrict__ blocks, const TcItem* __restrict__ items,
                   const HpsiTask* __restrict__ tasks, const int* __restrict__ cta_off,
                   const TcSlot* __restrict__ cta_task, double* __restrict__ scratch, int* __restrict__ err,
                   unsigned long long wait_ns, int drain_terms, int tile_n, int csize) {
  extern __shared__ unsigned char smraw[];
  __shared__ __align__(8) uint64_t bar[B_COUNT];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  __shared__ int consumed;  // stage fills the MMA warp has waited for
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t sraw = smem_u32(smraw);
  const uint32_t sbase = (sraw + 1023u) & ~1023u;  // the same offset in every CTA of the cluster
  unsigned char* const sgen = smraw + (sbase - sraw);
  const int rank = (int)cluster_rank();
  const uint16_t cmask = (uint16_t)((1u << csize) - 1);  // every CTA of the cluster
  const int t0 = cta_off[blockIdx.x], t1 = cta_off[blockIdx.x + 1];
  volatile int* abort = &abort_flag;
  // an aborting role stops the roles of every CTA of the cluster
  auto abort_all = [&]() {
    *abort = 1;
    for (int j = 0; j < csize; ++j)
      if (j != rank)
        asm volatile("st.relaxed.cluster.shared::cluster.u32 [%0], %1;" ::"r"(map_to(smem_u32(&abort_flag), j)),
                     "r"(1)
                     : "memory");
    atomicExch(err, 1);
  };

  if (tid == 0) {
    for (int i = 0; i < NSTAGE; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[B_FULL + i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[B_EMPTY + i])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[B_XPF])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(smem_u32(&bar[B_XPE])));
    for (int i = 0; i < 2; ++i) {
      // XF: one arrival (the converters of the CTA that owns the piece, or,
      // for a piece from the peer, this CTA's converters expecting its bytes);
      // XE: the MMA issuers of all CTAs of the cluster
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[B_XF + i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar[B_XE + i])), "r"(csize));
      // XA: this CTA's converter threads, once they have seen the reads of
      // two pieces back complete
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(smem_u32(&bar[B_XA + i])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[B_SF])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(smem_u32(&bar[B_SE])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[B_DONE])));
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_flag = 0;
    consumed = 0;
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  // the barriers of every CTA of the cluster are initialised before any
  // arrival from a peer
  cluster_sync();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tS = tmem_base + TCOL_S, tX = tmem_base + TCOL_X;
  int produced = 0;  // stage fills issued (producer lane)

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map32)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map64)) : "memory");
      int q = 0;
      bool ok = true;
      auto acquire = [&](int& s) -> bool {
        s = q % NSTAGE;
        return wait_bar(&bar[B_EMPTY + s], (uint32_t)(((q / NSTAGE) & 1) ^ 1), abort, wait_ns);
      };
      // k-blocks [k0, k1) of stage 1 of the super-chunk at w: per k-block of 16
      // of ka, the A tile (the tile's rows) and the P^T tile (256 rows from the
      // super-chunk's first)
      auto s1 = [&](const Walk& w, int k0, int k1) -> bool {
        for (int kk = k0; kk < k1; ++kk) {
          int s;
          if (!acquire(s)) return false;
          const uint32_t st = sbase + OFF_STAGE + s * STAGE;
          const int x = (kk & 1) * 128, kb32 = kk >> 1;
          arrive_expect(&bar[B_FULL + s], A_BYTES + P_BYTES);
          tma_load(st, &map32, x, w.it.A.unit + (kb32 * w.it.A.groups + (w.tk.r0 >> 3)) * 2, &bar[B_FULL + s]);
          tma_load(st + A_BYTES, &map64, x, w.it.Pt.unit + (kb32 * w.it.Pt.groups + (w.jc >> 3)) * 2,
                   &bar[B_FULL + s]);
          ++q;
        }
        return true;
      };
      // stage 2 of the piece at w: per k-block of 16 of the piece, the B tile
      // (the tile's columns, 256 rows)
      auto s2 = [&](const Walk& w) -> bool {
        const int nk = s2_kblocks(w);
        const int k16 = (w.jc + PW * w.p) >> 4;
        for (int kk = 0; kk < nk; ++kk) {
          int s;
          if (!acquire(s)) return false;
          const uint32_t st = sbase + OFF_STAGE + s * STAGE;
          const int kq = k16 + kk;
          arrive_expect(&bar[B_FULL + s], B_BYTES);
          tma_load(st, &map64, (kq & 1) * 128, w.it.B.unit + ((kq >> 1) * w.it.B.groups + (w.tk.c0 >> 3)) * 2,
                   &bar[B_FULL + s]);
          ++q;
        }
        return true;
      };
      // the fill order of the MMA issuer: stage 1 in the order of s1_now,
      // stage 2 of every piece of a tile
      Walk s2w;
      walk_start(s2w, blocks, items, tasks, cta_task, t0, t1, drain_terms, tile_n, rank);
      S1Order o;
      s1_order_start(o, s2w);
      while (ok && s2w.valid) {
        const int k = s1_now(o, s2w);
        if (k > 0) {
          if (!(ok = s1(o.w, o.done, o.done + k))) break;
          s1_issued(o, s2w, k);
        }
        if (!ghost(s2w) && !(ok = s2(s2w))) break;
        walk_next(s2w);
      }
      if (!ok) abort_all();
      produced = q;
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int q = 0, nd = 0, nsc = 0, g = 0;  // stage fills consumed, drains, super-chunks issued, pieces issued
      int xfu0 = 0, xfu1 = 0;             // pieces received in buffers 0 and 1
      bool need_se = false, fresh = true, ok = true;
      auto take = [&](int& s) -> bool {
        s = q % NSTAGE;
        if (!wait_bar(&bar[B_FULL + s], (uint32_t)((q / NSTAGE) & 1), abort, wait_ns)) return false;
        asm volatile("tcgen05.fence::after_thread_sync;");
        return true;
      };
      // k-blocks [k0, k1) of stage 1 of the super-chunk at w
      auto s1 = [&](const Walk& w, int k0, int k1) -> bool {
        // X' must have been read by the converters (every piece of this CTA's last super-chunk)
        if (k0 == 0 && nsc >= 1 && !wait_bar(&bar[B_XPE], (uint32_t)((nsc - 1) & 1), abort, wait_ns)) return false;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t id = idesc_tf32(TM, (sc_width(w) + 15) & ~15);
        const int nb = s1_blocks(w);
        for (int kk = k0; kk < k1; ++kk) {
          int s;
          if (!take(s)) return false;
          const uint32_t st = sbase + OFF_STAGE + s * STAGE;
          // descriptors of the stage; a k-step of 8 moves the start address by
          // 256 B (16 in the address field, which stays inside its 14 bits)
          const uint64_t ah0 = desc(st, SBO_OP), al0 = desc(st + LO_OP, SBO_OP);
          const uint64_t ph0 = desc(st + A_BYTES, SBO_OP), pl0 = desc(st + A_BYTES + LO_OP, SBO_OP);
#pragma unroll
          for (int k8 = 0; k8 < 2; ++k8) {
            const uint64_t ko = (uint64_t)(k8 * 2 * LBO) >> 4;
            mma_tf32(tX, al0 + ko, ph0 + ko, id, (kk > 0 || k8 > 0) ? 1u : 0u);
            mma_tf32(tX, ah0 + ko, pl0 + ko, id, 1u);
            mma_tf32(tX, ah0 + ko, ph0 + ko, id, 1u);
          }
          commit(&bar[B_EMPTY + s]);
          ++q;
        }
        if (k1 == nb) {
          commit(&bar[B_XPF]);
          ++nsc;
        }
        return true;
      };
      auto s2 = [&](const Walk& w) -> bool {
        const int b = g & 1;
        // the converters have seen piece g - 2 read everywhere, and the piece is
        // in this CTA's buffer b (written by whichever CTA of the group owns it)
        if (!wait_bar(&bar[B_XA + b], (uint32_t)((g >> 1) & 1), abort, wait_ns)) return false;
        int& xfu = b ? xfu1 : xfu0;
        if (!wait_bar<true>(&bar[B_XF + b], (uint32_t)(xfu & 1), abort, wait_ns)) return false;
        ++xfu;
        if (need_se) {
          if (!wait_bar(&bar[B_SE], (uint32_t)((nd - 1) & 1), abort, wait_ns)) return false;
          need_se = false;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t id = idesc_tf32(TM, w.N);
        const uint32_t xh = sbase + OFF_X + b * XBUF, xl = xh + XLO;
        const int nk = s2_kblocks(w);
        for (int kk = 0; kk < nk; ++kk) {
          int s;
          if (!take(s)) return false;
          const uint32_t st = sbase + OFF_STAGE + s * STAGE;
          const uint32_t xo = (uint32_t)kk * 4 * LBO;
          const uint64_t xh0 = desc(xh + xo, SBO_X), xl0 = desc(xl + xo, SBO_X);
          const uint64_t bh0 = desc(st, SBO_OP), bl0 = desc(st + LO_OP, SBO_OP);
#pragma unroll
          for (int k8 = 0; k8 < 2; ++k8) {
            const uint64_t ko = (uint64_t)(k8 * 2 * LBO) >> 4;
            mma_tf32(tS, xl0 + ko, bh0 + ko, id, fresh ? 0u : 1u);
            fresh = false;
            mma_tf32(tS, xh0 + ko, bl0 + ko, id, 1u);
            mma_tf32(tS, xh0 + ko, bh0 + ko, id, 1u);
          }
          commit(&bar[B_EMPTY + s]);
          ++q;
        }
        // buffer b of every CTA may be rewritten once all of them have read it
        commit_all(&bar[B_XE + b], cmask);
        ++g;
        if (drain_point(w)) {
          commit(&bar[B_SF]);
          ++nd;
          need_se = true;
          fresh = true;
        }
        return true;
      };
      // a ghost entry computes nothing but keeps the cluster's count of the
      // reads of every piece buffer: one arrival per piece, each once this
      // CTA's converters have seen the previous use of the buffer complete
      // (so that no phase takes two)
      auto ghost_piece = [&]() -> bool {
        const int b = g & 1;
        if (!wait_bar(&bar[B_XA + b], (uint32_t)((g >> 1) & 1), abort, wait_ns)) return false;
        commit_all(&bar[B_XE + b], cmask);
        ++g;
        return true;
      };
      Walk s2w;
      walk_start(s2w, blocks, items, tasks, cta_task, t0, t1, drain_terms, tile_n, rank);
      S1Order o;
      s1_order_start(o, s2w);
      while (ok && s2w.valid) {
        const int k = s1_now(o, s2w);
        if (k > 0) {
          if (!(ok = s1(o.w, o.done, o.done + k))) break;
          s1_issued(o, s2w, k);
        }
        if (!(ok = ghost(s2w) ? ghost_piece() : s2(s2w))) break;
        walk_next(s2w);
      }
      if (!ok) abort_all();
      consumed = q;
      // every MMA issued by this thread has completed once B_DONE fires
      // (waited for also after an abort, bounded)
      commit(&bar[B_DONE]);
      const unsigned long long t0w = global_ns();
      while (!test_wait<false>(&bar[B_DONE], 0u) && global_ns() - t0w < kWaitNs) __nanosleep(64);
    }
  } else {
    // ------------------------------------------------------------ converters
    const int quarter = warp & 3;
    const int r = quarter * 32 + lane;  // TMEM lane = tile row
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    float2* const part_base = reinterpret_cast<float2*>(scratch);
    int nd = 0, nsc = 0, g = 0;  // drains done, super-chunks converted, pieces walked
    bool ok = true;
    // the piece at w (this CTA's stage 1) into buffer g & 1 of every CTA of the group
    auto convert = [&](const Walk& w) -> bool {
      if (w.p == 0) {
        // X' of this super-chunk complete
        if (!wait_bar_warp(&bar[B_XPF], (uint32_t)(nsc & 1), abort, wait_ns)) return false;
        asm volatile("tcgen05.fence::after_thread_sync;");
      }
      uint32_t q[32];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3]), "=r"(q[4]), "=r"(q[5]), "=r"(q[6]), "=r"(q[7]),
            "=r"(q[8]), "=r"(q[9]), "=r"(q[10]), "=r"(q[11]), "=r"(q[12]), "=r"(q[13]), "=r"(q[14]), "=r"(q[15]),
            "=r"(q[16]), "=r"(q[17]), "=r"(q[18]), "=r"(q[19]), "=r"(q[20]), "=r"(q[21]), "=r"(q[22]), "=r"(q[23]),
            "=r"(q[24]), "=r"(q[25]), "=r"(q[26]), "=r"(q[27]), "=r"(q[28]), "=r"(q[29]), "=r"(q[30]), "=r"(q[31])
          : "r"(tX + lane_base + (uint32_t)(PW * w.p)));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (last_piece(w)) {
        // every piece of the super-chunk is read: X' may be overwritten
        asm volatile("tcgen05.fence::before_thread_sync;");
        arrive(&bar[B_XPE]);
        ++nsc;
      }
      const int b = g & 1;
      const float al = (float)w.it.alpha;
      unsigned char* const xl = sgen + OFF_X + b * XBUF;
#pragma unroll
      for (int j = 0; j < PW; j += 4) {
        float4 hv, lv;
        const float x0 = al * __uint_as_float(q[j]), x1 = al * __uint_as_float(q[j + 1]);
        const float x2 = al * __uint_as_float(q[j + 2]), x3 = al * __uint_as_float(q[j + 3]);
        hv.x = __uint_as_float(tf32(x0));
        hv.y = __uint_as_float(tf32(x1));
        hv.z = __uint_as_float(tf32(x2));
        hv.w = __uint_as_float(tf32(x3));
        lv.x = __uint_as_float(tf32(x0 - hv.x));
        lv.y = __uint_as_float(tf32(x1 - hv.y));
        lv.z = __uint_as_float(tf32(x2 - hv.z));
        lv.w = __uint_as_float(tf32(x3 - hv.w));
        const uint32_t o = x_off(r, j);
        *reinterpret_cast<float4*>(xl + o) = hv;
        *reinterpret_cast<float4*>(xl + XLO + o) = lv;
      }
      // the writes are seen by the async proxy (this CTA's tensor core and the
      // bulk copy to the group's other CTA, if any)
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (tid == 64) {
        // one copy into every other CTA of the group
        const uint32_t xb = sbase + OFF_X + b * XBUF;
        for (int peer = w.sl.grp0; peer < w.sl.grp0 + w.sl.grpn; ++peer)
          if (peer != rank)
            copy_to_peer(map_to(xb, (uint32_t)peer), xb, XBUF, map_to(smem_u32(&bar[B_XF + b]), (uint32_t)peer));
        arrive(&bar[B_XF + b]);
      }
      return true;
    };
    // S (FP32, TMEM) is added to the task's partial tile of float pairs (hi,
    // lo), stored column by column (element (r, c) at c * 128 + r, so a warp's
    // lanes touch consecutive pairs), by a TwoSum (Knuth) on the FP32 pipe;
    // the first drain of a task stores.  N columns are written; the reduction
    // reads the valid rows and columns only.
    auto drain = [&](long long part, int N, bool first) -> bool {
      if (!wait_bar_warp(&bar[B_SF], (uint32_t)(nd & 1), abort, wait_ns)) return false;
      asm volatile("tcgen05.fence::after_thread_sync;");
      float2* d = part_base + part + r;
      for (int c0 = 0; c0 < N; c0 += 32) {
        // N is a multiple of 16: the chunk has 16 or 32 valid columns.  The
        // partials of the chunk are all loaded before they are used, so their
        // latencies overlap (and overlap the TMEM load).
        const bool two = N - c0 > 16;
        float2 a[32];
        if (!first) {
#pragma unroll
          for (int j = 0; j < 16; ++j) a[j] = d[(size_t)(c0 + j) * TM];
          if (two) {
#pragma unroll
            for (int j = 16; j < 32; ++j) a[j] = d[(size_t)(c0 + j) * TM];
          }
        }
        uint32_t v[32];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
              "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
              "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
              "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
            : "r"(tS + lane_base + (uint32_t)c0));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        auto put = [&](int j) {
          const float x = __uint_as_float(v[j]);
          if (first) {
            d[(size_t)(c0 + j) * TM] = make_float2(x, 0.0f);
          } else {
            const float sum = __fadd_rn(a[j].x, x);
            const float bv = __fsub_rn(sum, a[j].x);
            const float e = __fadd_rn(__fsub_rn(a[j].x, __fsub_rn(sum, bv)), __fsub_rn(x, bv));
            d[(size_t)(c0 + j) * TM] = make_float2(sum, __fadd_rn(a[j].y, e));
          }
        };
#pragma unroll
        for (int j = 0; j < 16; ++j) put(j);
        if (two) {
#pragma unroll
          for (int j = 16; j < 32; ++j) put(j);
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      arrive(&bar[B_SE]);
      ++nd;
      return true;
    };
    Walk w;
    walk_start(w, blocks, items, tasks, cta_task, t0, t1, drain_terms, tile_n, rank);
    int drains_in_task = 0, last_t = -1;
    bool pend = false, pend_first = false;
    long long pend_part = 0;
    int pend_N = 0;
    while (ok && w.valid) {
      if (w.t != last_t) {
        last_t = w.t;
        drains_in_task = 0;
      }
      // every CTA's MMAs have read piece g - 2 (buffer g & 1 is free in the
      // whole cluster); waited for at every piece, in order, and acknowledged
      // to this CTA's MMA issuer, which waits for the acknowledgement before
      // its own reads of piece g: so no converter is two phases behind when
      // it waits
      const int b = g & 1;
      if (g >= 2 && !(ok = wait_bar_warp<true>(&bar[B_XE + b], (uint32_t)(((g >> 1) - 1) & 1), abort, wait_ns)))
        break;
      arrive(&bar[B_XA + b]);
      if (owned(w)) {
        if (!(ok = convert(w))) break;
      } else if (!ghost(w) && w.sl.grpn > 1 && tid == 64) {
        // the piece comes from the CTA of the group that owns it: its bytes complete the phase
        arrive_expect(&bar[B_XF + b], XBUF);
      }
      if (pend && !(ok = drain(pend_part, pend_N, pend_first))) break;
      pend = !ghost(w) && drain_point(w);
      if (pend) {
        pend_part = w.tk.part;
        pend_N = w.N;
        pend_first = drains_in_task == 0;
        ++drains_in_task;
      }
      ++g;
      walk_next(w);
    }
    if (ok && pend) ok = drain(pend_part, pend_N, pend_first);
    if (!ok) {
      *abort = 1;
      if (lane == 0) abort_all();
    }
  }
  __syncthreads();
  if (warp == 0 && lane == 0 && *abort) {
    // copies still in flight land before the CTA exits
    for (int q = consumed; q < produced; ++q) {
      uint32_t par = (uint32_t)((q / NSTAGE) & 1);
      const unsigned long long t0w = global_ns();
      while (!test_wait<false>(&bar[B_FULL + q % NSTAGE], par) && global_ns() - t0w < kWaitNs) __nanosleep(64);
    }
  }
  if (*abort) {
    // after an abort a bulk copy from the peer may still be in flight into
    // this CTA's piece buffers: give it time to land before the cluster exits
    const unsigned long long t0w = global_ns();
    while (global_ns() - t0w < kDrainCopiesNs) __nanosleep(1000);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(512));
  // no CTA leaves while a peer may still write into its shared memory or
  // arrive on its barriers
  cluster_sync();
}

// partial tiles are TM x TNMAX float pairs stored column by column (element
// (r, c) at c * TM + r); CTA (tile, y) sums columns [32 y, 32 y + 32) of a
// tile over its chunks in fixed order, thread t taking row t % 128 of every
// second column
__global__ void hpsi_tc_reduce(const HpsiBlock* __restrict__ blocks, const HpsiReduce* __restrict__ reds,
                               const double* __restrict__ scratch, int tile_n) {
  const HpsiReduce rd = reds[blockIdx.x];
  const HpsiBlock bk = blocks[rd.block];
  const int nvalid = min(tile_n, bk.n - rd.c0);
  const int r = threadIdx.x & (TM - 1), gr = rd.r0 + r;
  if (gr >= bk.m) return;
  const int cend = min(nvalid, (int)blockIdx.y * 32 + 32);
  for (int c = blockIdx.y * 32 + (int)(threadIdx.x >> 7); c < cend; c += 2) {
    const float2* part = reinterpret_cast<const float2*>(scratch + rd.part0) + (size_t)c * TM + r;
    double acc = 0.0;
    for (int p = 0; p < rd.nparts; ++p) {
      const float2 v = part[(long long)p * TM * TNMAX];
      acc += (double)v.x + (double)v.y;
    }
    bk.C[(size_t)gr * bk.ldc + rd.c0 + c] += acc;
  }
}

// unit pairs of job j: pair p = kblock * G + g holds hi (unit 2p) and lo
// (unit 2p + 1) of rows [8g, 8g + 8) x cols [32 kblock, 32 kblock + 32)
__global__ void split_kernel(const SplitJob* __restrict__ jobs, int n, float* __restrict__ pool) {
  for (int j = blockIdx.x; j < n; j += gridDim.x) {
    const SplitJob jb = jobs[j];
    const int G = (jb.rows + 7) >> 3;
    const size_t pairs = (size_t)G * ((jb.cols + 31) >> 5);
    float* const base = pool + (size_t)jb.unit * kTcUnitFloats;
    for (size_t e = threadIdx.x; e < pairs * kTcUnitFloats; e += blockDim.x) {
      const size_t pr = e / kTcUnitFloats;
      const int w = (int)(e % kTcUnitFloats);
      const int kbk = (int)(pr / G), g = (int)(pr % G);
      const int r = 8 * g + ((w >> 2) & 7);
      const int k = 32 * kbk + 4 * (w >> 5) + (w & 3);
      double v = 0.0;
      if (r < jb.rows && k < jb.cols) {
        if (jb.src == nullptr) v = (r == k) ? 1.0 : 0.0;
        else v = jb.trans ? jb.src[(size_t)k * jb.ld + r] : jb.src[(size_t)r * jb.ld + k];
      }
      const float h = __uint_as_float(tf32((float)v));
      float* u = base + pr * 2 * kTcUnitFloats;
      u[w] = h;
      u[kTcUnitFloats + w] = __uint_as_float(tf32((float)(v - (double)h)));
    }
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// 2D map over the pool: 256 floats (one unit) per row; a box is 128 floats
// (half a unit: one k-block of 16) by `rows` units
void make_map(CUtensorMap* m, const void* pool, size_t units, int rows) {
  auto fn = encode_fn();
  if (!fn) throw std::runtime_error("cuda: cuTensorMapEncodeTiled is not available");
  cuuint64_t dims[2] = {(cuuint64_t)kTcUnitFloats, (cuuint64_t)units};
  cuuint64_t strides[1] = {(cuuint64_t)kTcUnitFloats * sizeof(float)};
  cuuint32_t box[2] = {(cuuint32_t)(kTcUnitFloats / 2), (cuuint32_t)rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(pool), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw std::runtime_error("cuda: tensor map encoding failed (" + std::to_string((int)r) + ")");
}

}  // namespace

void split_launch(const SplitJob* jobs, int n, float* pool, cudaStream_t st) {
  if (n <= 0) return;
  split_kernel<<<std::min(n, 152 * 8), 256, 0, st>>>(jobs, n, pool);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw std::runtime_error(std::string("cuda: split launch: ") + cudaGetErrorString(e));
}

namespace {
// launch of whole clusters of `cluster` CTAs along x
void launch_config(cudaLaunchConfig_t& cfg, cudaLaunchAttribute* attr, int ncta, cudaStream_t st, int cluster) {
  cfg.gridDim = dim3((unsigned)ncta, 1, 1);
  cfg.blockDim = dim3(NTHREADS, 1, 1);
  cfg.dynamicSmemBytes = SMEM_BYTES;
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
}
}  // namespace

int hpsi_tc_max_ctas(int cluster) {
  static std::mutex mu;
  static int cached[64][kTcClusterMax + 1];
  static bool have[64][kTcClusterMax + 1];
  int dev = 0;
  if (cluster < 1 || cluster > kTcClusterMax) return 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  std::lock_guard<std::mutex> lk(mu);
  if (!have[dev][cluster]) {
    int n = 0;
    if (ensure_smem_attr((const void*)hpsi_tc_kernel, SMEM_BYTES) == cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute attr[1];
      launch_config(cfg, attr, cluster, nullptr, cluster);
      if (cudaOccupancyMaxActiveClusters(&n, (const void*)hpsi_tc_kernel, &cfg) != cudaSuccess) n = 0;
    }
    cudaGetLastError();
    cached[dev][cluster] = n * cluster;
    have[dev][cluster] = true;
  }
  return cached[dev][cluster];
}

void hpsi_tc_launch(const TcLaunch& L, int* err, unsigned long long wait_ns, cudaStream_t st) {
  {
    cudaError_t e = ensure_smem_attr((const void*)hpsi_tc_kernel, SMEM_BYTES);
    if (e != cudaSuccess) throw std::runtime_error(std::string("cuda: hpsi tc attribute: ") + cudaGetErrorString(e));
  }
  if (L.tile_n < 16 || L.tile_n > TNMAX || L.tile_n % 16)
    throw std::runtime_error("internal: tcgen05 tile width not a multiple of 16 in [16, 256]");
  if (L.ncta > 0) {
    if (!L.pool || L.units == 0) throw std::runtime_error("internal: tcgen05 contraction without a split pool");
    if (((uintptr_t)L.pool & 15) != 0) throw std::runtime_error("internal: split pool not 16-byte aligned");
    CUtensorMap m32, m64;
    make_map(&m32, L.pool, L.units, 32);
    make_map(&m64, L.pool, L.units, 64);
    if (L.cluster < 1 || L.cluster > kTcClusterMax || L.ncta % L.cluster)
      throw std::runtime_error("internal: tcgen05 launch not in whole clusters");
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    launch_config(cfg, attr, L.ncta, st, L.cluster);
    cudaError_t e = cudaLaunchKernelEx(&cfg, hpsi_tc_kernel, m32, m64, L.blocks, L.items, L.tasks, L.cta_off,
                                       L.cta_task, L.scratch, err, wait_ns, L.drain_terms, L.tile_n, L.cluster);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) throw std::runtime_error(std::string("cuda: hpsi tc launch: ") + cudaGetErrorString(e));
  }
  if (L.nreds > 0) {
    hpsi_tc_reduce<<<dim3(L.nreds, (L.tile_n + 31) / 32), 256, 0, st>>>(L.blocks, L.reds, L.scratch, L.tile_n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw std::runtime_error(std::string("cuda: hpsi tc reduce: ") + cudaGetErrorString(e));
  }
}

}  // namespace dmrg
