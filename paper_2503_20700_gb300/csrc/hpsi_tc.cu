// tcgen05 fused H_eff psi contraction (see hpsi_tc.cuh).
//
// Shared memory (bytes): X hi/lo planes (2 x 32 KB, 128 x 64, K-major) and
// three 48 KB slots, each holding the operand tiles of one k-block of 32:
//   stage 1: A hi | A lo (128 x 32 each, 16 KB) | P^T hi | P^T lo (64 x 32, 8 KB)
//   stage 2: B hi | B lo (up to 128 x 32 each, 16 KB): one column half of
//            the sigma tile (columns [0, 128) or [128, N))
// all in the canonical no-swizzle K-major layout (8-row x 16-byte core
// matrices; 128 B between K-adjacent cores, 1 KB between 8-row groups for
// 32-wide tiles, 2 KB for the 64-wide X).  TMEM: S in columns [0, 256), X' in
// [256, 320).  The k-blocks of a task form one sequence: the MMAs of block b
// are issued once its copies have landed (blocks b and b+1 are in flight),
// then the copies of block b+2 refill the slot of block b-1 after its MMAs
// completed.  Each slot has its own mbarrier (tcgen05.commit after the
// block's MMAs) and every wait is bounded by 2 s of wall clock.  The FP32
// accumulator S is drained into the task's partial tile of float pairs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <stdexcept>
#include <string>

#include "hpsi_tc.cuh"
#include "kattr.hpp"

namespace dmrg {

namespace {

constexpr int TM = kTcTileM, TNMAX = kTcTileN, KB = 32, JC = 64;
constexpr uint32_t LBO = 128;
constexpr uint32_t SBO32 = 1024;  // 8-row group stride of a 32-wide tile
constexpr uint32_t SBO64 = 2048;  // of the 64-wide X tile
constexpr int NSLOT = 3;
constexpr int OFF_XH = 0, OFF_XL = 32768, OFF_SLOT = 65536, SLOT = 49152;
constexpr int SMEM_BYTES = OFF_SLOT + NSLOT * SLOT;  // 208 KB
constexpr int HALF = 128;  // column half of the sigma tile per stage-2 block
constexpr int kDrainItems = 4;  // items accumulated in FP32 before a float64 drain
constexpr uint32_t TCOL_S = 0, TCOL_X = 256;
constexpr unsigned long long kWaitNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ int roundup32(int x) { return (x + 31) & ~31; }

__device__ __forceinline__ uint64_t desc(uint32_t saddr, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((LBO >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
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
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar)));
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity) {
  // a short spin first (the MMAs of a k-block take about a microsecond), then
  // probes with a sleep between them, bounded by kWaitNs of wall clock
  for (int i = 0; i < 128; ++i) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity));
    if (done) return true;
  }
  const unsigned long long t0 = global_ns();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity));
    if (done) return true;
    if (global_ns() - t0 > kWaitNs) return false;
    __nanosleep(64);
  }
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}
// 16-byte async copy; src_bytes = 0 fills the destination with zeros
__device__ __forceinline__ void cp16(uint32_t dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes));
}
// byte offset of element (r, k) (k multiple of 4) in a K-major tile with 8-row group stride sbo
__device__ __forceinline__ uint32_t core_off(int r, int k, uint32_t sbo) {
  return (uint32_t)(r >> 3) * sbo + (uint32_t)(k >> 2) * LBO + (uint32_t)(r & 7) * 16;
}
__device__ __forceinline__ uint32_t word_off(int r, int k, uint32_t sbo) {
  return core_off(r, k & ~3, sbo) + (uint32_t)(k & 3) * 4;
}

// copies rows [row0, min(row0 + nrows, rmax)) x cols [k0, k0 + 32) of a
// split matrix into a K-major tile (both planes).  A thread keeps one 16-byte
// column chunk and steps 16 rows at a time.  Tile rows at or beyond rmax are
// not copied and keep earlier slot contents (zero at kernel start, later
// finite operand values): rows of A or B there only reach output rows or
// columns outside the block, which are never stored, and rows of P^T beyond
// kb only reach columns of X that meet the zero padding of B's planes (or
// zeros of a generated identity tile).
__device__ __forceinline__ void load_tile(uint32_t dhi, uint32_t dlo, const TcMat& m, int row0, int nrows, int rmax,
                                          int k0, int tid) {
  const int rows = min(nrows, rmax - row0);
  const int kc = (tid & 7) * 4;
  int r = tid >> 3;
  if (r >= rows) return;
  const size_t step = (size_t)16 * m.ld;
  size_t off = (size_t)(row0 + r) * m.ld + k0 + kc;
  uint32_t o = core_off(r, kc, SBO32);
  for (; r < rows; r += 16) {  // 16 rows = two 8-row core-matrix groups
    cp16(dhi + o, m.hi + off, 16);
    cp16(dlo + o, m.lo + off, 16);
    off += step;
    o += 2 * SBO32;
  }
}

struct Cursor {
  int ii, jc, jc_end, stage, k0, half;
};

__device__ __forceinline__ void cursor_item(Cursor& c, const TcItem& it, int c0, int N) {
  c.jc = 0;
  c.jc_end = it.kb;
  if (it.B.hi == nullptr) {
    c.jc = c0;
    c.jc_end = min(it.kb, c0 + N);
  }
  c.stage = it.A.hi ? 1 : 2;
  c.k0 = 0;
  c.half = 0;
}
__device__ __forceinline__ int chunk_kspan(const Cursor& c) { return min(JC, roundup32(c.jc_end - c.jc)); }
// advance to the next k-block; false at the end of the task
// `it` is the cursor's current item (kept in registers): reloaded from the
// item list only when the cursor moves to the next item
__device__ __forceinline__ bool cursor_next(Cursor& c, TcItem& it, const TcItem* __restrict__ items, int it_end,
                                            int c0, int N) {
  if (c.stage == 1) {
    c.k0 += KB;
    if (c.k0 < roundup32(it.ka)) return true;
    c.stage = 2;
    c.k0 = 0;
    return true;
  }
  if (c.half == 0 && N > HALF) {
    c.half = 1;
    return true;
  }
  c.half = 0;
  c.k0 += KB;
  if (c.k0 < chunk_kspan(c)) return true;
  c.jc += JC;
  if (c.jc < c.jc_end) {
    c.stage = it.A.hi ? 1 : 2;
    c.k0 = 0;
    return true;
  }
  if (++c.ii >= it_end) return false;
  it = items[c.ii];
  cursor_item(c, it, c0, N);
  return true;
}

__global__ void __launch_bounds__(128, 1)
    hpsi_tc_kernel(const HpsiBlock* __restrict__ blocks, const TcItem* __restrict__ items,
                   const HpsiTask* __restrict__ tasks, double* __restrict__ scratch, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  __shared__ __align__(8) uint64_t bar[NSLOT];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5;
  const HpsiTask tk = tasks[blockIdx.x];
  const HpsiBlock bk = blocks[tk.block];
  const int nvalid = min(TNMAX, bk.n - tk.c0);
  const int N = (nvalid + 15) & ~15;  // MMA N: multiple of 16
  const int it_end = tk.it_begin + tk.it_count;
  const uint32_t sbase = smem_u32(smraw);
  const uint32_t xh = sbase + OFF_XH, xl = sbase + OFF_XL;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // slots start at zero: tile rows that are never copied hold finite values
  for (int e = tid; e < NSLOT * SLOT / 16; e += 128)
    reinterpret_cast<uint4*>(smraw + OFF_SLOT)[e] = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) {
    for (int i = 0; i < NSLOT; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[i])));
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_flag = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tS = tmem_base + TCOL_S, tX = tmem_base + TCOL_X;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  const int N1 = min(N, HALF), N2 = N - N1;  // MMA widths of the two column halves
  const uint32_t id1 = idesc_tf32(TM, JC), id2a = idesc_tf32(TM, N1), id2b = idesc_tf32(TM, N2 > 0 ? N2 : 16);

  // issue the operand copies of the block at cursor c (item it) into slot s
  auto produce = [&](const Cursor& c, const TcItem& it, int s) {
    const uint32_t sl = sbase + OFF_SLOT + s * SLOT;
    if (c.stage == 1) {
      load_tile(sl, sl + 16384, it.A, tk.r0, TM, bk.m, c.k0, tid);
      load_tile(sl + 32768, sl + 40960, it.Pt, c.jc, JC, it.kb, c.k0, tid);
    } else if (it.B.hi != nullptr) {
      load_tile(sl, sl + 16384, it.B, tk.c0 + c.half * HALF, c.half ? N2 : N1, bk.n, c.jc + c.k0, tid);
    } else {
      // identity on the right: B(n, k) = [c0 + n == jc + k0 + k]
      float* bh = (float*)(smraw + OFF_SLOT + s * SLOT);
      float* bl = (float*)(smraw + OFF_SLOT + s * SLOT + 16384);
      const int n0 = c.half * HALF, nn = c.half ? N2 : N1;
      for (int e = tid; e < nn * KB; e += 128) {
        int n = e / KB, k = e % KB;
        bool one = (tk.c0 + n0 + n == c.jc + c.k0 + k) && (tk.c0 + n0 + n < bk.n);
        uint32_t o = word_off(n, k, SBO32) >> 2;
        bh[o] = one ? 1.0f : 0.0f;
        bl[o] = 0.0f;
      }
    }
    asm volatile("cp.async.commit_group;");
  };
  // bounded wait on the commit of block b; failure sets the abort flag
  auto wait_block = [&](int b) {
    if (b < 0) return;
    if (!wait_bar(&bar[b % NSLOT], (uint32_t)((b / NSLOT) & 1))) abort_flag = 1;
  };

  // S (FP32, TMEM) is added to the task's partial tile every kDrainItems
  // items and at the end, so FP32 accumulation spans a few items only.
  // The first drain stores, later ones add.
  bool s_started = false, s_started_b = false;  // first / second column half written since the last drain
  bool drained = false;
  auto drain = [&]() {
    // the task's partial tile holds float pairs (hi, lo): a TwoSum (Knuth)
    // adds each FP32 value of S with its rounding error kept in lo, on the
    // FP32 pipe (the float64 conversion happens once, in the reduction)
    const int r = tid;
    float2* d = reinterpret_cast<float2*>(scratch + tk.part) + (size_t)r * TNMAX;
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      if (s_started) {
        tmem_ld16(tS + lane_base + c0, v);
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = 0.0f;
      }
      if (!drained) {
#pragma unroll
        for (int j = 0; j < 16; ++j) d[c0 + j] = make_float2(v[j], 0.0f);
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const float2 a = d[c0 + j];
          const float sum = __fadd_rn(a.x, v[j]);
          const float bv = __fsub_rn(sum, a.x);
          const float err = __fadd_rn(__fsub_rn(a.x, __fsub_rn(sum, bv)), __fsub_rn(v[j], bv));
          d[c0 + j] = make_float2(sum, __fadd_rn(a.y, err));
        }
      }
    }
    drained = true;
  };

  Cursor cur;
  cur.ii = tk.it_begin;
  TcItem it_cur = items[cur.ii];
  cursor_item(cur, it_cur, tk.c0, N);
  // blocks b+1 and b+2 (n1, n2) are prefetched ahead of block b
  Cursor n1 = cur, n2;
  TcItem it_n1 = it_cur, it_n2;
  bool has1 = cursor_next(n1, it_n1, items, it_end, tk.c0, N), has2 = false;
  n2 = n1;
  it_n2 = it_n1;
  if (has1) has2 = cursor_next(n2, it_n2, items, it_end, tk.c0, N);
  int b = 0;
  produce(cur, it_cur, 0);
  if (has1) produce(n1, it_n1, 1);
  for (;;) {
    // copies in flight: blocks b and b+1 (b+2 is issued after the MMAs of b)
    if (has1) {
      asm volatile("cp.async.wait_group 1;");
    } else {
      asm volatile("cp.async.wait_group 0;");
    }
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (abort_flag) break;
    const TcItem& it = it_cur;
    if (cur.stage == 2 && cur.k0 == 0 && cur.half == 0) {
      // X = alpha X' (or alpha P for an identity left operand) -> hi/lo planes;
      // the commit of block b-1 covers every earlier MMA (stage 1 of this
      // chunk, stage 2 of the previous one that read X)
      if (b >= 1) wait_block(b - 1);
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int r = tid;
      float* xhp = (float*)(smraw + OFF_XH);
      float* xlp = (float*)(smraw + OFF_XL);
      if (it.A.hi != nullptr) {
        // the four 16-column loads of the row are issued before one wait
        uint32_t q[64];
#pragma unroll
        for (int c4 = 0; c4 < 4; ++c4)
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
              : "=r"(q[16 * c4 + 0]), "=r"(q[16 * c4 + 1]), "=r"(q[16 * c4 + 2]), "=r"(q[16 * c4 + 3]),
                "=r"(q[16 * c4 + 4]), "=r"(q[16 * c4 + 5]), "=r"(q[16 * c4 + 6]), "=r"(q[16 * c4 + 7]),
                "=r"(q[16 * c4 + 8]), "=r"(q[16 * c4 + 9]), "=r"(q[16 * c4 + 10]), "=r"(q[16 * c4 + 11]),
                "=r"(q[16 * c4 + 12]), "=r"(q[16 * c4 + 13]), "=r"(q[16 * c4 + 14]), "=r"(q[16 * c4 + 15])
              : "r"(tX + lane_base + 16 * c4));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        const float al = (float)it.alpha;
#pragma unroll
        for (int j = 0; j < JC; ++j) {
          float x = al * __uint_as_float(q[j]);
          uint32_t h = tf32(x);
          uint32_t o = word_off(r, j, SBO64) >> 2;
          xhp[o] = __uint_as_float(h);
          xlp[o] = __uint_as_float(tf32(x - __uint_as_float(h)));
        }
      } else {
        const int gr = tk.r0 + r;
        for (int c = 0; c < JC; ++c) {
          int gc = cur.jc + c;
          double x = (gr < bk.m && gc < it.kb) ? it.alpha * it.P[(size_t)gr * it.ldp + gc] : 0.0;
          uint32_t h = tf32((float)x);
          uint32_t o = word_off(r, c, SBO64) >> 2;
          xhp[o] = __uint_as_float(h);
          xlp[o] = __uint_as_float(tf32((float)(x - (double)__uint_as_float(h))));
        }
      }
      asm volatile("fence.proxy.async.shared::cta;");
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;");
      if (abort_flag) break;
    }
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t sl = sbase + OFF_SLOT + (b % NSLOT) * SLOT;
      if (cur.stage == 1) {
#pragma unroll
        for (int s = 0; s < KB / 8; ++s) {
          const uint32_t ko = (uint32_t)s * 2 * LBO;
          uint64_t ah = desc(sl + ko, SBO32), al = desc(sl + 16384 + ko, SBO32);
          uint64_t ph = desc(sl + 32768 + ko, SBO32), pl = desc(sl + 40960 + ko, SBO32);
          mma_tf32(tX, al, ph, id1, (cur.k0 > 0 || s > 0) ? 1u : 0u);
          mma_tf32(tX, ah, pl, id1, 1u);
          mma_tf32(tX, ah, ph, id1, 1u);
        }
      } else {
        const uint32_t xo = (uint32_t)(cur.k0 / 4) * LBO;
        const uint32_t dS = tS + (uint32_t)(cur.half * HALF);
        const uint32_t id2 = cur.half ? id2b : id2a;
        // the first MMA into each column half overwrites it
        const bool fresh = cur.half == 0 ? !s_started : !s_started_b;
#pragma unroll
        for (int s = 0; s < KB / 8; ++s) {
          const uint32_t ko = (uint32_t)s * 2 * LBO;
          uint64_t ah = desc(xh + xo + ko, SBO64), al = desc(xl + xo + ko, SBO64);
          uint64_t bh = desc(sl + ko, SBO32), bl = desc(sl + 16384 + ko, SBO32);
          mma_tf32(dS, al, bh, id2, (!fresh || s > 0) ? 1u : 0u);
          mma_tf32(dS, ah, bl, id2, 1u);
          mma_tf32(dS, ah, bh, id2, 1u);
        }
      }
      commit(&bar[b % NSLOT]);
    }
    // uniform over the CTA
    if (cur.stage == 2) {
      if (cur.half == 0) s_started = true;
      else s_started_b = true;
    }
    // prefetch block b+2 into the slot of block b-1 once its MMAs are done;
    // the MMAs of b are already queued behind them
    if (has2) {
      wait_block(b - 1);
      produce(n2, it_n2, (b + 2) % NSLOT);
    }
    if (!has1) break;
    if (n1.ii != cur.ii && ((n1.ii - tk.it_begin) % kDrainItems) == 0 && s_started) {
      // item boundary: drain S once its MMAs are done, then let the next
      // stage-2 MMA overwrite it
      wait_block(b);
      asm volatile("tcgen05.fence::after_thread_sync;");
      __syncthreads();
      if (abort_flag) break;
      drain();
      s_started = s_started_b = false;
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
    }
    cur = n1;
    it_cur = it_n1;
    n1 = n2;
    it_n1 = it_n2;
    has1 = has2;
    if (has1) {
      has2 = cursor_next(n2, it_n2, items, it_end, tk.c0, N);
    } else {
      has2 = false;
    }
    ++b;
  }
  // wait for the last blocks (after an abort, whatever may be in flight)
  wait_block(b);
  wait_block(b - 1);
  wait_block(b - 2);
  asm volatile("cp.async.wait_group 0;");
  asm volatile("tcgen05.fence::after_thread_sync;");
  __syncthreads();
  if (abort_flag) {
    if (tid == 0) atomicExch(err, 1);
  } else if (s_started || !drained) {
    drain();
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(512));
}

// partial tiles are TM x TNMAX (row stride TNMAX)
__global__ void hpsi_tc_reduce(const HpsiBlock* __restrict__ blocks, const HpsiReduce* __restrict__ reds,
                               const double* __restrict__ scratch) {
  const HpsiReduce rd = reds[blockIdx.x];
  const HpsiBlock bk = blocks[rd.block];
  const int nvalid = min(TNMAX, bk.n - rd.c0);
  for (int e = threadIdx.x; e < TM * TNMAX; e += blockDim.x) {
    int r = e / TNMAX, c = e % TNMAX;
    int gr = rd.r0 + r;
    if (gr >= bk.m || c >= nvalid) continue;
    const float2* part = reinterpret_cast<const float2*>(scratch + rd.part0) + e;
    double acc = 0.0;
    for (int p = 0; p < rd.nparts; ++p) {
      const float2 v = part[(long long)p * TM * TNMAX];
      acc += (double)v.x + (double)v.y;
    }
    bk.C[(size_t)gr * bk.ldc + rd.c0 + c] += acc;
  }
}

__global__ void split_kernel(const SplitJob* __restrict__ jobs, int n) {
  for (int j = blockIdx.x; j < n; j += gridDim.x) {
    const SplitJob jb = jobs[j];
    const size_t total = (size_t)jb.rows * jb.ldd;
    for (size_t e = threadIdx.x; e < total; e += blockDim.x) {
      int r = (int)(e / jb.ldd), c = (int)(e % jb.ldd);
      double v = 0.0;
      if (c < jb.cols) v = jb.trans ? jb.src[(size_t)c * jb.ld + r] : jb.src[(size_t)r * jb.ld + c];
      float h = __uint_as_float(tf32((float)v));
      jb.hi[e] = h;
      jb.lo[e] = __uint_as_float(tf32((float)(v - (double)h)));
    }
  }
}

}  // namespace

void split_launch(const SplitJob* jobs, int n, cudaStream_t st) {
  if (n <= 0) return;
  split_kernel<<<std::min(n, 152 * 8), 256, 0, st>>>(jobs, n);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw std::runtime_error(std::string("cuda: split launch: ") + cudaGetErrorString(e));
}

void hpsi_tc_launch(const HpsiBlock* blocks, const TcItem* items, const HpsiTask* tasks, int ntasks,
                    const HpsiReduce* reds, int nreds, double* scratch, int* err, cudaStream_t st) {
  {
    cudaError_t e = ensure_smem_attr((const void*)hpsi_tc_kernel, SMEM_BYTES);
    if (e != cudaSuccess) throw std::runtime_error(std::string("cuda: hpsi tc attribute: ") + cudaGetErrorString(e));
  }
  if (ntasks > 0) {
    hpsi_tc_kernel<<<ntasks, 128, SMEM_BYTES, st>>>(blocks, items, tasks, scratch, err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw std::runtime_error(std::string("cuda: hpsi tc launch: ") + cudaGetErrorString(e));
  }
  if (nreds > 0) {
    hpsi_tc_reduce<<<nreds, 256, 0, st>>>(blocks, reds, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw std::runtime_error(std::string("cuda: hpsi tc reduce: ") + cudaGetErrorString(e));
  }
}

}  // namespace dmrg
