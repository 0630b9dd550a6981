// tcgen05 (5th-generation tensor core) version of the fused H_eff psi
// contraction of hpsi_fused.cuh for sm_103a, 3xTF32 split precision:
//
//   sigma(a', b') += sum_i alpha_i op(A_i) P_i op(B_i)^T
//
// One CTA (128 threads) owns a 128 x 64 tile of one sigma block and a chunk of
// its items.  Per item and per 64-wide column chunk of P:
//   stage 1  X (128 x 64, TMEM)  = alpha op(A) P(:, chunk)        [3 MMAs per k-step]
//   X: TMEM -> registers -> hi/lo TF32 -> shared memory (K-major)
//   stage 2  S (128 x 64, TMEM) += X op(B)(tile cols, chunk)^T     [3 MMAs per k-step]
// Operands are staged from float64 into the canonical no-swizzle K-major
// shared-memory layout (8-row x 16-byte core matrices), split into hi/lo
// TF32 planes; one elected thread issues tcgen05.mma and commits to an
// mbarrier.  S accumulates in FP32 in TMEM across the items of the chunk and
// is written as a float64 partial tile (reduced by hpsi_reduce) or added into
// sigma.  Every wait is bounded; a wait that runs out sets *err and the CTA
// skips the rest of its work, after a second bounded wait for the MMAs still
// in flight, and releases its TMEM columns.
#include <cuda_runtime.h>

#include <cstdint>
#include <stdexcept>
#include <string>

#include "hpsi_fused.cuh"

namespace dmrg {

namespace {

constexpr int TM = 128, TN = 64, KS = 32, JC = 64;
constexpr uint32_t LBO = 128;                 // bytes between K-adjacent core matrices
constexpr uint32_t SBO_K32 = (KS / 4) * 128;  // bytes between M-adjacent cores, K = 32 tiles
constexpr uint32_t SBO_K64 = (JC / 4) * 128;  // same for the X tile (K = 64)
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s of wall clock per wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t desc(uint32_t saddr, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((LBO >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // sm_100-family descriptor version; no swizzle
  return d;
}

__device__ __forceinline__ uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// word offset of element (r, k) in a canonical K-major tile with K-extent kext
__device__ __forceinline__ int koff(int r, int k, int kext) {
  return (r >> 3) * (kext * 8) + (k >> 2) * 32 + (r & 7) * 4 + (k & 3);
}

__device__ __forceinline__ uint32_t tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void split64(double x, uint32_t& hi, uint32_t& lo) {
  hi = tf32((float)x);
  lo = tf32((float)(x - (double)__uint_as_float(hi)));
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

// wait for the completion of phase `parity` of the mbarrier, bounded by
// kWaitNs of wall clock (non-blocking probes with a short sleep between them)
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity) {
  const unsigned long long t0 = global_ns();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity));
    if (done) return true;
    if (global_ns() - t0 > kWaitNs) return false;
    __nanosleep(32);
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

__device__ __forceinline__ double ldA(const HpsiItem& it, int r, int c) {
  if (it.A == nullptr) return r == c ? 1.0 : 0.0;
  return it.transA ? it.A[(size_t)c * it.lda + r] : it.A[(size_t)r * it.lda + c];
}
__device__ __forceinline__ double ldB(const HpsiItem& it, int n, int k) {
  if (it.B == nullptr) return n == k ? 1.0 : 0.0;
  return it.transB ? it.B[(size_t)k * it.ldb + n] : it.B[(size_t)n * it.ldb + k];
}

// shared memory (bytes)
constexpr int SZ_A = TM * KS * 4;   // 16 KB per plane
constexpr int SZ_P = JC * KS * 4;   //  8 KB
constexpr int SZ_X = TM * JC * 4;   // 32 KB
constexpr int SZ_B = TN * KS * 4;   //  8 KB
constexpr int OFF_AH = 0, OFF_AL = OFF_AH + SZ_A, OFF_PH = OFF_AL + SZ_A, OFF_PL = OFF_PH + SZ_P;
constexpr int OFF_XH = OFF_PL + SZ_P, OFF_XL = OFF_XH + SZ_X, OFF_BH = OFF_XL + SZ_X, OFF_BL = OFF_BH + SZ_B;
constexpr int SMEM_BYTES = OFF_BL + SZ_B;  // 128 KB

__global__ void __launch_bounds__(128, 1)
    hpsi_tc_kernel(const HpsiBlock* __restrict__ blocks, const HpsiItem* __restrict__ items,
                   const HpsiTask* __restrict__ tasks, double* __restrict__ scratch, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  uint32_t* Ah = (uint32_t*)(smraw + OFF_AH);
  uint32_t* Al = (uint32_t*)(smraw + OFF_AL);
  uint32_t* Ph = (uint32_t*)(smraw + OFF_PH);
  uint32_t* Pl = (uint32_t*)(smraw + OFF_PL);
  uint32_t* Xh = (uint32_t*)(smraw + OFF_XH);
  uint32_t* Xl = (uint32_t*)(smraw + OFF_XL);
  uint32_t* Bh = (uint32_t*)(smraw + OFF_BH);
  uint32_t* Bl = (uint32_t*)(smraw + OFF_BL);
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5;
  const HpsiTask tk = tasks[blockIdx.x];
  const HpsiBlock bk = blocks[tk.block];
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)), "r"(128));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_flag = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tX = tmem_base;       // columns [0, 64): X accumulator
  const uint32_t tS = tmem_base + 64;  // columns [64, 128): sigma accumulator
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  const uint32_t id1 = idesc_tf32(TM, JC);
  const uint32_t id2 = idesc_tf32(TM, TN);
  uint32_t phase = 0;
  bool s_started = false;  // sigma accumulator holds data
  // issue the MMAs of one staged k-block (32 wide) and wait for them
  auto run_k32 = [&](uint32_t dtm, uint32_t a_h, uint32_t a_l, uint32_t a_sbo, uint32_t b_h, uint32_t b_l,
                     uint32_t idesc, bool& started) -> bool {
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid == 0) {
#pragma unroll
      for (int s = 0; s < KS / 8; ++s) {
        uint32_t ko = (uint32_t)s * 2 * LBO;
        uint64_t ah = desc(a_h + ko, a_sbo), al = desc(a_l + ko, a_sbo);
        uint64_t bh = desc(b_h + s * 2 * LBO, SBO_K32), bl = desc(b_l + s * 2 * LBO, SBO_K32);
        mma_tf32(dtm, al, bh, idesc, (started || s > 0) ? 1u : 0u);
        mma_tf32(dtm, ah, bl, idesc, 1u);
        mma_tf32(dtm, ah, bh, idesc, 1u);
      }
      commit(&bar);
    }
    started = true;  // uniform over the CTA: the epilogue's tcgen05.ld is warp-collective
    bool ok = wait_bar(&bar, phase & 1);
    if (!ok) {
      ok = false;
      wait_bar(&bar, phase & 1);  // second bounded window for the MMAs in flight
      abort_flag = 1;
    }
    phase ^= 1;
    asm volatile("tcgen05.fence::after_thread_sync;");
    __syncthreads();
    if (abort_flag != 0 && tid == 0) atomicExch(err, 1);
    return abort_flag == 0;
  };
  bool alive = true;
  for (int ii = tk.it_begin; ii < tk.it_begin + tk.it_count && alive; ++ii) {
    const HpsiItem it = items[ii];
    int jc_begin = 0, jc_end = it.kb;
    if (it.B == nullptr) {
      jc_begin = tk.c0;
      jc_end = min(it.kb, tk.c0 + TN);
    }
    for (int jc = jc_begin; jc < jc_end && alive; jc += JC) {
      // ---- stage 1: X = alpha op(A) P(:, jc chunk)
      bool x_started = false;
      for (int k0 = 0; k0 < it.ka && alive; k0 += KS) {
        for (int e = tid; e < TM * KS; e += 128) {
          int r = e / KS, k = e % KS;
          int gr = tk.r0 + r, gk = k0 + k;
          double v = (gr < bk.m && gk < it.ka) ? it.alpha * ldA(it, gr, gk) : 0.0;
          uint32_t h, l;
          split64(v, h, l);
          int o = koff(r, k, KS);
          Ah[o] = h;
          Al[o] = l;
        }
        for (int e = tid; e < JC * KS; e += 128) {
          int n = e % JC, k = e / JC;  // P^T (n, k) = P(k, n)
          int gk = k0 + k, gn = jc + n;
          double v = (gk < it.ka && gn < jc_end) ? it.P[(size_t)gk * it.ldp + gn] : 0.0;
          uint32_t h, l;
          split64(v, h, l);
          int o = koff(n, k, KS);
          Ph[o] = h;
          Pl[o] = l;
        }
        alive = run_k32(tX, smem_u32(Ah), smem_u32(Al), SBO_K32, smem_u32(Ph), smem_u32(Pl), id1, x_started);
      }
      if (!alive) break;
      // ---- X: TMEM -> registers -> hi/lo K-major tile (row = thread)
      {
        const int r = tid;
#pragma unroll
        for (int c0 = 0; c0 < JC; c0 += 16) {
          float v[16];
          tmem_ld16(tX + lane_base + c0, v);
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            uint32_t h = tf32(v[j]);
            int o = koff(r, c0 + j, JC);
            Xh[o] = h;
            Xl[o] = tf32(v[j] - __uint_as_float(h));
          }
        }
      }
      // ---- stage 2: S += X op(B)(tile cols, chunk)^T
      for (int k0 = 0; k0 < JC && jc + k0 < jc_end && alive; k0 += KS) {
        for (int e = tid; e < TN * KS; e += 128) {
          int n = e / KS, k = e % KS;
          int gn = tk.c0 + n, gk = jc + k0 + k;
          double v = (gn < bk.n && gk < jc_end) ? ldB(it, gn, gk) : 0.0;
          uint32_t h, l;
          split64(v, h, l);
          int o = koff(n, k, KS);
          Bh[o] = h;
          Bl[o] = l;
        }
        uint32_t xoff = (uint32_t)(k0 / 4) * LBO;
        alive = run_k32(tS, smem_u32(Xh) + xoff, smem_u32(Xl) + xoff, SBO_K64, smem_u32(Bh), smem_u32(Bl), id2,
                        s_started);
      }
    }
  }
  // ---- write the sigma tile (row = thread)
  if (alive) {
    const int r = tid;
    for (int c0 = 0; c0 < TN; c0 += 16) {
      float v[16];
      if (s_started) tmem_ld16(tS + lane_base + c0, v);
      else
        for (int j = 0; j < 16; ++j) v[j] = 0.f;
      for (int j = 0; j < 16; ++j) {
        int c = c0 + j;
        if (tk.part >= 0) {
          scratch[tk.part + (long long)r * TN + c] = (double)v[j];
        } else {
          int gr = tk.r0 + r, gc = tk.c0 + c;
          if (gr < bk.m && gc < bk.n) bk.C[(size_t)gr * bk.ldc + gc] += (double)v[j];
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(128));
}

// partial tiles of the tcgen05 kernel are TM x TN
__global__ void hpsi_tc_reduce(const HpsiBlock* __restrict__ blocks, const HpsiReduce* __restrict__ reds,
                               const double* __restrict__ scratch) {
  const HpsiReduce rd = reds[blockIdx.x];
  const HpsiBlock bk = blocks[rd.block];
  for (int e = threadIdx.x; e < TM * TN; e += blockDim.x) {
    int r = e / TN, c = e % TN;
    int gr = rd.r0 + r, gc = rd.c0 + c;
    if (gr >= bk.m || gc >= bk.n) continue;
    double acc = 0.0;
    for (int p = 0; p < rd.nparts; ++p) acc += scratch[rd.part0 + (long long)p * TM * TN + e];
    bk.C[(size_t)gr * bk.ldc + gc] += acc;
  }
}

}  // namespace

void hpsi_tc_launch(const HpsiBlock* blocks, const HpsiItem* items, const HpsiTask* tasks, int ntasks,
                    const HpsiReduce* reds, int nreds, double* scratch, int* err, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(hpsi_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    attr = true;
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
