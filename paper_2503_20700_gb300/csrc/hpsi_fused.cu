// Fused H_eff psi kernels (see hpsi_fused.cuh).
#include <stdexcept>
#include <string>

#include "hpsi_fused.cuh"
#include "kattr.hpp"

namespace dmrg {

namespace {

constexpr int T = 64;   // tile edge of sigma and of the psi column chunk
constexpr int KS = 16;  // k-step of the staged operand tiles

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ uint32_t tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void split64(double x, uint32_t& hi, uint32_t& lo) {
  hi = tf32((float)x);
  lo = tf32((float)(x - (double)__uint_as_float(hi)));
}
__device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// element (r, c) of op(A) (m x k); op = identity when trans == 0
__device__ __forceinline__ double ldA(const HpsiItem& it, int r, int c) {
  return it.transA ? it.A[(size_t)c * it.lda + r] : it.A[(size_t)r * it.lda + c];
}
// element (n, k) of the right operand as used in X B^T
__device__ __forceinline__ double ldB(const HpsiItem& it, int n, int k) {
  return it.transB ? it.B[(size_t)k * it.ldb + n] : it.B[(size_t)n * it.ldb + k];
}

// shared-memory layout (32-bit words) of the TF32 kernel
constexpr int LDS = KS + 4;      // padded row of a 16-wide staged tile
constexpr int LDX = T + 4;       // padded row of the X tile
constexpr int SM_AH = 0;
constexpr int SM_AL = SM_AH + T * LDS;
constexpr int SM_PH = SM_AL + T * LDS;  // P stored n-major: [n][k]
constexpr int SM_PL = SM_PH + T * LDS;
constexpr int SM_BH = SM_PL + T * LDS;  // B stored n-major: [n][k]
constexpr int SM_BL = SM_BH + T * LDS;
constexpr int SM_XH = SM_BL + T * LDS;  // X stored m-major: [m][k]
constexpr int SM_XL = SM_XH + T * LDX;
constexpr int SM_WORDS = SM_XL + T * LDX;

// warp tile: 16 rows x 32 cols of the 64 x 64 tile; acc[nt][q] per mma.sync fragment
__device__ __forceinline__ void warp_mma_k16(float (&acc)[4][4], const uint32_t* Ah, const uint32_t* Al,
                                             int lda_s, const uint32_t* Bh, const uint32_t* Bl, int ldb_s,
                                             int kofs, int wm, int wn, int gid, int tig) {
#pragma unroll
  for (int ks = 0; ks < KS; ks += 8) {
    const int r = wm * 16 + gid;
    const int k = kofs + ks + tig;
    uint32_t ah[4] = {Ah[r * lda_s + k], Ah[(r + 8) * lda_s + k], Ah[r * lda_s + k + 4], Ah[(r + 8) * lda_s + k + 4]};
    uint32_t al[4] = {Al[r * lda_s + k], Al[(r + 8) * lda_s + k], Al[r * lda_s + k + 4], Al[(r + 8) * lda_s + k + 4]};
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int c = wn * 32 + nt * 8 + gid;
      const int kb = ks + tig;
      uint32_t bh[2] = {Bh[c * ldb_s + kb], Bh[c * ldb_s + kb + 4]};
      uint32_t bl[2] = {Bl[c * ldb_s + kb], Bl[c * ldb_s + kb + 4]};
      mma(acc[nt], al, bh);
      mma(acc[nt], ah, bl);
      mma(acc[nt], ah, bh);
    }
  }
}

__global__ void __launch_bounds__(256) hpsi_tf32x3_kernel(const HpsiBlock* __restrict__ blocks,
                                                          const HpsiItem* __restrict__ items,
                                                          const HpsiTask* __restrict__ tasks,
                                                          double* __restrict__ scratch) {
  extern __shared__ uint32_t sm[];
  uint32_t* Ah = sm + SM_AH;
  uint32_t* Al = sm + SM_AL;
  uint32_t* Ph = sm + SM_PH;
  uint32_t* Pl = sm + SM_PL;
  uint32_t* Bh = sm + SM_BH;
  uint32_t* Bl = sm + SM_BL;
  uint32_t* Xh = sm + SM_XH;
  uint32_t* Xl = sm + SM_XL;
  const HpsiTask tk = tasks[blockIdx.x];
  const HpsiBlock bk = blocks[tk.block];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = warp & 3, wn = warp >> 2;
  const int gid = lane >> 2, tig = lane & 3;
  double s64[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) s64[i][j] = 0.0;
  for (int ii = tk.it_begin; ii < tk.it_begin + tk.it_count; ++ii) {
    const HpsiItem it = items[ii];
    float sacc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) sacc[i][j] = 0.0f;
    // column chunks of psi (the k dimension of the second product)
    int jc_begin = 0, jc_end = it.kb;
    if (it.B == nullptr) {  // identity on the right: only sigma's own columns
      jc_begin = tk.c0;
      jc_end = min(it.kb, tk.c0 + T);
    }
    for (int jc = jc_begin; jc < jc_end; jc += T) {
      float xacc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) xacc[i][j] = 0.0f;
      if (it.A == nullptr) {
        // X = alpha P(rows of the tile, jc chunk): written straight to the X tile
        for (int e = threadIdx.x; e < T * T; e += 256) {
          int r = e / T, c = e % T;
          int gr = tk.r0 + r, gc = jc + c;
          double v = (gr < bk.m && gr < it.ka && gc < jc_end) ? it.alpha * it.P[(size_t)gr * it.ldp + gc] : 0.0;
          uint32_t h, l;
          split64(v, h, l);
          Xh[r * LDX + c] = h;
          Xl[r * LDX + c] = l;
        }
        __syncthreads();
      } else {
        for (int k0 = 0; k0 < it.ka; k0 += KS) {
          for (int e = threadIdx.x; e < T * KS; e += 256) {
            int r, c;
            if (!it.transA) { r = e / KS; c = e % KS; }
            else { c = e / T; r = e % T; }
            int gr = tk.r0 + r, gk = k0 + c;
            double v = (gr < bk.m && gk < it.ka) ? it.alpha * ldA(it, gr, gk) : 0.0;
            uint32_t h, l;
            split64(v, h, l);
            Ah[r * LDS + c] = h;
            Al[r * LDS + c] = l;
          }
          for (int e = threadIdx.x; e < T * KS; e += 256) {
            int kk = e / T, n = e % T;
            int gk = k0 + kk, gn = jc + n;
            double v = (gk < it.ka && gn < jc_end) ? it.P[(size_t)gk * it.ldp + gn] : 0.0;
            uint32_t h, l;
            split64(v, h, l);
            Ph[n * LDS + kk] = h;
            Pl[n * LDS + kk] = l;
          }
          __syncthreads();
          warp_mma_k16(xacc, Ah, Al, LDS, Ph, Pl, LDS, 0, wm, wn, gid, tig);
          __syncthreads();
        }
        if (it.B == nullptr) {
          // identity on the right: sigma += X for the tile's own columns
#pragma unroll
          for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int q = 0; q < 4; ++q) sacc[nt][q] += xacc[nt][q];
          continue;
        }
        // X fragments -> X tile in shared memory (hi / lo planes)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            int r = wm * 16 + gid + ((q >> 1) ? 8 : 0);
            int c = wn * 32 + nt * 8 + 2 * tig + (q & 1);
            float x = xacc[nt][q];
            uint32_t h = tf32(x);
            Xh[r * LDX + c] = h;
            Xl[r * LDX + c] = tf32(x - __uint_as_float(h));
          }
        __syncthreads();
      }
      if (it.B == nullptr) {
        // identity on the right with identity on the left: sigma += X tile
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            int r = wm * 16 + gid + ((q >> 1) ? 8 : 0);
            int c = wn * 32 + nt * 8 + 2 * tig + (q & 1);
            sacc[nt][q] += __uint_as_float(Xh[r * LDX + c]) + __uint_as_float(Xl[r * LDX + c]);
          }
        __syncthreads();
        continue;
      }
      // sigma tile += X (64 x chunk) B(tile cols, chunk)^T
      for (int k0 = 0; k0 < T && jc + k0 < jc_end; k0 += KS) {
        for (int e = threadIdx.x; e < T * KS; e += 256) {
          int n, kk;
          if (!it.transB) { n = e / KS; kk = e % KS; }
          else { kk = e / T; n = e % T; }
          int gn = tk.c0 + n, gk = jc + k0 + kk;
          double v = (gn < bk.n && gk < jc_end) ? ldB(it, gn, gk) : 0.0;
          uint32_t h, l;
          split64(v, h, l);
          Bh[n * LDS + kk] = h;
          Bl[n * LDS + kk] = l;
        }
        __syncthreads();
        warp_mma_k16(sacc, Xh, Xl, LDX, Bh, Bl, LDS, k0, wm, wn, gid, tig);
        __syncthreads();
      }
    }
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) s64[nt][q] += (double)sacc[nt][q];
  }
  // write: partial tile or direct add
#pragma unroll
  for (int nt = 0; nt < 4; ++nt)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int r = wm * 16 + gid + ((q >> 1) ? 8 : 0);
      int c = wn * 32 + nt * 8 + 2 * tig + (q & 1);
      if (tk.part >= 0) {
        scratch[tk.part + r * T + c] = s64[nt][q];
      } else {
        int gr = tk.r0 + r, gc = tk.c0 + c;
        if (gr < bk.m && gc < bk.n) bk.C[(size_t)gr * bk.ldc + gc] += s64[nt][q];
      }
    }
}

// ---------------------------------------------------------------- FP64 variant
// 16 x 16 threads, each owning a 4 x 4 register tile of the 64 x 64 tile
__global__ void __launch_bounds__(256) hpsi_f64_kernel(const HpsiBlock* __restrict__ blocks,
                                                       const HpsiItem* __restrict__ items,
                                                       const HpsiTask* __restrict__ tasks,
                                                       double* __restrict__ scratch) {
  extern __shared__ double smd[];
  double* As = smd;                 // [KS][T+1]   (k-major)
  double* Ps = As + KS * (T + 1);   // [KS][T+1]
  double* Bs = Ps + KS * (T + 1);   // [KS][T+1]   (k-major, n fast)
  double* Xs = Bs + KS * (T + 1);   // [T][T+1]    (m rows, k fast)
  const HpsiTask tk = tasks[blockIdx.x];
  const HpsiBlock bk = blocks[tk.block];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double s[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) s[i][j] = 0.0;
  for (int ii = tk.it_begin; ii < tk.it_begin + tk.it_count; ++ii) {
    const HpsiItem it = items[ii];
    int jc_begin = 0, jc_end = it.kb;
    if (it.B == nullptr) {
      jc_begin = tk.c0;
      jc_end = min(it.kb, tk.c0 + T);
    }
    for (int jc = jc_begin; jc < jc_end; jc += T) {
      double x[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) x[i][j] = 0.0;
      if (it.A == nullptr) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            int gr = tk.r0 + ty + 16 * i, gc = jc + tx + 16 * j;
            x[i][j] = (gr < bk.m && gr < it.ka && gc < jc_end) ? it.alpha * it.P[(size_t)gr * it.ldp + gc] : 0.0;
          }
      } else {
        for (int k0 = 0; k0 < it.ka; k0 += KS) {
          for (int e = threadIdx.x; e < T * KS; e += 256) {
            int r, c;
            if (!it.transA) { r = e / KS; c = e % KS; }
            else { c = e / T; r = e % T; }
            int gr = tk.r0 + r, gk = k0 + c;
            As[c * (T + 1) + r] = (gr < bk.m && gk < it.ka) ? it.alpha * ldA(it, gr, gk) : 0.0;
          }
          for (int e = threadIdx.x; e < T * KS; e += 256) {
            int kk = e / T, n = e % T;
            int gk = k0 + kk, gn = jc + n;
            Ps[kk * (T + 1) + n] = (gk < it.ka && gn < jc_end) ? it.P[(size_t)gk * it.ldp + gn] : 0.0;
          }
          __syncthreads();
#pragma unroll
          for (int kk = 0; kk < KS; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk * (T + 1) + ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Ps[kk * (T + 1) + tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
              for (int j = 0; j < 4; ++j) x[i][j] = fma(a[i], b[j], x[i][j]);
          }
          __syncthreads();
        }
      }
      if (it.B == nullptr) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) s[i][j] += x[i][j];
        continue;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) Xs[(ty + 16 * i) * (T + 1) + tx + 16 * j] = x[i][j];
      __syncthreads();
      for (int k0 = 0; k0 < T && jc + k0 < jc_end; k0 += KS) {
        for (int e = threadIdx.x; e < T * KS; e += 256) {
          int n, kk;
          if (!it.transB) { n = e / KS; kk = e % KS; }
          else { kk = e / T; n = e % T; }
          int gn = tk.c0 + n, gk = jc + k0 + kk;
          Bs[kk * (T + 1) + n] = (gn < bk.n && gk < jc_end) ? ldB(it, gn, gk) : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < KS; ++kk) {
          double a[4], b[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) a[i] = Xs[(ty + 16 * i) * (T + 1) + k0 + kk];
#pragma unroll
          for (int j = 0; j < 4; ++j) b[j] = Bs[kk * (T + 1) + tx + 16 * j];
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) s[i][j] = fma(a[i], b[j], s[i][j]);
        }
        __syncthreads();
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int r = ty + 16 * i, c = tx + 16 * j;
      if (tk.part >= 0) {
        scratch[tk.part + r * T + c] = s[i][j];
      } else {
        int gr = tk.r0 + r, gc = tk.c0 + c;
        if (gr < bk.m && gc < bk.n) bk.C[(size_t)gr * bk.ldc + gc] += s[i][j];
      }
    }
}

// sum the partial tiles of one sigma tile in a fixed order and add into C
__global__ void hpsi_reduce_kernel(const HpsiBlock* __restrict__ blocks, const HpsiReduce* __restrict__ reds,
                                   const double* __restrict__ scratch) {
  const HpsiReduce rd = reds[blockIdx.x];
  const HpsiBlock bk = blocks[rd.block];
  for (int e = threadIdx.x; e < T * T; e += blockDim.x) {
    int r = e / T, c = e % T;
    int gr = rd.r0 + r, gc = rd.c0 + c;
    if (gr >= bk.m || gc >= bk.n) continue;
    double acc = 0.0;
    for (int p = 0; p < rd.nparts; ++p) acc += scratch[rd.part0 + (long long)p * T * T + e];
    bk.C[(size_t)gr * bk.ldc + gc] += acc;
  }
}

}  // namespace

void hpsi_tile(Precision prec, int* tile_m, int* tile_n) {
  (void)prec;
  *tile_m = T;
  *tile_n = T;
}

size_t hpsi_plan_tasks(const std::vector<HpsiBlock>& blocks, Precision prec, std::vector<HpsiTask>& tasks,
                       std::vector<HpsiReduce>& reds) {
  tasks.clear();
  reds.clear();
  int tm, tn;
  hpsi_tile(prec, &tm, &tn);
  long long tile_items = 0;
  for (auto& b : blocks) tile_items += (long long)b.item_count * ((b.m + tm - 1) / tm) * ((b.n + tn - 1) / tn);
  const int max_items = (int)std::max<long long>(4, tile_items / (8 * 152) + 1);
  long long part = 0;
  for (size_t b = 0; b < blocks.size(); ++b) {
    const HpsiBlock& bk = blocks[b];
    if (bk.item_count == 0 || bk.m == 0 || bk.n == 0) continue;
    int nch = (bk.item_count + max_items - 1) / max_items;
    int per = (bk.item_count + nch - 1) / nch;
    for (int r0 = 0; r0 < bk.m; r0 += tm)
      for (int c0 = 0; c0 < bk.n; c0 += tn) {
        if (nch == 1) {
          tasks.push_back({(int)b, r0, c0, bk.item_begin, bk.item_count, -1});
        } else {
          reds.push_back({(int)b, r0, c0, nch, part});
          for (int c = 0; c < nch; ++c) {
            int i0 = bk.item_begin + c * per;
            int cnt = std::min(per, bk.item_begin + bk.item_count - i0);
            tasks.push_back({(int)b, r0, c0, i0, cnt, part});
            part += (long long)tm * tn;
          }
        }
      }
  }
  return (size_t)part;
}

void hpsi_launch(const HpsiBlock* blocks, const HpsiItem* items, const HpsiTask* tasks, int ntasks,
                 const HpsiReduce* reds, int nreds, double* scratch, Precision prec, int* err,
                 cudaStream_t st) {
  (void)err;
  if (prec == Precision::TC_TF32X3)
    throw std::runtime_error("internal: the tcgen05 contraction runs on pre-split operands (hpsi_tc_launch)");
  if (ntasks > 0) {
    if (prec == Precision::FP64) {
      size_t smem = (size_t)(3 * KS * (T + 1) + T * (T + 1)) * sizeof(double);
      cudaError_t ea = ensure_smem_attr((const void*)hpsi_f64_kernel, (int)smem);
      if (ea != cudaSuccess)
        throw std::runtime_error(std::string("cuda: hpsi f64 attribute: ") + cudaGetErrorString(ea));
      hpsi_f64_kernel<<<ntasks, 256, smem, st>>>(blocks, items, tasks, scratch);
    } else {
      size_t smem = (size_t)SM_WORDS * sizeof(uint32_t);
      cudaError_t ea = ensure_smem_attr((const void*)hpsi_tf32x3_kernel, (int)smem);
      if (ea != cudaSuccess)
        throw std::runtime_error(std::string("cuda: hpsi tf32x3 attribute: ") + cudaGetErrorString(ea));
      hpsi_tf32x3_kernel<<<ntasks, 256, smem, st>>>(blocks, items, tasks, scratch);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw std::runtime_error(std::string("cuda: hpsi launch: ") + cudaGetErrorString(e));
  }
  if (nreds > 0) {
    hpsi_reduce_kernel<<<nreds, 256, 0, st>>>(blocks, reds, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw std::runtime_error(std::string("cuda: hpsi reduce: ") + cudaGetErrorString(e));
  }
}

}  // namespace dmrg
