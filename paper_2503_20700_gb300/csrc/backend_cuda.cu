// CUDA implementation of the device primitives (backend.hpp) for sm_103a.
//
// Kernels:
//   place_kernel        C += sum_s alpha_s op(S_s)            (HBM-bound block copies)
//   gemm_f64_kernel     C += sum_s alpha_s op(A_s) op(B_s)    (FP64 reference path, DFMA)
//   gemm_tf32x3 (gemm_split.cu)                                (split-FP32 tensor-core path)
//   dots/combine/axpby  Davidson vector algebra (FP64, deterministic two-stage reductions)
//   jacobi_smem_kernel  parallel cyclic Jacobi eigensolver (FP64) of one matrix in shared memory, one CTA
//   jacobi_coop_kernel  a batch of matrices on one CTA per SM, each on a group of CTAs sized to its work
// All kernels are bounded loops over their inputs; the one wait on other CTAs,
// the group barrier of jacobi_coop_kernel, gives up after the backend's wait
// bound (2 s by default) and sets the error flag.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <stdexcept>
#include <string>
#include <vector>

#include "backend.hpp"
#include "gemm_split.cuh"
#include "hpsi_fused.cuh"
#include "hpsi_tc.cuh"
#include "jacobi_plan.hpp"

namespace dmrg {

#define CK(x)                                                                          \
  do {                                                                                 \
    cudaError_t e_ = (x);                                                              \
    if (e_ != cudaSuccess)                                                             \
      throw std::runtime_error(std::string("cuda: ") + #x + ": " + cudaGetErrorString(e_)); \
  } while (0)

// ------------------------------------------------------------------ place
struct PlaceTile {
  int group, r0, c0, pad;
};

__global__ void place_kernel(const PlaceGroup* __restrict__ groups, const PlaceSeg* __restrict__ segs,
                             const PlaceTile* __restrict__ tiles) {
  const PlaceTile t = tiles[blockIdx.x];
  const PlaceGroup g = groups[t.group];
  // 32 x 32 tile, 256 threads: 4 rows per thread
  const int c = t.c0 + (threadIdx.x & 31);
  const int rb = t.r0 + (threadIdx.x >> 5);
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  if (c < g.cols) {
    for (int s = g.seg_begin; s < g.seg_begin + g.seg_count; ++s) {
      const PlaceSeg sg = segs[s];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        int r = rb + 8 * i;
        if (r >= g.rows) break;
        double v;
        if (sg.src == nullptr) v = (r == c) ? 1.0 : 0.0;
        else v = sg.trans ? sg.src[(size_t)c * sg.ld + r] : sg.src[(size_t)r * sg.ld + c];
        acc[i] += sg.alpha * v;
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int r = rb + 8 * i;
      if (r >= g.rows) break;
      g.dst[(size_t)r * g.ld + c] += acc[i];
    }
  }
}

// ------------------------------------------------------------------ FP64 GEMM
struct GemmTile {
  int group, r0, c0, pad;
};

constexpr int kTM = 64, kTN = 64, kTK = 16;

__device__ __forceinline__ void gemm_f64_step(const double (*As)[kTM + 1], const double (*Bs)[kTN + 1], int kk,
                                              int tx, int ty, double (&acc)[4][4]) {
  double a[4], b[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
  for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
}

__global__ void __launch_bounds__(256) gemm_f64_kernel(const GemmGroup* __restrict__ groups,
                                                       const GemmSeg* __restrict__ segs,
                                                       const GemmTile* __restrict__ tiles) {
  __shared__ double As[kTK][kTM + 1];
  __shared__ double Bs[kTK][kTN + 1];
  const GemmTile t = tiles[blockIdx.x];
  const GemmGroup g = groups[t.group];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (int s = g.seg_begin; s < g.seg_begin + g.seg_count; ++s) {
    const GemmSeg sg = segs[s];
    for (int k0 = 0; k0 < sg.k; k0 += kTK) {
      // A tile (kTM x kTK) -> As[kk][i], scaled by alpha
      for (int e = threadIdx.x; e < kTM * kTK; e += 256) {
        int i, kk;
        if (!sg.transA) { i = e / kTK; kk = e % kTK; }
        else { kk = e / kTM; i = e % kTM; }
        int gi = t.r0 + i, gk = k0 + kk;
        double v = 0.0;
        if (gi < g.m && gk < sg.k)
          v = sg.transA ? sg.A[(size_t)gk * sg.lda + gi] : sg.A[(size_t)gi * sg.lda + gk];
        As[kk][i] = sg.alpha * v;
      }
      for (int e = threadIdx.x; e < kTN * kTK; e += 256) {
        int j, kk;
        if (!sg.transB) { kk = e / kTN; j = e % kTN; }
        else { j = e / kTK; kk = e % kTK; }
        int gj = t.c0 + j, gk = k0 + kk;
        double v = 0.0;
        if (gj < g.n && gk < sg.k)
          v = sg.transB ? sg.B[(size_t)gj * sg.ldb + gk] : sg.B[(size_t)gk * sg.ldb + gj];
        Bs[kk][j] = v;
      }
      __syncthreads();
      // a ragged last step (k = 1 outer products, k tails) runs only its valid kk
      const int kn = min(kTK, sg.k - k0);
      if (kn == kTK) {
#pragma unroll
        for (int kk = 0; kk < kTK; ++kk) gemm_f64_step(As, Bs, kk, tx, ty, acc);
      } else {
        for (int kk = 0; kk < kn; ++kk) gemm_f64_step(As, Bs, kk, tx, ty, acc);
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int gi = t.r0 + ty + 16 * i;
    if (gi >= g.m) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gj = t.c0 + tx + 16 * j;
      if (gj < g.n) g.C[(size_t)gi * g.ldc + gj] += acc[i][j];
    }
  }
}

// ------------------------------------------------------------------ vectors
constexpr int kRedBlocks = 152;  // one partial per SM for the reductions

__global__ void dots_partial(const double* __restrict__ V, int m, size_t len, size_t ld,
                             const double* __restrict__ x, double* __restrict__ part) {
  // blockIdx.y = vector index, blockIdx.x = chunk
  __shared__ double sh[256];
  const int i = blockIdx.y;
  double s = 0.0;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < len;
       t += (size_t)gridDim.x * blockDim.x)
    s = fma(V[(size_t)i * ld + t], x[t], s);
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(size_t)i * gridDim.x + blockIdx.x] = sh[0];
}

__global__ void dots_final(const double* __restrict__ part, int nparts, double* __restrict__ out) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int t = threadIdx.x; t < nparts; t += blockDim.x) s += part[(size_t)blockIdx.x * nparts + t];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

__global__ void combine_kernel(double* __restrict__ y, double beta, const double* __restrict__ V,
                               int m, size_t len, size_t ld, const double* __restrict__ c) {
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < len;
       t += (size_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < m; ++i) s = fma(c[i], V[(size_t)i * ld + t], s);
    y[t] = (beta == 0.0) ? s : fma(beta, y[t], s);
  }
}

__global__ void axpby_kernel(double* __restrict__ y, double a, const double* __restrict__ x, double b,
                             size_t len) {
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < len;
       t += (size_t)gridDim.x * blockDim.x)
    y[t] = (a == 0.0) ? b * x[t] : fma(a, y[t], b * x[t]);
}

__global__ void precond_kernel(double* __restrict__ y, const double* __restrict__ x,
                               const double* __restrict__ d, double e, size_t len) {
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < len;
       t += (size_t)gridDim.x * blockDim.x) {
    double den = d[t] - e;
    if (fabs(den) < 1e-8) den = den < 0 ? -1e-8 : 1e-8;
    y[t] = x[t] / den;
  }
}

// ------------------------------------------------------------------ Jacobi
// Parallel cyclic Jacobi (round-robin pairing) on a symmetric n x n matrix
// (destroyed).  Eigenvalues descending in w, the eigenvectors as rows of V.
// One round rotates n/2 disjoint pairs.  The matrix is updated as 2x2 blocks
// (rows of pair i, columns of pair j) R_i X R_j^T for i <= j only, each
// result stored at both symmetric positions: 2n^2 FP64 operations a round on
// A instead of 4n^2, plus 2n^2 on the eigenvector rows p, q of V.  A pair is
// skipped when its off-diagonal entry is negligible next to both diagonal
// entries, or below 1e-16 ||A||_F: the rounding noise of a GEMM-formed
// density matrix, whose (near) null space would otherwise keep rotating noise
// for every sweep.  The iteration stops after a sweep without rotations, or
// after kMaxSweeps sweeps.
//
// The work is FP64-bound (GB300 has few FP64 units per SM), so a batch of
// matrices is spread over the SMs: one cooperative launch with one CTA per
// SM, each matrix on a group of g CTAs sized to its share of the work (g = 1:
// A and V in shared memory; g > 1: A and V in global memory, one group
// barrier per round).
constexpr int kMaxSweeps = 30;
constexpr int kSmemN = kJacSmemN;  // largest matrix of the shared-memory path
constexpr int kJacThreads = 512;  // threads of a batched-launch CTA

__host__ __device__ constexpr size_t jacobi_smem_bytes(int n) {
  return ((size_t)n * (n + 1) + (size_t)n * n + (size_t)((n + 1) & ~1)) * sizeof(double) +
         (size_t)((n + 1) & ~1) * 2 * sizeof(int) + 64;
}

// pair i of a round, closed form of the round-robin schedule: (round, M) and
// (round + i, round - i) mod M, M = np - 1
__device__ __forceinline__ void jac_pair(int round, int i, int np, int& p, int& q) {
  const int M = np - 1;
  p = i == 0 ? round : (round + i) % M;
  q = i == 0 ? M : (round - i + M) % M;
  if (p > q) {
    int t = p;
    p = q;
    q = t;
  }
}

// (c, s) of the rotation that annihilates a_pq; false when the pair is skipped
__device__ __forceinline__ bool jac_rotation(double apq, double app, double aqq, double floor_abs, double& c,
                                             double& s) {
  c = 1.0;
  s = 0.0;
  const double g = 100.0 * fabs(apq);
  if (fabs(apq) <= floor_abs || (fabs(app) + g == fabs(app) && fabs(aqq) + g == fabs(aqq))) return false;
  const double theta = (aqq - app) / (2.0 * apq);
  const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
  c = 1.0 / sqrt(t * t + 1.0);
  s = t * c;
  return true;
}

// block (i, j), i <= j < h, of linear index e in the row-major upper triangle;
// row i starts at i h - i (i - 1) / 2
__device__ __forceinline__ void tri_index(int e, int h, int& i, int& j) {
  const float b = 2.0f * (float)h + 1.0f;
  int r = (int)((b - sqrtf(fmaxf(b * b - 8.0f * (float)e, 0.0f))) * 0.5f);
  r = max(0, min(r, h - 1));
  while (r > 0 && r * h - r * (r - 1) / 2 > e) --r;
  while (r + 1 < h && (r + 1) * h - (r + 1) * r / 2 <= e) ++r;
  i = r;
  j = r + (e - (r * h - r * (r - 1) / 2));
}

template <bool kGlobal>
__device__ __forceinline__ double jac_ld(const double* p) {
  if constexpr (kGlobal) return __ldcg(p);
  else return *p;
}

struct JacRound {
  const double* cs;
  const double* sn;
  const int* pp;
  const int* qq;
};

// R_i X R_j^T on block (i, j), i <= j, stored at both symmetric positions
template <bool kGlobal>
__device__ __forceinline__ void jac_block(double* a, int lda, int n, int i, int j, const JacRound& R) {
  const double ci = R.cs[i], si = R.sn[i], cj = R.cs[j], sj = R.sn[j];
  if (si == 0.0 && sj == 0.0) return;
  const int p = R.pp[i], q = R.qq[i], r = R.pp[j], t = R.qq[j];
  const bool qv = q < n, tv = t < n;
  const double x00 = jac_ld<kGlobal>(a + (size_t)p * lda + r);
  const double x01 = tv ? jac_ld<kGlobal>(a + (size_t)p * lda + t) : 0.0;
  const double x10 = qv ? jac_ld<kGlobal>(a + (size_t)q * lda + r) : 0.0;
  const double x11 = (qv && tv) ? jac_ld<kGlobal>(a + (size_t)q * lda + t) : 0.0;
  const double y00 = ci * x00 - si * x10, y01 = ci * x01 - si * x11;
  const double y10 = si * x00 + ci * x10, y11 = si * x01 + ci * x11;
  const double n00 = cj * y00 - sj * y01, n01 = sj * y00 + cj * y01;
  if (i == j) {  // r = p, t = q: the diagonal block, (p, q) and (q, p) from one value
    a[(size_t)p * lda + p] = n00;
    if (qv) {
      a[(size_t)p * lda + q] = n01;
      a[(size_t)q * lda + p] = n01;
      a[(size_t)q * lda + q] = sj * y10 + cj * y11;
    }
    return;
  }
  const double n10 = cj * y10 - sj * y11, n11 = sj * y10 + cj * y11;
  a[(size_t)p * lda + r] = n00;
  a[(size_t)r * lda + p] = n00;
  if (tv) {
    a[(size_t)p * lda + t] = n01;
    a[(size_t)t * lda + p] = n01;
  }
  if (qv) {
    a[(size_t)q * lda + r] = n10;
    a[(size_t)r * lda + q] = n10;
  }
  if (qv && tv) {
    a[(size_t)q * lda + t] = n11;
    a[(size_t)t * lda + q] = n11;
  }
}

// element k of the eigenvector rows p, q of pair i
template <bool kGlobal>
__device__ __forceinline__ void jac_vrot(double* v, int n, int i, int k, const JacRound& R) {
  const double s = R.sn[i];
  if (s == 0.0) return;
  const double c = R.cs[i];
  const int p = R.pp[i], q = R.qq[i];
  const double vp = jac_ld<kGlobal>(v + (size_t)p * n + k), vq = jac_ld<kGlobal>(v + (size_t)q * n + k);
  v[(size_t)p * n + k] = c * vp - s * vq;
  v[(size_t)q * n + k] = s * vp + c * vq;
}

// rotation parameters of every pair of the round (threads < h); nrot counts
// the rotations of the sweep
template <bool kGlobal>
__device__ __forceinline__ void jac_params(const double* a, int lda, int n, int np, int round, double floor_abs,
                                           double* cs, double* sn, int* pp, int* qq, int* nrot) {
  const int h = np / 2;
  for (int i = threadIdx.x; i < h; i += blockDim.x) {
    int p, q;
    jac_pair(round, i, np, p, q);
    pp[i] = p;
    qq[i] = q;
    double c = 1.0, s = 0.0;
    if (q < n &&
        jac_rotation(jac_ld<kGlobal>(a + (size_t)p * lda + q), jac_ld<kGlobal>(a + (size_t)p * lda + p),
                     jac_ld<kGlobal>(a + (size_t)q * lda + q), floor_abs, c, s))
      atomicAdd(nrot, 1);
    cs[i] = c;
    sn[i] = s;
  }
}

// sum over the CTA (blockDim a power of two, red holds blockDim values)
__device__ double jac_block_sum(double x, double* red) {
  red[threadIdx.x] = x;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

// rank of the diagonal entries, descending (NaN last, ties by index): perm[rank] = i
template <bool kGlobal>
__device__ void jac_order(const double* a, int lda, int n, int* perm) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double di = jac_ld<kGlobal>(a + (size_t)i * lda + i);
    if (!(di == di)) di = -INFINITY;
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      double dj = jac_ld<kGlobal>(a + (size_t)j * lda + j);
      if (!(dj == dj)) dj = -INFINITY;
      rank += (dj > di) || (dj == di && j < i);
    }
    perm[rank] = i;
  }
}

// one matrix on one CTA, A (row stride n+1) and V in shared memory
__device__ void jacobi_one(const EighTask& tk, double* sm, double* red, int* nrot) {
  const int n = tk.n;
  const int lda = n + 1;
  const int np = (n + 1) & ~1, h = np / 2;
  double* a = sm;                   // n x (n+1)
  double* v = a + (size_t)n * lda;  // n x n, row p = eigenvector p
  double* cs = v + (size_t)n * n;   // h
  double* sn = cs + h;              // h
  int* pp = (int*)(sn + h);
  int* qq = pp + h;
  int* perm = qq + h;  // np
  const JacRound R{cs, sn, pp, qq};
  double fro = 0.0;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int r = e / n, c = e % n;
    const double x = tk.A[e];
    a[r * lda + c] = x;
    v[e] = (r == c) ? 1.0 : 0.0;
    fro += x * x;
  }
  const double floor_abs = 1e-16 * sqrt(jac_block_sum(fro, red));
  const int nb = h * (h + 1) / 2;
  for (int sweep = 0; sweep < kMaxSweeps && n > 1; ++sweep) {
    if (threadIdx.x == 0) *nrot = 0;
    __syncthreads();
    for (int round = 0; round < np - 1; ++round) {
      jac_params<false>(a, lda, n, np, round, floor_abs, cs, sn, pp, qq, nrot);
      __syncthreads();
      for (int e = threadIdx.x; e < nb; e += blockDim.x) {
        int i, j;
        tri_index(e, h, i, j);
        jac_block<false>(a, lda, n, i, j, R);
      }
      for (int e = threadIdx.x; e < h * n; e += blockDim.x) jac_vrot<false>(v, n, e / n, e % n, R);
      __syncthreads();
    }
    if (*nrot == 0) break;
    __syncthreads();
  }
  jac_order<false>(a, lda, n, perm);
  __syncthreads();
  for (int r = threadIdx.x; r < n; r += blockDim.x) tk.w[r] = a[perm[r] * lda + perm[r]];
  // eigenvector rows in descending order, largest-magnitude component positive
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    const double* src = v + (size_t)perm[r] * n;
    double best = 0.0;
    int bi = 0;
    for (int k = 0; k < n; ++k) {
      double x = fabs(src[k]);
      if (x > best + 1e-12) {
        best = x;
        bi = k;
      }
    }
    const double sg = src[bi] < 0 ? -1.0 : 1.0;
    for (int k = 0; k < n; ++k) tk.V[(size_t)r * n + k] = sg * src[k];
  }
}

__global__ void __launch_bounds__(256) jacobi_smem_kernel(const EighTask* __restrict__ tasks) {
  extern __shared__ double sm[];
  __shared__ double red[256];
  __shared__ int nrot;
  jacobi_one(tasks[blockIdx.x], sm, red, &nrot);
}

// A matrix on a group of g CTAs: every CTA of the group computes the round's
// rotation parameters from the same entries (identical values, so no
// exchange is needed) and updates its own contiguous share of the triangle
// blocks and of the eigenvector elements; one group barrier per round
// publishes the updates.  The barrier's wait is bounded by the backend's
// wait bound (wall clock) and sets the error flag on timeout; with a bound of
// 0 a barrier not complete at its first probe gives up.
struct CoopEigh {
  EighTask t;
  int g, cta0;
  unsigned* bar;  // (arrivals, generation), zero at launch
};

__device__ __forceinline__ unsigned long long jac_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned x;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(x) : "l"(p) : "memory");
  return x;
}

// returns false when the wait ran out
__device__ bool group_sync(unsigned* bar, int g, unsigned& gen, int* ok_s, unsigned long long wait_ns) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned target = gen + 1;
    if (atomicAdd(&bar[0], 1u) == (unsigned)g - 1) {
      atomicExch(&bar[0], 0u);
      __threadfence();
      atomicExch(&bar[1], target);
    } else {
      const unsigned long long t0 = jac_ns();
      const int spin = wait_ns > 0 ? 256 : 1;
      for (int probe = 0; (int)(ld_acquire(&bar[1]) - target) < 0; ++probe) {
        if (probe >= spin) {
          if (jac_ns() - t0 >= wait_ns) {
            *ok_s = 0;
            break;
          }
          __nanosleep(32);
        }
      }
    }
    gen = target;
    __threadfence();
  }
  __syncthreads();
  return *ok_s != 0;
}

__device__ void jacobi_group(const CoopEigh& ct, int me, double* sm, double* red, int* nrot, int* ok_s,
                             int* err, unsigned long long wait_ns) {
  const int g = ct.g;
  const int n = ct.t.n;
  double* a = const_cast<double*>(ct.t.A);
  double* v = ct.t.V;
  const int np = (n + 1) & ~1, h = np / 2;
  double* cs = sm;
  double* sn = sm + h;
  int* pp = (int*)(sm + np);
  int* qq = pp + h;
  int* perm = qq + h;
  const JacRound R{cs, sn, pp, qq};
  unsigned gen = 0;
  if (threadIdx.x == 0) *ok_s = 1;
  for (int r = me; r < n; r += g)
    for (int k = threadIdx.x; k < n; k += blockDim.x) v[(size_t)r * n + k] = (r == k) ? 1.0 : 0.0;
  double fro = 0.0;
  for (size_t e = threadIdx.x; e < (size_t)n * n; e += blockDim.x) {
    const double x = __ldcg(a + e);
    fro += x * x;
  }
  const double floor_abs = 1e-16 * sqrt(jac_block_sum(fro, red));
  // this CTA's shares: triangle blocks [b0, b1), eigenvector elements [v0, v1)
  const long long nb = (long long)h * (h + 1) / 2, nv = (long long)h * n;
  const int b0 = (int)(nb * me / g), b1 = (int)(nb * (me + 1) / g);
  const int v0 = (int)(nv * me / g), v1 = (int)(nv * (me + 1) / g);
  if (!group_sync(ct.bar, g, gen, ok_s, wait_ns)) goto fail;
  for (int sweep = 0; sweep < kMaxSweeps && n > 1; ++sweep) {
    if (threadIdx.x == 0) *nrot = 0;
    __syncthreads();
    for (int round = 0; round < np - 1; ++round) {
      jac_params<true>(a, n, n, np, round, floor_abs, cs, sn, pp, qq, nrot);
      __syncthreads();
      for (int e = b0 + (int)threadIdx.x; e < b1; e += blockDim.x) {
        int i, j;
        tri_index(e, h, i, j);
        jac_block<true>(a, n, n, i, j, R);
      }
      for (int e = v0 + (int)threadIdx.x; e < v1; e += blockDim.x) jac_vrot<true>(v, n, e / n, e % n, R);
      if (!group_sync(ct.bar, g, gen, ok_s, wait_ns)) goto fail;
    }
    if (*nrot == 0) break;
    __syncthreads();
  }
  if (me != 0) return;
  // CTA 0: eigenvalues descending, rows of V permuted, largest component positive
  jac_order<true>(a, n, n, perm);
  __syncthreads();
  for (int r = threadIdx.x; r < n; r += blockDim.x) ct.t.w[r] = __ldcg(a + (size_t)perm[r] * n + perm[r]);
  __syncthreads();
  for (size_t e = threadIdx.x; e < (size_t)n * n; e += blockDim.x) a[e] = __ldcg(v + e);
  __syncthreads();
  for (size_t e = threadIdx.x; e < (size_t)n * n; e += blockDim.x) {
    const int r = (int)(e / n), k = (int)(e % n);
    v[e] = a[(size_t)perm[r] * n + k];
  }
  __syncthreads();
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    double best = 0.0;
    int bi = 0;
    for (int k = 0; k < n; ++k) {
      double x = fabs(v[(size_t)r * n + k]);
      if (x > best + 1e-12) {
        best = x;
        bi = k;
      }
    }
    if (v[(size_t)r * n + bi] < 0)
      for (int k = 0; k < n; ++k) v[(size_t)r * n + k] = -v[(size_t)r * n + k];
  }
  return;
fail:
  if (threadIdx.x == 0) atomicExch(err, 1);
}

// The batched launch: CTA b belongs to the last task whose cta0 <= b.
__global__ void __launch_bounds__(kJacThreads) jacobi_coop_kernel(const CoopEigh* __restrict__ tasks, int ntasks,
                                                                  int* __restrict__ err,
                                                                  unsigned long long wait_ns) {
  int lo = 0, hi = ntasks - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (tasks[mid].cta0 <= (int)blockIdx.x) lo = mid;
    else hi = mid - 1;
  }
  const CoopEigh ct = tasks[lo];
  extern __shared__ double sm[];
  __shared__ double red[kJacThreads];
  __shared__ int nrot, ok_s;
  if (ct.g == 1) jacobi_one(ct.t, sm, red, &nrot);
  else jacobi_group(ct, (int)blockIdx.x - ct.cta0, sm, red, &nrot, &ok_s, err, wait_ns);
}

// ------------------------------------------------------------------ backend
class CudaBackend : public Backend {
 public:
  int dev = 0;
  cudaStream_t st = nullptr;
  size_t used = 0;
  std::vector<std::pair<void*, size_t>> live;
  // staging for task lists
  void* dtask = nullptr;
  size_t dtask_cap = 0;
  void* htask = nullptr;
  size_t htask_cap = 0;
  double* part = nullptr;
  size_t part_cap = 0;
  // profiling
  bool profiling = false;
  struct Rec {
    cudaEvent_t a, b;
    double flops;
    int tag;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  // categories: 0 GEMMs, 1 H_eff psi (with its operand splits), 2 blocking
  // placement, 3 eigensolver (shared-memory kernel), 4 eigensolver
  // (cooperative kernel)
  static constexpr int kTags = 6;
  double acc_ms[kTags] = {0, 0, 0, 0, 0, 0}, acc_flops[kTags] = {0, 0, 0, 0, 0, 0};
  long acc_launch[kTags] = {0, 0, 0, 0, 0, 0};
  cudaEvent_t ev() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    return e;
  }
  void drain() {
    for (auto& r : recs) {
      CK(cudaEventSynchronize(r.b));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, r.a, r.b));
      int t = std::min(kTags - 1, std::max(0, r.tag));
      acc_ms[t] += ms;
      acc_flops[t] += r.flops;
      acc_launch[t] += 1;
      pool.push_back(r.a);
      pool.push_back(r.b);
    }
    recs.clear();
  }
  cudaEvent_t mb_[2] = {nullptr, nullptr}, me_[2] = {nullptr, nullptr};
  void mark_begin(int slot) override {
    if (slot < 0 || slot > 1) throw std::logic_error("internal: event slot out of range");
    if (!mb_[slot]) {
      CK(cudaEventCreate(&mb_[slot]));
      CK(cudaEventCreate(&me_[slot]));
    }
    CK(cudaEventRecord(mb_[slot], st));
  }
  double mark_end(int slot) override {
    if (slot < 0 || slot > 1 || !mb_[slot]) throw std::logic_error("internal: event slot not started");
    CK(cudaEventRecord(me_[slot], st));
    CK(cudaEventSynchronize(me_[slot]));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, mb_[slot], me_[slot]));
    return ms;
  }
  void set_profile(bool on) override {
    drain();
    profiling = on;
    for (int t = 0; t < kTags; ++t) acc_ms[t] = acc_flops[t] = 0, acc_launch[t] = 0;
  }
  void kernel_stats(int t, double* ms, double* flops, long* launches) override {
    drain();
    t = std::min(kTags - 1, std::max(0, t));
    if (ms) *ms = acc_ms[t];
    if (flops) *flops = acc_flops[t];
    if (launches) *launches = acc_launch[t];
  }

  explicit CudaBackend(int device) : dev(device) {
    CK(cudaSetDevice(dev));
    CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    cudaMemPool_t pool;
    CK(cudaDeviceGetDefaultMemPool(&pool, dev));
    uint64_t thr = UINT64_MAX;
    CK(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
    size_t fr = 0;
    CK(cudaMemGetInfo(&fr, &total_mem));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  int sms = 152;
  int sm_count() const override { return sms; }
  ~CudaBackend() override {
    cudaStreamSynchronize(st);
    if (side) {
      cudaStreamSynchronize(side);
      cudaStreamDestroy(side);
    }
    for (auto& r : recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : pool) cudaEventDestroy(e);
    for (int k = 0; k < 2; ++k)
      if (mb_[k]) {
        cudaEventDestroy(mb_[k]);
        cudaEventDestroy(me_[k]);
      }
    if (dtask) cudaFreeAsync(dtask, st);
    if (part) cudaFreeAsync(part, st);
    if (dflag) cudaFreeAsync(dflag, st);
    if (htask) cudaFreeHost(htask);
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  std::string name() const override { return "cuda"; }
  void* alloc(size_t b) override {
    void* p = nullptr;
    if (b == 0) b = 8;
    while (budget_ && used + b > budget_ && make_room && make_room()) {
    }
    if (budget_ && used + b > budget_)
      throw std::runtime_error("out of device memory (budget of " + std::to_string(budget_) + " bytes: " +
                               std::to_string(used) + " held, " + std::to_string(b) + " requested)");
    cudaError_t e = cudaMallocAsync(&p, b, st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw std::runtime_error("out of device memory (" + std::to_string(b) + " bytes)");
    }
    used += b;
    peak_bytes = std::max(peak_bytes, used);
    window_peak = std::max(window_peak, used);
    live.push_back({p, b});
    return p;
  }
  void free(void* p) override {
    if (!p) return;
    for (size_t i = 0; i < live.size(); ++i)
      if (live[i].first == p) {
        used -= live[i].second;
        live[i] = live.back();
        live.pop_back();
        break;
      }
    CK(cudaFreeAsync(p, st));
  }
  size_t bytes_in_use() const override { return used; }
  // ---- staging to pinned host memory on the side stream
  cudaStream_t side = nullptr;
  cudaStream_t side_stream() {
    if (!side) CK(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
    return side;
  }
  void* stage_out(void* dev, size_t bytes) override {
    if (!dev || bytes == 0) return nullptr;
    cudaStream_t sd = side_stream();
    void* h = nullptr;
    if (cudaMallocHost(&h, bytes) != cudaSuccess) {
      cudaGetLastError();
      throw std::runtime_error("out of pinned host memory (" + std::to_string(bytes) + " bytes)");
    }
    cudaEvent_t e;
    CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    CK(cudaEventRecord(e, st));
    CK(cudaStreamWaitEvent(sd, e, 0));
    CK(cudaEventDestroy(e));
    CK(cudaMemcpyAsync(h, dev, bytes, cudaMemcpyDeviceToHost, sd));
    // the device buffer goes back to the pool after the copy (side-stream order)
    for (size_t i = 0; i < live.size(); ++i)
      if (live[i].first == dev) {
        used -= live[i].second;
        live[i] = live.back();
        live.pop_back();
        break;
      }
    CK(cudaFreeAsync(dev, sd));
    staged_bytes += bytes;
    staged_out_bytes += bytes;
    return h;
  }
  void* stage_in(const void* host, size_t bytes) override {
    if (!host || bytes == 0) return nullptr;
    cudaStream_t sd = side_stream();
    void* d = alloc(bytes);  // main-stream ordered allocation
    cudaEvent_t e;
    CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    CK(cudaEventRecord(e, st));
    CK(cudaStreamWaitEvent(sd, e, 0));
    CK(cudaEventDestroy(e));
    CK(cudaMemcpyAsync(d, host, bytes, cudaMemcpyHostToDevice, sd));
    staged_in_bytes += bytes;
    return d;
  }
  void stage_join() override {
    if (!side) return;
    cudaEvent_t e;
    CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    CK(cudaEventRecord(e, side));
    CK(cudaStreamWaitEvent(st, e, 0));
    CK(cudaEventDestroy(e));
  }
  void host_release(void* host) override {
    if (!host) return;
    if (side) CK(cudaStreamSynchronize(side));
    CK(cudaFreeHost(host));
  }
  size_t total_mem = 0;
  size_t capacity() const override { return total_mem; }
  size_t device_free() const override {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return fr;
  }
  void memset0(void* p, size_t b) override { if (b) CK(cudaMemsetAsync(p, 0, b, st)); }
  void copy_d2d(void* d, const void* s, size_t b) override {
    if (b) CK(cudaMemcpyAsync(d, s, b, cudaMemcpyDeviceToDevice, st));
  }
  void copy_h2d(void* d, const void* s, size_t b) override {
    if (b) {
      CK(cudaMemcpyAsync(d, s, b, cudaMemcpyHostToDevice, st));
      CK(cudaStreamSynchronize(st));
    }
  }
  void copy_d2h(void* d, const void* s, size_t b) override {
    if (b) {
      CK(cudaMemcpyAsync(d, s, b, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
    }
  }
  void sync() override { CK(cudaStreamSynchronize(st)); }
  int* dflag = nullptr;  // device error flag of the bounded waits
  int* flag() {
    if (!dflag) {
      CK(cudaMallocAsync((void**)&dflag, sizeof(int), st));
      CK(cudaMemsetAsync(dflag, 0, sizeof(int), st));
    }
    return dflag;
  }
  void check_device_flag() override {
    if (!dflag) return;
    int h = 0;
    CK(cudaMemcpyAsync(&h, dflag, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h != 0) {
      CK(cudaMemsetAsync(dflag, 0, sizeof(int), st));
      throw std::runtime_error("timeout: a bounded wait in the tcgen05 H_eff psi kernel ran out");
    }
  }
  void* stream() override { return (void*)st; }

  // upload a packed task buffer; returns the device base pointer
  char* upload(const std::vector<std::pair<const void*, size_t>>& parts, std::vector<size_t>& offs) {
    size_t tot = 0;
    offs.clear();
    for (auto& p : parts) {
      offs.push_back(tot);
      tot += (p.second + 255) & ~size_t(255);
    }
    if (tot > htask_cap) {
      CK(cudaStreamSynchronize(st));
      if (htask) CK(cudaFreeHost(htask));
      htask_cap = std::max(tot, htask_cap * 2);
      CK(cudaMallocHost(&htask, htask_cap));
    }
    if (tot > dtask_cap) {
      if (dtask) CK(cudaFreeAsync(dtask, st));
      dtask_cap = std::max(tot, dtask_cap * 2);
      CK(cudaMallocAsync(&dtask, dtask_cap, st));
    }
    // the pinned staging buffer may still be in use by a previous copy
    CK(cudaStreamSynchronize(st));
    for (size_t i = 0; i < parts.size(); ++i)
      std::memcpy((char*)htask + offs[i], parts[i].first, parts[i].second);
    CK(cudaMemcpyAsync(dtask, htask, tot, cudaMemcpyHostToDevice, st));
    return (char*)dtask;
  }

  void place(const std::vector<PlaceGroup>& groups, const std::vector<PlaceSeg>& segs) override {
    std::vector<PlaceTile> tiles;
    for (size_t gi = 0; gi < groups.size(); ++gi) {
      auto& g = groups[gi];
      for (int r = 0; r < g.rows; r += 32)
        for (int c = 0; c < g.cols; c += 32) tiles.push_back({(int)gi, r, c, 0});
      place_bytes += 16.0 * g.rows * g.cols * std::max(1, g.seg_count);
    }
    if (tiles.empty()) return;
    std::vector<size_t> off;
    char* d = upload({{groups.data(), groups.size() * sizeof(PlaceGroup)},
                      {segs.data(), segs.size() * sizeof(PlaceSeg)},
                      {tiles.data(), tiles.size() * sizeof(PlaceTile)}},
                     off);
    Rec* rec = nullptr;
    if (profiling) {
      recs.push_back(Rec{ev(), ev(), 0.0, 2});
      rec = &recs.back();
      CK(cudaEventRecord(rec->a, st));
    }
    place_kernel<<<(unsigned)tiles.size(), 256, 0, st>>>((const PlaceGroup*)(d + off[0]),
                                                          (const PlaceSeg*)(d + off[1]),
                                                          (const PlaceTile*)(d + off[2]));
    if (rec) CK(cudaEventRecord(rec->b, st));
    if (recs.size() > 4096) drain();
    ++launches;
    CK(cudaGetLastError());
  }

  void gemm(const std::vector<GemmGroup>& groups, const std::vector<GemmSeg>& segs,
            Precision prec) override {
    if (groups.empty()) return;
    double fl = 0.0;
    for (auto& g : groups)
      for (int s = g.seg_begin; s < g.seg_begin + g.seg_count; ++s)
        fl += 2.0 * g.m * g.n * segs[s].k;
    gemm_flops += fl;
    if (profiling) {
      // upload first so the events bracket the kernel only
      Rec r{ev(), ev(), fl, tag};
      recs.push_back(r);
      gemm_impl(groups, segs, prec, &recs.back());
      if (recs.size() > 4096) drain();
      return;
    }
    gemm_impl(groups, segs, prec, nullptr);
  }

  void gemm_impl(const std::vector<GemmGroup>& groups, const std::vector<GemmSeg>& segs,
                 Precision prec, Rec* rec) {
    if (prec != Precision::FP64) {
      gemm_split_launch(groups, segs, prec, st,
                        [&](const std::vector<std::pair<const void*, size_t>>& parts,
                            std::vector<size_t>& offs) {
                          char* d = upload(parts, offs);
                          if (rec) CK(cudaEventRecord(rec->a, st));
                          return d;
                        });
      ++launches;
      if (rec) CK(cudaEventRecord(rec->b, st));
      return;
    }
    std::vector<GemmTile> tiles;
    for (size_t gi = 0; gi < groups.size(); ++gi) {
      auto& g = groups[gi];
      for (int r = 0; r < g.m; r += kTM)
        for (int c = 0; c < g.n; c += kTN) tiles.push_back({(int)gi, r, c, 0});
    }
    std::vector<size_t> off;
    char* d = upload({{groups.data(), groups.size() * sizeof(GemmGroup)},
                      {segs.data(), segs.size() * sizeof(GemmSeg)},
                      {tiles.data(), tiles.size() * sizeof(GemmTile)}},
                     off);
    if (rec) CK(cudaEventRecord(rec->a, st));
    // grid.x is limited to 2^31-1; task lists stay far below
    gemm_f64_kernel<<<(unsigned)tiles.size(), 256, 0, st>>>((const GemmGroup*)(d + off[0]),
                                                             (const GemmSeg*)(d + off[1]),
                                                             (const GemmTile*)(d + off[2]));
    ++launches;
    CK(cudaGetLastError());
    if (rec) CK(cudaEventRecord(rec->b, st));
  }

  void hpsi(const HpsiBlock* blocks, const HpsiItem* items, const HpsiTask* tasks, int ntasks,
            const HpsiReduce* reds, int nreds, double* scratch, Precision prec, double flops) override {
    gemm_flops += flops;
    Rec* rec = nullptr;
    if (profiling) {
      recs.push_back(Rec{ev(), ev(), flops, 1});
      rec = &recs.back();
      CK(cudaEventRecord(rec->a, st));
    }
    hpsi_launch(blocks, items, tasks, ntasks, reds, nreds, scratch, prec, flag(), st);
    launches += (ntasks > 0) + (nreds > 0);
    if (rec) CK(cudaEventRecord(rec->b, st));
    if (recs.size() > 4096) drain();
  }

  void hpsi_tc(const TcLaunch& L, double flops, int tag) override {
    gemm_flops += flops;
    Rec* rec = nullptr;
    if (profiling) {
      recs.push_back(Rec{ev(), ev(), flops, tag});
      rec = &recs.back();
      CK(cudaEventRecord(rec->a, st));
    }
    hpsi_tc_launch(L, flag(), wait_ns_, st);
    launches += (L.ncta > 0) + (L.nreds > 0);
    if (rec) CK(cudaEventRecord(rec->b, st));
    if (recs.size() > 4096) drain();
  }
  void split(const SplitJob* jobs, int n, float* pool) override {
    if (n <= 0) return;
    // the operand splits of the tcgen05 path (tag 5)
    Rec* rec = nullptr;
    if (profiling) {
      recs.push_back(Rec{ev(), ev(), 0.0, 5});
      rec = &recs.back();
      CK(cudaEventRecord(rec->a, st));
    }
    split_launch(jobs, n, pool, st);
    ++launches;
    if (rec) CK(cudaEventRecord(rec->b, st));
    if (recs.size() > 4096) drain();
  }

  void ensure_part(size_t n) {
    if (n <= part_cap) return;
    if (part) CK(cudaFreeAsync(part, st));
    part_cap = std::max(n, 2 * part_cap);
    CK(cudaMallocAsync((void**)&part, part_cap * sizeof(double), st));
  }
  void dots(const double* V, int m, size_t len, size_t ld, const double* x, double* out) override {
    if (m <= 0) return;
    int nb = (int)std::min<size_t>(kRedBlocks, (len + 255) / 256);
    if (nb < 1) nb = 1;
    ensure_part((size_t)m * nb);
    dots_partial<<<dim3(nb, m), 256, 0, st>>>(V, m, len, ld, x, part);
    ++launches;
    dots_final<<<m, 256, 0, st>>>(part, nb, out);
    ++launches;
    CK(cudaGetLastError());
  }
  void combine(double* y, double beta, const double* V, int m, size_t len, size_t ld,
               const double* c) override {
    int nb = (int)std::min<size_t>(152 * 8, (len + 255) / 256);
    if (nb < 1) nb = 1;
    combine_kernel<<<nb, 256, 0, st>>>(y, beta, V, m, len, ld, c);
    ++launches;
    CK(cudaGetLastError());
  }
  void axpby(double* y, double a, const double* x, double b, size_t len) override {
    int nb = (int)std::min<size_t>(152 * 8, (len + 255) / 256);
    if (nb < 1) nb = 1;
    axpby_kernel<<<nb, 256, 0, st>>>(y, a, x, b, len);
    ++launches;
    CK(cudaGetLastError());
  }
  void precondition(double* y, const double* x, const double* d, double e, size_t len) override {
    int nb = (int)std::min<size_t>(152 * 8, (len + 255) / 256);
    if (nb < 1) nb = 1;
    precond_kernel<<<nb, 256, 0, st>>>(y, x, d, e, len);
    ++launches;
    CK(cudaGetLastError());
  }
  // One small matrix (the Davidson subspace problem): one CTA.  A batch (the
  // density-matrix sectors of a decimation): cooperative launches of one CTA
  // per SM (the shared memory of the n <= kSmemN path admits one CTA per SM),
  // largest matrices first, group sizes from jac_assign_groups.
  bool jac_init = false;
  int jac_cap = 0;
  void eigh(const std::vector<EighTask>& tasks) override {
    if (tasks.empty()) return;
    const size_t smem = jacobi_smem_bytes(kSmemN);
    if (!jac_init) {
      CK(cudaFuncSetAttribute(jacobi_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      CK(cudaFuncSetAttribute(jacobi_coop_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      int per_sm = 0, sms = 0;
      CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_coop_kernel, kJacThreads, smem));
      CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
      jac_cap = per_sm * sms;
      if (jac_cap < 2) throw std::runtime_error("cuda: eigensolver needs two co-resident CTAs");
      jac_init = true;
    }
    if (tasks.size() == 1 && tasks[0].n <= kSmemN) {
      std::vector<size_t> off;
      char* d = upload({{tasks.data(), sizeof(EighTask)}}, off);
      Rec* rec = nullptr;
      if (profiling) {
        recs.push_back(Rec{ev(), ev(), 0.0, 3});
        rec = &recs.back();
        CK(cudaEventRecord(rec->a, st));
      }
      jacobi_smem_kernel<<<1, 256, jacobi_smem_bytes(tasks[0].n), st>>>((const EighTask*)(d + off[0]));
      if (rec) CK(cudaEventRecord(rec->b, st));
      ++launches;
      CK(cudaGetLastError());
      return;
    }
    std::vector<EighTask> order(tasks);
    std::stable_sort(order.begin(), order.end(), [](const EighTask& x, const EighTask& y) { return x.n > y.n; });
    std::vector<int> n_desc;
    for (auto& t : order) n_desc.push_back(t.n);
    for (const JacBatch& jb : jac_plan_batches(n_desc, jac_cap)) {
      std::vector<CoopEigh> ct;
      int ctas = 0;
      for (size_t k = jb.begin; k < jb.end; ++k) {
        ct.push_back({order[k], jb.g[k - jb.begin], ctas, nullptr});
        ctas += jb.g[k - jb.begin];
      }
      std::vector<unsigned> bars(2 * ct.size(), 0u);
      std::vector<size_t> off;
      char* d = upload({{ct.data(), ct.size() * sizeof(CoopEigh)}, {bars.data(), bars.size() * sizeof(unsigned)}},
                       off);
      unsigned* dbar = (unsigned*)(d + off[1]);
      for (size_t k = 0; k < ct.size(); ++k) ct[k].bar = dbar + 2 * k;
      CK(cudaMemcpyAsync(d + off[0], ct.data(), ct.size() * sizeof(CoopEigh), cudaMemcpyHostToDevice, st));
      const CoopEigh* dt = (const CoopEigh*)(d + off[0]);
      int nt = (int)ct.size();
      int* fl = flag();
      unsigned long long wns = wait_ns_;
      void* args[] = {(void*)&dt, (void*)&nt, (void*)&fl, (void*)&wns};
      Rec* rec = nullptr;
      if (profiling) {
        recs.push_back(Rec{ev(), ev(), 0.0, 4});
        rec = &recs.back();
        CK(cudaEventRecord(rec->a, st));
      }
      CK(cudaLaunchCooperativeKernel((const void*)jacobi_coop_kernel, dim3(ctas), dim3(kJacThreads), args, smem, st));
      if (rec) CK(cudaEventRecord(rec->b, st));
      ++launches;
    }
  }
};

Backend* make_cuda_backend(int device, std::string* err) {
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess || count == 0) {
    if (err) *err = std::string("cuda: no usable device (") + cudaGetErrorString(e) + ")";
    cudaGetLastError();
    return nullptr;
  }
  if (device < 0 || device >= count) {
    if (err) *err = "cuda: device ordinal out of range";
    return nullptr;
  }
  try {
    return new CudaBackend(device);
  } catch (const std::exception& ex) {
    if (err) *err = ex.what();
    return nullptr;
  }
}

}  // namespace dmrg
