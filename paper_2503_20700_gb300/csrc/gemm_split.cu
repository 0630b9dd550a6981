// 3xTF32 grouped GEMM on the warp-level tensor-core path (mma.sync m16n8k8).
#include <stdexcept>
#include <string>

#include "gemm_split.cuh"

namespace dmrg {

namespace {

constexpr int SM = 64, SN = 64, SK = 16;

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// split a float64 into two TF32 words: hi = tf32(x), lo = tf32(x - hi)
__device__ __forceinline__ void split(double x, uint32_t& hi, uint32_t& lo) {
  float xf = (float)x;
  hi = to_tf32(xf);
  double r = x - (double)__uint_as_float(hi);
  lo = to_tf32((float)r);
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// 256 threads = 8 warps as 4 (M) x 2 (N); a warp owns 16 x 32 of the 64 x 64 tile.
__global__ void __launch_bounds__(256) gemm_tf32x3_mma(const GemmGroup* __restrict__ groups,
                                                       const GemmSeg* __restrict__ segs,
                                                       const SplitTile* __restrict__ tiles) {
  __shared__ uint32_t Ah[SM][SK + 4], Al[SM][SK + 4];
  __shared__ uint32_t Bh[SN][SK + 4], Bl[SN][SK + 4];  // B stored n-major: Bs[n][k]
  const SplitTile t = tiles[blockIdx.x];
  const GemmGroup g = groups[t.group];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = warp & 3, wn = warp >> 2;
  const int gid = lane >> 2, tig = lane & 3;
  double acc64[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc64[i][j] = 0.0;
  for (int s = g.seg_begin; s < g.seg_begin + g.seg_count; ++s) {
    const GemmSeg sg = segs[s];
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
    for (int k0 = 0; k0 < sg.k; k0 += SK) {
      for (int e = threadIdx.x; e < SM * SK; e += 256) {
        int i, kk;
        if (!sg.transA) { i = e / SK; kk = e % SK; }
        else { kk = e / SM; i = e % SM; }
        int gi = t.r0 + i, gk = k0 + kk;
        double v = 0.0;
        if (gi < g.m && gk < sg.k)
          v = sg.transA ? sg.A[(size_t)gk * sg.lda + gi] : sg.A[(size_t)gi * sg.lda + gk];
        uint32_t h, l;
        split(sg.alpha * v, h, l);
        Ah[i][kk] = h;
        Al[i][kk] = l;
      }
      for (int e = threadIdx.x; e < SN * SK; e += 256) {
        int j, kk;
        if (!sg.transB) { kk = e / SN; j = e % SN; }
        else { j = e / SK; kk = e % SK; }
        int gj = t.c0 + j, gk = k0 + kk;
        double v = 0.0;
        if (gj < g.n && gk < sg.k)
          v = sg.transB ? sg.B[(size_t)gj * sg.ldb + gk] : sg.B[(size_t)gk * sg.ldb + gj];
        uint32_t h, l;
        split(v, h, l);
        Bh[j][kk] = h;
        Bl[j][kk] = l;
      }
      __syncthreads();
#pragma unroll
      for (int ks = 0; ks < SK; ks += 8) {
        uint32_t ah[4], al[4];
        const int r = wm * 16 + gid;
        ah[0] = Ah[r][ks + tig];
        ah[1] = Ah[r + 8][ks + tig];
        ah[2] = Ah[r][ks + tig + 4];
        ah[3] = Ah[r + 8][ks + tig + 4];
        al[0] = Al[r][ks + tig];
        al[1] = Al[r + 8][ks + tig];
        al[2] = Al[r][ks + tig + 4];
        al[3] = Al[r + 8][ks + tig + 4];
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          const int c = wn * 32 + nt * 8 + gid;
          uint32_t bh[2] = {Bh[c][ks + tig], Bh[c][ks + tig + 4]};
          uint32_t bl[2] = {Bl[c][ks + tig], Bl[c][ks + tig + 4]};
          mma_tf32(acc[nt], al, bh);
          mma_tf32(acc[nt], ah, bl);
          mma_tf32(acc[nt], ah, bh);
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc64[nt][q] += (double)acc[nt][q];
  }
  // C fragment: c0 (gid, 2tig), c1 (gid, 2tig+1), c2 (gid+8, 2tig), c3 (gid+8, 2tig+1)
#pragma unroll
  for (int nt = 0; nt < 4; ++nt)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int gi = t.r0 + wm * 16 + gid + ((q >> 1) ? 8 : 0);
      int gj = t.c0 + wn * 32 + nt * 8 + 2 * tig + (q & 1);
      if (gi < g.m && gj < g.n) g.C[(size_t)gi * g.ldc + gj] += acc64[nt][q];
    }
}

}  // namespace

void gemm_split_launch(const std::vector<GemmGroup>& groups, const std::vector<GemmSeg>& segs,
                       Precision prec, cudaStream_t st, const UploadFn& upload) {
  if (prec != Precision::SPLIT_TF32) throw std::invalid_argument("unsupported precision");
  std::vector<SplitTile> tiles;
  for (size_t gi = 0; gi < groups.size(); ++gi) {
    auto& g = groups[gi];
    for (int r = 0; r < g.m; r += SM)
      for (int c = 0; c < g.n; c += SN) tiles.push_back({(int)gi, r, c, 0});
  }
  if (tiles.empty()) return;
  std::vector<size_t> off;
  char* d = upload({{groups.data(), groups.size() * sizeof(GemmGroup)},
                    {segs.data(), segs.size() * sizeof(GemmSeg)},
                    {tiles.data(), tiles.size() * sizeof(SplitTile)}},
                   off);
  gemm_tf32x3_mma<<<(unsigned)tiles.size(), 256, 0, st>>>((const GemmGroup*)(d + off[0]),
                                                          (const GemmSeg*)(d + off[1]),
                                                          (const SplitTile*)(d + off[2]));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw std::runtime_error(std::string("cuda: split gemm launch: ") + cudaGetErrorString(e));
}

}  // namespace dmrg
