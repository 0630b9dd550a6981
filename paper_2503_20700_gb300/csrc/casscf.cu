// CAS-SCF side of the hot path (Sec. II.A): orbital rotation U = exp(-kappa),
// integral transformation in Cholesky form, the active-space problem handed to
// DMRG, and the orbital gradient from the one- and two-particle RDMs.
//
// Everything runs on the device in float64.  The contractions over the
// Cholesky index go through the grouped segment-sum GEMM of the backend; the
// small elementwise / reduction steps are the kernels below.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "backend.hpp"
#include "casscf.hpp"

namespace dmrg {

namespace {

// v[k] = sum_{i<ncore} L[k,i,i];  w[k] = sum_{t,u} gamma[t,u] L[k,c+t,c+u]
__global__ void k_diag_contract(const double* __restrict__ L, int nb, int ncore, int ncas,
                                const double* __restrict__ gamma, double* __restrict__ v,
                                double* __restrict__ w) {
  const int k = blockIdx.x;
  const double* Lk = L + (size_t)k * nb * nb;
  __shared__ double s1[256], s2[256];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < ncore; i += blockDim.x) a += Lk[(size_t)i * nb + i];
  if (gamma)
    for (int e = threadIdx.x; e < ncas * ncas; e += blockDim.x) {
      int t = e / ncas, u = e % ncas;
      b += gamma[e] * Lk[(size_t)(ncore + t) * nb + ncore + u];
    }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) {
      s1[threadIdx.x] += s1[threadIdx.x + st];
      s2[threadIdx.x] += s2[threadIdx.x + st];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    v[k] = s1[0];
    if (w) w[k] = s2[0];
  }
}

// gather the active block of every Cholesky vector: La[k, t*ncas+u] = L[k, c+t, c+u]
__global__ void k_gather_active(const double* __restrict__ L, int rank, int nb, int ncore, int ncas,
                                double* __restrict__ La) {
  size_t tot = (size_t)rank * ncas * ncas;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (size_t)gridDim.x * blockDim.x) {
    size_t k = e / ((size_t)ncas * ncas);
    int r = (int)(e % ((size_t)ncas * ncas));
    int t = r / ncas, u = r % ncas;
    La[e] = L[(k * nb + ncore + t) * nb + ncore + u];
  }
}

// d[t,u,v,w] = Gamma[t,v,w,u] (paper operator order -> chemists' order)
__global__ void k_permute_rdm2(const double* __restrict__ G, int n, double* __restrict__ d) {
  size_t tot = (size_t)n * n * n * n;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (size_t)gridDim.x * blockDim.x) {
    size_t r = e;
    int w = (int)(r % n); r /= n;
    int v = (int)(r % n); r /= n;
    int u = (int)(r % n); r /= n;
    int t = (int)r;
    d[e] = G[(((size_t)t * n + v) * n + w) * n + u];
  }
}

// out = a*X + b*Y + c*Z elementwise (any pointer may be null)
__global__ void k_axpbypcz(double* __restrict__ out, size_t len, double a, const double* X, double b,
                           const double* Y, double c, const double* Z) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < len;
       e += (size_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    if (X) s += a * X[e];
    if (Y) s += b * Y[e];
    if (Z) s += c * Z[e];
    out[e] = s;
  }
}

// generalised Fock F (nb x nb) from its pieces; rows: core, active, virtual
//   F[i,q] = 2 (FI[q,i] + FA[q,i]);  F[t,q] = sum_u gamma[t,u] FI[q,c+u] + F2[t,q];  F[a,q] = 0
__global__ void k_assemble_fock(const double* __restrict__ FI, const double* __restrict__ FA,
                                const double* __restrict__ gamma, const double* __restrict__ F2,
                                int nb, int ncore, int ncas, double* __restrict__ F) {
  size_t tot = (size_t)nb * nb;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (size_t)gridDim.x * blockDim.x) {
    int p = (int)(e / nb), q = (int)(e % nb);
    double v = 0.0;
    if (p < ncore) {
      v = 2.0 * (FI[(size_t)q * nb + p] + FA[(size_t)q * nb + p]);
    } else if (p < ncore + ncas) {
      int t = p - ncore;
      for (int u = 0; u < ncas; ++u) v += gamma[(size_t)t * ncas + u] * FI[(size_t)q * nb + ncore + u];
      v += F2[(size_t)t * nb + q];
    }
    F[e] = v;
  }
}

// grad = 2 (F - F^T) with the active-active block zeroed
__global__ void k_gradient(const double* __restrict__ F, int nb, int ncore, int ncas,
                           double* __restrict__ g) {
  size_t tot = (size_t)nb * nb;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (size_t)gridDim.x * blockDim.x) {
    int p = (int)(e / nb), q = (int)(e % nb);
    bool aa = p >= ncore && p < ncore + ncas && q >= ncore && q < ncore + ncas;
    g[e] = aa ? 0.0 : 2.0 * (F[e] - F[(size_t)q * nb + p]);
  }
}

// e = sum_i (h[i,i] + FI[i,i]) over core orbitals (single block)
__global__ void k_core_energy(const double* __restrict__ h, const double* __restrict__ FI, int nb,
                              int ncore, double* __restrict__ e) {
  __shared__ double s[256];
  double a = 0.0;
  for (int i = threadIdx.x; i < ncore; i += blockDim.x) a += h[(size_t)i * nb + i] + FI[(size_t)i * nb + i];
  s[threadIdx.x] = a;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) s[threadIdx.x] += s[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) *e = s[0];
}

// copy a sub-block: out[r*lo + c] = in[(r0+r)*li + c0 + c]
__global__ void k_subblock(const double* __restrict__ in, int li, int r0, int c0, int rows, int cols,
                           double* __restrict__ out, int lo) {
  size_t tot = (size_t)rows * cols;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (size_t)gridDim.x * blockDim.x) {
    int r = (int)(e / cols), c = (int)(e % cols);
    out[(size_t)r * lo + c] = in[(size_t)(r0 + r) * li + c0 + c];
  }
}

// A[i,i] += s
__global__ void k_add_diag(double* A, int n, double s) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    A[(size_t)i * n + i] += s;
}

// out[0] = max_c sum_r |A[r, c]| (1-norm; single block)
__global__ void k_norm1(const double* __restrict__ A, int n, double* __restrict__ out) {
  __shared__ double s[256];
  double m = 0.0;
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    double a = 0.0;
    for (int r = 0; r < n; ++r) a += fabs(A[(size_t)r * n + c]);
    m = fmax(m, a);
  }
  s[threadIdx.x] = m;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) s[threadIdx.x] = fmax(s[threadIdx.x], s[threadIdx.x + st]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

// B (2n x 2n) = [[K, G], [0, K]]
__global__ void k_block_upper(const double* __restrict__ K, const double* __restrict__ G, int n,
                              double* __restrict__ B) {
  const size_t m = 2 * (size_t)n, tot = m * m;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / m), c = (int)(e % m);
    double v = 0.0;
    if (r < n && c < n) v = K[(size_t)r * n + c];
    else if (r >= n && c >= n) v = K[(size_t)(r - n) * n + (c - n)];
    else if (r < n && c >= n) v = G[(size_t)r * n + (c - n)];
    B[e] = v;
  }
}

// dK[r, c] = scale * (L[c, r] - L[r, c]) with L the upper-right block of E (2n x 2n)
__global__ void k_antisym_from_upper(const double* __restrict__ E, int n, double scale, double* __restrict__ dK) {
  const size_t tot = (size_t)n * n, m = 2 * (size_t)n;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / n), c = (int)(e % n);
    dK[e] = scale * (E[(size_t)c * m + r + n] - E[(size_t)r * m + c + n]);
  }
}

// Upstream weights of the active-space functional to RDM-shaped inputs of the
// generalised Fock matrix: gamma = sym(g_h) / c, and Gamma[t,v,w,u] =
// (2 / c) * (8-fold average of g_eri)[t,u,v,w] (E holds 1/2 (tu|vw) Gamma_tvwu)
__global__ void k_weights_to_rdms(const double* __restrict__ gh, const double* __restrict__ ge, int n, double c,
                                  double* __restrict__ gamma, double* __restrict__ Gamma) {
  const size_t n2 = (size_t)n * n, tot = n2 * n2;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    size_t q = e;
    const int w = (int)(q % n); q /= n;
    const int v = (int)(q % n); q /= n;
    const int u = (int)(q % n); q /= n;
    const int t = (int)q;
    auto at = [&](int a, int b, int cc, int d) { return ge[(((size_t)a * n + b) * n + cc) * n + d]; };
    const double sym = (at(t, u, v, w) + at(u, t, v, w) + at(t, u, w, v) + at(u, t, w, v) + at(v, w, t, u) +
                        at(w, v, t, u) + at(v, w, u, t) + at(w, v, u, t)) / 8.0;
    Gamma[(((size_t)t * n + v) * n + w) * n + u] = (2.0 / c) * sym;
    if (v == 0 && w == 0) gamma[(size_t)t * n + u] = 0.5 * (gh[(size_t)t * n + u] + gh[(size_t)u * n + t]) / c;
  }
}

// mask[p, q] = 1 for the non-redundant rotations p > q between different
// orbital classes (core, active, virtual), else 0
__global__ void k_rotation_mask(int nb, int ncore, int ncas, double* __restrict__ m) {
  const size_t tot = (size_t)nb * nb;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(e / nb), q = (int)(e % nb);
    const int cp = p < ncore ? 0 : (p < ncore + ncas ? 1 : 2), cq = q < ncore ? 0 : (q < ncore + ncas ? 1 : 2);
    m[e] = (p > q && cp != cq) ? 1.0 : 0.0;
  }
}

__global__ void k_mul(const double* __restrict__ a, const double* __restrict__ b, size_t n, double* __restrict__ out) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    out[e] = a[e] * b[e];
}

// out[0] = max |a| (single block)
__global__ void k_maxabs(const double* __restrict__ a, size_t n, double* __restrict__ out) {
  __shared__ double s[256];
  double m = 0.0;
  for (size_t e = threadIdx.x; e < n; e += blockDim.x) m = fmax(m, fabs(a[e]));
  s[threadIdx.x] = m;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) s[threadIdx.x] = fmax(s[threadIdx.x], s[threadIdx.x + st]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

// r = mask ? q / h : 0  (h > 0 by the floor)
__global__ void k_div_mask(const double* __restrict__ q, const double* __restrict__ h, const double* __restrict__ m,
                           size_t n, double* __restrict__ r) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    r[e] = (m[e] != 0.0 && h[e] > 0.0) ? q[e] / h[e] : 0.0;
}

// K = x - x^T
__global__ void k_antisym(const double* __restrict__ x, int nb, double* __restrict__ K) {
  const size_t tot = (size_t)nb * nb;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(e / nb), q = (int)(e % nb);
    K[e] = x[e] - x[(size_t)q * nb + p];
  }
}

// fd[p] = F^I_pp + F^A_pp (FA may be null)
__global__ void k_fock_diag(const double* __restrict__ FI, const double* __restrict__ FA, int nb, double* __restrict__ fd) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nb; p += gridDim.x * blockDim.x)
    fd[p] = FI[(size_t)p * nb + p] + (FA ? FA[(size_t)p * nb + p] : 0.0);
}

// Approximate diagonal orbital Hessian of the closed-shell-core CAS-SCF
// energy for the rotations p > q, floored: virtual-core 4 (f_p - f_q),
// virtual-active 2 n_t f_p - 2 F_tt, active-core 4 (f_p - f_q) + 2 n_t f_q -
// 2 F_tt (f = F^I + F^A, n_t = gamma~_tt, F the generalised Fock matrix)
__global__ void k_diag_hessian(const double* __restrict__ f, const double* __restrict__ F,
                               const double* __restrict__ gamma, int nb, int ncore, int ncas, double floor_v,
                               double* __restrict__ H) {
  const size_t tot = (size_t)nb * nb;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(e / nb), q = (int)(e % nb);
    const bool pc = p < ncore, pa = p >= ncore && p < ncore + ncas;
    const bool qc = q < ncore, qa = q >= ncore && q < ncore + ncas;
    double v = 0.0;
    bool set = false;
    if (p > q && !pc && !(pa && qa)) {
      if (!pa && qc) {
        v = 4.0 * (f[p] - f[q]);
        set = true;
      } else if (!pa && qa) {
        const int t = q - ncore;
        v = 2.0 * gamma[(size_t)t * ncas + t] * f[p] - 2.0 * F[(size_t)q * nb + q];
        set = true;
      } else if (pa && qc) {
        const int t = p - ncore;
        v = 4.0 * (f[p] - f[q]) + 2.0 * gamma[(size_t)t * ncas + t] * f[q] - 2.0 * F[(size_t)p * nb + p];
        set = true;
      }
    }
    H[e] = set ? fmax(v, floor_v) : 0.0;
  }
}

#define ST ((cudaStream_t)be_->stream())
int grid_for(size_t n) { return (int)std::min<size_t>(152 * 16, std::max<size_t>(1, (n + 255) / 256)); }

}  // namespace

// ---------------------------------------------------------------- helpers
struct Casscf::Dev {
  Backend* be;
  std::vector<void*> mem;
  explicit Dev(Backend* b) : be(b) {}
  ~Dev() {
    be->sync();
    for (void* p : mem) be->free(p);
  }
  double* alloc(size_t n) {
    double* p = (double*)be->alloc(std::max<size_t>(n, 1) * sizeof(double));
    be->memset0(p, std::max<size_t>(n, 1) * sizeof(double));
    mem.push_back(p);
    return p;
  }
  double* upload(const double* h, size_t n) {
    double* p = alloc(n);
    be->copy_h2d(p, h, n * sizeof(double));
    return p;
  }
};

static void gemm1(Backend* be, double* C, int m, int n, int ldc, const double* A, int lda, int ta,
                  const double* B, int ldb, int tb, int k, double alpha) {
  std::vector<GemmGroup> g{{C, m, n, ldc, 0, 1}};
  std::vector<GemmSeg> s{{A, B, k, lda, ldb, ta, tb, alpha}};
  be->gemm(g, s, Precision::FP64);
}

Casscf::Casscf(Backend* be) : be_(be) {}

// R = expm(-K): scaling and squaring with a degree-18 Taylor polynomial
// (Horner form) of the scaled matrix.
void Casscf::expm_neg(const double* dK, int n, double* dR, double sign) {
  // 1-norm on the device; the number of squarings makes the scaled
  // argument's norm at most 1/4
  double nrm = 0.0;
  {
    Dev d0(be_);
    double* dn = d0.alloc(1);
    k_norm1<<<1, 256, 0, ST>>>(dK, n, dn);
    be_->copy_d2h(&nrm, dn, sizeof(double));
    be_->sync();
  }
  int sq = 0;
  while (nrm / std::ldexp(1.0, sq) > 0.25 && sq < 60) ++sq;
  double scale = sign / std::ldexp(1.0, sq);
  Dev d(be_);
  double* X = d.alloc((size_t)n * n);
  double* T = d.alloc((size_t)n * n);
  k_axpbypcz<<<grid_for((size_t)n * n), 256, 0, ST>>>(X, (size_t)n * n, scale, dK, 0, nullptr, 0, nullptr);
  // Horner: P = I + X/18;  P = I + X P / j  for j = 17 .. 1
  const int deg = 18;
  be_->memset0(dR, (size_t)n * n * sizeof(double));
  k_add_diag<<<grid_for(n), 256, 0, ST>>>(dR, n, 1.0);
  for (int j = deg; j >= 1; --j) {
    be_->memset0(T, (size_t)n * n * sizeof(double));
    gemm1(be_, T, n, n, n, X, n, 0, dR, n, 0, n, 1.0 / j);
    k_add_diag<<<grid_for(n), 256, 0, ST>>>(T, n, 1.0);
    be_->copy_d2d(dR, T, (size_t)n * n * sizeof(double));
  }
  for (int s = 0; s < sq; ++s) {
    be_->memset0(T, (size_t)n * n * sizeof(double));
    gemm1(be_, T, n, n, n, dR, n, 0, dR, n, 0, n, 1.0);
    be_->copy_d2d(dR, T, (size_t)n * n * sizeof(double));
  }
  be_->sync();
}

void Casscf::matmul(const double* A, const double* B, int n, double* C) {
  Dev d(be_);
  const size_t nn = (size_t)n * n;
  double* dA = d.upload(A, nn);
  double* dB = d.upload(B, nn);
  double* dC = d.alloc(nn);
  gemm1(be_, dC, n, n, n, dA, n, 0, dB, n, 0, n, 1.0);
  be_->copy_d2h(C, dC, nn * sizeof(double));
}

void Casscf::rotation(const double* K, int nb, double* R) {
  Dev d(be_);
  double* dK = d.upload(K, (size_t)nb * nb);
  double* dR = d.alloc((size_t)nb * nb);
  expm_neg(dK, nb, dR, -1.0);
  be_->copy_d2h(R, dR, (size_t)nb * nb * sizeof(double));
}

// dE/dK for R = expm(-K) given G = dE/dR: with X = -K, dE/dX = L_exp(X^T, G)
// = upper-right block of expm([[K, G], [0, K]]) (X^T = K for antisymmetric K),
// so dE/dK = -L and the parameter gradient is antisymmetrised.
void Casscf::rotation_backward_dev(const double* dKin, const double* dG, int nb, double scale, double* ddK) {
  const size_t n2 = 2 * (size_t)nb;
  Dev d(be_);
  double* dB = d.alloc(n2 * n2);
  double* dE = d.alloc(n2 * n2);
  k_block_upper<<<grid_for(n2 * n2), 256, 0, ST>>>(dKin, dG, nb, dB);
  expm_neg(dB, (int)n2, dE, 1.0);
  // dK = -(L - L^T) with L = dE/dX = upper-right block (X = -K, X^T = K)
  k_antisym_from_upper<<<grid_for((size_t)nb * nb), 256, 0, ST>>>(dE, nb, scale, ddK);
  be_->sync();
}

void Casscf::rotation_backward(const double* K, const double* G, int nb, double* dK) {
  Dev d(be_);
  const size_t nn = (size_t)nb * nb;
  double* dKin = d.upload(K, nn);
  double* dG = d.upload(G, nn);
  double* dout = d.alloc(nn);
  rotation_backward_dev(dKin, dG, nb, 1.0, dout);
  be_->copy_d2h(dK, dout, nn * sizeof(double));
}

// h' = R^T h R and L'^k = R^T L^k R (batched over the Cholesky index)
void Casscf::transform(const double* R, const double* h, const double* L, int rank, int nb,
                       double* h_out, double* L_out) {
  Dev d(be_);
  size_t nn = (size_t)nb * nb;
  double* dR = d.upload(R, nn);
  double* dh = d.upload(h, nn);
  double* dL = d.upload(L, nn * rank);
  double* T = d.alloc(nn * (rank + 1));
  double* out = d.alloc(nn * (rank + 1));
  std::vector<GemmGroup> g1, g2;
  std::vector<GemmSeg> s1, s2;
  for (int k = 0; k <= rank; ++k) {
    const double* Mk = (k == 0) ? dh : dL + nn * (k - 1);
    g1.push_back({T + nn * k, nb, nb, nb, (int)s1.size(), 1});
    s1.push_back({Mk, dR, nb, nb, nb, 0, 0, 1.0});
    g2.push_back({out + nn * k, nb, nb, nb, (int)s2.size(), 1});
    s2.push_back({dR, T + nn * k, nb, nb, nb, 1, 0, 1.0});
  }
  be_->gemm(g1, s1, Precision::FP64);
  be_->gemm(g2, s2, Precision::FP64);
  be_->copy_d2h(h_out, out, nn * sizeof(double));
  be_->copy_d2h(L_out, out + nn, nn * rank * sizeof(double));
}

// Pieces shared by the active-space problem and the gradient.
struct FockParts {
  double *FI, *FA, *La, *v, *w;
};

static FockParts fock_parts(Backend* be, Casscf::Dev& d, const double* dh, const double* dL, int rank,
                            int nb, int ncore, int ncas, const double* dgamma) {
  size_t nn = (size_t)nb * nb;
  Backend* be_ = be;  // stream of the launches below
  FockParts f{};
  f.v = d.alloc(rank);
  f.w = d.alloc(rank);
  k_diag_contract<<<rank, 256, 0, ST>>>(dL, nb, ncore, ncas, dgamma, f.v, f.w);
  // J = sum_k v_k L^k  (1 x rank) x (rank x nb^2)
  double* J = d.alloc(nn);
  gemm1(be, J, 1, (int)nn, (int)nn, f.v, rank, 0, dL, (int)nn, 0, rank, 1.0);
  // Kc = sum_k L^k[:, core] L^k[core, :]
  double* Kc = d.alloc(nn);
  if (ncore > 0) {
    std::vector<GemmGroup> g{{Kc, nb, nb, nb, 0, rank}};
    std::vector<GemmSeg> s;
    for (int k = 0; k < rank; ++k) s.push_back({dL + nn * k, dL + nn * k, ncore, nb, nb, 0, 0, 1.0});
    be->gemm(g, s, Precision::FP64);
  }
  f.FI = d.alloc(nn);
  k_axpbypcz<<<grid_for(nn), 256, 0, ST>>>(f.FI, nn, 1.0, dh, 2.0, J, -1.0, Kc);
  f.FA = nullptr;
  if (dgamma) {
    double* JA = d.alloc(nn);
    gemm1(be, JA, 1, (int)nn, (int)nn, f.w, rank, 0, dL, (int)nn, 0, rank, 1.0);
    // M^k = L^k[:, act] gamma ; KA = sum_k M^k L^k[act, :]
    double* M = d.alloc((size_t)rank * nb * ncas);
    std::vector<GemmGroup> g1;
    std::vector<GemmSeg> s1;
    for (int k = 0; k < rank; ++k) {
      g1.push_back({M + (size_t)k * nb * ncas, nb, ncas, ncas, (int)s1.size(), 1});
      s1.push_back({dL + nn * k + ncore, dgamma, ncas, nb, ncas, 0, 0, 1.0});
    }
    be->gemm(g1, s1, Precision::FP64);
    double* KA = d.alloc(nn);
    std::vector<GemmGroup> g2{{KA, nb, nb, nb, 0, rank}};
    std::vector<GemmSeg> s2;
    for (int k = 0; k < rank; ++k)
      s2.push_back({M + (size_t)k * nb * ncas, dL + nn * k + (size_t)ncore * nb, ncas, ncas, nb, 0, 0, 1.0});
    be->gemm(g2, s2, Precision::FP64);
    f.FA = d.alloc(nn);
    k_axpbypcz<<<grid_for(nn), 256, 0, ST>>>(f.FA, nn, 1.0, JA, -0.5, KA, 0.0, nullptr);
  }
  f.La = d.alloc((size_t)rank * ncas * ncas);
  k_gather_active<<<grid_for((size_t)rank * ncas * ncas), 256, 0, ST>>>(dL, rank, nb, ncore, ncas, f.La);
  return f;
}

void Casscf::active_space(const double* h, const double* L, int rank, int nb, int ncore, int ncas,
                          double* e_core, double* h_act, double* eri_act) {
  Dev d(be_);
  size_t nn = (size_t)nb * nb;
  double* dh = d.upload(h, nn);
  double* dL = d.upload(L, nn * rank);
  FockParts f = fock_parts(be_, d, dh, dL, rank, nb, ncore, ncas, nullptr);
  double* de = d.alloc(1);
  k_core_energy<<<1, 256, 0, ST>>>(dh, f.FI, nb, ncore, de);
  double* ha = d.alloc((size_t)ncas * ncas);
  k_subblock<<<grid_for((size_t)ncas * ncas), 256, 0, ST>>>(f.FI, nb, ncore, ncore, ncas, ncas, ha, ncas);
  // (tu|vw) = sum_k La[k,tu] La[k,vw]
  int a2 = ncas * ncas;
  double* eri = d.alloc((size_t)a2 * a2);
  gemm1(be_, eri, a2, a2, a2, f.La, a2, 1, f.La, a2, 0, rank, 1.0);
  be_->copy_d2h(e_core, de, sizeof(double));
  be_->copy_d2h(h_act, ha, (size_t)ncas * ncas * sizeof(double));
  be_->copy_d2h(eri_act, eri, (size_t)a2 * a2 * sizeof(double));
}

void Casscf::gradient(const double* h, const double* L, int rank, int nb, int ncore, int ncas,
                      const double* gamma, const double* Gamma, double* grad, double* fock) {
  Dev d(be_);
  size_t nn = (size_t)nb * nb;
  int a2 = ncas * ncas;
  double* dh = d.upload(h, nn);
  double* dL = d.upload(L, nn * rank);
  double* dg = d.upload(gamma, (size_t)a2);
  double* dG = d.upload(Gamma, (size_t)a2 * a2);
  double* F = d.alloc(nn);
  fock_dev(dh, dL, rank, nb, ncore, ncas, dg, dG, F);
  double* dgr = d.alloc(nn);
  k_gradient<<<grid_for(nn), 256, 0, ST>>>(F, nb, ncore, ncas, dgr);
  be_->copy_d2h(grad, dgr, nn * sizeof(double));
  if (fock) be_->copy_d2h(fock, F, nn * sizeof(double));
}

// Backward of (e_core, h_act, eri_act) = active_space(transform(expm(-K), h, L))
// for upstream weights (c, g_h, g_eri): the weighted sum is a CAS-SCF energy
// functional with RDMs (g_h / c, 2 g_eri / c), whose derivative with respect
// to the rotated orbitals is 2 R F^T (F its generalised Fock matrix); the
// core part of F scales with c, so for c = 0 the functional is evaluated with
// c = 1 and the pure-core F(0, 0) subtracted.  The adjoint Frechet derivative
// of expm carries dE/dR to K; half of it is the gradient with respect to the
// full antisymmetric input matrix.
void Casscf::transform_backward(const double* K, const double* R, const double* h, const double* L, int rank,
                                int nb, int ncore, int ncas, double g_core, const double* g_h,
                                const double* g_eri, double* dK) {
  Dev d(be_);
  const size_t nn = (size_t)nb * nb;
  const int a2 = ncas * ncas;
  double* dKin = d.upload(K, nn);
  double* dR = d.upload(R, nn);
  double* dh = d.upload(h, nn);
  double* dL = d.upload(L, nn * rank);
  double* dgh = d.upload(g_h, (size_t)a2);
  double* dge = d.upload(g_eri, (size_t)a2 * a2);
  const double c_eff = g_core != 0.0 ? g_core : 1.0;
  double* dgam = d.alloc((size_t)a2);
  double* dGam = d.alloc((size_t)a2 * a2);
  k_weights_to_rdms<<<grid_for((size_t)a2 * a2), 256, 0, ST>>>(dgh, dge, ncas, c_eff, dgam, dGam);
  double* F = d.alloc(nn);
  fock_dev(dh, dL, rank, nb, ncore, ncas, dgam, dGam, F);
  double* Ft = d.alloc(nn);
  if (g_core != 0.0) {
    k_axpbypcz<<<grid_for(nn), 256, 0, ST>>>(Ft, nn, g_core, F, 0.0, nullptr, 0.0, nullptr);
  } else {
    double* z1 = d.alloc((size_t)a2);
    double* z2 = d.alloc((size_t)a2 * a2);
    double* F0 = d.alloc(nn);
    fock_dev(dh, dL, rank, nb, ncore, ncas, z1, z2, F0);
    k_axpbypcz<<<grid_for(nn), 256, 0, ST>>>(Ft, nn, 1.0, F, -1.0, F0, 0.0, nullptr);
  }
  // G = dE/dR = 2 R Ft^T
  double* G = d.alloc(nn);
  gemm1(be_, G, nb, nb, nb, dR, nb, 0, Ft, nb, 1, nb, 2.0);
  double* out = d.alloc(nn);
  rotation_backward_dev(dKin, G, nb, 0.5, out);
  be_->copy_d2h(dK, out, nn * sizeof(double));
}

// generalised Fock matrix F (device, nb x nb) from device integrals and RDMs
void Casscf::fock_dev(const double* dh, const double* dL, int rank, int nb, int ncore, int ncas,
                      const double* dg, const double* dG, double* F, double* fdiag) {
  Dev d(be_);
  size_t nn = (size_t)nb * nb;
  int a2 = ncas * ncas;
  FockParts f = fock_parts(be_, d, dh, dL, rank, nb, ncore, ncas, dg);
  // d[t,u,v,w] = Gamma[t,v,w,u];  W (rank x a2) = La (rank x a2) d^T (a2 x a2)
  double* dd = d.alloc((size_t)a2 * a2);
  k_permute_rdm2<<<grid_for((size_t)a2 * a2), 256, 0, ST>>>(dG, ncas, dd);
  double* W = d.alloc((size_t)rank * a2);
  gemm1(be_, W, rank, a2, a2, f.La, a2, 0, dd, a2, 1, a2, 1.0);
  // F2[t, q] = sum_k sum_u W^k[t,u] L^k[q, c+u]
  double* F2 = d.alloc((size_t)ncas * nb);
  std::vector<GemmGroup> g{{F2, ncas, nb, nb, 0, rank}};
  std::vector<GemmSeg> s;
  for (int k = 0; k < rank; ++k)
    s.push_back({W + (size_t)k * a2, dL + nn * k + ncore, ncas, ncas, nb, 0, 1, 1.0});
  be_->gemm(g, s, Precision::FP64);
  k_assemble_fock<<<grid_for(nn), 256, 0, ST>>>(f.FI, f.FA, dg, F2, nb, ncore, ncas, F);
  if (fdiag) k_fock_diag<<<grid_for(nb), 256, 0, ST>>>(f.FI, f.FA, nb, fdiag);
  be_->sync();
}

// ---------------------------------------------------------------- DMRG-SCF step
ScfStepper::ScfStepper(Backend* be, int nb, int ncore, int ncas, int memory, double max_step)
    : be_(be), nb_(nb), ncore_(ncore), ncas_(ncas), memory_(std::max(0, memory)), max_step_(max_step) {
  const size_t nn = (size_t)nb * nb;
  auto al = [&](size_t n) {
    double* p = (double*)be_->alloc(std::max<size_t>(n, 1) * sizeof(double));
    be_->memset0(p, std::max<size_t>(n, 1) * sizeof(double));
    mem_.push_back(p);
    return p;
  };
  mask_ = al(nn);
  g_ = al(nn);
  gprev_ = al(nn);
  xprev_ = al(nn);
  q_ = al(nn);
  r_ = al(nn);
  hd_ = al(nn);
  scal_ = al(4);
  S_.resize(memory_);
  Y_.resize(memory_);
  for (int i = 0; i < memory_; ++i) {
    S_[i] = al(nn);
    Y_[i] = al(nn);
  }
  k_rotation_mask<<<grid_for(nn), 256, 0, (cudaStream_t)be_->stream()>>>(nb, ncore, ncas, mask_);
}

ScfStepper::~ScfStepper() {
  be_->sync();
  for (double* p : mem_) be_->free(p);
}

double ScfStepper::dot(const double* a, const double* b) {
  be_->dots(a, 1, (size_t)nb_ * nb_, (size_t)nb_ * nb_, b, scal_);
  double v;
  be_->copy_d2h(&v, scal_, sizeof(double));
  return v;
}

double ScfStepper::gradient_max(const double* g_host) {
  const size_t nn = (size_t)nb_ * nb_;
  be_->copy_h2d(q_, g_host, nn * sizeof(double));
  cudaStream_t st = (cudaStream_t)be_->stream();
  k_mul<<<grid_for(nn), 256, 0, st>>>(q_, mask_, nn, g_);
  k_maxabs<<<1, 256, 0, st>>>(g_, nn, scal_ + 1);
  double v;
  be_->copy_d2h(&v, scal_ + 1, sizeof(double));
  return v;
}

void ScfStepper::step(Casscf& cas, const double* h, const double* L, int rank, const double* gamma,
                      const double* Gamma, double* K_host) {
  const size_t nn = (size_t)nb_ * nb_;
  cudaStream_t st = (cudaStream_t)be_->stream();
  // curvature pair of the last step
  if (have_prev_) {
    double* y = q_;
    be_->copy_d2d(y, g_, nn * sizeof(double));
    be_->axpby(y, 1.0, gprev_, -1.0, nn);
    if (dot(xprev_, y) > 1e-12 && memory_ > 0) {
      const int slot = pairs_ % memory_;
      be_->copy_d2d(S_[slot], xprev_, nn * sizeof(double));
      be_->copy_d2d(Y_[slot], y, nn * sizeof(double));
      ++pairs_;
    }
  }
  // diagonal Hessian of the current orbitals
  {
    Casscf::Dev d(be_);
    const int a2 = ncas_ * ncas_;
    double* dh = d.upload(h, nn);
    double* dL = d.upload(L, nn * rank);
    double* dg = d.upload(gamma, (size_t)a2);
    double* dG = d.upload(Gamma, (size_t)a2 * a2);
    double* F = d.alloc(nn);
    double* fd = d.alloc(nb_);
    cas.fock_dev(dh, dL, rank, nb_, ncore_, ncas_, dg, dG, F, fd);
    k_diag_hessian<<<grid_for(nn), 256, 0, st>>>(fd, F, dg, nb_, ncore_, ncas_, 0.05, hd_);
    be_->sync();
  }
  // two-loop recursion, newest pair first
  const int np = std::min(pairs_, memory_);
  std::vector<double> rho(np), alpha(np);
  be_->copy_d2d(q_, g_, nn * sizeof(double));
  for (int k = 0; k < np; ++k) {
    const int slot = (pairs_ - 1 - k) % memory_;
    rho[k] = 1.0 / dot(Y_[slot], S_[slot]);
    alpha[k] = rho[k] * dot(S_[slot], q_);
    be_->axpby(q_, 1.0, Y_[slot], -alpha[k], nn);
  }
  k_div_mask<<<grid_for(nn), 256, 0, st>>>(q_, hd_, mask_, nn, r_);
  for (int k = np - 1; k >= 0; --k) {
    const int slot = (pairs_ - 1 - k) % memory_;
    const double beta = rho[k] * dot(Y_[slot], r_);
    be_->axpby(r_, 1.0, S_[slot], alpha[k] - beta, nn);
  }
  // x = -r, largest entry capped
  k_maxabs<<<1, 256, 0, st>>>(r_, nn, scal_ + 2);
  double big;
  be_->copy_d2h(&big, scal_ + 2, sizeof(double));
  const double sc = big > max_step_ ? -max_step_ / big : -1.0;
  be_->axpby(r_, sc, r_, 0.0, nn);
  be_->copy_d2d(xprev_, r_, nn * sizeof(double));
  be_->copy_d2d(gprev_, g_, nn * sizeof(double));
  have_prev_ = true;
  k_antisym<<<grid_for(nn), 256, 0, st>>>(r_, nb_, q_);
  be_->copy_d2h(K_host, q_, nn * sizeof(double));
}

}  // namespace dmrg
