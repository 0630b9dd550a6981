// SU(2) recoupling coefficients and the reduced matrix elements of one site.
//
// The spin-adapted DMRG of the paper (Sec. II.C: D counts SU(2) multiplets,
// the Clebsch-Gordan layer is decoupled from the tensor algebra) needs, on
// the host only:
//   * Wigner 6j symbols (Racah's closed form) and 9j symbols (sum of 6j's),
//   * Clebsch-Gordan coefficients (Racah's closed form),
//   * reduced matrix elements of the site operators a+, a~ and their
//     products on the three site multiplets (N,2S) = (0,0), (1,1), (2,0).
// All angular momenta are passed doubled (integers).
//
// Reduced matrix elements use the Clebsch-Gordan convention
//   <j' m'| T^k_q |j m> = <j m k q | j' m'> T(j', j).
#pragma once
#include <array>
#include <cmath>
#include <map>
#include <tuple>
#include <vector>

namespace dmrg {

inline bool triangle(int a, int b, int c) {
  return c >= std::abs(a - b) && c <= a + b && ((a + b + c) & 1) == 0;
}

double log_factorial(int n);
double clebsch(int j1, int m1, int j2, int m2, int J, int M);
double wigner6j(int a, int b, int c, int d, int e, int f);
double wigner9j(int a, int b, int c, int d, int e, int f, int g, int h, int i);

// Sign (-1)^(x/2) for an even doubled exponent x.
inline double phase2(int x2) { return ((x2 / 2) & 1) ? -1.0 : 1.0; }

// Coefficient of the tensor product [X^{kx} (x) Y^{ky}]^k between coupled
// states |(j1' j2') J'> and |(j1 j2) J> of two subsystems (first factor on
// the first subsystem); fermion signs are applied by the caller.
double tensor_product_coef(int j1p, int j1, int kx, int j2p, int j2, int ky,
                           int Jp, int J, int k);

// Coefficient of a scalar term [O^L(k) (x) O^R(k)]^0 acting on the two-block
// wavefunction coupled to total spin S:
//   sigma(jL',jR') += coef * O^L(jL',jL) psi(jL,jR) O^R(jR',jR).
double hpsi_coef(int jLp, int jRp, int jL, int jR, int k, int S);

// Reduced elements of the adjoint tensor  T~_q = (-1)^(k-q) (T_{-q})^+ :
//   T~(j, j') = adjoint_coef(j, j', k) * T(j', j).
inline double adjoint_coef(int j, int jp, int k) {
  return phase2(jp + k - j) * std::sqrt((jp + 1.0) / (j + 1.0));
}

// ------------------------------------------------------------------ site
// Site multiplets: 0 = (N=0, 2S=0), 1 = (N=1, 2S=1), 2 = (N=2, 2S=0).
constexpr int kSiteN[3] = {0, 1, 2};
constexpr int kSiteJ[3] = {0, 1, 0};

// A reduced site operator: rank k (doubled), particle change dn, fermion
// parity, and the 3x3 reduced matrix  m[bra][ket].
struct SiteOp {
  int k2 = 0, dn = 0, parity = 0;
  std::array<std::array<double, 3>, 3> m{};
  SiteOp scaled(double s) const {
    SiteOp o = *this;
    for (auto& r : o.m) for (auto& x : r) x *= s;
    return o;
  }
  bool zero() const {
    for (auto& r : m) for (double x : r) if (x != 0.0) return false;
    return true;
  }
};

// Library of site operators derived from explicit 4x4 fermion matrices
// (digits 0 empty, 1 down, 2 up, 3 double; a+_up a+_dn |0> = |3>).
struct SiteAlgebra {
  SiteOp I, C, D, N;          // identity, a+ (rank 1/2), a~ (rank 1/2), number
  SiteOp CC0, DD0;            // [a+ a+]^0, [a~ a~]^0 on the site
  SiteOp CD[2];               // [a+ a~]^k, k = 0, 1
  SiteOp NnD;                 // S~-form of sum_t a+_t a_t a_s  (three operators on the site)
  SiteOp Hu;                  // n_up n_dn (on-site pair)
  SiteAlgebra();
};

const SiteAlgebra& site_algebra();

}  // namespace dmrg

namespace dmrg {

// ------------------------------------------------------------------ strings
// Coupled tensor of a string of spinor operators on ONE site, written left to
// right (dag[i]: a+ spinor, else a~ spinor), coupled sequentially
// (((o0 o1)^{k2[0]} o2)^{k2[1]} ...): k2 holds the doubled intermediate ranks,
// its last entry the rank of the whole string.  An empty string is the
// identity.  Used for the on-site parts of the reduced density matrices.
SiteOp site_string(const std::vector<int>& dag, const std::vector<int>& k2);

// Invariant 4-index (or 2-index) tensors over the spinor components of a
// string of rank-1/2 operators o_0 .. o_{n-1} (n = 2 or 4), entries indexed
// by the bit mask of the components (bit i set: component -1/2 of o_i).
//
// A coupling tree is a list of nodes; node i is a leaf (slot >= 0) or joins
// nodes l and r (l, r < i) to rank k2.  The last node is the root (rank 0).
struct TreeNode {
  int slot = -1;
  int l = -1, r = -1, k2 = 0;
};
// T[mask] with  [tree]^0 = sum_mask T[mask] o_0(m_0) ... o_{n-1}(m_{n-1}).
std::vector<double> tree_tensor(const std::vector<TreeNode>& tree, int n);
// Spin-free pairing: sum over sigma of a+_{i sigma} ... a_{j sigma} for each
// pair (i, j) of creator slot i and annihilator slot j, written in spinor
// components (a+_up = o(+1/2), a+_dn = o(-1/2); a_dn = o~(+1/2), a_up = -o~(-1/2)).
std::vector<double> pairing_tensor(const std::vector<int>& dag,
                                   const std::vector<std::pair<int, int>>& pairs, int n);
// Least-squares coefficients c with  target = sum_a c_a basis[a]  (exact when
// target lies in the span; the residual is returned in *res if given).
std::vector<double> expand_invariant(const std::vector<double>& target,
                                     const std::vector<std::vector<double>>& basis, double* res = nullptr);

}  // namespace dmrg
