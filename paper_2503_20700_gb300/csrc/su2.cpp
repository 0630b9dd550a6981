// SU(2) coefficients (Racah closed forms) and the explicit one-site algebra.
#include "su2.hpp"

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <mutex>
#include <vector>

namespace dmrg {

double log_factorial(int n) {
  static std::vector<double> table;
  static std::once_flag once;
  std::call_once(once, [] {
    table.resize(512);
    table[0] = 0.0;
    for (int i = 1; i < 512; ++i) table[i] = table[i - 1] + std::log((double)i);
  });
  return table.at(n);
}

// Racah's formula for <j1 m1 j2 m2 | J M> (doubled arguments).
double clebsch(int j1, int m1, int j2, int m2, int J, int M) {
  if (m1 + m2 != M) return 0.0;
  if (std::abs(m1) > j1 || std::abs(m2) > j2 || std::abs(M) > J) return 0.0;
  if (((j1 + m1) & 1) || ((j2 + m2) & 1) || ((J + M) & 1)) return 0.0;
  if (!triangle(j1, j2, J)) return 0.0;
  auto f = [](int x2) { return log_factorial(x2 / 2); };
  double lpre = std::log(J + 1.0) + f(J + j1 - j2) + f(J - j1 + j2) + f(j1 + j2 - J) -
                f(j1 + j2 + J + 2) + f(J + M) + f(J - M) + f(j1 - m1) + f(j1 + m1) +
                f(j2 - m2) + f(j2 + m2);
  double s = 0.0;
  for (int k = 0;; ++k) {
    int a = j1 + j2 - J - 2 * k, b = j1 - m1 - 2 * k, c = j2 + m2 - 2 * k;
    int d = J - j2 + m1 + 2 * k, e = J - j1 - m2 + 2 * k;
    if (a < 0 || b < 0 || c < 0) break;
    if (d < 0 || e < 0) continue;
    double t = std::exp(0.5 * lpre - log_factorial(k) - f(a) - f(b) - f(c) - f(d) - f(e));
    s += (k & 1) ? -t : t;
  }
  return s;
}

namespace {
double log_delta(int a, int b, int c) {
  return 0.5 * (log_factorial((a + b - c) / 2) + log_factorial((a - b + c) / 2) +
                log_factorial((-a + b + c) / 2) - log_factorial((a + b + c) / 2 + 1));
}
// Memo of coefficients under a packed integer key: open addressing with
// linear probing, at most half full, one table per thread.  The planners ask
// for the same few thousand coefficients millions of times.
class FlatMemo {
 public:
  bool find(uint64_t key, double& v) const {
    if (n_ == 0) return false;
    for (size_t h = mix(key) & mask_;; h = (h + 1) & mask_) {
      if (!used_[h]) return false;
      if (keys_[h] == key) {
        v = vals_[h];
        return true;
      }
    }
  }
  void put(uint64_t key, double v) {
    if (2 * (n_ + 1) > keys_.size()) grow();
    size_t h = mix(key) & mask_;
    while (used_[h] && keys_[h] != key) h = (h + 1) & mask_;
    if (!used_[h]) ++n_;
    used_[h] = 1;
    keys_[h] = key;
    vals_[h] = v;
  }

 private:
  static uint64_t mix(uint64_t x) {
    x ^= x >> 31;
    x *= 0x9e3779b97f4a7c15ull;
    return x ^ (x >> 29);
  }
  void grow() {
    std::vector<uint64_t> k = std::move(keys_);
    std::vector<double> v = std::move(vals_);
    std::vector<uint8_t> u = std::move(used_);
    const size_t cap = std::max<size_t>(1024, 2 * k.size());
    keys_.assign(cap, 0);
    vals_.assign(cap, 0.0);
    used_.assign(cap, 0);
    mask_ = cap - 1;
    n_ = 0;
    for (size_t i = 0; i < k.size(); ++i)
      if (u[i]) put(k[i], v[i]);
  }
  std::vector<uint64_t> keys_;
  std::vector<double> vals_;
  std::vector<uint8_t> used_;
  size_t n_ = 0, mask_ = 0;
};

// packs small non-negative arguments (doubled spins below 128), 7 bits each
template <size_t K>
bool pack7(const int (&v)[K], uint64_t& key) {
  key = 0;
  for (int x : v) {
    if (x < 0 || x >= 128) return false;
    key = (key << 7) | (uint64_t)x;
  }
  return true;
}
}  // namespace

// Racah's closed form for {a b c; d e f} (doubled arguments).
double wigner6j(int a, int b, int c, int d, int e, int f) {
  if (!triangle(a, b, c) || !triangle(a, e, f) || !triangle(d, b, f) || !triangle(d, e, c))
    return 0.0;
  static thread_local FlatMemo cache;
  const int args[6] = {a, b, c, d, e, f};
  uint64_t key;
  const bool packed = pack7(args, key);
  double hit;
  if (packed && cache.find(key, hit)) return hit;
  double ld = log_delta(a, b, c) + log_delta(a, e, f) + log_delta(d, b, f) + log_delta(d, e, c);
  int t1 = (a + b + c) / 2, t2 = (a + e + f) / 2, t3 = (d + b + f) / 2, t4 = (d + e + c) / 2;
  int u1 = (a + b + d + e) / 2, u2 = (b + c + e + f) / 2, u3 = (c + a + f + d) / 2;
  int tmin = std::max(std::max(t1, t2), std::max(t3, t4));
  int tmax = std::min(u1, std::min(u2, u3));
  double s = 0.0;
  for (int t = tmin; t <= tmax; ++t) {
    double lt = log_factorial(t + 1) - log_factorial(t - t1) - log_factorial(t - t2) -
                log_factorial(t - t3) - log_factorial(t - t4) - log_factorial(u1 - t) -
                log_factorial(u2 - t) - log_factorial(u3 - t);
    double term = std::exp(lt + ld);
    s += (t & 1) ? -term : term;
  }
  if (packed) cache.put(key, s);
  return s;
}

// 9j symbol as a sum over x of (-1)^(2x) (2x+1) {a b c; f i x}{d e f; b x h}{g h i; x a d}.
double wigner9j(int a, int b, int c, int d, int e, int f, int g, int h, int i) {
  if (!triangle(a, b, c) || !triangle(d, e, f) || !triangle(g, h, i) || !triangle(a, d, g) ||
      !triangle(b, e, h) || !triangle(c, f, i))
    return 0.0;
  int lo = std::max(std::max(std::abs(a - i), std::abs(d - h)), std::abs(b - f));
  int hi = std::min(std::min(a + i, d + h), b + f);
  double s = 0.0;
  for (int x = lo; x <= hi; x += 2) {
    double t = wigner6j(a, b, c, f, i, x) * wigner6j(d, e, f, b, x, h) * wigner6j(g, h, i, x, a, d);
    s += ((x & 1) ? -1.0 : 1.0) * (x + 1) * t;
  }
  return s;
}

double tensor_product_coef(int j1p, int j1, int kx, int j2p, int j2, int ky, int Jp, int J, int k) {
  // memoised: the blocking and RDM planners ask for the same few thousand
  // combinations millions of times; doubled spins here are far below 128
  const int v[9] = {j1p, j1, kx, j2p, j2, ky, Jp, J, k};
  uint64_t key;
  const bool packed = pack7(v, key);
  static thread_local FlatMemo cache;
  double hit;
  if (packed && cache.find(key, hit)) return hit;
  double n9 = wigner9j(j1p, j1, kx, j2p, j2, ky, Jp, J, k);
  double r = n9 == 0.0 ? 0.0 : std::sqrt((J + 1.0) * (k + 1.0) * (j1p + 1.0) * (j2p + 1.0)) * n9;
  if (packed) cache.put(key, r);
  return r;
}

double hpsi_coef(int jLp, int jRp, int jL, int jR, int k, int S) {
  double s6 = wigner6j(jLp, jL, k, jR, jRp, S);
  if (s6 == 0.0) return 0.0;
  return std::sqrt((jLp + 1.0) * (jRp + 1.0) / (k + 1.0)) * phase2(jL + jRp + k + S) * s6;
}

// ------------------------------------------------------------------ site
namespace {
using Mat4 = std::array<std::array<double, 4>, 4>;
// Site digits: 0 empty, 1 down, 2 up, 3 double.  Jordan-Wigner order inside
// the site: up before down, |3> = a+_up a+_dn |0>.
Mat4 zero4() { Mat4 m{}; return m; }
Mat4 mul(const Mat4& a, const Mat4& b) {
  Mat4 c = zero4();
  for (int i = 0; i < 4; ++i)
    for (int k = 0; k < 4; ++k)
      if (a[i][k] != 0.0)
        for (int j = 0; j < 4; ++j) c[i][j] += a[i][k] * b[k][j];
  return c;
}
Mat4 add(const Mat4& a, const Mat4& b, double s = 1.0) {
  Mat4 c = a;
  for (int i = 0; i < 4; ++i) for (int j = 0; j < 4; ++j) c[i][j] += s * b[i][j];
  return c;
}
Mat4 transpose(const Mat4& a) {
  Mat4 c;
  for (int i = 0; i < 4; ++i) for (int j = 0; j < 4; ++j) c[i][j] = a[j][i];
  return c;
}
// creation operators on the site
Mat4 cdag(bool up) {
  Mat4 m = zero4();
  if (up) {
    m[2][0] = 1.0;   // a+_up |0> = |up>
    m[3][1] = 1.0;   // a+_up |dn> = a+_up a+_dn |0> = |3>
  } else {
    m[1][0] = 1.0;   // a+_dn |0> = |dn>
    m[3][2] = -1.0;  // a+_dn |up> = a+_dn a+_up|0> = -|3>
  }
  return m;
}
// spherical components indexed by q2 + k2 (component q2 in -k2..k2)
using Tensor = std::map<int, Mat4>;
Tensor couple(const Tensor& A, int ka, const Tensor& B, int kb, int k) {
  Tensor out;
  for (int q = -k; q <= k; q += 2) {
    Mat4 m = zero4();
    for (auto& [qa, ma] : A) {
      int qb = q - qa;
      auto it = B.find(qb);
      if (it == B.end()) continue;
      double c = clebsch(ka, qa, kb, qb, k, q);
      if (c != 0.0) m = add(m, mul(ma, it->second), c);
    }
    out[q] = m;
  }
  return out;
}
// explicit multiplet states: (multiplet index, 2m) -> digit
int state_digit(int mult, int m2) {
  if (mult == 0) return 0;
  if (mult == 2) return 3;
  return m2 > 0 ? 2 : 1;
}
SiteOp reduce(const Tensor& T, int k2, int dn, int parity) {
  SiteOp o;
  o.k2 = k2;
  o.dn = dn;
  o.parity = parity;
  for (int b = 0; b < 3; ++b)
    for (int a = 0; a < 3; ++a) {
      int jb = kSiteJ[b], ja = kSiteJ[a];
      if (kSiteN[b] != kSiteN[a] + dn) continue;
      double val = 0.0;
      bool found = false;
      for (int ma = -ja; ma <= ja && !found; ma += 2)
        for (int q = -k2; q <= k2 && !found; q += 2) {
          int mb = ma + q;
          if (std::abs(mb) > jb) continue;
          double c = clebsch(ja, ma, k2, q, jb, mb);
          if (std::abs(c) < 1e-12) continue;
          val = T.at(q)[state_digit(b, mb)][state_digit(a, ma)] / c;
          found = true;
        }
      o.m[b][a] = found ? val : 0.0;
    }
  return o;
}
}  // namespace

SiteAlgebra::SiteAlgebra() {
  Mat4 cu = cdag(true), cd = cdag(false);
  Mat4 au = transpose(cu), ad = transpose(cd);
  Tensor C{{1, cu}, {-1, cd}};
  Mat4 mau = au;
  for (auto& r : mau) for (auto& x : r) x = -x;
  Tensor D{{1, ad}, {-1, mau}};  // a~ = (a_dn, -a_up)
  Mat4 eye = zero4();
  for (int i = 0; i < 4; ++i) eye[i][i] = 1.0;
  Mat4 num = add(mul(cu, au), mul(cd, ad));
  this->I = reduce(Tensor{{0, eye}}, 0, 0, 0);
  this->C = reduce(C, 1, 1, 1);
  this->D = reduce(D, 1, -1, 1);
  this->N = reduce(Tensor{{0, num}}, 0, 0, 0);
  this->CC0 = reduce(couple(C, 1, C, 1, 0), 0, 2, 0);
  this->DD0 = reduce(couple(D, 1, D, 1, 0), 0, -2, 0);
  this->CD[0] = reduce(couple(C, 1, D, 1, 0), 0, 0, 0);
  this->CD[1] = reduce(couple(C, 1, D, 1, 2), 2, 0, 0);
  // sum_t a+_t a_t a_sigma in the a~ arrangement: components (+1/2: sigma=dn, -1/2: -(sigma=up))
  Mat4 nn = num;
  Tensor T3{{1, mul(nn, ad)}, {-1, mul(nn, mau)}};
  this->NnD = reduce(T3, 1, -1, 1);
  this->Hu = reduce(Tensor{{0, mul(mul(cu, au), mul(cd, ad))}}, 0, 0, 0);
}

const SiteAlgebra& site_algebra() {
  static SiteAlgebra alg;
  return alg;
}

}  // namespace dmrg

namespace dmrg {

SiteOp site_string(const std::vector<int>& dag, const std::vector<int>& k2) {
  Mat4 cu = cdag(true), cd = cdag(false);
  Mat4 au = transpose(cu), ad = transpose(cd);
  Mat4 mau = au;
  for (auto& r : mau) for (auto& x : r) x = -x;
  const Tensor C{{1, cu}, {-1, cd}};
  const Tensor D{{1, ad}, {-1, mau}};
  if (dag.empty()) {
    Mat4 eye = zero4();
    for (int i = 0; i < 4; ++i) eye[i][i] = 1.0;
    return reduce(Tensor{{0, eye}}, 0, 0, 0);
  }
  Tensor T = dag[0] ? C : D;
  int kt = 1, dn = dag[0] ? 1 : -1;
  for (size_t i = 1; i < dag.size(); ++i) {
    int k = k2.at(i - 1);
    T = couple(T, kt, dag[i] ? C : D, 1, k);
    kt = k;
    dn += dag[i] ? 1 : -1;
  }
  return reduce(T, kt, dn, (int)(dag.size() & 1));
}

std::vector<double> tree_tensor(const std::vector<TreeNode>& tree, int n) {
  // per node: map (M2, mask) -> value
  std::vector<std::map<std::pair<int, int>, double>> val(tree.size());
  std::vector<int> rank(tree.size(), 1);
  for (size_t i = 0; i < tree.size(); ++i) {
    const TreeNode& t = tree[i];
    if (t.slot >= 0) {
      val[i][{1, 0}] = 1.0;                  // component +1/2
      val[i][{-1, 1 << t.slot}] = 1.0;       // component -1/2
      rank[i] = 1;
      continue;
    }
    rank[i] = t.k2;
    for (auto& [ka, va] : val[t.l])
      for (auto& [kb, vb] : val[t.r]) {
        int M = ka.first + kb.first;
        if (std::abs(M) > t.k2) continue;
        double c = clebsch(rank[t.l], ka.first, rank[t.r], kb.first, t.k2, M);
        if (c == 0.0) continue;
        val[i][{M, ka.second | kb.second}] += c * va * vb;
      }
  }
  std::vector<double> out((size_t)1 << n, 0.0);
  for (auto& [k, v] : val.back())
    if (k.first == 0) out[k.second] += v;
  return out;
}

std::vector<double> pairing_tensor(const std::vector<int>& dag,
                                   const std::vector<std::pair<int, int>>& pairs, int n) {
  std::vector<double> out((size_t)1 << n, 0.0);
  const int np = (int)pairs.size();
  for (int sp = 0; sp < (1 << np); ++sp) {  // spin of each pair: bit set = down
    int mask = 0;
    double f = 1.0;
    for (int p = 0; p < np; ++p) {
      bool down = (sp >> p) & 1;
      int i = pairs[p].first, j = pairs[p].second;
      for (int slot : {i, j}) {
        if (dag[slot]) {
          if (down) mask |= 1 << slot;      // a+_dn = o(-1/2)
        } else {
          if (!down) {                      // a_up = -o~(-1/2)
            mask |= 1 << slot;
            f = -f;
          }                                 // a_dn = o~(+1/2)
        }
      }
    }
    out[mask] += f;
  }
  return out;
}

std::vector<double> expand_invariant(const std::vector<double>& target,
                                     const std::vector<std::vector<double>>& basis, double* res) {
  const size_t m = basis.size(), L = target.size();
  // normal equations (m <= 4), solved by Gaussian elimination with pivoting
  std::vector<std::vector<double>> A(m, std::vector<double>(m + 1, 0.0));
  for (size_t a = 0; a < m; ++a) {
    for (size_t b = 0; b < m; ++b)
      for (size_t e = 0; e < L; ++e) A[a][b] += basis[a][e] * basis[b][e];
    for (size_t e = 0; e < L; ++e) A[a][m] += basis[a][e] * target[e];
  }
  std::vector<double> c(m, 0.0);
  std::vector<int> piv_col;
  std::vector<size_t> rows(m);
  for (size_t i = 0; i < m; ++i) rows[i] = i;
  // eliminate; dependent basis tensors get coefficient 0
  std::vector<int> pivot_of_col(m, -1);
  size_t r = 0;
  for (size_t col = 0; col < m && r < m; ++col) {
    size_t best = r;
    for (size_t i = r; i < m; ++i)
      if (std::abs(A[i][col]) > std::abs(A[best][col])) best = i;
    if (std::abs(A[best][col]) < 1e-12) continue;
    std::swap(A[r], A[best]);
    for (size_t i = 0; i < m; ++i) {
      if (i == r) continue;
      double f = A[i][col] / A[r][col];
      for (size_t j = col; j <= m; ++j) A[i][j] -= f * A[r][j];
    }
    pivot_of_col[col] = (int)r;
    ++r;
  }
  for (size_t col = 0; col < m; ++col)
    if (pivot_of_col[col] >= 0) c[col] = A[pivot_of_col[col]][m] / A[pivot_of_col[col]][col];
  if (res) {
    double s = 0.0;
    for (size_t e = 0; e < L; ++e) {
      double v = target[e];
      for (size_t a = 0; a < m; ++a) v -= c[a] * basis[a][e];
      s += v * v;
    }
    *res = std::sqrt(s);
  }
  return c;
}

}  // namespace dmrg
