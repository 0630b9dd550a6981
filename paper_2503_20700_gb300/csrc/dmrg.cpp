// Host planner of the spin-adapted two-site DMRG (see dmrg.hpp).
#include "dmrg.hpp"
#include "hpsi_fused.cuh"
#include "hpsi_tc.cuh"
#include "host_pool.hpp"

#include <algorithm>
#include <functional>
#include <array>
#include <chrono>
#include <thread>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <set>
#include <stdexcept>

namespace dmrg {

static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}


namespace {
thread_local std::string g_last_error;
const double kSqrt2 = std::sqrt(2.0);
const double kSqrt3 = std::sqrt(3.0);
// Spinor recoupling constants in the Clebsch-Gordan convention of su2.hpp
// (verified against explicit fermion matrices; see the test suite):
//   sum_{st} a+_ps a+_qt a_rt a_ss = sum_k alpha_k [[a+_p a+_q]^k [a~_r a~_s]^k]^0
//   sum_{st} a+_ps a_rt a+_qt a_ss = sum_k beta_k  [[a+_p a~_r]^k [a+_q a~_s]^k]^0
const double kAlpha[2] = {-1.0, std::sqrt(3.0)};
const double kBeta[2] = {1.0, -std::sqrt(3.0)};
// Mixed terms of the three-index complementary operator S~_p when a block
// grows by one site s (L: block left of s; R: block right of s):
//   M2: sum_t a+_qt a_st a_t'sigma      ->  c2  [[a+_q a~_t']^k (x) a~_s]
//   M3: sum_t a+_st a_rt a_t'sigma      ->  c3  [[a~_r a~_t']^k (x) a+_s]
//   M5: sum_t a+_st a_rt a_s sigma      ->  c5  [a~_r (x) [a+_s a~_s]^k]
const double kC2L[2] = {1.0 / std::sqrt(2.0), std::sqrt(1.5)};
const double kC2R[2] = {1.0 / std::sqrt(2.0), -std::sqrt(1.5)};
const double kC5L[2] = {1.0 / std::sqrt(2.0), -std::sqrt(1.5)};
const double kC5R[2] = {1.0 / std::sqrt(2.0), std::sqrt(1.5)};
const double kC6 = 1.0 / std::sqrt(2.0);
// [a+_s a~_r]^k = kSwapB[k] [a~_r (x) a+_s]^k for two distinct sites (either order)
const double kSwapB[2] = {1.0, -1.0};
// adj([a+_a a~_b]^k) = kAdjB[k] [a+_b a~_a]^k ;  adj([a+_a a+_b]^k) = -[a~_a a~_b]^k
const double kAdjB[2] = {1.0, -1.0};
}  // namespace

std::string last_error() { return g_last_error; }
void set_last_error(const std::string& e) { g_last_error = e; }

// ============================================================ op sets
OpSet::~OpSet() {
  if (!be) return;
  if (!pending.empty()) {
    be->stage_join();
    release_pending();
  }
  if (on_host) {
    for (void* h : host) be->host_release(h);
    be->staged_bytes -= device_bytes();
  } else {
    for (void* p : mem) be->free(p);
  }
}

size_t OpSet::device_bytes() const {
  size_t b = 0;
  for (size_t x : mem_bytes) b += x;
  return b;
}

void OpSet::stage_out() {
  if (on_host || mem.empty()) return;
  host.assign(mem.size(), nullptr);
  for (size_t i = 0; i < mem.size(); ++i) host[i] = be->stage_out(mem[i], mem_bytes[i]);
  on_host = true;
}

void OpSet::stage_in() {
  if (!on_host) return;
  // operator pointers are offsets into the allocations: rebase them
  std::vector<double*> old(mem.size());
  for (size_t i = 0; i < mem.size(); ++i) old[i] = (double*)mem[i];
  std::vector<double*> fresh(mem.size());
  for (size_t i = 0; i < mem.size(); ++i) fresh[i] = (double*)be->stage_in(host[i], mem_bytes[i]);
  for (auto& [k, p] : ops) {
    for (size_t i = 0; i < mem.size(); ++i) {
      const size_t n = mem_bytes[i] / sizeof(double);
      if (p >= old[i] && p < old[i] + n) {
        p = fresh[i] + (p - old[i]);
        break;
      }
    }
  }
  for (size_t i = 0; i < mem.size(); ++i) mem[i] = fresh[i];
  // the copies are in flight on the side stream: the main stream waits for
  // them at the next join, and the pinned copies are released after it
  pending.insert(pending.end(), host.begin(), host.end());
  be->staged_bytes -= device_bytes();
  host.clear();
  on_host = false;
  arriving = true;
}

void OpSet::release_pending() {
  for (void* h : pending) be->host_release(h);
  pending.clear();
}

static Layout make_layout(const Basis& bra, const Basis& ket, int dn, int k2) {
  Layout L;
  L.dn = dn;
  L.k2 = k2;
  L.nket = (int)ket.sec.size();
  L.lut.assign(bra.sec.size() * ket.sec.size(), -1);
  size_t off = 0;
  for (size_t kb = 0; kb < ket.sec.size(); ++kb)
    for (size_t bb = 0; bb < bra.sec.size(); ++bb) {
      const Sector& K = ket.sec[kb];
      const Sector& B = bra.sec[bb];
      if (B.n != K.n + dn || !triangle(K.j, k2, B.j)) continue;
      L.lut[bb * ket.sec.size() + kb] = (int)L.blk.size();
      L.blk.push_back({(int)bb, (int)kb, B.dim, K.dim, off});
      off += (size_t)B.dim * K.dim;
    }
  L.size = off;
  return L;
}

const Layout& OpSet::layout(int dn, int k2) {
  auto key = std::make_pair(dn, k2);
  auto it = layouts.find(key);
  if (it != layouts.end()) return it->second;
  return layouts.emplace(key, make_layout(basis, basis, dn, k2)).first->second;
}

void OpSet::allocate(const std::vector<OpKey>& keys) {
  std::map<std::pair<int, int>, std::vector<OpKey>> by;
  for (auto& k : keys) by[{kind_dn(k.kind), k.k2}].push_back(k);
  for (auto& [lk, ks] : by) {
    const Layout& L = layout(lk.first, lk.second);
    if (L.size == 0) continue;
    size_t bytes = L.size * ks.size() * sizeof(double);
    double* p = (double*)be->alloc(bytes);
    be->memset0(p, bytes);
    mem.push_back(p);
    mem_bytes.push_back(bytes);
    for (size_t i = 0; i < ks.size(); ++i) ops[ks[i]] = p + i * L.size;
  }
}

size_t OpSet::bytes() const {
  size_t b = 0;
  for (auto& [k, p] : ops) {
    auto it = layouts.find({kind_dn(k.kind), k.k2});
    if (it != layouts.end()) b += it->second.size * sizeof(double);
  }
  return b;
}

// ============================================================ operands
struct Operand {
  enum T { ID, BLK, SITE } t = ID;
  OpKey key{0, 0, 0, 0};
  int adj = 0;
  SiteOp s;
  int k2 = 0, dn = 0, par = 0;
};

Operand op_id() { return Operand(); }
Operand op_blk(int kind, int i, int j, int k2, int adj = 0) {
  Operand o;
  o.t = Operand::BLK;
  o.key = {kind, i, j, k2};
  o.adj = adj;
  o.k2 = k2;
  o.dn = adj ? -kind_dn(kind) : kind_dn(kind);
  o.par = kind_parity(kind);
  return o;
}
Operand op_site(const SiteOp& s) {
  Operand o;
  o.t = Operand::SITE;
  o.s = s;
  o.k2 = s.k2;
  o.dn = s.dn;
  o.par = s.parity;
  return o;
}
// adjoint of an operand
Operand op_adj(const Operand& x) {
  Operand o = x;
  if (x.t == Operand::BLK) {
    o.adj = !x.adj;
    o.dn = -x.dn;
  } else if (x.t == Operand::SITE) {
    SiteOp s;
    s.k2 = x.s.k2;
    s.dn = -x.s.dn;
    s.parity = x.s.parity;
    for (int b = 0; b < 3; ++b)
      for (int a = 0; a < 3; ++a)
        s.m[b][a] = adjoint_coef(kSiteJ[b], kSiteJ[a], x.s.k2) * x.s.m[a][b];
    o.s = s;
    o.dn = s.dn;
  }
  return o;
}
SiteOp site_add(const SiteOp& a, const SiteOp& b, double cb) {
  SiteOp o = a;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) o.m[i][j] += cb * b.m[i][j];
  return o;
}

struct Term {
  Operand x, y;  // x acts on the left part, y on the right part
  int k2;        // coupled rank of [x (x) y]
  double coef;
};

// A member of a bipartition: a single site or a block.
struct Side {
  bool is_site = false;
  int site = -1;
  const Block* blk = nullptr;
  std::vector<int> sites;
  bool normal = true;
  bool has(int p) const { return std::find(sites.begin(), sites.end(), p) != sites.end(); }
};

// Operands of a side; integral-dependent site operators are built here.
struct SideOps {
  const Engine* e;
  const SiteAlgebra& sa = site_algebra();
  const Side& s;
  double (*gfun)(const Engine*, int, int, int, int);
  double (*hfun)(const Engine*, int, int);
  SideOps(const Engine* e_, const Side& s_, double (*g_)(const Engine*, int, int, int, int),
          double (*h_)(const Engine*, int, int))
      : e(e_), s(s_), gfun(g_), hfun(h_) {}
  double g(int p, int q, int r, int t) const { return gfun(e, p, q, r, t); }
  Operand C(int p) const { return s.is_site ? op_site(sa.C) : op_blk(K_C, p, 0, 1); }
  Operand S(int p) const {  // S~_p, p outside the side
    if (!s.is_site) return op_blk(K_S, p, 0, 1);
    int t = s.site;
    SiteOp o = sa.D.scaled(0.5 * hfun(e, p, t));
    o = site_add(o, sa.NnD, g(p, t, t, t));
    return op_site(o);
  }
  // normal pair operators (p <= q inside the side)
  Operand A(int p, int q, int k) const {
    if (s.is_site) return k == 0 ? op_site(sa.CC0) : op_site(SiteOp());
    return op_blk(K_A, p, q, 2 * k);
  }
  Operand B(int p, int q, int k) const {
    if (s.is_site) return op_site(sa.CD[k]);
    return op_blk(K_B, p, q, 2 * k);
  }
  // complementary pair operators (p <= q outside the side)
  Operand P(int p, int q, int k) const {
    if (s.is_site) {
      int t = s.site;
      if (k == 1) return op_site(SiteOp());
      return op_site(sa.DD0.scaled(g(p, q, t, t)));
    }
    return op_blk(K_P, p, q, 2 * k);
  }
  Operand QJ(int p, int q) const {
    if (s.is_site) {
      int t = s.site;
      return op_site(sa.CD[0].scaled(g(p, t, t, q)));
    }
    return op_blk(K_QJ, p, q, 0);
  }
  Operand QK(int p, int q, int k) const {
    if (s.is_site) {
      int t = s.site;
      return op_site(sa.CD[k].scaled(g(p, t, q, t)));
    }
    return op_blk(K_QK, p, q, 2 * k);
  }
};

static double g_acc(const Engine* e, int p, int q, int r, int s);
static double h_acc(const Engine* e, int p, int q);

namespace {
bool operand_zero(const Operand& o) {
  return o.t == Operand::SITE && o.s.zero();
}
void push(std::vector<Term>& out, const Operand& x, const Operand& y, int k2, double c) {
  if (c == 0.0 || operand_zero(x) || operand_zero(y)) return;
  out.push_back({x, y, k2, c});
}
// h.c. of a scalar term: ([x (x) y]^0)^+ = (-1)^(px py) [x~ (x) y~]^0
void push_hc(std::vector<Term>& out, const Operand& x, const Operand& y, double c) {
  push(out, x, y, 0, c);
  double eps = (x.par && y.par) ? -1.0 : 1.0;
  push(out, op_adj(x), op_adj(y), 0, eps * c);
}
}  // namespace

// Interaction terms between a left part X and a right part Y (X left of Y in
// the Jordan-Wigner order), as scalar couplings [x (x) y]^0.
static void emit_cross(const Engine* e, const Side& X, const Side& Y, std::vector<Term>& out) {
  SideOps ox(e, X, g_acc, h_acc), oy(e, Y, g_acc, h_acc);
  // one-index / three-index terms
  for (int p : X.sites) push_hc(out, ox.C(p), oy.S(p), -kSqrt2);
  for (int p : Y.sites) push_hc(out, ox.S(p), oy.C(p), -kSqrt2);
  // pair terms: normal operators on side N, complementary on the other
  bool x_normal;
  if (!X.is_site && !Y.is_site) {
    if (X.normal == Y.normal) throw std::runtime_error("both sides have the same pair type");
    x_normal = X.normal;
  } else if (X.is_site && Y.is_site) {
    x_normal = true;
  } else if (X.is_site) {
    x_normal = !Y.normal;  // site normal iff the block is complementary
  } else {
    x_normal = X.normal;
  }
  const SideOps& on = x_normal ? ox : oy;
  const SideOps& oc = x_normal ? oy : ox;
  const Side& N = x_normal ? X : Y;
  for (size_t a = 0; a < N.sites.size(); ++a)
    for (size_t b = a; b < N.sites.size(); ++b) {
      int p = N.sites[a], q = N.sites[b];
      double w = (p == q) ? 1.0 : 2.0;
      for (int k = 0; k < 2; ++k) {
        if (p == q && k == 1) continue;
        Operand nA = on.A(p, q, k), cP = oc.P(p, q, k);
        double c = w * 0.5 * kAlpha[k];
        if (x_normal) push_hc(out, nA, cP, c);
        else push_hc(out, cP, nA, c);
      }
      // B-type (Coulomb + exchange)
      for (int k = 0; k < 2; ++k) {
        Operand nB = on.B(p, q, k);
        std::vector<std::pair<Operand, double>> comp;
        if (k == 0) comp.push_back({oc.QJ(p, q), 2.0});
        comp.push_back({oc.QK(p, q, k), -kBeta[k]});
        for (auto& [cq, c] : comp) {
          if (p == q) {
            if (x_normal) push(out, nB, cq, 0, c);
            else push(out, cq, nB, 0, c);
          } else {
            if (x_normal) push_hc(out, nB, cq, c);
            else push_hc(out, cq, nB, c);
          }
        }
      }
    }
}

// ============================================================ engine basics
struct EngineAccess {
  static double g(const Engine* e, int p, int q, int r, int s) { return e->g(p, q, r, s); }
  static double h(const Engine* e, int p, int q) { return e->hh(p, q); }
};
static double g_acc(const Engine* e, int p, int q, int r, int s) {
  return EngineAccess::g(e, p, q, r, s);
}
static double h_acc(const Engine* e, int p, int q) { return EngineAccess::h(e, p, q); }

namespace {
std::vector<int> block_sites(const Block& b, int n) {
  std::vector<int> s;
  if (b.left)
    for (int p = 0; p < b.nsites; ++p) s.push_back(p);
  else
    for (int p = n - b.nsites; p < n; ++p) s.push_back(p);
  return s;
}
bool in_sites(const std::vector<int>& v, int p) { return std::find(v.begin(), v.end(), p) != v.end(); }

// Keys of all operators a block with the given sites carries.
std::vector<OpKey> op_keys(const std::vector<int>& sites, int n, bool normal) {
  std::vector<OpKey> k;
  k.push_back({K_H, 0, 0, 0});
  std::vector<int> out;
  for (int p = 0; p < n; ++p)
    if (!in_sites(sites, p)) out.push_back(p);
  for (int p : sites) k.push_back({K_C, p, 0, 1});
  for (int p : out) k.push_back({K_S, p, 0, 1});
  const std::vector<int>& ps = normal ? sites : out;
  for (size_t a = 0; a < ps.size(); ++a)
    for (size_t b = a; b < ps.size(); ++b) {
      int p = ps[a], q = ps[b];
      if (normal) {
        k.push_back({K_A, p, q, 0});
        if (p != q) k.push_back({K_A, p, q, 2});
        k.push_back({K_B, p, q, 0});
        k.push_back({K_B, p, q, 2});
      } else {
        k.push_back({K_P, p, q, 0});
        if (p != q) k.push_back({K_P, p, q, 2});
        k.push_back({K_QJ, p, q, 0});
        k.push_back({K_QK, p, q, 0});
        k.push_back({K_QK, p, q, 2});
      }
    }
  return k;
}

// Collects place segments grouped by destination sub-block.
// Collects place segments and groups them by destination sub-block (one
// destination pointer always has the same shape): a flat list sorted by
// destination at run time, in insertion order within a destination.
struct PlaceBuilder {
  struct Entry {
    double* dst;
    int rows, cols, ld;
    PlaceSeg seg;
  };
  std::vector<Entry> entries;
  void add(double* dst, int rows, int cols, int ld, const PlaceSeg& s) {
    if (s.alpha == 0.0 || rows == 0 || cols == 0) return;
    entries.push_back({dst, rows, cols, ld, s});
  }
  void run(Backend* be) {
    std::stable_sort(entries.begin(), entries.end(),
                     [](const Entry& a, const Entry& b) { return std::less<double*>()(a.dst, b.dst); });
    std::vector<PlaceGroup> g;
    std::vector<PlaceSeg> segs;
    segs.reserve(entries.size());
    for (size_t i = 0; i < entries.size();) {
      size_t j = i;
      PlaceGroup pg;
      pg.dst = entries[i].dst;
      pg.rows = entries[i].rows;
      pg.cols = entries[i].cols;
      pg.ld = entries[i].ld;
      pg.seg_begin = (int)segs.size();
      while (j < entries.size() && entries[j].dst == entries[i].dst) segs.push_back(entries[j++].seg);
      pg.seg_count = (int)(j - i);
      g.push_back(pg);
      i = j;
    }
    if (!g.empty()) be->place(g, segs);
    entries.clear();
  }
};

struct GemmBuilder {
  std::map<double*, std::pair<std::array<int, 3>, std::vector<GemmSeg>>> groups;
  void add(double* C, int m, int n, int ldc, const GemmSeg& s) {
    if (s.alpha == 0.0 || m == 0 || n == 0 || s.k == 0) return;
    auto& g = groups[C];
    g.first = {m, n, ldc};
    g.second.push_back(s);
  }
  void run(Backend* be, Precision prec) {
    std::vector<GemmGroup> gs;
    std::vector<GemmSeg> segs;
    for (auto& [C, v] : groups) {
      GemmGroup gg;
      gg.C = C;
      gg.m = v.first[0];
      gg.n = v.first[1];
      gg.ldc = v.first[2];
      gg.seg_begin = (int)segs.size();
      gg.seg_count = (int)v.second.size();
      segs.insert(segs.end(), v.second.begin(), v.second.end());
      gs.push_back(gg);
    }
    if (!gs.empty()) be->gemm(gs, segs, prec);
    groups.clear();
  }
};
}  // namespace

Engine::~Engine() {
  if (be_) be_->make_room = nullptr;
  if (solve_psi_ && be_) be_->free(solve_psi_);
  if (prev_.psi && be_) be_->free(prev_.psi);
  if (ones_ && be_) be_->free(ones_);
}

int Engine::left_dim(int m) const {
  if (m < 0 || m >= (int)L_.size() || !L_[m]) return -1;
  int t = 0;
  for (auto& s : L_[m]->ops->basis.sec) t += s.dim;
  return t;
}
int Engine::right_dim(int m) const {
  if (m < 0 || m >= (int)R_.size() || !R_[m]) return -1;
  int t = 0;
  for (auto& s : R_[m]->ops->basis.sec) t += s.dim;
  return t;
}
int Engine::left_dim_u1(int m) const {
  if (m < 0 || m >= (int)L_.size() || !L_[m]) return -1;
  int t = 0;
  for (auto& s : L_[m]->ops->basis.sec) t += s.dim * (s.j + 1);
  return t;
}
int Engine::right_dim_u1(int m) const {
  if (m < 0 || m >= (int)R_.size() || !R_[m]) return -1;
  int t = 0;
  for (auto& s : R_[m]->ops->basis.sec) t += s.dim * (s.j + 1);
  return t;
}

std::unique_ptr<Block> Engine::vacuum(bool left) {
  auto b = std::make_unique<Block>();
  b->left = left;
  b->nsites = 0;
  b->normal = true;
  b->ops = std::make_unique<OpSet>();
  b->ops->be = be_;
  b->ops->basis.sec.push_back({0, 0, 1, 0});
  b->ops->basis.total = 1;
  b->ops->allocate(op_keys({}, n_, true));
  return b;
}

// Blocking: enlarged block = b (x) site (left) or site (x) b (right).
namespace {
// Single-orbital operator strings of the orbital-entanglement pass: the
// spinors a+ (dag 1) and a~ (dag 0) of one orbital coupled sequentially to
// the doubled intermediate ranks kl.  Together with the identity they span
// the SU(2) tensor operators of one orbital: number and double occupancy
// (rank 0), spin (rank 1), a+ and a+ n (rank 1/2), pair creation (rank 0),
// and the adjoints.
struct OrbStr {
  std::vector<int> dag, kl;
};
const std::vector<OrbStr>& orb_strings() {
  static const std::vector<OrbStr> t = {
      {{1}, {}},                  // 0  a+
      {{0}, {}},                  // 1  a~
      {{1, 0}, {0}},              // 2  [a+ a~]^0
      {{1, 0}, {2}},              // 3  [a+ a~]^1
      {{1, 1}, {0}},              // 4  [a+ a+]^0
      {{0, 0}, {0}},              // 5  [a~ a~]^0
      {{1, 1, 0}, {0, 1}},        // 6  [[a+ a+]^0 a~]^1/2
      {{0, 0, 1}, {0, 1}},        // 7  [[a~ a~]^0 a+]^1/2
      {{1, 1, 0, 0}, {0, 1, 0}},  // 8  [[[a+ a+]^0 a~]^1/2 a~]^0
  };
  return t;
}
int orb_rank(int a) { return orb_strings()[a].kl.empty() ? 1 : orb_strings()[a].kl.back(); }
int orb_dn(int a) {
  int d = 0;
  for (int x : orb_strings()[a].dag) d += x ? 1 : -1;
  return d;
}
constexpr int kOrbSite0 = 3000;  // OpKey.i of the strings of site p: kOrbSite0 + p
OpKey orb_key(int site, int a) { return OpKey{K_T0 + orb_dn(a), kOrbSite0 + site, a, orb_rank(a)}; }
bool is_orb_key(const OpKey& k) { return k.kind >= K_TM2 && k.i >= kOrbSite0; }
}  // namespace

std::unique_ptr<Block> Engine::enlarge(const Block& b, int site) {
  const SiteAlgebra& sa = site_algebra();
  const double t_start = now_s();
  auto e = std::make_unique<Block>();
  e->left = b.left;
  e->nsites = b.nsites + 1;
  e->normal = b.normal;
  e->parent = &b.ops->basis;
  e->ops = std::make_unique<OpSet>();
  e->ops->be = be_;
  const Basis& bb = b.ops->basis;
  // enlarged sectors: collect (n, j) -> list of (bsec, site)
  std::map<std::pair<int, int>, std::vector<std::pair<int, int>>> es;
  for (size_t s = 0; s < bb.sec.size(); ++s)
    for (int t = 0; t < 3; ++t) {
      int jb = bb.sec[s].j, jt = kSiteJ[t];
      for (int J = std::abs(jb - jt); J <= jb + jt; J += 2)
        es[{bb.sec[s].n + kSiteN[t], J}].push_back({(int)s, t});
    }
  Basis& eb = e->ops->basis;
  int off = 0;
  for (auto& [key, list] : es) {
    Sector sec{key.first, key.second, 0, off};
    int loc = 0;
    int esec = (int)eb.sec.size();
    for (auto& [s, t] : list) {
      e->comps.push_back({s, t, esec, loc});
      loc += bb.sec[s].dim;
    }
    sec.dim = loc;
    off += loc;
    eb.sec.push_back(sec);
  }
  eb.total = off;
  std::vector<int> bsites = block_sites(b, n_);
  std::vector<int> esites = bsites;
  if (b.left) esites.push_back(site);
  else esites.insert(esites.begin(), site);
  const double t_alloc0 = now_s();
  std::vector<OpKey> keys;
  if (rdm_mode_ && orb_mode_) {
    // orbital-entanglement blocks: on the left, the single-orbital strings of
    // every site (carried, and created for the new site); nothing on the right
    if (b.left) {
      for (auto& [k, ptr] : b.ops->ops)
        if (is_orb_key(k)) keys.push_back(k);
      for (int a = 0; a < (int)orb_strings().size(); ++a) keys.push_back(orb_key(site, a));
    }
  } else if (rdm_mode_) {
    // measurement blocks: the single spinors and, on normal blocks, the pairs
    for (const OpKey& k : op_keys(esites, n_, e->normal))
      if (k.kind == K_C || (e->normal && (k.kind == K_A || k.kind == K_B))) keys.push_back(k);
  } else {
    keys = op_keys(esites, n_, e->normal);
  }
  e->ops->allocate(keys);
  stats_.t_enl_alloc += now_s() - t_alloc0;

  // ---- blocking terms, target by target
  Side bs;
  bs.blk = &b;
  bs.sites = bsites;
  bs.normal = b.normal;
  Side ss;
  ss.is_site = true;
  ss.site = site;
  ss.sites = {site};
  const bool L = b.left;
  std::vector<std::pair<OpKey, Term>> terms;
  auto T = [&](const OpKey& tk, const Operand& blk_op, const Operand& site_op, double c) {
    if (c == 0.0 || operand_zero(site_op)) return;
    // left part = block for L growth, site for R growth
    Term t;
    t.k2 = tk.k2;
    t.coef = c;
    if (L) { t.x = blk_op; t.y = site_op; }
    else { t.x = site_op; t.y = blk_op; }
    terms.push_back({tk, t});
  };
  Operand I = op_id();
  const int s = site;
  if (rdm_mode_ && orb_mode_) {
    if (L) {
      for (auto& [k, ptr] : b.ops->ops)
        if (is_orb_key(k)) T(k, op_blk(k.kind, k.i, k.j, k.k2), op_site(sa.I), 1.0);
      for (int a = 0; a < (int)orb_strings().size(); ++a)
        T(orb_key(s, a), I, op_site(site_string(orb_strings()[a].dag, orb_strings()[a].kl)), 1.0);
    }
    stats_.t_enl_terms += now_s() - t_start;
    place_terms(b, nullptr, *e, terms);
    return e;
  }
  std::vector<int> outs;
  for (int p = 0; p < n_; ++p)
    if (!in_sites(esites, p)) outs.push_back(p);

  // H
  if (!rdm_mode_) {
    OpKey tk{K_H, 0, 0, 0};
    T(tk, op_blk(K_H, 0, 0, 0), op_site(sa.I), 1.0);
    SiteOp hs = site_add(sa.N.scaled(hh(s, s)), sa.Hu, g(s, s, s, s));
    T(tk, I, op_site(hs), 1.0);
    std::vector<Term> cr;
    if (L) emit_cross(this, bs, ss, cr);
    else emit_cross(this, ss, bs, cr);
    for (auto& t : cr) terms.push_back({tk, t});
  }
  // C_p
  for (int p : esites) {
    OpKey tk{K_C, p, 0, 1};
    if (p == s) T(tk, I, op_site(sa.C), 1.0);
    else T(tk, op_blk(K_C, p, 0, 1), op_site(sa.I), 1.0);
  }
  // temporaries for the S recurrence when the block holds normal pairs
  std::unique_ptr<OpSet> tmp;
  auto comp_op = [&](int kind, int p, int q, int k2) -> Operand {
    // complementary operator of the block for the pair (p, q), any order
    if (!b.normal) {
      if (p <= q) return op_blk(kind, p, q, k2);
      // (p, q) from (q, p): P^k_pq = (-1)^k P^k_qp, QJ symmetric, QK^k_pq = c_k adj(QK^k_qp)
      Operand o = op_blk(kind, q, p, k2);
      if (kind == K_QK) return o;  // adjoint handled by caller through flag below
      return o;
    }
    return op_blk(kind, p, q, k2);  // looked up in tmp
  };
  if (b.normal && b.nsites > 0 && !rdm_mode_) {
    tmp = std::make_unique<OpSet>();
    tmp->be = be_;
    tmp->basis = bb;
    std::vector<OpKey> tk;
    for (int p : outs) {
      tk.push_back({K_QJ, p, s, 0});
      tk.push_back({K_QK, p, s, 0});
      tk.push_back({K_QK, p, s, 2});
      tk.push_back({K_P, p, s, 0});
      tk.push_back({K_P, p, s, 2});
    }
    tmp->allocate(tk);
    const double tc0 = now_s();
    build_comp_from_normal(b, *tmp, tk);
    stats_.t_enl_comp += now_s() - tc0;
  }
  // S_p, p outside the enlarged block
  for (int p : rdm_mode_ ? std::vector<int>() : outs) {
    OpKey tk{K_S, p, 0, 1};
    T(tk, op_blk(K_S, p, 0, 1), op_site(sa.I), 1.0);
    SiteOp so = site_add(sa.D.scaled(0.5 * hh(p, s)), sa.NnD, g(p, s, s, s));
    T(tk, I, op_site(so), 1.0);
    if (b.nsites == 0) continue;
    // pair operators of the block for (p, s), with the sign/adjoint fixes of a stored (s, p)
    auto pair = [&](int kind, int k2, double& sign, int& adj) -> Operand {
      sign = 1.0;
      adj = 0;
      if (b.normal || p <= s) return op_blk(kind, p, s, k2);
      if (kind == K_P && k2 == 2) sign = -1.0;
      if (kind == K_QK) {
        adj = 1;
        sign = kAdjB[k2 / 2];
      }
      return op_blk(kind, s, p, k2, adj);
    };
    double sg;
    int ad;
    // M1: -sqrt2 [QJ_ps (x) a~_s]
    {
      Operand q = pair(K_QJ, 0, sg, ad);
      T(tk, q, op_site(sa.D), -kSqrt2 * sg);
    }
    // M2: c2_k [QK^k_ps (x) a~_s]
    for (int k = 0; k < 2; ++k) {
      Operand q = pair(K_QK, 2 * k, sg, ad);
      T(tk, q, op_site(sa.D), (L ? kC2L[k] : kC2R[k]) * sg);
    }
    // M3: c3_k [P^k_ps (x) a+_s]   (c3 equals c2 on both sides)
    for (int k = 0; k < 2; ++k) {
      Operand q = pair(K_P, 2 * k, sg, ad);
      T(tk, q, op_site(sa.C), (L ? kC2L[k] : kC2R[k]) * sg);
    }
    for (int r : bsites) {
      // M4: g_psst [a~_t (x) n_s]
      T(tk, op_blk(K_C, r, 0, 1, 1), op_site(sa.N), g(p, s, s, r));
      // M5: g_psrs c5_k [a~_r (x) [a+_s a~_s]^k]
      for (int k = 0; k < 2; ++k)
        T(tk, op_blk(K_C, r, 0, 1, 1), op_site(sa.CD[k]), g(p, s, r, s) * (L ? kC5L[k] : kC5R[k]));
      // M6: g_pqss c6 [a+_q (x) [a~_s a~_s]^0]
      T(tk, op_blk(K_C, r, 0, 1), op_site(sa.DD0), g(p, r, s, s) * kC6);
    }
  }
  (void)comp_op;
  if (e->normal) {
    for (size_t a = 0; a < esites.size(); ++a)
      for (size_t c = a; c < esites.size(); ++c) {
        int p = esites[a], q = esites[c];
        for (int k = 0; k < 2; ++k) {
          OpKey ta{K_A, p, q, 2 * k}, tb{K_B, p, q, 2 * k};
          if (p != s && q != s) {
            if (!(p == q && k == 1)) T(ta, op_blk(K_A, p, q, 2 * k), op_site(sa.I), 1.0);
            T(tb, op_blk(K_B, p, q, 2 * k), op_site(sa.I), 1.0);
          } else if (p == s && q == s) {
            if (k == 0) T(ta, I, op_site(sa.CC0), 1.0);
            T(tb, I, op_site(sa.CD[k]), 1.0);
          } else {
            // one index on the site: L growth has q == s, R growth has p == s
            int r = (p == s) ? q : p;
            T(ta, op_blk(K_C, r, 0, 1), op_site(sa.C), 1.0);
            T(tb, op_blk(K_C, r, 0, 1, L ? 0 : 1), op_site(L ? sa.D : sa.C), 1.0);
          }
        }
      }
  } else if (!rdm_mode_) {
    for (size_t a = 0; a < outs.size(); ++a)
      for (size_t c = a; c < outs.size(); ++c) {
        int p = outs[a], q = outs[c];
        for (int k = 0; k < 2; ++k) {
          double sk = k ? -1.0 : 1.0;
          OpKey tp{K_P, p, q, 2 * k}, tq{K_QK, p, q, 2 * k};
          if (!(p == q && k == 1)) {
            T(tp, op_blk(K_P, p, q, 2 * k), op_site(sa.I), 1.0);
            if (k == 0) T(tp, I, op_site(sa.DD0), g(p, q, s, s));
            for (int r : bsites) {
              double c = L ? (g(p, q, r, s) + sk * g(p, q, s, r)) : (sk * g(p, q, r, s) + g(p, q, s, r));
              T(tp, op_blk(K_C, r, 0, 1, 1), op_site(sa.D), c);
            }
          }
          T(tq, op_blk(K_QK, p, q, 2 * k), op_site(sa.I), 1.0);
          T(tq, I, op_site(sa.CD[k]), g(p, s, q, s));
          for (int r : bsites) {
            if (L) {
              T(tq, op_blk(K_C, r, 0, 1), op_site(sa.D), g(p, r, q, s));
              T(tq, op_blk(K_C, r, 0, 1, 1), op_site(sa.C), g(p, s, q, r) * kSwapB[k]);
            } else {
              T(tq, op_blk(K_C, r, 0, 1, 1), op_site(sa.C), g(p, s, q, r));
              T(tq, op_blk(K_C, r, 0, 1), op_site(sa.D), g(p, r, q, s) * kSwapB[k]);
            }
          }
        }
        OpKey tj{K_QJ, p, q, 0};
        T(tj, op_blk(K_QJ, p, q, 0), op_site(sa.I), 1.0);
        T(tj, I, op_site(sa.CD[0]), g(p, s, s, q));
        for (int r : bsites) {
          if (L) {
            T(tj, op_blk(K_C, r, 0, 1), op_site(sa.D), g(p, r, s, q));
            T(tj, op_blk(K_C, r, 0, 1, 1), op_site(sa.C), g(p, s, r, q) * kSwapB[0]);
          } else {
            T(tj, op_blk(K_C, r, 0, 1, 1), op_site(sa.C), g(p, s, r, q));
            T(tj, op_blk(K_C, r, 0, 1), op_site(sa.D), g(p, r, s, q) * kSwapB[0]);
          }
        }
      }
  }
  stats_.t_enl_terms += now_s() - t_start;
  place_terms(b, tmp.get(), *e, terms);
  return e;
}

// ============================================================ place_terms
namespace {
struct SrcBlock {
  const double* ptr = nullptr;  // nullptr: identity
  int trans = 0;
  int ld = 0;
  double coef = 1.0;
  bool ok = false;
};
// Block (bra, ket) of a block operand on `basis`, honouring the adjoint flag.
SrcBlock find_block(OpSet& set, const OpSet* tmp, const Operand& x, int bra, int ket) {
  SrcBlock r;
  const Basis& B = set.basis;
  if (x.t == Operand::ID) {
    if (bra != ket) return r;
    r.ok = true;
    r.ld = B.sec[bra].dim;
    return r;
  }
  double* base = set.get(x.key);
  OpSet* owner = &set;
  if (!base && tmp) {
    base = tmp->get(x.key);
    owner = const_cast<OpSet*>(tmp);
  }
  if (!base) return r;
  int dn = kind_dn(x.key.kind);
  const Layout& L = owner->layout(dn, x.key.k2);
  if (!x.adj) {
    int bi = L.find(bra, ket);
    if (bi < 0) return r;
    r.ptr = base + L.blk[bi].off;
    r.ld = L.blk[bi].cols;
    r.ok = true;
  } else {
    int bi = L.find(ket, bra);
    if (bi < 0) return r;
    r.ptr = base + L.blk[bi].off;
    r.ld = L.blk[bi].cols;
    r.trans = 1;
    r.coef = adjoint_coef(B.sec[bra].j, B.sec[ket].j, x.key.k2);
    r.ok = true;
  }
  return r;
}
// find_block with the operand's storage resolved once (base and layout of a
// block operand; both null for the identity)
struct ResolvedOperand {
  const double* base = nullptr;
  const Layout* lay = nullptr;
  bool ok = false;
};
ResolvedOperand resolve(OpSet& set, const OpSet* tmp, const Operand& x) {
  ResolvedOperand r;
  if (x.t == Operand::ID) {
    r.ok = true;
    return r;
  }
  const double* base = set.get(x.key);
  OpSet* owner = &set;
  if (!base && tmp) {
    base = tmp->get(x.key);
    owner = const_cast<OpSet*>(tmp);
  }
  if (!base) return r;
  r.base = base;
  r.lay = &owner->layout(kind_dn(x.key.kind), x.key.k2);
  r.ok = true;
  return r;
}
SrcBlock block_of(const Basis& B, const ResolvedOperand& ro, const Operand& x, int bra, int ket) {
  SrcBlock r;
  if (x.t == Operand::ID) {
    if (bra != ket) return r;
    r.ok = true;
    r.ld = B.sec[bra].dim;
    return r;
  }
  if (!x.adj) {
    int bi = ro.lay->find(bra, ket);
    if (bi < 0) return r;
    r.ptr = ro.base + ro.lay->blk[bi].off;
    r.ld = ro.lay->blk[bi].cols;
    r.ok = true;
  } else {
    int bi = ro.lay->find(ket, bra);
    if (bi < 0) return r;
    r.ptr = ro.base + ro.lay->blk[bi].off;
    r.ld = ro.lay->blk[bi].cols;
    r.trans = 1;
    r.coef = adjoint_coef(B.sec[bra].j, B.sec[ket].j, x.key.k2);
    r.ok = true;
  }
  return r;
}
double site_val(const Operand& y, int bra, int ket) {
  if (y.t == Operand::ID) return bra == ket ? 1.0 : 0.0;
  return y.s.m[bra][ket];
}
}  // namespace

void Engine::place_terms(const Block& b, const OpSet* tmp, Block& e,
                         const std::vector<std::pair<OpKey, Term>>& terms) {
  OpSet& bo = *b.ops;
  OpSet& eo = *e.ops;
  const Basis& bb = bo.basis;
  const Basis& eb = eo.basis;
  std::vector<std::vector<const EnlComp*>> by(eb.sec.size());
  for (auto& c : e.comps) by[c.esec].push_back(&c);
  const bool L = e.left;
  const double t_host = now_s();
  // Every destination sub-block of a target operator has a dense index
  // (layout block, bra component, ket component); the segments of one
  // target are grouped by it with a counting sort, in term order.
  struct LayoutIndex {
    std::vector<size_t> base;  // per layout block
    size_t total = 0;
  };
  // The layouts of the targets and operands are created first, so that the
  // threaded passes below only read the layout maps.
  {
    std::set<std::pair<int, int>> used;
    for (const auto& [tk, t] : terms) {
      used.insert({kind_dn(tk.kind), tk.k2});
      const Operand& bop = L ? t.x : t.y;
      if (bop.t != Operand::ID) used.insert({kind_dn(bop.key.kind), bop.key.k2});
    }
    for (auto& [dn, k2] : used) {
      eo.layout(dn, k2);
      bo.layout(dn, k2);
      if (tmp) const_cast<OpSet*>(tmp)->layout(dn, k2);
    }
  }
  std::map<const Layout*, LayoutIndex> lidx;
  for (auto& [key, lay] : eo.layouts) {
    LayoutIndex li;
    for (auto& blk : lay.blk) {
      li.base.push_back(li.total);
      li.total += by[blk.bra].size() * by[blk.ket].size();
    }
    lidx.emplace(&lay, std::move(li));
  }
  struct TermCtx {
    double* dst = nullptr;
    const Layout* TL = nullptr;
    const LayoutIndex* LI = nullptr;
    ResolvedOperand rop;
  };
  std::vector<TermCtx> ctx(terms.size());
  struct Entry {
    uint32_t li;
    double* d;
    int rows, cols, ld;
    PlaceSeg seg;
  };
  // term chunks: context, then placement segments (pure host arithmetic)
  const size_t nterm = terms.size();
  const size_t chunk = std::max<size_t>(16, nterm / (8 * host_threads()) + 1);
  const size_t nchunk = (nterm + chunk - 1) / chunk;
  std::vector<std::vector<Entry>> parts(nchunk);
  std::vector<std::pair<const Entry*, const Entry*>> range(nterm, {nullptr, nullptr});
  host_parallel_for(nchunk, [&](size_t c) {
    const size_t t0 = c * chunk, t1 = std::min(nterm, t0 + chunk);
    std::vector<size_t> ends;
    std::vector<Entry>& out = parts[c];
    for (size_t i = t0; i < t1; ++i) {
      TermCtx& cx = ctx[i];
      const auto& [tk, t] = terms[i];
      cx.dst = eo.get(tk);
      if (cx.dst) {
        cx.TL = &eo.layout(kind_dn(tk.kind), tk.k2);
        cx.LI = &lidx.at(cx.TL);
        const Operand& bop = L ? t.x : t.y;
        if (bop.t == Operand::SITE) throw std::runtime_error("site operand on block part");
        cx.rop = resolve(bo, tmp, bop);
      }
      if (cx.dst && cx.rop.ok) {
        const Operand& bop = L ? t.x : t.y;   // operand on the block part
        const Operand& sop = L ? t.y : t.x;   // operand on the site part
        for (size_t bi = 0; bi < cx.TL->blk.size(); ++bi) {
          const auto& blk = cx.TL->blk[bi];
          int Jp = eb.sec[blk.bra].j, J = eb.sec[blk.ket].j;
          const auto& cps = by[blk.bra];
          const auto& cs = by[blk.ket];
          for (size_t ia = 0; ia < cps.size(); ++ia)
            for (size_t ic = 0; ic < cs.size(); ++ic) {
              const EnlComp* cp = cps[ia];
              const EnlComp* c = cs[ic];
              double sv = site_val(sop, cp->site, c->site);
              if (sv == 0.0) continue;
              SrcBlock src = block_of(bb, cx.rop, bop, cp->bsec, c->bsec);
              if (!src.ok) continue;
              int jb_p = bb.sec[cp->bsec].j, jb = bb.sec[c->bsec].j;
              int js_p = kSiteJ[cp->site], js = kSiteJ[c->site];
              double tp;
              int nleft, pright;
              if (L) {
                tp = tensor_product_coef(jb_p, jb, bop.k2, js_p, js, sop.k2, Jp, J, t.k2);
                nleft = bb.sec[c->bsec].n;
                pright = sop.par;
              } else {
                tp = tensor_product_coef(js_p, js, sop.k2, jb_p, jb, bop.k2, Jp, J, t.k2);
                nleft = kSiteN[c->site];
                pright = bop.par;
              }
              if (tp == 0.0) continue;
              double sign = ((pright & nleft) & 1) ? -1.0 : 1.0;
              double alpha = t.coef * tp * sv * sign * src.coef;
              int rows = bb.sec[cp->bsec].dim, cols = bb.sec[c->bsec].dim;
              if (alpha == 0.0 || rows == 0 || cols == 0) continue;
              double* d = cx.dst + blk.off + (size_t)cp->eoff * blk.cols + c->eoff;
              out.push_back({(uint32_t)(cx.LI->base[bi] + ia * cs.size() + ic), d, rows, cols, blk.cols,
                             PlaceSeg{src.ptr, src.ld, src.trans, alpha}});
            }
        }
      }
      ends.push_back(out.size());
    }
    // entry range of every term of the chunk (out no longer grows)
    size_t prev = 0;
    for (size_t k = 0; k < ends.size(); ++k) {
      range[t0 + k] = {out.data() + prev, out.data() + ends[k]};
      prev = ends[k];
    }
  });
  // terms with segments grouped by target (targets in key order, terms in
  // term order within a target)
  std::vector<uint32_t> tord;
  for (size_t i = 0; i < nterm; ++i)
    if (ctx[i].dst && range[i].first != range[i].second) tord.push_back((uint32_t)i);
  std::stable_sort(tord.begin(), tord.end(),
                   [&](uint32_t a, uint32_t b) { return terms[a].first < terms[b].first; });
  std::vector<std::pair<size_t, size_t>> tgt;  // [begin, end) of a target's terms in tord
  for (size_t k = 0; k < tord.size();) {
    size_t j = k + 1;
    while (j < tord.size() && !(terms[tord[k]].first < terms[tord[j]].first)) ++j;
    tgt.push_back({k, j});
    k = j;
  }
  // the segments of one target ordered by destination sub-block, stably
  // (term order within a sub-block): a counting sort when the target has
  // many segments for its layout, else a comparison sort of its few
  // segments; target chunks in parallel, concatenated in target order
  const size_t tchunk = std::max<size_t>(1, tgt.size() / (4 * host_threads()) + 1);
  const size_t ntchunk = (tgt.size() + tchunk - 1) / tchunk;
  std::vector<std::vector<PlaceGroup>> cgroups(ntchunk);
  std::vector<std::vector<PlaceSeg>> csegs(ntchunk);
  host_parallel_for(ntchunk, [&](size_t c) {
    std::vector<uint32_t> count;
    std::vector<const Entry*> order;
    auto& groups = cgroups[c];
    auto& segs = csegs[c];
    for (size_t g = c * tchunk; g < std::min(tgt.size(), (c + 1) * tchunk); ++g) {
      const LayoutIndex& LI = *ctx[tord[tgt[g].first]].LI;
      size_t ne = 0;
      for (size_t k = tgt[g].first; k < tgt[g].second; ++k) ne += range[tord[k]].second - range[tord[k]].first;
      order.clear();
      if (4 * ne >= LI.total) {
        count.assign(LI.total + 1, 0);
        for (size_t k = tgt[g].first; k < tgt[g].second; ++k)
          for (const Entry* x = range[tord[k]].first; x != range[tord[k]].second; ++x) ++count[x->li + 1];
        for (size_t k = 1; k <= LI.total; ++k) count[k] += count[k - 1];
        order.assign(ne, nullptr);
        for (size_t k = tgt[g].first; k < tgt[g].second; ++k)
          for (const Entry* x = range[tord[k]].first; x != range[tord[k]].second; ++x) order[count[x->li]++] = x;
      } else {
        for (size_t k = tgt[g].first; k < tgt[g].second; ++k)
          for (const Entry* x = range[tord[k]].first; x != range[tord[k]].second; ++x) order.push_back(x);
        std::stable_sort(order.begin(), order.end(), [](const Entry* a, const Entry* b) { return a->li < b->li; });
      }
      for (size_t k = 0; k < ne;) {
        size_t j = k;
        PlaceGroup pg;
        pg.dst = order[k]->d;
        pg.rows = order[k]->rows;
        pg.cols = order[k]->cols;
        pg.ld = order[k]->ld;
        pg.seg_begin = (int)segs.size();
        while (j < ne && order[j]->li == order[k]->li) segs.push_back(order[j++]->seg);
        pg.seg_count = (int)(j - k);
        groups.push_back(pg);
        k = j;
      }
    }
  });
  std::vector<PlaceGroup> groups;
  std::vector<PlaceSeg> segs;
  for (size_t c = 0; c < ntchunk; ++c) {
    const int base = (int)segs.size();
    for (PlaceGroup pg : cgroups[c]) {
      pg.seg_begin += base;
      groups.push_back(pg);
    }
    segs.insert(segs.end(), csegs[c].begin(), csegs[c].end());
  }
  stats_.t_enl_place_host += now_s() - t_host;
  const double t_run = now_s();
  if (!groups.empty()) be_->place(groups, segs);
  stats_.t_enl_place_run += now_s() - t_run;
}

// ============================================================ complementary from normal
// P^k_pq = sum_{a,b in blk} g_pqab [a~_a a~_b]^k,  QJ_pq = sum g_pabq B^0_ab,
// QK^k_pq = sum g_paqb B^k_ab, built from the stored normal operators
// (A^k_ab, B^k_ab with a <= b) by one dense GEMM per source layout
// (coefficient matrix times the stacked operators) and an adjoint placement.
void Engine::build_comp_from_normal(const Block& b, OpSet& dst, const std::vector<OpKey>& keys) {
  OpSet& src = *b.ops;
  std::vector<int> bs = block_sites(b, n_);
  // source ops of a layout in allocation order
  auto stacked = [&](int dn, int k2, std::vector<OpKey>& order) -> const double* {
    const double* base = nullptr;
    std::vector<std::pair<const double*, OpKey>> v;
    for (auto& [k, p] : src.ops)
      if (kind_dn(k.kind) == dn && k.k2 == k2) v.push_back({p, k});
    std::sort(v.begin(), v.end(), [](auto& x, auto& y) { return x.first < y.first; });
    for (auto& [p, k] : v) order.push_back(k);
    if (!v.empty()) base = v.front().first;
    return base;
  };
  for (int kind : {K_P, K_QJ, K_QK})
    for (int k2 : {0, 2}) {
      if (kind == K_QJ && k2 == 2) continue;
      std::vector<OpKey> tk;
      for (auto& k : keys)
        if (k.kind == kind && k.k2 == k2 && dst.get(k)) tk.push_back(k);
      if (tk.empty()) continue;
      int sdn = (kind == K_P) ? 2 : 0;
      std::vector<OpKey> order;
      const double* X = stacked(sdn, k2, order);
      if (!X) continue;
      const Layout& SL = src.layout(sdn, k2);
      int K = (int)order.size(), M = (int)tk.size();
      std::map<OpKey, int> col;
      for (int i = 0; i < K; ++i) col[order[i]] = i;
      std::vector<double> Gd((size_t)M * K, 0.0), Ga((size_t)M * K, 0.0);
      double sk = (k2 == 2) ? -1.0 : 1.0;
      for (int m = 0; m < M; ++m) {
        int p = tk[m].i, q = tk[m].j;
        for (size_t ia = 0; ia < bs.size(); ++ia)
          for (size_t ib = ia; ib < bs.size(); ++ib) {
            int a = bs[ia], c = bs[ib];
            if (kind == K_P) {
              if (a == c && k2 == 2) continue;
              auto it = col.find({K_A, a, c, k2});
              if (it == col.end()) continue;
              double v = g(p, q, a, c) + (a != c ? sk * g(p, q, c, a) : 0.0);
              Ga[(size_t)m * K + it->second] += -v;  // P = -adj(sum v A)
            } else {
              auto it = col.find({K_B, a, c, k2});
              if (it == col.end()) continue;
              if (kind == K_QJ) {
                Gd[(size_t)m * K + it->second] += g(p, a, c, q);
                if (a != c) Ga[(size_t)m * K + it->second] += g(p, c, a, q);
              } else {
                Gd[(size_t)m * K + it->second] += g(p, a, q, c);
                if (a != c) Ga[(size_t)m * K + it->second] += kAdjB[k2 / 2] * g(p, c, q, a);
              }
            }
          }
      }
      size_t N = SL.size;
      for (int pass = 0; pass < 2; ++pass) {
        std::vector<double>& G = pass == 0 ? Gd : Ga;
        bool any = false;
        for (double v : G) if (v != 0.0) { any = true; break; }
        if (!any) continue;
        double* Gdev = (double*)be_->alloc(G.size() * sizeof(double));
        be_->copy_h2d(Gdev, G.data(), G.size() * sizeof(double));
        double* Y = (double*)be_->alloc((size_t)M * N * sizeof(double));
        be_->memset0(Y, (size_t)M * N * sizeof(double));
        GemmBuilder gb;
        // the N dimension can be large: split into column panels
        const size_t panel = 1 << 20;
        for (size_t c0 = 0; c0 < N; c0 += panel) {
          int nc = (int)std::min(panel, N - c0);
          gb.add(Y + c0, M, nc, (int)N, GemmSeg{Gdev, X + c0, K, K, (int)N, 0, 0, 1.0});
        }
        // complementary operators stay float64 under the tcgen05 renormalisation
        gb.run(be_, opt_.prec_renorm == Precision::TC_TF32X3 ? Precision::FP64 : opt_.prec_renorm);
        // place rows of Y into the targets (directly, or as adjoint)
        PlaceBuilder pb;
        const Layout& DL = dst.layout(kind_dn(kind), k2);
        for (int m = 0; m < M; ++m) {
          double* d = dst.get(tk[m]);
          const double* y = Y + (size_t)m * N;
          for (auto& blk : DL.blk) {
            if (pass == 0) {
              int si = SL.find(blk.bra, blk.ket);
              if (si < 0) continue;
              pb.add(d + blk.off, blk.rows, blk.cols, blk.cols,
                     PlaceSeg{y + SL.blk[si].off, SL.blk[si].cols, 0, 1.0});
            } else {
              int si = SL.find(blk.ket, blk.bra);
              if (si < 0) continue;
              double c = adjoint_coef(dst.basis.sec[blk.bra].j, dst.basis.sec[blk.ket].j, k2);
              pb.add(d + blk.off, blk.rows, blk.cols, blk.cols,
                     PlaceSeg{y + SL.blk[si].off, SL.blk[si].cols, 1, c});
            }
          }
        }
        pb.run(be_);
        be_->sync();
        be_->free(Y);
        be_->free(Gdev);
      }
    }
}

// ============================================================ renormalisation
// One tcgen05 contraction sigma_b += sum alpha op(A) P op(B)^T over the given
// blocks and items (device pointers): plan, split planes, launch, wait.
// Counted as "other GEMM work" (profiling tag 0).
void Engine::tc_contract(const std::vector<HpsiBlock>& blocks, const std::vector<HpsiItem>& items, double flops) {
  if (blocks.empty() || items.empty()) return;
  TcPlan tp;
  void* pool = nullptr;
  const int tc_ctas = hpsi_tc_max_ctas();
  hpsi_tc_prepare(blocks, items, [&](size_t bytes) { return pool = be_->alloc(bytes); }, tp,
                  tc_ctas > 0 ? tc_ctas : be_->sm_count());
  if (opt_.debug_bounds) {
    const std::string bad = tc_plan_check(tp, blocks);
    if (!bad.empty()) {
      if (pool) be_->free(pool);
      throw std::logic_error("internal: tcgen05 plan: " + bad);
    }
  }
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  std::vector<SplitJob> jobs = tp.op_jobs;
  jobs.insert(jobs.end(), tp.psi_jobs.begin(), tp.psi_jobs.end());
  const size_t ob = 0, oc = al(blocks.size() * sizeof(HpsiBlock));
  const size_t ot = al(oc + tp.items.size() * sizeof(TcItem));
  const size_t orr = al(ot + tp.tasks.size() * sizeof(HpsiTask));
  const size_t oj = al(orr + tp.reds.size() * sizeof(HpsiReduce));
  const size_t oco = al(oj + jobs.size() * sizeof(SplitJob));
  const size_t oct = al(oco + tp.cta_off.size() * sizeof(int));
  const size_t os = al(oct + tp.cta_task.size() * sizeof(TcSlot));
  char* d = (char*)be_->alloc(os + tp.scratch * sizeof(double) + 256);
  be_->copy_h2d(d + ob, blocks.data(), blocks.size() * sizeof(HpsiBlock));
  if (!tp.items.empty()) be_->copy_h2d(d + oc, tp.items.data(), tp.items.size() * sizeof(TcItem));
  if (!tp.tasks.empty()) be_->copy_h2d(d + ot, tp.tasks.data(), tp.tasks.size() * sizeof(HpsiTask));
  if (!tp.reds.empty()) be_->copy_h2d(d + orr, tp.reds.data(), tp.reds.size() * sizeof(HpsiReduce));
  if (!jobs.empty()) {
    be_->copy_h2d(d + oj, jobs.data(), jobs.size() * sizeof(SplitJob));
    be_->split((const SplitJob*)(d + oj), (int)jobs.size(), (float*)pool);
  }
  if (!tp.cta_off.empty()) be_->copy_h2d(d + oco, tp.cta_off.data(), tp.cta_off.size() * sizeof(int));
  if (!tp.cta_task.empty()) be_->copy_h2d(d + oct, tp.cta_task.data(), tp.cta_task.size() * sizeof(TcSlot));
  TcLaunch L;
  L.blocks = (const HpsiBlock*)(d + ob);
  L.items = (const TcItem*)(d + oc);
  L.tasks = (const HpsiTask*)(d + ot);
  L.cta_off = (const int*)(d + oco);
  L.cta_task = (const TcSlot*)(d + oct);
  L.ncta = tp.cta_off.empty() ? 0 : (int)tp.cta_off.size() - 1;
  L.reds = (const HpsiReduce*)(d + orr);
  L.nreds = (int)tp.reds.size();
  L.scratch = (double*)(d + os);
  L.pool = pool;
  L.units = tp.units;
  L.drain_terms = opt_.tc_drain_terms;
  be_->hpsi_tc(L, flops, 0);
  be_->sync();
  be_->check_device_flag();
  be_->free(d);
  if (pool) be_->free(pool);
}

// O'(a', a) = U_a'^T O(a', a) U_a with Ut[a] = kept eigenvectors as rows.
std::unique_ptr<Block> Engine::renormalize(Block& enl, const SavedU& U, bool switch_to_comp) {
  const std::vector<int>& kept = U.kept;
  std::vector<const double*> ut(U.off.size(), nullptr);
  for (size_t s = 0; s < U.off.size(); ++s)
    if (kept[s] > 0) ut[s] = U.ut((int)s);
  auto nb = std::make_unique<Block>();
  nb->left = enl.left;
  nb->nsites = enl.nsites;
  nb->normal = enl.normal;
  nb->ops = std::make_unique<OpSet>();
  nb->ops->be = be_;
  const Basis& eb = enl.ops->basis;
  Basis& b = nb->ops->basis;
  std::vector<int> map(eb.sec.size(), -1);
  int off = 0;
  for (size_t s = 0; s < eb.sec.size(); ++s) {
    if (kept[s] <= 0) continue;
    map[s] = (int)b.sec.size();
    b.sec.push_back({eb.sec[s].n, eb.sec[s].j, kept[s], off});
    off += kept[s];
  }
  b.total = off;
  std::vector<OpKey> keys;
  for (auto& [k, p] : enl.ops->ops) keys.push_back(k);
  nb->ops->allocate(keys);
  // per layout: T = E U (temp), O' = U^T T
  std::map<std::pair<int, int>, std::vector<OpKey>> by;
  for (auto& k : keys) by[{kind_dn(k.kind), k.k2}].push_back(k);
  if (opt_.prec_renorm == Precision::TC_TF32X3) {
    // each block O'(a', a) = Ut_a' E(a', a) Ut_a^T is one item of a tcgen05
    // contraction (op(A) = Ut_a', P = E block, op(B) = Ut_a), the operators
    // of a layout in groups that bound the plan
    for (auto& [lk, ks] : by) {
      const Layout& EL = enl.ops->layout(lk.first, lk.second);
      const Layout& NL = nb->ops->layout(lk.first, lk.second);
      if (NL.size == 0) continue;
      std::vector<HpsiBlock> blocks;
      std::vector<HpsiItem> items;
      double flops = 0.0;
      auto flush = [&]() {
        tc_contract(blocks, items, flops);
        blocks.clear();
        items.clear();
        flops = 0.0;
      };
      for (size_t oi = 0; oi < ks.size(); ++oi) {
        const double* E = enl.ops->get(ks[oi]);
        double* O = nb->ops->get(ks[oi]);
        if (!E || !O) continue;
        for (size_t i = 0; i < EL.blk.size(); ++i) {
          auto& bl = EL.blk[i];
          const int na = map[bl.bra], nk = map[bl.ket];
          if (na < 0 || nk < 0) continue;
          const int ka = kept[bl.ket], kap = kept[bl.bra];
          const int ni = NL.find(na, nk);
          auto& nbk = NL.blk[ni];
          HpsiBlock hb{};
          hb.C = O + nbk.off;
          hb.m = kap;
          hb.n = ka;
          hb.ldc = ka;
          hb.item_begin = (int)items.size();
          hb.item_count = 1;
          HpsiItem it{};
          it.A = ut[bl.bra];
          it.lda = bl.rows;
          it.transA = 0;
          it.P = E + bl.off;
          it.ldp = bl.cols;
          it.B = ut[bl.ket];
          it.ldb = bl.cols;
          it.transB = 0;
          it.ka = bl.rows;
          it.kb = bl.cols;
          it.alpha = 1.0;
          items.push_back(it);
          blocks.push_back(hb);
          flops += 2.0 * kap * bl.rows * bl.cols + 2.0 * kap * bl.cols * ka;
        }
        if (items.size() >= 200000) flush();
      }
      flush();
    }
  }
  for (auto& [lk, ks] : by) {
    if (opt_.prec_renorm == Precision::TC_TF32X3) break;
    const Layout& EL = enl.ops->layout(lk.first, lk.second);
    const Layout& NL = nb->ops->layout(lk.first, lk.second);
    if (NL.size == 0) continue;
    // temp layout sizes: block (a', a) -> m_a' x kept_a
    std::vector<size_t> toff(EL.blk.size(), 0);
    size_t tsz = 0;
    for (size_t i = 0; i < EL.blk.size(); ++i) {
      auto& bl = EL.blk[i];
      toff[i] = tsz;
      if (map[bl.bra] >= 0 && map[bl.ket] >= 0) tsz += (size_t)bl.rows * kept[bl.ket];
    }
    if (tsz == 0) continue;
    // chunk operators to bound the temporary
    size_t per = std::max<size_t>(1, (size_t)(256u << 20) / (tsz * sizeof(double)));
    double* T = (double*)be_->alloc(std::min(per, ks.size()) * tsz * sizeof(double));
    for (size_t c0 = 0; c0 < ks.size(); c0 += per) {
      size_t c1 = std::min(ks.size(), c0 + per);
      be_->memset0(T, (c1 - c0) * tsz * sizeof(double));
      GemmBuilder g1, g2;
      for (size_t oi = c0; oi < c1; ++oi) {
        const double* E = enl.ops->get(ks[oi]);
        double* O = nb->ops->get(ks[oi]);
        if (!E || !O) continue;
        double* Tb = T + (oi - c0) * tsz;
        for (size_t i = 0; i < EL.blk.size(); ++i) {
          auto& bl = EL.blk[i];
          int na = map[bl.bra], nk = map[bl.ket];
          if (na < 0 || nk < 0) continue;
          int ka = kept[bl.ket], kap = kept[bl.bra];
          // T(a',a) = E(a',a) * Ut_a^T
          g1.add(Tb + toff[i], bl.rows, ka, ka,
                 GemmSeg{E + bl.off, ut[bl.ket], bl.cols, bl.cols, bl.cols, 0, 1, 1.0});
          int ni = NL.find(na, nk);
          auto& nbk = NL.blk[ni];
          // O'(a',a) = Ut_a' * T(a',a)
          g2.add(O + nbk.off, kap, ka, ka,
                 GemmSeg{ut[bl.bra], Tb + toff[i], bl.rows, bl.rows, ka, 0, 0, 1.0});
        }
      }
      g1.run(be_, opt_.prec_renorm);
      g2.run(be_, opt_.prec_renorm);
    }
    be_->sync();
    be_->free(T);
  }
  if (switch_to_comp) {
    // new complementary block: H, C, S copied, P/QJ/QK built from the normal pairs
    auto cb = std::make_unique<Block>();
    cb->left = nb->left;
    cb->nsites = nb->nsites;
    cb->normal = false;
    cb->ops = std::make_unique<OpSet>();
    cb->ops->be = be_;
    cb->ops->basis = nb->ops->basis;
    std::vector<int> sites = block_sites(*nb, n_);
    auto ck = op_keys(sites, n_, false);
    cb->ops->allocate(ck);
    for (auto& k : ck) {
      if (k.kind == K_H || k.kind == K_C || k.kind == K_S) {
        double* d = cb->ops->get(k);
        const double* s = nb->ops->get(k);
        if (d && s) {
          size_t sz = cb->ops->layout(kind_dn(k.kind), k.k2).size;
          be_->copy_d2d(d, s, sz * sizeof(double));
        }
      }
    }
    build_comp_from_normal(*nb, *cb->ops, ck);
    be_->sync();
    return cb;
  }
  return nb;
}

// ============================================================ bond: psi, H psi
struct PsiLayout {
  struct Blk {
    int a, b, rows, cols;
    size_t off;
  };
  std::vector<Blk> blk;
  std::vector<int> lut;  // a * nb + b
  int nb = 0;
  size_t size = 0;
  int find(int a, int b) const { return lut[(size_t)a * nb + b]; }
};
PsiLayout make_psi(const Basis& L, const Basis& R, int N, int S) {
  PsiLayout P;
  P.nb = (int)R.sec.size();
  P.lut.assign(L.sec.size() * R.sec.size(), -1);
  for (size_t a = 0; a < L.sec.size(); ++a)
    for (size_t b = 0; b < R.sec.size(); ++b) {
      if (L.sec[a].n + R.sec[b].n != N || !triangle(L.sec[a].j, R.sec[b].j, S)) continue;
      P.lut[a * R.sec.size() + b] = (int)P.blk.size();
      P.blk.push_back({(int)a, (int)b, L.sec[a].dim, R.sec[b].dim, P.size});
      P.size += (size_t)L.sec[a].dim * R.sec[b].dim;
    }
  return P;
}
// bra sectors reachable from ket sector `ket` through operand x on basis B
void reach(const Basis& B, const ResolvedOperand& ro, const Operand& x, int ket,
           std::vector<std::pair<int, SrcBlock>>& out) {
  out.clear();
  if (!ro.ok) return;
  if (x.t == Operand::ID) {
    SrcBlock s;
    s.ok = true;
    s.ld = B.sec[ket].dim;
    out.push_back({ket, s});
    return;
  }
  for (size_t bra = 0; bra < B.sec.size(); ++bra) {
    if (B.sec[bra].n != B.sec[ket].n + x.dn || !triangle(B.sec[ket].j, x.k2, B.sec[bra].j)) continue;
    SrcBlock s = block_of(B, ro, x, (int)bra, ket);
    if (s.ok) out.push_back({(int)bra, s});
  }
}

// H_eff psi as one fused launch: per sigma block, the list of items
// alpha op(A) P op(B)^T (left operator block, psi block, right operator block).
struct HPsiPlan {
  PsiLayout psi;
  double* in = nullptr;   // psi input buffer
  double* out = nullptr;  // sigma output buffer
  // device copies of the task lists (built once per bond)
  void* dev = nullptr;
  HpsiBlock* d_blocks = nullptr;
  HpsiItem* d_items = nullptr;
  HpsiTask* d_tasks = nullptr;
  HpsiReduce* d_reds = nullptr;
  double* scratch = nullptr;
  Precision prec = Precision::FP64;  // kernel the task list was planned for
  // tcgen05 path: split planes, items on them, and the per-product psi splits
  void* tc_pool = nullptr;
  TcItem* d_tcitems = nullptr;
  SplitJob* d_psi_jobs = nullptr;
  int n_psi_jobs = 0;
  TcLaunch tc;  // device lists of the persistent contraction
  // operands and schedule on the host (rescheduled while autotuning), the
  // device lists and scratch of the current schedule, and the tuning state
  std::unique_ptr<TcPlan> tcp;
  std::vector<HpsiBlock> tc_blocks;
  int tc_ncta = 0;
  void* sched = nullptr;
  bool tuning = false;
  uint64_t tune_key = 0;
  int tc_cand = 0;  // candidate of the current schedule (index into the candidate list)
  int ntasks = 0, nreds = 0;
  size_t nitems = 0;
  double flops = 0.0;
  double* diag = nullptr;  // diagonal of H_eff (Davidson preconditioner)
};

void Engine::plan_hpsi(Block& Le, Block& Re, HPsiPlan& plan) {
  const double tp0 = now_s();
  OpSet& lo = *Le.ops;
  OpSet& ro = *Re.ops;
  plan.psi = make_psi(lo.basis, ro.basis, n_elec_, two_s_);
  const PsiLayout& P = plan.psi;
  std::vector<Term> terms;
  terms.push_back({op_blk(K_H, 0, 0, 0), op_id(), 0, 1.0});
  terms.push_back({op_id(), op_blk(K_H, 0, 0, 0), 0, 1.0});
  Side ls, rs;
  ls.blk = &Le;
  ls.sites = block_sites(Le, n_);
  ls.normal = Le.normal;
  rs.blk = &Re;
  rs.sites = block_sites(Re, n_);
  rs.normal = Re.normal;
  emit_cross(this, ls, rs, terms);
  std::vector<std::vector<HpsiItem>> per(P.blk.size());
  std::vector<std::pair<int, HpsiItem>> diag_items;
  plan.flops = 0.0;
  // operand layouts created first (the threaded pass only reads the layout
  // maps); items of term chunks generated on the host pool and merged in term
  // order, so the item order (and the summation order) does not depend on
  // the number of threads
  {
    std::set<std::pair<int, int>> used;
    for (const Term& t : terms) {
      if (t.x.t != Operand::ID) used.insert({kind_dn(t.x.key.kind), t.x.key.k2});
      if (t.y.t != Operand::ID) used.insert({kind_dn(t.y.key.kind), t.y.key.k2});
    }
    for (auto& [dn, k2] : used) {
      lo.layout(dn, k2);
      ro.layout(dn, k2);
    }
  }
  std::vector<std::pair<ResolvedOperand, ResolvedOperand>> rop(terms.size());
  struct Gen {
    std::vector<std::pair<int, HpsiItem>> items;  // (sigma block, item) in term order
    std::vector<std::pair<int, HpsiItem>> diag;
    double flops = 0.0;
  };
  auto generate = [&](size_t t0, size_t t1, Gen& out) {
    std::vector<std::pair<int, SrcBlock>> lr, rr;
    for (size_t ti = t0; ti < t1; ++ti) {
      const Term& t = terms[ti];
      // rank k of the two factors of the scalar coupling [x^k (x) y^k]^0
      int kop = (t.x.t != Operand::ID) ? t.x.k2 : t.y.k2;
      rop[ti] = {resolve(lo, nullptr, t.x), resolve(ro, nullptr, t.y)};
      const ResolvedOperand& rx = rop[ti].first;
      const ResolvedOperand& ry = rop[ti].second;
      if (!rx.ok || !ry.ok) continue;
      for (auto& kb : P.blk) {
        reach(lo.basis, rx, t.x, kb.a, lr);
        if (lr.empty()) continue;
        reach(ro.basis, ry, t.y, kb.b, rr);
        if (rr.empty()) continue;
        const Sector& sa = lo.basis.sec[kb.a];
        const Sector& sb = ro.basis.sec[kb.b];
        double sign = ((t.y.par & sa.n) & 1) ? -1.0 : 1.0;
        for (auto& [ap, xs] : lr)
          for (auto& [bp, ys] : rr) {
            int pi = P.find(ap, bp);
            if (pi < 0) continue;
            const Sector& sap = lo.basis.sec[ap];
            const Sector& sbp = ro.basis.sec[bp];
            double hc = hpsi_coef(sap.j, sbp.j, sa.j, sb.j, kop, two_s_);
            if (hc == 0.0) continue;
            HpsiItem it;
            it.A = (t.x.t == Operand::ID) ? nullptr : xs.ptr;
            it.lda = xs.ld;
            it.transA = xs.trans;
            it.P = plan.in + kb.off;
            it.ldp = sb.dim;
            it.B = (t.y.t == Operand::ID) ? nullptr : ys.ptr;
            it.ldb = ys.ld;
            it.transB = ys.trans;
            it.ka = sa.dim;
            it.kb = sb.dim;
            it.alpha = t.coef * hc * sign * xs.coef * ys.coef;
            out.items.push_back({pi, it});
            if (it.A) out.flops += 2.0 * sap.dim * sa.dim * sb.dim;
            if (it.B) out.flops += 2.0 * sap.dim * sbp.dim * sb.dim;
            if (ap == kb.a && bp == kb.b) out.diag.push_back({pi, it});
          }
      }
    }
  };
  const size_t nterm = terms.size();
  const size_t chunk = std::max<size_t>(4, nterm / (8 * host_threads()) + 1);
  const size_t nchunk = (nterm + chunk - 1) / chunk;
  std::vector<Gen> gens(nchunk);
  host_parallel_for(nchunk, [&](size_t c) { generate(c * chunk, std::min(nterm, (c + 1) * chunk), gens[c]); });
  for (auto& g : gens) {
    for (auto& [pi, it] : g.items) per[pi].push_back(it);
    diag_items.insert(diag_items.end(), g.diag.begin(), g.diag.end());
    plan.flops += g.flops;
  }
  if (opt_.verbose >= 2) {
    // shape statistics of the contraction, weighted by flops: the smallest
    // GEMM dimension bounds the tensor-core tile efficiency
    const double edges[] = {16, 32, 64, 128, 256, 512, 1e30};
    double hist[7] = {0}, tot = 0.0;
    size_t nit = 0;
    for (size_t b = 0; b < P.blk.size(); ++b)
      for (auto& it : per[b]) {
        ++nit;
        int m = P.blk[b].rows, n = P.blk[b].cols;
        double f = (it.A ? 2.0 * m * it.ka * it.kb : 0.0) + (it.B ? 2.0 * m * n * it.kb : 0.0);
        int d = std::min({m, n, it.ka, it.kb});
        int k = 0;
        while (d > edges[k]) ++k;
        hist[k] += f;
        tot += f;
      }
    std::fprintf(stderr, "hpsi shapes: terms %zu blocks %zu items %zu flops %.3e | min-dim<=16 %.2f <=32 %.2f "
                 "<=64 %.2f <=128 %.2f <=256 %.2f <=512 %.2f >512 %.2f\n",
                 terms.size(), P.blk.size(), nit, tot, hist[0] / tot, hist[1] / tot, hist[2] / tot,
                 hist[3] / tot, hist[4] / tot, hist[5] / tot, hist[6] / tot);
    // tensor work of the tcgen05 blocking (128 x 256 sigma tiles, stage 1 in
    // 256-column super-chunks, k-blocks of 16) over the algorithmic work
    // (stage 1 once per row tile and group of g column tiles, g = 1, 2, 4)
    double a1 = 0.0, a2 = 0.0, e1[3] = {0.0, 0.0, 0.0}, e2 = 0.0;
    auto r16 = [](int x) { return (double)((x + 15) & ~15); };
    for (size_t b = 0; b < P.blk.size(); ++b)
      for (auto& it : per[b]) {
        const int m = P.blk[b].rows, n = P.blk[b].cols;
        const double mt = 128.0 * ((m + 127) / 128);
        const int nt = (n + 255) / 256;
        const int ka = it.A ? it.ka : m, kb = it.B ? it.kb : n;
        a1 += (double)m * ka * kb;
        a2 += (double)m * kb * n;
        const double s1 = mt * r16(ka) * ((kb / 256) * 256.0 + (kb % 256 ? r16(kb % 256) : 0.0));
        for (int q = 0; q < 3; ++q) e1[q] += s1 * ((nt + (1 << q) - 1) >> q);
        e2 += mt * r16(kb) * (256.0 * (n / 256) + (n % 256 ? r16(n % 256) : 0.0));
      }
    const double am = std::max(a1, 1.0);
    std::fprintf(stderr, "hpsi tc blocking: stage-1 work x%.2f (x%.2f, x%.2f shared by 2, 4 column tiles), stage-2 "
                 "work x%.2f of algorithmic (stage-1 flops / all %.2f)\n", e1[0] / am, e1[1] / am, e1[2] / am,
                 e2 / std::max(a2, 1.0), a1 / std::max(a1 + a2, 1.0));
  }
  const double tp1 = now_s();
  stats_.t_plan_items += tp1 - tp0;
  std::vector<HpsiBlock> blocks;
  std::vector<HpsiItem> items;
  for (size_t b = 0; b < P.blk.size(); ++b) {
    HpsiBlock hb;
    hb.C = plan.out + P.blk[b].off;
    hb.m = P.blk[b].rows;
    hb.n = P.blk[b].cols;
    hb.ldc = P.blk[b].cols;
    hb.item_begin = (int)items.size();
    hb.item_count = (int)per[b].size();
    items.insert(items.end(), per[b].begin(), per[b].end());
    blocks.push_back(hb);
  }
  std::vector<HpsiTask> tasks;
  std::vector<HpsiReduce> reds;
  plan.prec = opt_.prec;
  const bool tc = plan.prec == Precision::TC_TF32X3;
  TcPlan tp_local;
  TcPlan& tp = tc ? *(plan.tcp = std::make_unique<TcPlan>()) : tp_local;
  size_t scr = 0;
  if (tc) {
    if (plan.tc_pool) be_->free(plan.tc_pool);
    plan.tc_pool = nullptr;
    const int tc_ctas = hpsi_tc_max_ctas();
    plan.tc_ncta = tc_ctas > 0 ? tc_ctas : be_->sm_count();
    hpsi_tc_operands(blocks, items, [&](size_t bytes) { return plan.tc_pool = be_->alloc(bytes); }, tp);
    plan.tc_blocks = blocks;
    // the schedule: the default shape, or with autotuning the fastest shape
    // of this sector histogram, or the next candidate still to be timed
    plan.tc_cand = 0;
    plan.tuning = false;
    if (opt_.tc_autotune) {
      const size_t nc = tc_shape_candidates().size();
      plan.tune_key = tc_histogram_key(blocks, plan.tc_ncta);
      TuneRec& rec = tune_cache_[plan.tune_key];
      if (rec.ms.size() != nc) rec.ms.assign(nc, -1.0);
      if (rec.best >= 0) {
        plan.tc_cand = rec.best;
      } else {
        plan.tuning = true;
        while (plan.tc_cand < (int)nc && rec.ms[plan.tc_cand] >= 0) ++plan.tc_cand;
      }
    }
    hpsi_tc_schedule(blocks, tp, tc_shape_candidates()[plan.tc_cand],
                     tc_ctas_for(tc_shape_candidates()[plan.tc_cand].cluster));
    if (opt_.debug_bounds) {
      const std::string bad = tc_plan_check(tp, blocks);
      if (!bad.empty()) throw std::logic_error("internal: tcgen05 plan: " + bad);
    }
    last_tc_key_ = opt_.tc_autotune ? plan.tune_key : 0;
    last_tc_cand_ = plan.tc_cand;
    have_tc_plan_ = true;
  } else {
    scr = hpsi_plan_tasks(blocks, plan.prec, tasks, reds);
  }
  const double tp2 = now_s();
  stats_.t_plan_tasks += tp2 - tp1;
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  size_t ob = 0, oi = al(ob + blocks.size() * sizeof(HpsiBlock));
  // the tcgen05 path reads its own item descriptors only
  size_t oc = al(oi + (tc ? 0 : items.size()) * sizeof(HpsiItem));
  size_t ot = al(oc + tp.items.size() * sizeof(TcItem));
  size_t orr = al(ot + tasks.size() * sizeof(HpsiTask));
  size_t oj = al(orr + reds.size() * sizeof(HpsiReduce));
  size_t opj = al(oj + tp.op_jobs.size() * sizeof(SplitJob));
  // (the tcgen05 schedule's lists and scratch live in plan.sched)
  size_t os = al(opj + tp.psi_jobs.size() * sizeof(SplitJob));
  size_t total = os + scr * sizeof(double) + 256;
  if (plan.dev) be_->free(plan.dev);
  plan.dev = nullptr;
  if (plan.sched) be_->free(plan.sched);
  plan.sched = nullptr;
  plan.dev = be_->alloc(total);
  char* d = (char*)plan.dev;
  plan.d_blocks = (HpsiBlock*)(d + ob);
  plan.d_items = (HpsiItem*)(d + oi);
  plan.d_tcitems = (TcItem*)(d + oc);
  plan.d_tasks = (HpsiTask*)(d + ot);
  plan.d_reds = (HpsiReduce*)(d + orr);
  plan.d_psi_jobs = (SplitJob*)(d + opj);
  plan.n_psi_jobs = (int)tp.psi_jobs.size();
  plan.scratch = (double*)(d + os);
  if (!blocks.empty()) be_->copy_h2d(plan.d_blocks, blocks.data(), blocks.size() * sizeof(HpsiBlock));
  if (!tc && !items.empty()) be_->copy_h2d(plan.d_items, items.data(), items.size() * sizeof(HpsiItem));
  if (!tp.items.empty()) be_->copy_h2d(plan.d_tcitems, tp.items.data(), tp.items.size() * sizeof(TcItem));
  if (!tasks.empty()) be_->copy_h2d(plan.d_tasks, tasks.data(), tasks.size() * sizeof(HpsiTask));
  if (!reds.empty()) be_->copy_h2d(plan.d_reds, reds.data(), reds.size() * sizeof(HpsiReduce));
  if (!tp.psi_jobs.empty())
    be_->copy_h2d(plan.d_psi_jobs, tp.psi_jobs.data(), tp.psi_jobs.size() * sizeof(SplitJob));
  if (tc) tc_upload_schedule(plan);
  if (!tp.op_jobs.empty()) {
    // operator blocks (and identities) are constant during Davidson: split them once
    be_->copy_h2d(d + oj, tp.op_jobs.data(), tp.op_jobs.size() * sizeof(SplitJob));
    be_->split((const SplitJob*)(d + oj), (int)tp.op_jobs.size(), (float*)plan.tc_pool);
  }
  if (!tc) {
    plan.ntasks = (int)tasks.size();
    plan.nreds = (int)reds.size();
  }
  plan.nitems = items.size();
  be_->sync();
  const double tp3 = now_s();
  stats_.t_plan_upload += tp3 - tp2;
  // diagonal: sigma_diag(a,b)[i,j] = sum alpha A(a,a)[i,i] B(b,b)[j,j] over the
  // items whose ket block equals their sigma block (outer products, k = 1)
  if (plan.diag) be_->free(plan.diag);
  plan.diag = (double*)be_->alloc(std::max<size_t>(P.size, 1) * sizeof(double));
  be_->memset0(plan.diag, std::max<size_t>(P.size, 1) * sizeof(double));
  int mx = 1;
  for (auto& b : P.blk) mx = std::max(mx, std::max(b.rows, b.cols));
  if (ones_len_ < (size_t)mx) {
    if (ones_) be_->free(ones_);
    std::vector<double> o(mx, 1.0);
    ones_ = (double*)be_->alloc(mx * sizeof(double));
    be_->copy_h2d(ones_, o.data(), mx * sizeof(double));
    ones_len_ = mx;
  }
  GemmBuilder gd;
  for (auto& [pi, it] : diag_items) {
    const auto& bl = P.blk[pi];
    const double* a = it.A ? it.A : ones_;
    const double* b = it.B ? it.B : ones_;
    int lda = it.A ? it.lda + 1 : 1;
    int ldb = it.B ? it.ldb + 1 : 1;
    gd.add(plan.diag + bl.off, bl.rows, bl.cols, bl.cols, GemmSeg{a, b, 1, lda, ldb, 0, 1, it.alpha});
  }
  gd.run(be_, Precision::FP64);
  be_->sync();
  stats_.t_plan_diag += now_s() - tp3;
}


// Device lists and scratch of the plan's current tcgen05 schedule, in an
// allocation of their own (replaced when the plan is rescheduled).
void Engine::tc_upload_schedule(HPsiPlan& plan) {
  const TcPlan& tp = *plan.tcp;
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t ot = 0;
  const size_t orr = al(ot + tp.tasks.size() * sizeof(HpsiTask));
  const size_t oco = al(orr + tp.reds.size() * sizeof(HpsiReduce));
  const size_t oct = al(oco + tp.cta_off.size() * sizeof(int));
  const size_t os = al(oct + tp.cta_task.size() * sizeof(TcSlot));
  const size_t total = os + tp.scratch * sizeof(double) + 256;
  if (plan.sched) be_->free(plan.sched);
  plan.sched = nullptr;
  plan.sched = be_->alloc(total);
  char* d = (char*)plan.sched;
  if (!tp.tasks.empty()) be_->copy_h2d(d + ot, tp.tasks.data(), tp.tasks.size() * sizeof(HpsiTask));
  if (!tp.reds.empty()) be_->copy_h2d(d + orr, tp.reds.data(), tp.reds.size() * sizeof(HpsiReduce));
  if (!tp.cta_off.empty()) be_->copy_h2d(d + oco, tp.cta_off.data(), tp.cta_off.size() * sizeof(int));
  if (!tp.cta_task.empty()) be_->copy_h2d(d + oct, tp.cta_task.data(), tp.cta_task.size() * sizeof(TcSlot));
  plan.d_tasks = (HpsiTask*)(d + ot);
  plan.d_reds = (HpsiReduce*)(d + orr);
  plan.scratch = (double*)(d + os);
  plan.tc = TcLaunch();
  plan.tc.blocks = plan.d_blocks;
  plan.tc.items = plan.d_tcitems;
  plan.tc.tasks = plan.d_tasks;
  plan.tc.cta_off = (const int*)(d + oco);
  plan.tc.cta_task = (const TcSlot*)(d + oct);
  plan.tc.ncta = (int)tp.cta_off.size() - 1;
  plan.tc.reds = plan.d_reds;
  plan.tc.nreds = (int)tp.reds.size();
  plan.tc.scratch = plan.scratch;
  plan.tc.pool = plan.tc_pool;
  plan.tc.units = tp.units;
  plan.tc.drain_terms = opt_.tc_drain_terms;
  plan.tc.tile_n = tp.shape.tile_n;
  plan.tc.cluster = tp.shape.cluster;
  plan.ntasks = (int)tp.tasks.size();
  plan.nreds = (int)tp.reds.size();
}

int Engine::tc_ctas_for(int cluster) const {
  const int m = hpsi_tc_max_ctas(cluster);
  return m > 0 ? m : std::max(cluster, be_->sm_count() / cluster * cluster);
}

void Engine::tc_reschedule(HPsiPlan& plan, int candidate) {
  be_->sync();  // the old lists and scratch may still be read by queued work
  hpsi_tc_schedule(plan.tc_blocks, *plan.tcp, tc_shape_candidates()[candidate],
                   tc_ctas_for(tc_shape_candidates()[candidate].cluster));
  if (opt_.debug_bounds) {
    const std::string bad = tc_plan_check(*plan.tcp, plan.tc_blocks);
    if (!bad.empty()) throw std::logic_error("internal: tcgen05 plan: " + bad);
  }
  plan.tc_cand = candidate;
  last_tc_cand_ = candidate;
  tc_upload_schedule(plan);
}

bool Engine::tc_schedule_info(int shape[4], std::vector<double>* ms) const {
  if (!have_tc_plan_ || last_tc_cand_ < 0) return false;
  const TcShape s = tc_shape_candidates()[last_tc_cand_];
  shape[0] = s.tile_n;
  shape[1] = s.chunks_per_cta;
  shape[2] = s.order;
  shape[3] = s.cluster;
  if (ms) {
    ms->assign(tc_shape_candidates().size(), -1.0);
    auto it = tune_cache_.find(last_tc_key_);
    if (last_tc_key_ && it != tune_cache_.end() && it->second.ms.size() == ms->size()) *ms = it->second.ms;
  }
  return true;
}

void Engine::apply_hpsi(HPsiPlan& plan) {
  be_->memset0(plan.out, plan.psi.size * sizeof(double));
  if (plan.prec == Precision::TC_TF32X3) {
    be_->split(plan.d_psi_jobs, plan.n_psi_jobs, (float*)plan.tc_pool);
    if (!plan.tuning) {
      be_->hpsi_tc(plan.tc, plan.flops);
      return;
    }
    // Autotuning: every candidate schedule of this sector histogram computes
    // one real product, timed on the device (contraction and chunk
    // reduction); once all were timed the fastest is kept for this plan and
    // every later plan with the same histogram.
    be_->mark_begin(1);
    be_->hpsi_tc(plan.tc, plan.flops);
    const double ms = be_->mark_end(1);
    be_->check_device_flag();
    TuneRec& rec = tune_cache_[plan.tune_key];
    if (rec.ms[plan.tc_cand] < 0) rec.ms[plan.tc_cand] = ms;
    int next = -1;
    for (size_t k = 0; k < rec.ms.size() && next < 0; ++k)
      if (rec.ms[k] < 0) next = (int)k;
    if (next < 0) {
      rec.best = (int)(std::min_element(rec.ms.begin(), rec.ms.end()) - rec.ms.begin());
      plan.tuning = false;
      next = rec.best;
    }
    if (next != plan.tc_cand) tc_reschedule(plan, next);
  } else {
    be_->hpsi(plan.d_blocks, plan.d_items, plan.d_tasks, plan.ntasks, plan.d_reds, plan.nreds,
              plan.scratch, plan.prec, plan.flops);
  }
}

// ============================================================ Davidson
namespace {
uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
}  // namespace

double Engine::davidson(HPsiPlan& plan, double* psi, int* iters) {
  const size_t len = plan.psi.size;
  const int M = std::max(4, opt_.max_space);
  double* V = (double*)be_->alloc((size_t)M * len * sizeof(double));
  double* HV = (double*)be_->alloc((size_t)M * len * sizeof(double));
  double* dv = (double*)be_->alloc((size_t)(M * M + 4 * M + 8) * sizeof(double));
  double* dA = dv;
  double* dw = dv + M * M;
  double* dZ = dw + M;        // reused for coefficient vectors (M)
  double* dc = dZ + M;
  double* dEv = (double*)be_->alloc((size_t)M * M * sizeof(double));
  std::vector<double> A((size_t)M * M, 0.0), w(M), Z((size_t)M * M), c(M), tmpv(M);
  // guess: provided psi (if nonzero) else a deterministic pseudo-random vector
  {
    std::vector<double> h(len);
    be_->copy_d2h(h.data(), psi, len * sizeof(double));
    double nrm = 0.0;
    for (double x : h) nrm += x * x;
    if (!(nrm > 1e-20)) {
      for (size_t i = 0; i < len; ++i)
        h[i] = ((splitmix64(i + 12345 + opt_.seed * 0x9E3779B97F4A7C15ull) >> 11) * (1.0 / 9007199254740992.0)) -
               0.5;
      nrm = 0.0;
      for (double x : h) nrm += x * x;
    }
    nrm = std::sqrt(nrm);
    for (double& x : h) x /= nrm;
    be_->copy_h2d(V, h.data(), len * sizeof(double));
  }
  auto dot_host = [&](const double* a, const double* b) {
    be_->dots(a, 1, len, len, b, dc);
    double r;
    be_->copy_d2h(&r, dc, sizeof(double));
    return r;
  };
  auto apply = [&](int i) {
    be_->copy_d2d(plan.in, V + (size_t)i * len, len * sizeof(double));
    auto t0 = std::chrono::steady_clock::now();
    if (call_ms_) be_->mark_begin();
    apply_hpsi(plan);
    if (call_ms_) call_ms_->push_back(be_->mark_end());
    be_->sync();
    if (plan.prec == Precision::TC_TF32X3) be_->check_device_flag();
    auto t1 = std::chrono::steady_clock::now();
    stats_.hpsi_seconds += std::chrono::duration<double>(t1 - t0).count();
    stats_.hpsi_flops += plan.flops;
    stats_.hpsi_calls += 1;
    be_->copy_d2d(HV + (size_t)i * len, plan.out, len * sizeof(double));
  };
  int m = 1;
  apply(0);
  double e = 0.0;
  double* x = psi;  // result vector
  double* r = plan.in;  // residual workspace (psi-in buffer reused between applies)
  int it = 0;
  double best_res = 1e300;
  int best_it = 0;
  double last_res = 1e300, last_tol = 0.0;
  for (it = 1; it <= opt_.max_davidson_iter; ++it) {
    // projected matrix: row/col m-1
    be_->dots(V, m, len, len, HV + (size_t)(m - 1) * len, dc);
    be_->copy_d2h(tmpv.data(), dc, m * sizeof(double));
    for (int i = 0; i < m; ++i) A[(size_t)i * M + (m - 1)] = A[(size_t)(m - 1) * M + i] = tmpv[i];
    // small eigenproblem on the device
    std::vector<double> Am((size_t)m * m);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) Am[(size_t)i * m + j] = 0.5 * (A[(size_t)i * M + j] + A[(size_t)j * M + i]);
    be_->copy_h2d(dA, Am.data(), Am.size() * sizeof(double));
    be_->eigh({EighTask{dA, dw, dEv, m}});
    be_->copy_d2h(w.data(), dw, m * sizeof(double));
    be_->copy_d2h(Z.data(), dEv, (size_t)m * m * sizeof(double));
    // lowest eigenpair = last row (eigenvalues descending)
    e = w[m - 1];
    last_gap_ = m >= 2 ? w[m - 2] - w[m - 1] : 0.0;
    for (int i = 0; i < m; ++i) c[i] = Z[(size_t)(m - 1) * m + i];
    be_->copy_h2d(dZ, c.data(), m * sizeof(double));
    be_->combine(x, 0.0, V, m, len, len, dZ);
    be_->combine(r, 0.0, HV, m, len, len, dZ);
    be_->axpby(r, 1.0, x, -e, len);
    double rn = std::sqrt(std::max(0.0, dot_host(r, r)));
    if (opt_.verbose > 1) std::fprintf(stderr, "  davidson it %d m %d E %.12f res %.3e\n", it, m, e, rn);
    // With split-precision H_eff psi the residual has a noise floor of about
    // 1e-7 |E| (TF32 pairs keep ~22 bits, FP32 accumulation): converge to
    // max(tol, 2e-7 |E|) and stop on stagnation (no 10% improvement in 8
    // iterations) in any mode.
    double tol_eff = opt_.davidson_tol;
    if (opt_.prec != Precision::FP64) tol_eff = std::max(tol_eff, 2e-7 * std::max(1.0, std::abs(e)));
    last_res = rn;
    last_tol = tol_eff;
    if (rn < tol_eff) break;
    if (rn < 0.9 * best_res) {
      best_res = rn;
      best_it = it;
    } else if (it - best_it >= 8 && rn < 1e3 * tol_eff) {
      break;
    }
    if (m >= M) {
      // restart with the lowest two Ritz vectors
      std::vector<double> c2((size_t)2 * m);
      for (int i = 0; i < m; ++i) {
        c2[i] = Z[(size_t)(m - 1) * m + i];
        c2[m + i] = Z[(size_t)(m - 2) * m + i];
      }
      double* nV = (double*)be_->alloc((size_t)2 * len * sizeof(double));
      double* nH = (double*)be_->alloc((size_t)2 * len * sizeof(double));
      for (int q = 0; q < 2; ++q) {
        be_->copy_h2d(dZ, c2.data() + (size_t)q * m, m * sizeof(double));
        be_->combine(nV + (size_t)q * len, 0.0, V, m, len, len, dZ);
        be_->combine(nH + (size_t)q * len, 0.0, HV, m, len, len, dZ);
      }
      be_->copy_d2d(V, nV, 2 * len * sizeof(double));
      be_->copy_d2d(HV, nH, 2 * len * sizeof(double));
      be_->free(nV);
      be_->free(nH);
      std::fill(A.begin(), A.end(), 0.0);
      A[0] = w[m - 1];
      A[(size_t)1 * M + 1] = w[m - 2];
      m = 2;
    }
    // new direction t = (D - E)^-1 r, orthogonalised twice against V
    double* t = V + (size_t)m * len;
    if (plan.diag) be_->precondition(t, r, plan.diag, e, len);
    else be_->copy_d2d(t, r, len * sizeof(double));
    for (int pass = 0; pass < 2; ++pass) {
      be_->dots(V, m, len, len, t, dc);
      be_->copy_d2h(tmpv.data(), dc, m * sizeof(double));
      for (int i = 0; i < m; ++i) tmpv[i] = -tmpv[i];
      be_->copy_h2d(dZ, tmpv.data(), m * sizeof(double));
      be_->combine(t, 1.0, V, m, len, len, dZ);
    }
    double tn = std::sqrt(std::max(0.0, dot_host(t, t)));
    if (tn < 1e-14) break;
    be_->axpby(t, 0.0, t, 1.0 / tn, len);
    apply(m);
    ++m;
  }
  if (iters) *iters = it;
  if (!(last_res < last_tol)) stats_.noconv_bonds += 1;
  be_->sync();
  be_->free(V);
  be_->free(HV);
  be_->free(dv);
  be_->free(dEv);
  return e;
}

// ============================================================ decimation
namespace {
struct Cand {
  double lam;
  int n, j, rank, sec;
};
std::vector<int> select(std::vector<Cand>& c, int D) {
  const double lam_min = 1e-12, tie = 1e-9;
  std::vector<int> idx;
  for (size_t i = 0; i < c.size(); ++i)
    if (c[i].lam >= lam_min) idx.push_back((int)i);
  auto key_less = [&](int a, int b) {
    if (c[a].lam != c[b].lam) return c[a].lam > c[b].lam;
    if (c[a].n != c[b].n) return c[a].n < c[b].n;
    if (c[a].j != c[b].j) return c[a].j < c[b].j;
    return c[a].rank < c[b].rank;
  };
  std::sort(idx.begin(), idx.end(), key_less);
  if ((int)idx.size() <= D) return idx;
  double ld = c[idx[D - 1]].lam;
  std::vector<int> hi, ti;
  for (int i : idx) {
    if (c[i].lam > ld * (1 + tie)) hi.push_back(i);
    else if (std::abs(c[i].lam - ld) <= ld * tie) ti.push_back(i);
  }
  std::sort(ti.begin(), ti.end(), [&](int a, int b) {
    if (c[a].n != c[b].n) return c[a].n < c[b].n;
    if (c[a].j != c[b].j) return c[a].j < c[b].j;
    return c[a].rank < c[b].rank;
  });
  for (int i : ti) {
    if ((int)hi.size() >= D) break;
    hi.push_back(i);
  }
  return hi;
}
}  // namespace

// rho per sector of the enlarged block being truncated, its eigenvectors, the
// selection of D multiplets; returns the kept eigenvectors (rows) per sector.
std::unique_ptr<SavedU> Engine::decimate(Block& enl, const HPsiPlan& plan, const double* psi,
                                         bool left, double* trunc) {
  const Basis& B = enl.ops->basis;
  const PsiLayout& P = plan.psi;
  size_t tot = 0;
  std::vector<size_t> roff(B.sec.size());
  for (size_t s = 0; s < B.sec.size(); ++s) {
    roff[s] = tot;
    tot += (size_t)B.sec[s].dim * B.sec[s].dim;
  }
  size_t wtot = B.total;
  double* buf = (double*)be_->alloc((2 * tot + wtot) * sizeof(double));
  be_->memset0(buf, (2 * tot + wtot) * sizeof(double));
  double* rho = buf;
  double* vec = buf + tot;
  double* wv = buf + 2 * tot;
  GemmBuilder gb;
  for (auto& bl : P.blk) {
    const double* pb = psi + bl.off;
    if (left) {
      int s = bl.a, m = bl.rows, k = bl.cols;
      gb.add(rho + roff[s], m, m, m, GemmSeg{pb, pb, k, k, k, 0, 1, 1.0});
    } else {
      int s = bl.b, m = bl.cols, k = bl.rows;
      gb.add(rho + roff[s], m, m, m, GemmSeg{pb, pb, k, m, m, 1, 0, 1.0});
    }
  }
  gb.run(be_, Precision::FP64);
  std::vector<EighTask> tasks;
  std::vector<size_t> woff(B.sec.size());
  size_t wo = 0;
  for (size_t s = 0; s < B.sec.size(); ++s) {
    woff[s] = wo;
    wo += B.sec[s].dim;
    if (B.sec[s].dim > 0) tasks.push_back({rho + roff[s], wv + woff[s], vec + roff[s], B.sec[s].dim});
  }
  be_->eigh(tasks);
  be_->check_device_flag();
  std::vector<double> w(wtot);
  be_->copy_d2h(w.data(), wv, wtot * sizeof(double));
  std::vector<Cand> cands;
  double total = 0.0;
  for (size_t s = 0; s < B.sec.size(); ++s)
    for (int r = 0; r < B.sec[s].dim; ++r) {
      double lam = w[woff[s] + r];
      total += lam;
      cands.push_back({lam, B.sec[s].n, B.sec[s].j, r, (int)s});
    }
  int Dk = opt_.D;
  if (opt_.trunc_target > 0.0) {
    // dynamic bond dimension: the fewest multiplets whose discarded weight is
    // at most trunc_target, between D_min and D
    std::vector<double> lams;
    lams.reserve(cands.size());
    for (auto& c : cands) lams.push_back(c.lam);
    std::sort(lams.begin(), lams.end(), std::greater<double>());
    double kept_w = 0.0;
    size_t k = 0;
    while (k < lams.size() && total - kept_w > opt_.trunc_target) kept_w += lams[k++];
    Dk = std::max(opt_.D_min, std::min(opt_.D, (int)k));
  }
  auto keep = select(cands, Dk);
  stats_.kept.push_back((int)keep.size());
  auto U = std::make_unique<SavedU>();
  U->be = be_;
  U->enl = B;
  U->comps = enl.comps;
  if (enl.parent) U->parent = *enl.parent;
  U->kept.assign(B.sec.size(), 0);
  double kw = 0.0;
  for (int i : keep) {
    U->kept[cands[i].sec] = std::max(U->kept[cands[i].sec], cands[i].rank + 1);
    kw += cands[i].lam;
  }
  // compact copy of the kept rows (eigenvalues descending: a prefix of rows)
  U->off.assign(B.sec.size(), 0);
  U->map.assign(B.sec.size(), -1);
  size_t uo = 0;
  int off = 0;
  for (size_t s = 0; s < B.sec.size(); ++s) {
    U->off[s] = uo;
    if (U->kept[s] > 0) {
      U->map[s] = (int)U->next.sec.size();
      U->next.sec.push_back({B.sec[s].n, B.sec[s].j, U->kept[s], off});
      off += U->kept[s];
    }
    uo += (size_t)U->kept[s] * B.sec[s].dim;
  }
  U->next.total = off;
  U->buf = (double*)be_->alloc(std::max<size_t>(uo, 1) * sizeof(double));
  for (size_t s = 0; s < B.sec.size(); ++s)
    if (U->kept[s] > 0)
      be_->copy_d2d(U->buf + U->off[s], vec + roff[s], (size_t)U->kept[s] * B.sec[s].dim * sizeof(double));
  be_->sync();
  be_->free(buf);
  *trunc = std::max(0.0, total - kw);
  return U;
}

// ============================================================ wavefunction guess
namespace {
// <((l s) a, r) S | (l, (s r) b) S>, all doubled
double recouple(int l, int s, int r, int a, int b, int S) {
  double six = wigner6j(l, s, a, r, S, b);
  if (six == 0.0) return 0.0;
  return phase2(l + s + r + S) * std::sqrt((a + 1.0) * (b + 1.0)) * six;
}
}  // namespace

void Engine::save_prev(int bond, const Block& Le, const Block& Re, const HPsiPlan& plan,
                       const double* psi) {
  if (prev_.psi) be_->free(prev_.psi);
  prev_.valid = true;
  prev_.bond = bond;
  prev_.Lb = Le.ops->basis;
  prev_.Rb = Re.ops->basis;
  prev_.Lc = Le.comps;
  prev_.Rc = Re.comps;
  prev_.blk.clear();
  for (auto& b : plan.psi.blk) prev_.blk.push_back({b.a, b.b, b.rows, b.cols, (int)b.off});
  prev_.len = plan.psi.size;
  prev_.psi = (double*)be_->alloc(std::max<size_t>(prev_.len, 1) * sizeof(double));
  be_->copy_d2d(prev_.psi, psi, prev_.len * sizeof(double));
}

// Moves the two-site wavefunction of bond b (from) to bond b+1: project the
// old enlarged left block onto its kept multiplets (U: L'(b) -> L(b+1)),
// recouple the site that changes side (6j), and expand the old right block
// R(b+2) into site (x) R(b+3) with its stored MPS tensor (V).  Exact when U
// keeps the whole support of the state.
void Engine::move_lr(const Prev& from, const SavedU& U, const SavedU& V, const Block& Le,
                     const Block& Re, const PsiLayout& P, double* psi) {
  const Basis& LB = Le.ops->basis;
  const Basis& RB = Re.ops->basis;
  const int S = two_s_;
  be_->memset0(psi, P.size * sizeof(double));
  const Basis& Lnew = U.next;            // L_[bond]
  const Basis& Rmid = V.next;            // R_[n-bond-1] = parent of prev R'
  // phi(l, b) = Ut_a psi(a, b)
  PsiLayout phiL = make_psi(Lnew, from.Rb, n_elec_, S);
  PsiLayout mid = make_psi(LB, Rmid, n_elec_, S);
  double* phi = (double*)be_->alloc(std::max<size_t>(phiL.size, 1) * sizeof(double));
  double* psm = (double*)be_->alloc(std::max<size_t>(mid.size, 1) * sizeof(double));
  be_->memset0(phi, std::max<size_t>(phiL.size, 1) * sizeof(double));
  be_->memset0(psm, std::max<size_t>(mid.size, 1) * sizeof(double));
  GemmBuilder g1;
  for (auto& b : from.blk) {
    int a = b[0], bb = b[1];
    int l = U.map[a];
    if (l < 0) continue;
    int pi = phiL.find(l, bb);
    if (pi < 0) continue;
    g1.add(phi + phiL.blk[pi].off, U.kept[a], b[3], b[3],
           GemmSeg{U.ut(a), from.psi + b[4], b[2], b[2], b[3], 0, 0, 1.0});
  }
  g1.run(be_, Precision::FP64);
  // recouple the site between the blocks
  PlaceBuilder pb;
  for (auto& pbk : phiL.blk) {
    int l = pbk.a, bb = pbk.b;
    for (auto& c : from.Rc) {
      if (c.esec != bb) continue;
      int sg = c.site, r = c.bsec;
      for (auto& cp : Le.comps) {
        if (cp.bsec != l || cp.site != sg) continue;
        int ap = cp.esec;
        int mi = mid.find(ap, r);
        if (mi < 0) continue;
        double co = recouple(Lnew.sec[l].j, kSiteJ[sg], Rmid.sec[r].j, LB.sec[ap].j,
                             from.Rb.sec[bb].j, S);
        if (co == 0.0) continue;
        double* d = psm + mid.blk[mi].off + (size_t)cp.eoff * mid.blk[mi].cols;
        const double* src = phi + pbk.off + c.eoff;
        pb.add(d, Lnew.sec[l].dim, Rmid.sec[r].dim, mid.blk[mi].cols,
               PlaceSeg{src, pbk.cols, 0, co});
      }
    }
  }
  pb.run(be_);
  // expand the right block: psi(a', e) = psm(a', r(e)) Ut_e
  GemmBuilder g2;
  for (size_t e = 0; e < V.enl.sec.size(); ++e) {
    int r = V.map[e];
    if (r < 0) continue;
    int eb = RB.find(V.enl.sec[e].n, V.enl.sec[e].j);
    if (eb < 0) continue;
    for (auto& mb : mid.blk) {
      if (mb.b != r) continue;
      int pi = P.find(mb.a, eb);
      if (pi < 0) continue;
      g2.add(psi + P.blk[pi].off, mb.rows, RB.sec[eb].dim, RB.sec[eb].dim,
             GemmSeg{psm + mb.off, V.ut((int)e), V.kept[e], mb.cols, RB.sec[eb].dim, 0, 0, 1.0});
    }
  }
  g2.run(be_, Precision::FP64);
  be_->sync();
  be_->free(phi);
  be_->free(psm);
}

// Predicted two-site wavefunction of bond `bond` from the state of the
// previous bond (one step of the sweep): project with the new block's kept
// eigenvectors, recouple the site that changes side (6j), expand the other
// block with its stored MPS tensor.  Falls back to zero (random start) when
// no previous state exists; the first bond uses the initial product state.
void Engine::guess(int bond, bool l2r, const Block& Le, const Block& Re, const HPsiPlan& plan,
                   double* psi) {
  be_->memset0(psi, plan.psi.size * sizeof(double));
  const PsiLayout& P = plan.psi;
  const Basis& LB = Le.ops->basis;
  const Basis& RB = Re.ops->basis;
  if (!prev_.valid) {
    // product state: L' = site 0 multiplet occ[0], R' = (site 1 (x) R(2)) multiplet path[1]
    if (bond != 0) return;
    int a = LB.find(occ_[0], kSiteJ[occ_[0]]);
    int nr = 0;
    for (int p = 1; p < n_; ++p) nr += occ_[p];
    int b = RB.find(nr, path_[1]);
    if (a < 0 || b < 0) return;
    int pi = P.find(a, b);
    if (pi < 0) return;
    int ca = -1, cb = -1;
    for (auto& c : Le.comps)
      if (c.esec == a && c.site == occ_[0]) ca = c.eoff;
    for (auto& c : Re.comps)
      if (c.esec == b && c.site == occ_[1] && c.bsec == 0) cb = c.eoff;
    if (ca < 0 || cb < 0) return;
    double one = 1.0;
    be_->copy_h2d(psi + P.blk[pi].off + (size_t)ca * P.blk[pi].cols + cb, &one, sizeof(double));
    return;
  }
  const int S = two_s_;
  (void)l2r;  // the move follows the position of the previous bond (turns included)
  if (prev_.bond == bond - 1) {
    move_lr(prev_, *LU_[bond], *RU_[n_ - bond - 1], Le, Re, P, psi);
  } else if (prev_.bond == bond + 1) {
    const SavedU& V = *RU_[n_ - bond - 2];  // R'(bond+1) -> R_[n-bond-2]
    const SavedU& U = *LU_[bond + 1];       // E ~ L'(bond) -> L_[bond+1]
    const Basis& Rnew = V.next;
    const Basis& Lmid = U.next;             // L_[bond+1] = parent of prev L'
    // phi(a, r) = psi(a, b) Ut_b^T
    PsiLayout phiL = make_psi(prev_.Lb, Rnew, n_elec_, S);
    PsiLayout mid = make_psi(Lmid, RB, n_elec_, S);
    double* phi = (double*)be_->alloc(std::max<size_t>(phiL.size, 1) * sizeof(double));
    double* psm = (double*)be_->alloc(std::max<size_t>(mid.size, 1) * sizeof(double));
    be_->memset0(phi, std::max<size_t>(phiL.size, 1) * sizeof(double));
    be_->memset0(psm, std::max<size_t>(mid.size, 1) * sizeof(double));
    GemmBuilder g1;
    for (auto& b : prev_.blk) {
      int a = b[0], bb = b[1];
      int r = V.map[bb];
      if (r < 0) continue;
      int pi = phiL.find(a, r);
      if (pi < 0) continue;
      g1.add(phi + phiL.blk[pi].off, b[2], V.kept[bb], V.kept[bb],
             GemmSeg{prev_.psi + b[4], V.ut(bb), b[3], b[3], b[3], 0, 1, 1.0});
    }
    g1.run(be_, Precision::FP64);
    PlaceBuilder pb;
    for (auto& pbk : phiL.blk) {
      int a = pbk.a, r = pbk.b;
      for (auto& c : prev_.Lc) {
        if (c.esec != a) continue;
        int l = c.bsec, sg = c.site;
        for (auto& cp : Re.comps) {
          if (cp.bsec != r || cp.site != sg) continue;
          int bp = cp.esec;
          int mi = mid.find(l, bp);
          if (mi < 0) continue;
          double co = recouple(Lmid.sec[l].j, kSiteJ[sg], Rnew.sec[r].j, prev_.Lb.sec[a].j,
                               RB.sec[bp].j, S);
          if (co == 0.0) continue;
          double* d = psm + mid.blk[mi].off + cp.eoff;
          const double* src = phi + pbk.off + (size_t)c.eoff * pbk.cols;
          pb.add(d, Lmid.sec[l].dim, Rnew.sec[r].dim, mid.blk[mi].cols,
                 PlaceSeg{src, pbk.cols, 0, co});
        }
      }
    }
    pb.run(be_);
    // expand the left block: psi(a'', b') = Ut_{a''}^T psm(l(a''), b')
    GemmBuilder g2;
    for (size_t e = 0; e < U.enl.sec.size(); ++e) {
      int l = U.map[e];
      if (l < 0) continue;
      int ea = LB.find(U.enl.sec[e].n, U.enl.sec[e].j);
      if (ea < 0) continue;
      for (auto& mb : mid.blk) {
        if (mb.a != l) continue;
        int pi = P.find(ea, mb.b);
        if (pi < 0) continue;
        g2.add(psi + P.blk[pi].off, LB.sec[ea].dim, mb.cols, mb.cols,
               GemmSeg{U.ut((int)e), psm + mb.off, U.kept[e], LB.sec[ea].dim, mb.cols, 1, 0, 1.0});
      }
    }
    g2.run(be_, Precision::FP64);
    be_->sync();
    be_->free(phi);
    be_->free(psm);
  }
}

// ============================================================ engine
Engine::Engine(Backend* be, int n, const double* h, const double* eri, double e_core, int n_elec,
               int two_s, const Options& opt, const int* occ, const int* two_s_right)
    : be_(be), n_(n), n_elec_(n_elec), two_s_(two_s), e_core_(e_core), opt_(opt) {
  if (n < 2) throw std::invalid_argument("need at least two orbitals");
  if (n_elec < 0 || n_elec > 2 * n) throw std::invalid_argument("n_elec out of range");
  if (two_s < 0 || ((n_elec - two_s) & 1)) throw std::invalid_argument("two_s parity");
  h_.assign(h, h + (size_t)n * n);
  g_.resize((size_t)n * n * n * n);
  // g_pqrs = (ps|qr) from chemists' integrals eri[p,q,r,s] = (pq|rs)
  for (int p = 0; p < n; ++p)
    for (int q = 0; q < n; ++q)
      for (int r = 0; r < n; ++r)
        for (int s = 0; s < n; ++s)
          g_[(((size_t)p * n + q) * n + r) * n + s] = eri[(((size_t)p * n + s) * n + q) * n + r];
  tL_ = (n - 1) / 2;
  tR_ = n - 1 - tL_;
  occ_.assign(occ, occ + n);
  path_.assign(two_s_right, two_s_right + n + 1);
  if (path_[0] != two_s || path_[n] != 0) throw std::invalid_argument("bad initial spin path");
  L_.resize(n + 1);
  R_.resize(n + 1);
  LU_.resize(n + 1);
  RU_.resize(n + 1);
  L_[0] = vacuum(true);
  L_[0]->normal = left_normal(0);
  if (!L_[0]->normal) {
    L_[0]->ops = std::make_unique<OpSet>();
    L_[0]->ops->be = be_;
    L_[0]->ops->basis.sec.push_back({0, 0, 1, 0});
    L_[0]->ops->basis.total = 1;
    L_[0]->ops->allocate(op_keys({}, n_, false));
  }
  build_initial_right();
}

void Engine::build_initial_right() {
  R_[0] = vacuum(false);
  R_[0]->normal = right_normal(0);
  if (!R_[0]->normal) {
    R_[0]->ops = std::make_unique<OpSet>();
    R_[0]->ops->be = be_;
    R_[0]->ops->basis.sec.push_back({0, 0, 1, 0});
    R_[0]->ops->basis.total = 1;
    R_[0]->ops->allocate(op_keys({}, n_, false));
  }
  int nr = 0;
  for (int r = 1; r <= n_ - 2; ++r) {
    int site = n_ - r;
    nr += occ_[site];
    auto e = enlarge(*R_[r - 1], site);
    const Basis& eb = e->ops->basis;
    int target = eb.find(nr, path_[site]);
    if (target < 0) throw std::runtime_error("initial state sector missing");
    std::vector<int> kept(eb.sec.size(), 0);
    kept[target] = 1;
    // the single multiplet: component (bsec 0, site occupation) of the target sector
    int eoff = -1;
    for (auto& c : e->comps)
      if (c.esec == target && c.site == occ_[site] && c.bsec == 0) eoff = c.eoff;
    if (eoff < 0) throw std::runtime_error("initial state component missing");
    int m = eb.sec[target].dim;
    std::vector<double> row(m, 0.0);
    row[eoff] = 1.0;
    auto U = std::make_unique<SavedU>();
    U->be = be_;
    U->enl = eb;
    U->comps = e->comps;
    U->parent = R_[r - 1]->ops->basis;
    U->kept = kept;
    U->map.assign(eb.sec.size(), -1);
    U->map[target] = 0;
    U->off.assign(eb.sec.size(), 0);
    U->next.sec.push_back({eb.sec[target].n, eb.sec[target].j, 1, 0});
    U->next.total = 1;
    U->buf = (double*)be_->alloc(m * sizeof(double));
    be_->copy_h2d(U->buf, row.data(), m * sizeof(double));
    bool sw = e->normal && !right_normal(r);
    R_[r] = renormalize(*e, *U, sw);
    RU_[r] = std::move(U);
    be_->sync();
  }
}

// ---- staging of stored blocks to pinned host memory (device budget)
// Bond b uses L(b) and R(n-b-2) in both directions; in sweep steps, L->R
// bond i is step i and R->L bond i is step (n-2) + (n-2-i), period 2n-4.
void Engine::memory_detail(size_t* dev, size_t* host, size_t* max_block, size_t* max_extra,
                           size_t* mps_bytes) const {
  size_t u = 0;
  for (auto* v : {&LU_, &RU_})
    for (auto& x : *v)
      if (x) {
        size_t n = 0;
        for (size_t s = 0; s < x->kept.size(); ++s) n += (size_t)x->kept[s] * x->enl.sec[s].dim;
        u += n * sizeof(double);
      }
  if (mps_bytes) *mps_bytes = u;
  size_t d = 0, h = 0, mb = 0;
  for (auto* v : {&L_, &R_})
    for (auto& b : *v) {
      if (!b || !b->ops) continue;
      const size_t x = b->ops->device_bytes();
      (b->ops->on_host ? h : d) += x;
      mb = std::max(mb, x);
    }
  if (dev) *dev = d;
  if (host) *host = h;
  if (max_block) *max_block = mb;
  if (max_extra) *max_extra = max_bond_extra_;
}

int Engine::next_use(bool left, int m, int step) const {
  const int b = left ? m : n_ - m - 2;
  const int P = 2 * n_ - 4;
  int best = INT32_MAX;
  for (int s : {b <= n_ - 3 ? b : -1, (b >= 1 && b <= n_ - 2) ? (n_ - 2) + (n_ - 2 - b) : -1}) {
    if (s < 0) continue;
    int t = s;
    while (t < step) t += P;
    best = std::min(best, t);
  }
  return best;
}

void Engine::resident(Block* b) {
  if (!b || !b->ops) return;
  if (b->ops->on_host) b->ops->stage_in();
  if (b->ops->arriving) {
    be_->stage_join();
    b->ops->arriving = false;
  }
}

// Before the bond of `step`: its two blocks on the device; when the stored
// blocks plus the bond's own working memory (measured at the previous bond)
// would exceed the budget, the blocks whose next use is farthest away are
// staged out; the blocks of the next step are brought back ahead of time.
bool Engine::stage_out_one() {
  const int step = cur_step_;
  auto bond_of = [&](int s) {
    const int P = 2 * n_ - 4;
    s %= P;
    return s <= n_ - 3 ? s : (n_ - 2) - (s - (n_ - 2));
  };
  std::vector<const Block*> busy;
  for (int s : {step, step + 1}) {
    const int b = bond_of(s);
    if (b >= 0 && b < (int)L_.size()) busy.push_back(L_[b].get());
    if (n_ - b - 2 >= 0 && n_ - b - 2 < (int)R_.size()) busy.push_back(R_[n_ - b - 2].get());
  }
  Block* best = nullptr;
  int best_next = -1;
  for (int side = 0; side < 2; ++side) {
    auto& v = side == 0 ? L_ : R_;
    for (int m = 0; m < (int)v.size(); ++m) {
      Block* b = v[m].get();
      if (!b || !b->ops || b->ops->on_host || b->ops->mem.empty() || b->ops->arriving) continue;
      if (std::find(busy.begin(), busy.end(), b) != busy.end()) continue;
      const int nu = next_use(side == 0, m, step);
      if (nu > best_next) {
        best_next = nu;
        best = b;
      }
    }
  }
  if (best) {
    best->ops->stage_out();
    return true;
  }
  if (!keep_L_.empty() || !keep_R_.empty()) {
    bool any = false;
    for (auto& b : keep_L_) any = any || b != nullptr;
    for (auto& b : keep_R_) any = any || b != nullptr;
    drop_kept();
    return any;
  }
  return false;
}

void Engine::stage_for_step(int step) {
  cur_step_ = step;
  const size_t budget = be_->budget();
  if (budget && !be_->make_room) be_->make_room = [this]() { return stage_out_one(); };
  auto bond_of = [&](int s) {
    const int P = 2 * n_ - 4;
    s %= P;
    return s <= n_ - 3 ? s : (n_ - 2) - (s - (n_ - 2));
  };
  auto blocks_of = [&](int s, Block** lb, Block** rb) {
    const int b = bond_of(s);
    *lb = (b >= 0 && b < (int)L_.size()) ? L_[b].get() : nullptr;
    *rb = (n_ - b - 2 >= 0 && n_ - b - 2 < (int)R_.size()) ? R_[n_ - b - 2].get() : nullptr;
  };
  Block *l0, *r0, *l1, *r1;
  blocks_of(step, &l0, &r0);
  blocks_of(step + 1, &l1, &r1);
  resident(l0);
  resident(r0);
  for (auto* v : {&L_, &R_})
    for (auto& b : *v)
      if (b && b->ops && !b->ops->pending.empty() && !b->ops->arriving) b->ops->release_pending();
  if (budget == 0) return;
  const size_t need = bond_extra_ + bond_extra_ * 3 / 10;
  if (be_->bytes_in_use() + need > budget) {
    struct Cand {
      int next;
      Block* b;
    };
    std::vector<Cand> c;
    for (int side = 0; side < 2; ++side) {
      auto& v = side == 0 ? L_ : R_;
      for (int m = 0; m < (int)v.size(); ++m) {
        Block* b = v[m].get();
        if (!b || !b->ops || b->ops->on_host || b == l0 || b == r0 || b == l1 || b == r1) continue;
        if (b->ops->mem.empty()) continue;
        c.push_back({next_use(side == 0, m, step), b});
      }
    }
    std::stable_sort(c.begin(), c.end(), [](const Cand& a, const Cand& b) { return a.next > b.next; });
    for (const Cand& x : c) {
      if (be_->bytes_in_use() + need <= budget) break;
      x.b->ops->stage_out();
    }
    // kept enlarged blocks are a cache: dropped (rebuilt when needed) rather
    // than staged
    if (be_->bytes_in_use() + need > budget) drop_kept();
  }
  // prefetch the next step's blocks
  for (Block* b : {l1, r1})
    if (b && b->ops && b->ops->on_host) b->ops->stage_in();
}

double Engine::optimize_bond(int i, bool l2r, double* trunc) {
  stage_for_step(step_of(i, l2r));
  const size_t bond_start = be_->bytes_in_use();
  be_->window_peak = bond_start;
  double t0 = now_s();
  // the environment side may have been enlarged at this bond on the way here
  auto take = [](std::vector<std::unique_ptr<Block>>& keep, int b) {
    std::unique_ptr<Block> e;
    if (b < (int)keep.size() && keep[b]) e = std::move(keep[b]);
    return e;
  };
  std::unique_ptr<Block> Le = l2r ? nullptr : take(keep_L_, i);
  std::unique_ptr<Block> Re = l2r ? take(keep_R_, i) : nullptr;
  if (!Le) Le = enlarge(*L_[i], i);
  if (!Re) Re = enlarge(*R_[n_ - i - 2], i + 1);
  be_->sync();
  double t1 = now_s();
  stats_.t_enlarge += t1 - t0;
  HPsiPlan plan;
  plan.psi = make_psi(Le->ops->basis, Re->ops->basis, n_elec_, two_s_);
  size_t len = plan.psi.size;
  if (len == 0) throw std::runtime_error("empty two-site space at bond " + std::to_string(i));
  plan.in = (double*)be_->alloc(len * sizeof(double));
  plan.out = (double*)be_->alloc(len * sizeof(double));
  double* psi = (double*)be_->alloc(len * sizeof(double));
  guess(i, l2r, *Le, *Re, plan, psi);
  be_->sync();
  double t2 = now_s();
  stats_.t_guess += t2 - t1;
  plan_hpsi(*Le, *Re, plan);
  be_->sync();
  double t3 = now_s();
  stats_.t_plan += t3 - t2;
  int its = 0;
  double e = davidson(plan, psi, &its) + e_core_;
  be_->check_device_flag();
  stats_.davidson_iters += its;
  if (opt_.prec != Precision::FP64 && ((!l2r && i == 1) || opt_.rq64_every_bond)) {
    // The sweep energy (last bond) of a split-precision run: the Rayleigh
    // quotient of the converged eigenvector with one float64 H_eff psi.  It is
    // second order in the eigenvector's error, while the split product's own
    // rounding (FP32 accumulation, ~1e-7 relative) would enter at first order.
    HPsiPlan p64;
    p64.in = plan.in;
    p64.out = plan.out;
    const Precision keep = opt_.prec;
    opt_.prec = Precision::FP64;
    plan_hpsi(*Le, *Re, p64);
    opt_.prec = keep;
    be_->copy_d2d(p64.in, psi, len * sizeof(double));
    apply_hpsi(p64);
    double* d2 = (double*)be_->alloc(2 * sizeof(double));
    be_->dots(psi, 1, len, len, p64.out, d2);
    be_->dots(psi, 1, len, len, psi, d2 + 1);
    double h2[2];
    be_->copy_d2h(h2, d2, sizeof(h2));
    be_->sync();
    be_->free(d2);
    if (p64.dev) be_->free(p64.dev);
    if (p64.diag) be_->free(p64.diag);
    e = h2[0] / h2[1] + e_core_;
  }
  double t4 = now_s();
  stats_.t_davidson += t4 - t3;
  std::unique_ptr<SavedU> U;
  if (l2r) U = decimate(*Le, plan, psi, true, trunc);
  else U = decimate(*Re, plan, psi, false, trunc);
  double t5 = now_s();
  stats_.t_decimate += t5 - t4;
  if (l2r) {
    bool sw = Le->normal && !left_normal(i + 1);
    L_[i + 1] = renormalize(*Le, *U, sw);
    LU_[i + 1] = std::move(U);
  } else {
    bool sw = Re->normal && !right_normal(n_ - i - 1);
    R_[n_ - i - 1] = renormalize(*Re, *U, sw);
    RU_[n_ - i - 1] = std::move(U);
  }
  be_->sync();
  const double t6 = now_s();
  stats_.t_renorm += t6 - t5;
  save_prev(i, *Le, *Re, plan, psi);
  be_->sync();
  be_->free(psi);
  be_->free(plan.in);
  be_->free(plan.out);
  if (plan.dev) be_->free(plan.dev);
  if (plan.sched) be_->free(plan.sched);
  if (plan.tc_pool) be_->free(plan.tc_pool);
  if (plan.diag) be_->free(plan.diag);
  bond_extra_ = be_->window_peak > bond_start ? be_->window_peak - bond_start : 0;
  max_bond_extra_ = std::max(max_bond_extra_, bond_extra_);
  size_t enl_bytes = 0;
  int enl_maxsec = 0;
  if (opt_.verbose) {
    for (const Block* b : {Le.get(), Re.get()})
      if (b && b->ops) enl_bytes += b->ops->bytes();
    const Block* tb = l2r ? Le.get() : Re.get();
    if (tb && tb->ops)
      for (auto& sc : tb->ops->basis.sec) enl_maxsec = std::max(enl_maxsec, sc.dim);
  }
  // keep this bond's system-side enlarged block for the way back
  const double cap = be_->budget() ? (double)std::min(be_->budget(), be_->capacity()) : (double)be_->capacity();
  // ... and only while the next bond's working memory still fits next to it
  if ((double)be_->bytes_in_use() <= kKeepFraction * cap &&
      (double)be_->bytes_in_use() + 1.3 * (double)bond_extra_ <= 0.85 * cap &&
      (double)be_->device_free() >= kKeepFreeFraction * (double)be_->capacity()) {
    auto& keep = l2r ? keep_L_ : keep_R_;
    if ((int)keep.size() < n_) keep.resize(n_);
    keep[i] = l2r ? std::move(Le) : std::move(Re);
  }
  last_bond_ = i;
  bond_e_.push_back(e);
  if (opt_.verbose) {
    // stored blocks of every bond, the two enlarged blocks of this one, and
    // the largest sector of the truncated enlarged basis (the eigensolver's
    // largest matrix)
    size_t stored = 0;
    for (auto& b : L_)
      if (b && b->ops) stored += b->ops->bytes();
    for (auto& b : R_)
      if (b && b->ops) stored += b->ops->bytes();
    std::fprintf(stderr,
                 "bond %d %s E %.12f trunc %.3e it %d len %zu flops %.3e | mem %.2f GB stored %.2f GB "
                 "enl %.2f GB maxsec %d | t enl %.3f plan %.3f dav %.3f dec %.3f ren %.3f\n",
                 i, l2r ? "LR" : "RL", e, *trunc, its, len, plan.flops, be_->bytes_in_use() / 1e9,
                 stored / 1e9, enl_bytes / 1e9, enl_maxsec, t1 - t0, t3 - t2, t4 - t3, t5 - t4, t6 - t5);
  }
  return e;
}

void Engine::end_bond_solves() {
  if (solve_bond_ < 0) return;
  // the enlarged blocks kept by bond solves are not those a sweep keeps
  drop_kept();
  if (solve_psi_) be_->free(solve_psi_);
  solve_psi_ = nullptr;
  solve_bond_ = -1;
}

SweepStats Engine::sweep_part(bool l2r, int last) {
  end_bond_solves();
  stats_ = SweepStats();
  auto t0 = std::chrono::steady_clock::now();
  be_->mark_begin();
  double e = 0.0, tr = 0.0, tmax = 0.0;
  if (l2r) {
    if (last < 0 || last > n_ - 3) throw std::invalid_argument("sweep part: last bond out of range");
    for (int i = 0; i <= last; ++i) {
      e = optimize_bond(i, true, &tr);
      tmax = std::max(tmax, tr);
      if (n_ - i - 2 > 0) R_[n_ - i - 2].reset();
    }
  } else {
    if (last < 1 || last > n_ - 2) throw std::invalid_argument("sweep part: last bond out of range");
    if (!L_[n_ - 2]) throw std::runtime_error("state: an R->L part needs a completed L->R half-sweep");
    for (int i = n_ - 2; i >= last; --i) {
      e = optimize_bond(i, false, &tr);
      tmax = std::max(tmax, tr);
      if (i > 0) L_[i].reset();
    }
  }
  sweep_device_ms = be_->mark_end();
  be_->sync();
  energy_ = e;
  stats_.energy = e;
  stats_.max_trunc = tmax;
  sweep_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return stats_;
}

Engine::BondSolve Engine::solve_bond(int bond, bool l2r, Precision p, int max_iter, double tol, int min_calls,
                                     bool check64) {
  if (bond < 0 || bond > n_ - 2) throw std::invalid_argument("bond out of range");
  if (!L_[bond] || !R_[n_ - bond - 2]) throw std::runtime_error("state: the blocks of this bond are not held");
  resident(L_[bond].get());
  resident(R_[n_ - bond - 2].get());
  BondSolve out;
  // the side that was enlarged on the way here may be kept; other kept
  // enlarged blocks are released
  std::unique_ptr<Block> Le, Re;
  if (!l2r && bond < (int)keep_L_.size() && keep_L_[bond]) Le = std::move(keep_L_[bond]);
  if (l2r && bond < (int)keep_R_.size() && keep_R_[bond]) Re = std::move(keep_R_[bond]);
  if (l2r && bond < (int)keep_L_.size() && keep_L_[bond]) Le = std::move(keep_L_[bond]);
  if (!l2r && bond < (int)keep_R_.size() && keep_R_[bond]) Re = std::move(keep_R_[bond]);
  drop_kept();
  if (solve_psi_) {
    be_->free(solve_psi_);
    solve_psi_ = nullptr;
  }
  if (!Le) Le = enlarge(*L_[bond], bond);
  if (!Re) Re = enlarge(*R_[n_ - bond - 2], bond + 1);
  HPsiPlan plan;
  plan.psi = make_psi(Le->ops->basis, Re->ops->basis, n_elec_, two_s_);
  const size_t len = plan.psi.size;
  if (len == 0) throw std::runtime_error("empty two-site space at bond " + std::to_string(bond));
  plan.in = (double*)be_->alloc(len * sizeof(double));
  plan.out = (double*)be_->alloc(len * sizeof(double));
  double* psi = (double*)be_->alloc(len * sizeof(double));
  guess(bond, l2r, *Le, *Re, plan, psi);
  const Options keep = opt_;
  opt_.prec = p;
  opt_.max_davidson_iter = std::max(1, max_iter);
  opt_.davidson_tol = tol;
  plan_hpsi(*Le, *Re, plan);
  std::vector<double> ms;
  call_ms_ = &ms;
  int its = 0;
  double e = 0.0;
  // kernel-class times of the products alone (the float64 evaluation below
  // is not counted)
  double c0 = 0.0, s0 = 0.0;
  long l0 = 0, ls = 0;
  be_->kernel_stats(1, &c0, nullptr, &l0);
  be_->kernel_stats(5, &s0, nullptr, &ls);
  try {
    e = davidson(plan, psi, &its);
    // pad with products on the result vector up to min_calls
    while ((int)ms.size() < min_calls) {
      be_->copy_d2d(plan.in, psi, len * sizeof(double));
      be_->mark_begin();
      apply_hpsi(plan);
      ms.push_back(be_->mark_end());
      if (plan.prec == Precision::TC_TF32X3) be_->check_device_flag();
    }
  } catch (...) {
    call_ms_ = nullptr;
    opt_ = keep;
    throw;
  }
  call_ms_ = nullptr;
  // the tcgen05 operand pool and schedule are not needed past the products
  if (plan.tc_pool) {
    be_->free(plan.tc_pool);
    plan.tc_pool = nullptr;
  }
  if (plan.sched) {
    be_->free(plan.sched);
    plan.sched = nullptr;
  }
  {
    double c1 = 0.0, s1 = 0.0;
    long l1 = 0;
    be_->kernel_stats(1, &c1, nullptr, &l1);
    be_->kernel_stats(5, &s1, nullptr, &ls);
    out.contraction_ms = c1 - c0;
    out.split_ms = s1 - s0;
    out.contraction_launches = l1 - l0;
  }
  out.gap = last_gap_;
  out.flops_per_call = plan.flops;
  opt_ = keep;
  out.energy = e + e_core_;
  out.iterations = its;
  out.calls = (int)ms.size();
  out.call_ms = std::move(ms);
  out.dim = len;
  be_->free(plan.in);
  be_->free(plan.out);
  if (plan.dev) be_->free(plan.dev);
  if (plan.diag) be_->free(plan.diag);
  // both enlarged blocks stay for the next call at this bond, and the vector
  // for check_bond64
  if ((int)keep_L_.size() < n_) keep_L_.resize(n_);
  if ((int)keep_R_.size() < n_) keep_R_.resize(n_);
  keep_L_[bond] = std::move(Le);
  keep_R_[bond] = std::move(Re);
  solve_psi_ = psi;
  solve_bond_ = bond;
  solve_l2r_ = l2r;
  if (check64) {
    double ms64 = 0.0, fl = 0.0;
    check_bond64(&out.energy_rq64, &out.residual64, &ms64, &fl);
  }
  return out;
}

size_t Engine::apply_bond(Precision p, const double* x, double* y) {
  const int bond = solve_bond_;
  if (!solve_psi_ || bond < 0 || bond >= (int)keep_L_.size() || !keep_L_[bond] || bond >= (int)keep_R_.size() ||
      !keep_R_[bond])
    throw std::runtime_error("state: no bond solve to apply H_eff at");
  Block& Le = *keep_L_[bond];
  Block& Re = *keep_R_[bond];
  HPsiPlan plan;
  plan.psi = make_psi(Le.ops->basis, Re.ops->basis, n_elec_, two_s_);
  const size_t len = plan.psi.size;
  if (!x || !y) return len;
  plan.in = (double*)be_->alloc(len * sizeof(double));
  plan.out = (double*)be_->alloc(len * sizeof(double));
  const Precision kp = opt_.prec;
  const bool kt = opt_.tc_autotune;
  opt_.prec = p;
  opt_.tc_autotune = false;
  try {
    plan_hpsi(Le, Re, plan);
    be_->copy_h2d(plan.in, x, len * sizeof(double));
    apply_hpsi(plan);
    if (plan.prec == Precision::TC_TF32X3) be_->check_device_flag();
    be_->copy_d2h(y, plan.out, len * sizeof(double));
    be_->sync();
  } catch (...) {
    opt_.prec = kp;
    opt_.tc_autotune = kt;
    for (void* q : {(void*)plan.in, (void*)plan.out, plan.dev, plan.sched, plan.tc_pool, (void*)plan.diag})
      if (q) be_->free(q);
    throw;
  }
  opt_.prec = kp;
  opt_.tc_autotune = kt;
  for (void* q : {(void*)plan.in, (void*)plan.out, plan.dev, plan.sched, plan.tc_pool, (void*)plan.diag})
    if (q) be_->free(q);
  return len;
}

void Engine::check_bond64(double* energy_rq64, double* residual64, double* ms, double* flops) {
  const int bond = solve_bond_;
  if (!solve_psi_ || bond < 0 || bond >= (int)keep_L_.size() || !keep_L_[bond] || bond >= (int)keep_R_.size() ||
      !keep_R_[bond])
    throw std::runtime_error("state: no bond solve to check");
  Block& Le = *keep_L_[bond];
  Block& Re = *keep_R_[bond];
  HPsiPlan p64;
  p64.psi = make_psi(Le.ops->basis, Re.ops->basis, n_elec_, two_s_);
  const size_t len = p64.psi.size;
  p64.in = (double*)be_->alloc(len * sizeof(double));
  p64.out = (double*)be_->alloc(len * sizeof(double));
  const Precision kp = opt_.prec;
  opt_.prec = Precision::FP64;
  plan_hpsi(Le, Re, p64);
  opt_.prec = kp;
  const double* psi = solve_psi_;
  be_->copy_d2d(p64.in, psi, len * sizeof(double));
  be_->mark_begin();
  apply_hpsi(p64);
  const double t = be_->mark_end();
  double* d3 = (double*)be_->alloc(3 * sizeof(double));
  be_->dots(psi, 1, len, len, p64.out, d3);
  be_->dots(psi, 1, len, len, psi, d3 + 1);
  double h2[2];
  be_->copy_d2h(h2, d3, 2 * sizeof(double));
  const double erq = h2[0] / h2[1];
  // r = H psi / |psi| - E_rq psi / |psi|
  be_->axpby(p64.out, 1.0 / std::sqrt(h2[1]), psi, -erq / std::sqrt(h2[1]), len);
  be_->dots(p64.out, 1, len, len, p64.out, d3 + 2);
  double r2;
  be_->copy_d2h(&r2, d3 + 2, sizeof(double));
  be_->sync();
  be_->free(d3);
  be_->free(p64.in);
  be_->free(p64.out);
  if (p64.dev) be_->free(p64.dev);
  if (p64.diag) be_->free(p64.diag);
  if (energy_rq64) *energy_rq64 = erq + e_core_;
  if (residual64) *residual64 = std::sqrt(std::max(0.0, r2));
  if (ms) *ms = t;
  if (flops) *flops = p64.flops;
}

SweepStats Engine::sweep() {
  end_bond_solves();
  stats_ = SweepStats();
  auto t0 = std::chrono::steady_clock::now();
  be_->mark_begin();
  double e = 0.0, tr = 0.0, tmax = 0.0;
  for (int i = 0; i <= n_ - 3; ++i) {
    e = optimize_bond(i, true, &tr);
    tmax = std::max(tmax, tr);
    if (n_ - i - 2 > 0) R_[n_ - i - 2].reset();
  }
  for (int i = n_ - 2; i >= 1; --i) {
    e = optimize_bond(i, false, &tr);
    tmax = std::max(tmax, tr);
    if (i > 0) L_[i].reset();
  }
  sweep_device_ms = be_->mark_end();
  be_->sync();
  energy_ = e;
  stats_.energy = e;
  stats_.max_trunc = tmax;
  sweep_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return stats_;
}

// ============================================================ reduced density matrices
// Spin-free RDMs of the final two-site state (Eqs. onerdm, twordm; the SU(2)
// channels of Sec. II.C are recoupled on the host).  A measurement pass walks
// the bonds left to right starting at bond 1: at every bond i the state is
// psi(L'(i), R'(i)) with L'(i) = L(i) (x) site i and R'(i) = site i+1 (x) R(i+2),
// where L(i) is an exact left basis of the state built in a measurement mode
// (single spinors and all normal pair operators) and R(i+2) the right block of
// the last sweep.  Moving to the next bond keeps every multiplet of nonzero
// weight (rho eigenvalue >= 1e-12), so the moved state is the same state.
//
// An element with operators at positions x1 <= x2 <= x3 (<= x4) is evaluated
// at bond i = min(n-2, x3) (2-RDM) or min(n-2, x2) (1-RDM): at most two of its
// operators lie in L(i), at most one to the right of site i (several on the
// last site at the last bond).  Its position-ordered operator string is
// a product  x_L . s . Y  of a normal operator of L(i) (identity, spinor or
// pair), a string on site i and an operator of R'(i), and the spin-free sum
// over the spins is expanded in the invariant couplings
//   [[x_L^{kx} (x) s^{ks}]^{kX} (x) Y^{kX}]^0
// that the pass can evaluate.  Their expectation values follow from
//   N_Y(a',a) = sum_{b',b} c(a',b',a,b) psi(a',b') Y(b',b) psi(a,b)^T
// (an operator-shaped object on L'), taken back to L(i) through the adjoint
// of the blocking placement (W), and one GEMM of all stored L(i) operators
// against all W.

struct Engine::RdmAcc {
  std::vector<double> g1, g2, orb;
};

namespace {

struct SortedOps {
  int n = 0;
  int pos[4] = {0, 0, 0, 0}, dag[4] = {0, 0, 0, 0};
  std::vector<std::pair<int, int>> pairs;
  double sign = 1.0;
};

// position order (stable: operators on one site keep their order); each
// exchange of operators on different orbitals gives a factor -1
SortedOps sort_ops(const int* pos, const int* dag, int n, const std::vector<std::pair<int, int>>& pairs) {
  SortedOps r;
  r.n = n;
  int ord[4] = {0, 1, 2, 3};
  int inv = 0;
  for (int i = 1; i < n; ++i)
    for (int j = i; j > 0 && pos[ord[j - 1]] > pos[ord[j]]; --j) {
      std::swap(ord[j - 1], ord[j]);
      ++inv;
    }
  int where[4] = {0, 0, 0, 0};
  for (int i = 0; i < n; ++i) {
    r.pos[i] = pos[ord[i]];
    r.dag[i] = dag[ord[i]];
    where[ord[i]] = i;
  }
  for (auto& pr : pairs) r.pairs.push_back({where[pr.first], where[pr.second]});
  r.sign = (inv & 1) ? -1.0 : 1.0;
  return r;
}

// sequences of doubled intermediate ranks of a sequential coupling of m spinors
void seq_ranks(int m, std::vector<std::vector<int>>& out) {
  out.clear();
  if (m == 0) { out.push_back({}); return; }
  std::vector<std::vector<int>> cur{{1}};  // rank after the first spinor
  for (int i = 1; i < m; ++i) {
    std::vector<std::vector<int>> nxt;
    for (auto& v : cur)
      for (int k : {v.back() - 1, v.back() + 1})
        if (k >= 0) {
          auto w = v;
          w.push_back(k);
          nxt.push_back(w);
        }
    cur = nxt;
  }
  for (auto& v : cur) out.push_back(std::vector<int>(v.begin() + 1, v.end()));  // drop the leading 1
}
int seq_rank(int m, const std::vector<int>& k) { return m == 0 ? 0 : (m == 1 ? 1 : k.back()); }

// One evaluable coupling of a split string (l ops | s ops | y ops).
struct Variant {
  int kx = 0;                 // rank of the L(i) part
  std::vector<int> kl;        // its sequential intermediates (pair: {kx})
  std::vector<int> ks, ky;    // sequential intermediates of the site / right parts
  int kX = 0;                 // rank of [x (x) s] (= rank of Y)
  double c = 0.0;             // coefficient in the spin-free sum
};

// builds the coupling tree of a variant over slots 0..n-1
std::vector<TreeNode> variant_tree(int l, int s, int y, const Variant& v) {
  std::vector<TreeNode> t;
  auto leaf = [&](int slot) { t.push_back(TreeNode{slot, -1, -1, 1}); return (int)t.size() - 1; };
  auto join = [&](int a, int b, int k) { t.push_back(TreeNode{-1, a, b, k}); return (int)t.size() - 1; };
  int xl = -1, xs = -1, xy = -1;
  for (int i = 0; i < l; ++i) {
    int f = leaf(i);
    xl = (i == 0) ? f : join(xl, f, v.kl[i - 1]);
  }
  for (int i = 0; i < s; ++i) {
    int f = leaf(l + i);
    xs = (i == 0) ? f : join(xs, f, v.ks[i - 1]);
  }
  for (int i = 0; i < y; ++i) {
    int f = leaf(l + s + i);
    xy = (i == 0) ? f : join(xy, f, v.ky[i - 1]);
  }
  int X = -1;
  if (xl >= 0 && xs >= 0) X = join(xl, xs, v.kX);
  else X = xl >= 0 ? xl : xs;
  if (X >= 0 && xy >= 0) join(X, xy, 0);
  return t;
}

// coefficients of the spin-free pairing in an independent set of variants
std::vector<Variant> expand_split(int l, int s, int y, const std::vector<int>& dag,
                                  const std::vector<std::pair<int, int>>& pairs) {
  const int n = l + s + y;
  std::vector<std::vector<int>> KL, KS, KY;
  seq_ranks(l, KL);
  seq_ranks(s, KS);
  seq_ranks(y, KY);
  std::vector<Variant> all;
  for (auto& kl : KL)
    for (auto& ks : KS)
      for (auto& ky : KY) {
        int kx = seq_rank(l, kl), rs = seq_rank(s, ks), ry = seq_rank(y, ky);
        for (int kX = 0; kX <= 4; ++kX) {
          if (l > 0 && s > 0) {
            if (!triangle(kx, rs, kX)) continue;
          } else if (kX != (l > 0 ? kx : rs)) {
            continue;
          }
          if (y > 0 ? kX != ry : kX != 0) continue;
          Variant v;
          v.kx = kx;
          v.kl = kl;
          v.ks = ks;
          v.ky = ky;
          v.kX = kX;
          all.push_back(v);
        }
      }
  // greedy independent subset
  std::vector<std::vector<double>> basis, ortho;
  std::vector<Variant> pick;
  for (auto& v : all) {
    auto T = tree_tensor(variant_tree(l, s, y, v), n);
    auto u = T;
    for (auto& o : ortho) {
      double d = 0.0, nn = 0.0;
      for (size_t e = 0; e < u.size(); ++e) { d += o[e] * u[e]; nn += o[e] * o[e]; }
      for (size_t e = 0; e < u.size(); ++e) u[e] -= d / nn * o[e];
    }
    double nrm = 0.0;
    for (double x : u) nrm += x * x;
    if (nrm < 1e-20) continue;
    ortho.push_back(u);
    basis.push_back(T);
    pick.push_back(v);
  }
  auto target = pairing_tensor(dag, pairs, n);
  double res = 0.0;
  auto c = expand_invariant(target, basis, &res);
  if (res > 1e-10) throw std::runtime_error("internal: spin-free pairing outside the coupling span");
  std::vector<Variant> out;
  for (size_t i = 0; i < pick.size(); ++i)
    if (std::abs(c[i]) > 1e-14) {
      pick[i].c = c[i];
      out.push_back(pick[i]);
    }
  return out;
}

// stored L(i) operator realising a position-ordered normal string (0-2 spinors)
struct XTerm {
  OpKey key;
  int adj = 0;
  double f = 1.0;
};
const OpKey kIdentityKey{K_T0, -1, -1, 0};
// key of an on-site string temporary (operators of L(1) for strings of three
// or four operators on site 0)
OpKey string_key(const std::vector<int>& dag, const std::vector<int>& k2, int k2tot) {
  int code = 0;
  for (int d : dag) code = code * 2 + d;
  for (int k : k2) code = code * 5 + k;
  int dn = 0;
  for (int d : dag) dn += d ? 1 : -1;
  return OpKey{K_T0 + dn, 1000 + (int)dag.size(), code, k2tot};
}
void x_terms(int l, const int* pos, const int* dag, const std::vector<int>& kl, std::vector<XTerm>& out) {
  out.clear();
  if (l == 0) { out.push_back({kIdentityKey, 0, 1.0}); return; }
  if (l >= 3) {
    std::vector<int> d(dag, dag + l);
    out.push_back({string_key(d, kl, kl.back()), 0, 1.0});
    return;
  }
  const int kx = l == 2 ? kl[0] : 1;
  if (l == 1) { out.push_back({OpKey{K_C, pos[0], 0, 1}, dag[0] ? 0 : 1, 1.0}); return; }
  int u = pos[0], v = pos[1];
  if (dag[0] && dag[1]) {
    if (!(u == v && kx == 2)) out.push_back({OpKey{K_A, u, v, kx}, 0, 1.0});
  } else if (!dag[0] && !dag[1]) {
    // [a~_u a~_v]^k = -adj(A^k_uv)
    if (!(u == v && kx == 2)) out.push_back({OpKey{K_A, u, v, kx}, 1, -1.0});
  } else if (dag[0]) {
    out.push_back({OpKey{K_B, u, v, kx}, 0, 1.0});
  } else if (u < v) {
    // [a~_u a+_v]^k = (-1)^k B^k_vu = adj(B^k_uv)
    out.push_back({OpKey{K_B, u, v, kx}, 1, 1.0});
  } else {
    // same orbital: [a~_u a+_u]^k = (-1)^k B^k_uu + sqrt2 delta_k0
    out.push_back({OpKey{K_B, u, u, kx}, 0, kx ? -1.0 : 1.0});
    if (kx == 0) out.push_back({kIdentityKey, 0, kSqrt2});
  }
}

// Request tables of the measurement pass at one bond (Engine::rdm_eval).
struct RdmVKey {
  int y, s, kX;
  OpKey x;
  int adj;
  bool operator<(const RdmVKey& o) const {
    if (y != o.y) return y < o.y;
    if (s != o.s) return s < o.s;
    if (kX != o.kX) return kX < o.kX;
    if (adj != o.adj) return adj < o.adj;
    return x < o.x;
  }
};
struct RdmContrib {
  size_t target;
  int order;
  double c;
  int v;
};

}  // namespace

struct Engine::RdmRequests {
  std::map<std::pair<std::vector<int>, std::vector<int>>, int> s_index;
  std::vector<SiteOp> s_ops;
  std::map<std::tuple<int, int, std::vector<int>, std::vector<int>>, int> y_index;
  std::vector<Operand> y_ops;
  std::vector<std::pair<OpKey, SiteOp>> y_temps;  // site strings on the last site
  std::map<RdmVKey, int> v_index;
  std::vector<RdmVKey> vkeys;
  std::vector<RdmContrib> contribs;
};

void Engine::rdm_bond(int i, Block& Lb, Block& Le, Block& Re, const Block& Rparent, const PsiLayout& P,
                      const double* psi, const std::vector<size_t>& elems, RdmAcc& acc) {
  const int n = n_;
  const size_t nn = (size_t)n * n;
  // ---------------------------------------------------------------- requests
  RdmRequests rq;
  auto& s_index = rq.s_index;
  auto& s_ops = rq.s_ops;
  auto& y_index = rq.y_index;
  auto& y_ops = rq.y_ops;
  auto& y_temps = rq.y_temps;
  auto& v_index = rq.v_index;
  auto& vkeys = rq.vkeys;
  auto& contribs = rq.contribs;
  using VKey = RdmVKey;
  std::map<std::tuple<int, int, int, int, std::vector<std::pair<int, int>>>, std::vector<Variant>> vcache;
  const bool last = (i == n - 2);
  std::vector<XTerm> xt;
  for (size_t e : elems) {
    int order, pos[4], dag[4];
    std::vector<std::pair<int, int>> pairs;
    size_t target;
    if (e < nn) {
      order = 1;
      pos[0] = (int)(e / n);
      pos[1] = (int)(e % n);
      dag[0] = 1;
      dag[1] = 0;
      pairs = {{0, 1}};
      target = e;
    } else {
      order = 2;
      size_t t = e - nn;
      target = t;
      pos[3] = (int)(t % n); t /= n;
      pos[2] = (int)(t % n); t /= n;
      pos[1] = (int)(t % n); t /= n;
      pos[0] = (int)t;
      dag[0] = dag[1] = 1;
      dag[2] = dag[3] = 0;
      pairs = {{0, 3}, {1, 2}};
    }
    const int m = order == 1 ? 2 : 4;
    SortedOps so = sort_ops(pos, dag, m, pairs);
    int l = 0, s = 0, y = 0;
    for (int k = 0; k < m; ++k) {
      if (so.pos[k] < i) ++l;
      else if (so.pos[k] == i) ++s;
      else ++y;
    }
    if ((l > 2 && (i != 1 || so.pos[l - 1] != 0)) || (!last && y > 1))
      throw std::runtime_error("internal: RDM element assigned to the wrong bond");
    int dmask = 0;
    for (int k = 0; k < m; ++k) dmask |= so.dag[k] << k;
    auto ck = std::make_tuple(l, s, y, dmask, so.pairs);
    auto it = vcache.find(ck);
    if (it == vcache.end())
      it = vcache.emplace(ck, expand_split(l, s, y, std::vector<int>(so.dag, so.dag + m), so.pairs)).first;
    for (const Variant& v : it->second) {
      x_terms(l, so.pos, so.dag, v.kl, xt);
      // site string
      std::vector<int> sd(so.dag + l, so.dag + l + s);
      auto sk = std::make_pair(sd, v.ks);
      auto si = s_index.find(sk);
      if (si == s_index.end()) {
        si = s_index.emplace(sk, (int)s_ops.size()).first;
        s_ops.push_back(site_string(sd, v.ks));
      }
      // right operand
      std::vector<int> yd(so.dag + l + s, so.dag + m);
      int ypos = y > 0 ? so.pos[l + s] : -1;
      auto yk = std::make_tuple(y, y == 1 ? ypos : -1, yd, v.ky);
      auto yi = y_index.find(yk);
      if (yi == y_index.end()) {
        yi = y_index.emplace(yk, (int)y_ops.size()).first;
        if (y == 0) {
          y_ops.push_back(op_id());
        } else if (y == 1) {
          y_ops.push_back(op_blk(K_C, ypos, 0, 1, yd[0] ? 0 : 1));
        } else {
          SiteOp so2 = site_string(yd, v.ky);
          OpKey key{K_T0 + so2.dn, (int)y_temps.size(), 0, so2.k2};
          y_temps.push_back({key, so2});
          y_ops.push_back(op_blk(key.kind, key.i, 0, key.k2));
        }
      }
      for (const XTerm& x : xt) {
        VKey vk{yi->second, si->second, v.kX, x.key, x.adj};
        auto vi = v_index.find(vk);
        if (vi == v_index.end()) {
          vi = v_index.emplace(vk, (int)vkeys.size()).first;
          vkeys.push_back(vk);
        }
        contribs.push_back({target, order, so.sign * v.c * x.f, vi->second});
      }
    }
  }
  rdm_eval(Lb, Le, Re, Rparent, P, psi, rq, acc);
}

// Evaluation of the requests of one bond: every distinct (right operand Y,
// site string s, coupling rank kX, stored L(i) operator x) gives
//   <[[x (x) s]^kX (x) Y]^0>,
// and each contribution adds c times its value to its target (order 1: the
// 1-RDM, 2: the 2-RDM, 3: the orbital-entanglement invariants).
void Engine::rdm_eval(Block& Lb, Block& Le, Block& Re, const Block& Rparent, const PsiLayout& P,
                      const double* psi, RdmRequests& rq, RdmAcc& acc) {
  auto& s_ops = rq.s_ops;
  auto& y_ops = rq.y_ops;
  auto& y_temps = rq.y_temps;
  auto& vkeys = rq.vkeys;
  auto& contribs = rq.contribs;
  using VKey = RdmVKey;
  if (vkeys.empty()) return;
  // site strings of the last site as operators of R'
  if (!y_temps.empty()) {
    std::vector<OpKey> keys;
    std::vector<std::pair<OpKey, Term>> terms;
    for (auto& [k, so2] : y_temps) {
      keys.push_back(k);
      Term t;
      t.x = op_site(so2);
      t.y = op_id();
      t.k2 = so2.k2;
      t.coef = 1.0;
      terms.push_back({k, t});
    }
    Re.ops->allocate(keys);
    place_terms(Rparent, nullptr, Re, terms);
  }
  // ---------------------------------------------------------------- N_Y on L'
  const Basis& LB = Le.ops->basis;
  const Basis& RB = Re.ops->basis;
  OpSet& ro = *Re.ops;
  std::vector<double*> Nbuf(y_ops.size(), nullptr);
  std::vector<int> Ndn(y_ops.size()), Nk(y_ops.size());
  std::vector<void*> scratch;
  for (size_t yi = 0; yi < y_ops.size(); ++yi) {
    const Operand& Y = y_ops[yi];
    const int dnX = -Y.dn, kY = Y.k2;
    Ndn[yi] = dnX;
    Nk[yi] = kY;
    const Layout& NL = Le.ops->layout(dnX, kY);
    if (NL.size == 0) continue;
    double* N = (double*)be_->alloc(NL.size * sizeof(double));
    be_->memset0(N, NL.size * sizeof(double));
    Nbuf[yi] = N;
    // T(a', b', b) = psi(a', b') op(Y)(b', b)
    struct TB { const double* ptr; int rows, cols, ld; int ap, bp, b; };
    std::vector<TB> tbs;
    size_t tsz = 0;
    std::vector<std::pair<size_t, int>> tdef;  // (offset, index into pending GEMMs)
    GemmBuilder g1;
    double* T = nullptr;
    std::vector<std::tuple<int, int, int, SrcBlock, int, size_t>> pend;  // ap, bp, b, Yblk, psi blk, toff
    for (auto& pb : P.blk) {
      int ap = pb.a, bp = pb.b;
      for (size_t b = 0; b < RB.sec.size(); ++b) {
        if (RB.sec[bp].n != RB.sec[b].n + Y.dn || !triangle(RB.sec[b].j, Y.k2, RB.sec[bp].j)) continue;
        SrcBlock yb = find_block(ro, nullptr, Y, bp, (int)b);
        if (!yb.ok) continue;
        pend.push_back({ap, bp, (int)b, yb, 0, tsz});
        if (Y.t != Operand::ID) tsz += (size_t)pb.rows * RB.sec[b].dim;
      }
    }
    if (tsz > 0) {
      T = (double*)be_->alloc(tsz * sizeof(double));
      be_->memset0(T, tsz * sizeof(double));
      scratch.push_back(T);
    }
    GemmBuilder g2;
    for (auto& [ap, bp, b, yb, unused, toff] : pend) {
      (void)unused;
      int pi = P.find(ap, bp);
      const auto& pbk = P.blk[pi];
      const double* Tp;
      int ldT;
      if (Y.t == Operand::ID) {
        Tp = psi + pbk.off;
        ldT = pbk.cols;
      } else {
        g1.add(T + toff, pbk.rows, RB.sec[b].dim, RB.sec[b].dim,
               GemmSeg{psi + pbk.off, yb.ptr, pbk.cols, pbk.cols, yb.ld, 0, yb.trans, yb.coef});
        Tp = T + toff;
        ldT = RB.sec[b].dim;
      }
      // N(a', a) += c * T psi(a, b)^T
      for (size_t a = 0; a < LB.sec.size(); ++a) {
        int ki = P.find((int)a, b);
        if (ki < 0) continue;
        int ni = NL.find(ap, (int)a);
        if (ni < 0) continue;
        double c = hpsi_coef(LB.sec[ap].j, RB.sec[bp].j, LB.sec[a].j, RB.sec[b].j, kY, two_s_);
        if (c == 0.0) continue;
        if ((Y.par & LB.sec[a].n) & 1) c = -c;
        if (Y.t == Operand::ID) c *= yb.coef;
        const auto& kb = P.blk[ki];
        g2.add(N + NL.blk[ni].off, pbk.rows, kb.rows, NL.blk[ni].cols,
               GemmSeg{Tp, psi + kb.off, kb.cols, ldT, kb.cols, 0, 1, c});
      }
    }
    g1.run(be_, Precision::FP64);
    g2.run(be_, Precision::FP64);
  }
  // ---------------------------------------------------------------- W = adjoint placement of N
  // group requests by (y, s, kX, adj, stored layout of x)
  struct WKey {
    int y, s, kX, adj, dn, k2;
    bool operator<(const WKey& o) const {
      return std::tie(dn, k2, y, s, kX, adj) < std::tie(o.dn, o.k2, o.y, o.s, o.kX, o.adj);
    }
  };
  std::map<WKey, int> w_col;                     // column within its layout's W stack
  std::map<std::pair<int, int>, int> w_count;    // per stored layout
  std::vector<int> v_col(vkeys.size());
  for (size_t v = 0; v < vkeys.size(); ++v) {
    const VKey& k = vkeys[v];
    WKey wk{k.y, k.s, k.kX, k.adj, kind_dn(k.x.kind), k.x.k2};
    auto it = w_col.find(wk);
    if (it == w_col.end()) it = w_col.emplace(wk, w_count[{wk.dn, wk.k2}]++).first;
    v_col[v] = it->second;
  }
  std::vector<std::vector<const EnlComp*>> by(LB.sec.size());
  for (auto& c : Le.comps) by[c.esec].push_back(&c);
  const Basis& bb = Lb.ops->basis;
  std::map<std::pair<int, int>, double*> wstack;
  for (auto& [lk, cnt] : w_count) {
    const Layout& XL = Lb.ops->layout(lk.first, lk.second);
    double* Wb = (double*)be_->alloc(std::max<size_t>(1, XL.size * cnt) * sizeof(double));
    be_->memset0(Wb, std::max<size_t>(1, XL.size * cnt) * sizeof(double));
    wstack[lk] = Wb;
    scratch.push_back(Wb);
  }
  PlaceBuilder pb;
  for (auto& [wk, col] : w_col) {
    double* N = Nbuf[wk.y];
    if (!N) continue;
    const Layout& NL = Le.ops->layout(Ndn[wk.y], Nk[wk.y]);
    const Layout& XL = Lb.ops->layout(wk.dn, wk.k2);
    if (XL.size == 0) continue;
    double* W = wstack[{wk.dn, wk.k2}] + (size_t)col * XL.size;
    const SiteOp& so = s_ops[wk.s];
    for (auto& blk : NL.blk) {
      int Jp = LB.sec[blk.bra].j, J = LB.sec[blk.ket].j;
      for (const EnlComp* cp : by[blk.bra])
        for (const EnlComp* c : by[blk.ket]) {
          double sv = so.m[cp->site][c->site];
          if (sv == 0.0) continue;
          int lp = cp->bsec, l = c->bsec;
          int xb;
          double ac = 1.0;
          if (!wk.adj) {
            if (bb.sec[lp].n != bb.sec[l].n + wk.dn) continue;
            xb = XL.find(lp, l);
          } else {
            if (bb.sec[l].n != bb.sec[lp].n + wk.dn) continue;
            xb = XL.find(l, lp);
            ac = adjoint_coef(bb.sec[lp].j, bb.sec[l].j, wk.k2);
          }
          if (xb < 0) continue;
          double tp = tensor_product_coef(bb.sec[lp].j, bb.sec[l].j, wk.k2, kSiteJ[cp->site], kSiteJ[c->site],
                                          so.k2, Jp, J, wk.kX);
          if (tp == 0.0) continue;
          double sign = ((so.parity & bb.sec[l].n) & 1) ? -1.0 : 1.0;
          double alpha = tp * sv * sign * ac;
          const auto& xbk = XL.blk[xb];
          const double* src = N + blk.off + (size_t)cp->eoff * blk.cols + c->eoff;
          pb.add(W + xbk.off, xbk.rows, xbk.cols, xbk.cols, PlaceSeg{src, blk.cols, wk.adj, alpha});
        }
    }
  }
  pb.run(be_);
  // ---------------------------------------------------------------- V = <x, W> for all stored x
  std::map<OpKey, std::pair<double*, int>> xrow;  // op -> (V run, row)
  std::vector<std::pair<double*, size_t>> vruns;  // host copies
  std::vector<std::tuple<double*, int, int>> runs_dev;  // (device V, rows, cols)
  GemmBuilder gv;
  std::vector<std::pair<std::vector<double>, std::tuple<double*, int, int>>> host_v;
  for (auto& [lk, cnt] : w_count) {
    const Layout& XL = Lb.ops->layout(lk.first, lk.second);
    if (XL.size == 0) continue;
    std::vector<std::pair<double*, OpKey>> ops;
    for (auto& [k, p] : Lb.ops->ops)
      if (kind_dn(k.kind) == lk.first && k.k2 == lk.second) ops.push_back({p, k});
    std::sort(ops.begin(), ops.end(), [](auto& a, auto& b) { return a.first < b.first; });
    size_t r0 = 0;
    while (r0 < ops.size()) {
      size_t r1 = r0 + 1;
      while (r1 < ops.size() && ops[r1].first == ops[r1 - 1].first + XL.size) ++r1;
      int rows = (int)(r1 - r0);
      double* V = (double*)be_->alloc((size_t)rows * cnt * sizeof(double));
      be_->memset0(V, (size_t)rows * cnt * sizeof(double));
      scratch.push_back(V);
      for (size_t r = r0; r < r1; ++r) xrow[ops[r].second] = {V, (int)(r - r0)};
      // V (rows x cnt) = X (rows x size) W^T, the K dimension in panels
      const size_t panel = 1 << 22;
      for (size_t c0 = 0; c0 < XL.size; c0 += panel) {
        int kc = (int)std::min(panel, XL.size - c0);
        gv.add(V, rows, cnt, cnt,
               GemmSeg{ops[r0].first + c0, wstack[lk] + c0, kc, (int)XL.size, (int)XL.size, 0, 1, 1.0});
      }
      runs_dev.push_back({V, rows, cnt});
      r0 = r1;
    }
  }
  gv.run(be_, Precision::FP64);
  std::map<double*, std::vector<double>> vhost;
  for (auto& [V, rows, cols] : runs_dev) {
    auto& h = vhost[V];
    h.resize((size_t)rows * cols);
    be_->copy_d2h(h.data(), V, h.size() * sizeof(double));
  }
  be_->sync();
  // ---------------------------------------------------------------- assemble
  std::vector<double> val(vkeys.size(), 0.0);
  for (size_t v = 0; v < vkeys.size(); ++v) {
    auto it = xrow.find(vkeys[v].x);
    if (it == xrow.end() || !Nbuf[vkeys[v].y]) continue;  // operator absent (zero by symmetry)
    const auto& h = vhost[it->second.first];
    int cnt = w_count[{kind_dn(vkeys[v].x.kind), vkeys[v].x.k2}];
    val[v] = h[(size_t)it->second.second * cnt + v_col[v]];
  }
  for (auto& c : contribs) {
    if (c.order == 1) acc.g1[c.target] += c.c * val[c.v];
    else if (c.order == 2) acc.g2[c.target] += c.c * val[c.v];
    else acc.orb[c.target] += c.c * val[c.v];
  }
  for (double* N : Nbuf)
    if (N) be_->free(N);
  for (void* p : scratch) be_->free(p);
}

void Engine::measurement_walk(const std::function<void(int, Block&, Block&, Block&, const Block&,
                                                        const PsiLayout&, const double*)>& at_bond) {
  const int n = n_;
  std::vector<void*> owned;
  auto add_identity = [&](Block& B) {
    B.ops->allocate({kIdentityKey});
    double* I = B.ops->get(kIdentityKey);
    const Layout& L = B.ops->layout(0, 0);
    if (!I || L.size == 0) return;
    std::vector<double> h(L.size, 0.0);
    for (auto& bl : L.blk)
      if (bl.bra == bl.ket)
        for (int r = 0; r < bl.rows; ++r) h[bl.off + (size_t)r * bl.cols + r] = 1.0;
    be_->copy_h2d(I, h.data(), h.size() * sizeof(double));
  };
  try {
    auto vac = vacuum(true);
    auto E0 = enlarge(*vac, 0);
    if (!orb_mode_) {
      // strings of three and four operators on site 0 (elements with x3 = 0)
      std::vector<OpKey> keys;
      std::vector<std::pair<OpKey, Term>> terms;
      for (int len = 3; len <= 4; ++len) {
        std::vector<std::vector<int>> KL;
        seq_ranks(len, KL);
        for (int mask = 0; mask < (1 << len); ++mask) {
          std::vector<int> d(len);
          for (int b = 0; b < len; ++b) d[b] = (mask >> (len - 1 - b)) & 1;
          for (auto& kl : KL) {
            SiteOp so = site_string(d, kl);
            if (so.zero()) continue;
            OpKey key = string_key(d, kl, kl.back());
            keys.push_back(key);
            Term t;
            t.x = op_id();
            t.y = op_site(so);
            t.k2 = so.k2;
            t.coef = 1.0;
            terms.push_back({key, t});
          }
        }
      }
      E0->ops->allocate(keys);
      place_terms(*vac, nullptr, *E0, terms);
    }
    std::unique_ptr<Block> Lb = renormalize(*E0, *LU_[1], false);
    add_identity(*Lb);
    auto Le = enlarge(*Lb, 1);
    resident(R_[n - 3].get());
    auto Re = enlarge(*R_[n - 3], 2);
    PsiLayout P = make_psi(Le->ops->basis, Re->ops->basis, n_elec_, two_s_);
    if (P.size != prev_.len) throw std::runtime_error("internal: measurement pass layout differs from the state");
    double* psi = (double*)be_->alloc(std::max<size_t>(P.size, 1) * sizeof(double));
    owned.push_back(psi);
    be_->copy_d2d(psi, prev_.psi, P.size * sizeof(double));
    for (int i = 1; i <= n - 2; ++i) {
      resident(R_[n - i - 2].get());
      at_bond(i, *Lb, *Le, *Re, *R_[n - i - 2], P, psi);
      if (i == n - 2) break;
      // move the state to bond i+1, keeping its whole support
      HPsiPlan plan;
      plan.psi = P;
      double tr = 0.0;
      auto U = decimate(*Le, plan, psi, true, &tr);
      auto Lnext = renormalize(*Le, *U, false);
      add_identity(*Lnext);
      auto Le2 = enlarge(*Lnext, i + 1);
      resident(R_[n - i - 3].get());
      auto Re2 = enlarge(*R_[n - i - 3], i + 2);
      PsiLayout P2 = make_psi(Le2->ops->basis, Re2->ops->basis, n_elec_, two_s_);
      Prev from;
      from.valid = true;
      from.bond = i;
      from.Lb = Le->ops->basis;
      from.Rb = Re->ops->basis;
      from.Lc = Le->comps;
      from.Rc = Re->comps;
      for (auto& b : P.blk) from.blk.push_back({b.a, b.b, b.rows, b.cols, (int)b.off});
      from.psi = psi;
      from.len = P.size;
      double* psi2 = (double*)be_->alloc(std::max<size_t>(P2.size, 1) * sizeof(double));
      owned.push_back(psi2);
      move_lr(from, *U, *RU_[n - i - 2], *Le2, *Re2, P2, psi2);
      from.psi = nullptr;
      be_->sync();
      be_->free(psi);
      owned.erase(std::find(owned.begin(), owned.end(), (void*)psi));
      psi = psi2;
      Lb = std::move(Lnext);
      Le = std::move(Le2);
      Re = std::move(Re2);
      P = P2;
    }
  } catch (...) {
    for (void* p : owned) be_->free(p);
    throw;
  }
  for (void* p : owned) be_->free(p);
}

void Engine::rdm12(double* gamma, double* Gamma) {
  if (!prev_.valid) throw std::runtime_error("state: no sweep has run");
  drop_kept();  // the measurement pass needs the memory more than the next sweep
  if (n_ < 3 || prev_.bond != 1 || (int)LU_.size() < 2 || !LU_[1])
    throw std::runtime_error("state: the RDMs are taken at bond 1, the end of a full sweep");
  const int n = n_;
  const size_t nn = (size_t)n * n, n4 = nn * nn;
  // bond of every element (1-RDM: index p*n+q; 2-RDM: nn + ((p*n+q)*n+r)*n+s)
  std::vector<std::vector<size_t>> at(n - 1);
  // (bond 0 is folded into bond 1, whose left block is site 0 itself)
  for (int p = 0; p < n; ++p)
    for (int q = 0; q < n; ++q) at[std::max(1, std::min(n - 2, std::max(p, q)))].push_back((size_t)p * n + q);
  for (size_t t = 0; t < n4; ++t) {
    int x[4] = {(int)(t / (nn * n)), (int)(t / nn % n), (int)(t / n % n), (int)(t % n)};
    std::sort(x, x + 4);
    at[std::max(1, std::min(n - 2, x[2]))].push_back(nn + t);
  }
  const Options saved = opt_;
  rdm_mode_ = true;
  orb_mode_ = false;
  opt_.prec_renorm = Precision::FP64;
  opt_.D = 1 << 30;  // keep the whole support when moving the state
  RdmAcc acc;
  acc.g1.assign(nn, 0.0);
  acc.g2.assign(n4, 0.0);
  try {
    measurement_walk([&](int i, Block& Lb, Block& Le, Block& Re, const Block& Rp, const PsiLayout& P,
                         const double* psi) { rdm_bond(i, Lb, Le, Re, Rp, P, psi, at[i], acc); });
  } catch (...) {
    rdm_mode_ = false;
    opt_ = saved;
    throw;
  }
  rdm_mode_ = false;
  opt_ = saved;
  std::copy(acc.g1.begin(), acc.g1.end(), gamma);
  std::copy(acc.g2.begin(), acc.g2.end(), Gamma);
}


// ============================================================ orbital entanglement
// The ordering step of Sec. II "Numerical procedure": one- and two-orbital
// reduced density matrices of the state, from expectation values of SU(2)
// invariants built from single-orbital strings.  For orbitals p < q the
// invariants are [X_p (x) Y_q]^0 over the pairs (X, Y) of orb_strings() with
// equal rank and opposite particle change, plus the single-orbital scalars
// (number, double occupancy) of p and of q and the identity: 20 operators
// spanning the operators of the two orbitals that commute with their total
// spin and particle number.  The SU(2)-invariant (multiplet-averaged)
// rho_pq is the unique matrix of that span with the measured expectation
// values, found from the fixed Gram matrix of the 20 operators.
namespace {
const std::vector<std::pair<int, int>>& orb_pair_invariants() {
  static const std::vector<std::pair<int, int>> t = {
      {2, 2}, {2, 8}, {8, 2}, {8, 8},          // rank 0, no particle change
      {3, 3},                                  // spin-spin
      {0, 1}, {0, 7}, {6, 1}, {6, 7},          // rank 1/2: p gains, q loses a particle
      {1, 0}, {1, 6}, {7, 0}, {7, 6},          // rank 1/2: q gains, p loses
      {4, 5}, {5, 4}};                         // pair transfer
  return t;
}
constexpr int kOrbScalar[2] = {2, 8};  // number and double occupancy

// Fock space of `orbs` orbitals (modes up, down per orbital, Jordan-Wigner
// order), state index sum_m occ_m 2^(M-1-m): for one orbital d = 2 n_up +
// n_dn, for two a = 4 d_p + d_q.
struct SmallFock {
  int M = 0, dim = 0;
  std::vector<std::vector<double>> cr;  // creator of each mode, dim x dim row-major
  explicit SmallFock(int orbs) : M(2 * orbs), dim(1 << (2 * orbs)) {
    cr.assign(M, std::vector<double>((size_t)dim * dim, 0.0));
    for (int m = 0; m < M; ++m)
      for (int a = 0; a < dim; ++a) {
        const int bit = 1 << (M - 1 - m);
        if (a & bit) continue;
        int before = 0;
        for (int k = 0; k < m; ++k) before += (a >> (M - 1 - k)) & 1;
        cr[m][(size_t)(a | bit) * dim + a] = (before & 1) ? -1.0 : 1.0;
      }
  }
  // spinor component (comp 0: +1/2, 1: -1/2) of a+ (dag) or a~ on orbital o:
  // a+(+1/2) = a+_up, a+(-1/2) = a+_dn, a~(+1/2) = a_dn, a~(-1/2) = -a_up
  std::vector<double> comp(int o, int dag, int c) const {
    std::vector<double> r((size_t)dim * dim);
    if (dag) return cr[2 * o + c];
    const auto& src = cr[2 * o + (c == 0 ? 1 : 0)];
    const double f = c == 0 ? 1.0 : -1.0;
    for (int i = 0; i < dim; ++i)
      for (int j = 0; j < dim; ++j) r[(size_t)i * dim + j] = f * src[(size_t)j * dim + i];
    return r;
  }
  // sum_mask T[mask] O_0(m_0) O_1(m_1) ... over the slots (orbital, dag)
  std::vector<double> invariant(const std::vector<int>& orb, const std::vector<int>& dag,
                                const std::vector<double>& T) const {
    const int L = (int)orb.size();
    std::vector<double> out((size_t)dim * dim, 0.0);
    for (int mask = 0; mask < (1 << L); ++mask) {
      if (T[mask] == 0.0) continue;
      std::vector<double> P((size_t)dim * dim, 0.0);
      for (int i = 0; i < dim; ++i) P[(size_t)i * dim + i] = 1.0;
      for (int sl = 0; sl < L; ++sl) {
        const std::vector<double> O = comp(orb[sl], dag[sl], (mask >> sl) & 1);
        std::vector<double> Q((size_t)dim * dim, 0.0);
        for (int i = 0; i < dim; ++i)
          for (int k = 0; k < dim; ++k) {
            const double pv = P[(size_t)i * dim + k];
            if (pv == 0.0) continue;
            for (int j = 0; j < dim; ++j) Q[(size_t)i * dim + j] += pv * O[(size_t)k * dim + j];
          }
        P.swap(Q);
      }
      for (size_t e = 0; e < out.size(); ++e) out[e] += T[mask] * P[e];
    }
    return out;
  }
};

// matrix of [X_a (x) Y_b]^0 (a or b < 0: that orbital carries the identity)
std::vector<double> orb_invariant_matrix(const SmallFock& F, int a, int b) {
  const auto& os = orb_strings();
  std::vector<int> orb, dag;
  Variant v;
  int la = 0, lb = 0;
  if (a >= 0) {
    la = (int)os[a].dag.size();
    v.kl = os[a].kl;
    for (int d : os[a].dag) orb.push_back(0), dag.push_back(d);
  }
  if (b >= 0) {
    lb = (int)os[b].dag.size();
    v.ks = os[b].kl;
    for (int d : os[b].dag) orb.push_back(F.M == 4 ? 1 : 0), dag.push_back(d);
  }
  v.kX = 0;
  if (la + lb == 0) {
    std::vector<double> I((size_t)F.dim * F.dim, 0.0);
    for (int i = 0; i < F.dim; ++i) I[(size_t)i * F.dim + i] = 1.0;
    return I;
  }
  return F.invariant(orb, dag, tree_tensor(variant_tree(la, lb, 0, v), la + lb));
}

// inverse of a small symmetric positive definite matrix (Gauss-Jordan with
// partial pivoting)
std::vector<double> small_inverse(std::vector<double> A, int K) {
  std::vector<double> X((size_t)K * K, 0.0);
  for (int i = 0; i < K; ++i) X[(size_t)i * K + i] = 1.0;
  double scale = 0.0;
  for (double x : A) scale = std::max(scale, std::abs(x));
  for (int c = 0; c < K; ++c) {
    int piv = c;
    for (int r = c + 1; r < K; ++r)
      if (std::abs(A[(size_t)r * K + c]) > std::abs(A[(size_t)piv * K + c])) piv = r;
    if (std::abs(A[(size_t)piv * K + c]) < 1e-12 * scale)
      throw std::logic_error("internal: orbital invariants are linearly dependent");
    for (int j = 0; j < K; ++j) {
      std::swap(A[(size_t)c * K + j], A[(size_t)piv * K + j]);
      std::swap(X[(size_t)c * K + j], X[(size_t)piv * K + j]);
    }
    const double d = A[(size_t)c * K + c];
    for (int j = 0; j < K; ++j) {
      A[(size_t)c * K + j] /= d;
      X[(size_t)c * K + j] /= d;
    }
    for (int r = 0; r < K; ++r) {
      if (r == c) continue;
      const double f = A[(size_t)r * K + c];
      if (f == 0.0) continue;
      for (int j = 0; j < K; ++j) {
        A[(size_t)r * K + j] -= f * A[(size_t)c * K + j];
        X[(size_t)r * K + j] -= f * X[(size_t)c * K + j];
      }
    }
  }
  return X;
}

// The invariants of one and of two orbitals with their matrices and the
// inverse Gram matrices (fixed tables, built once).
struct OrbTables {
  int K1 = 0, K2 = 0;
  std::vector<std::vector<double>> M1, M2;
  std::vector<double> G1inv, G2inv;
  OrbTables() {
    SmallFock F1(1), F2(2);
    M1.push_back(orb_invariant_matrix(F1, -1, -1));
    for (int a : kOrbScalar) M1.push_back(orb_invariant_matrix(F1, a, -1));
    M2.push_back(orb_invariant_matrix(F2, -1, -1));
    for (int a : kOrbScalar) M2.push_back(orb_invariant_matrix(F2, a, -1));
    for (int b : kOrbScalar) M2.push_back(orb_invariant_matrix(F2, -1, b));
    for (auto& [a, b] : orb_pair_invariants()) M2.push_back(orb_invariant_matrix(F2, a, b));
    K1 = (int)M1.size();
    K2 = (int)M2.size();
    auto gram = [](const std::vector<std::vector<double>>& M) {
      const int K = (int)M.size();
      std::vector<double> G((size_t)K * K, 0.0);
      for (int i = 0; i < K; ++i)
        for (int j = 0; j < K; ++j)
          for (size_t e = 0; e < M[i].size(); ++e) G[(size_t)i * K + j] += M[i][e] * M[j][e];
      return G;
    };
    G1inv = small_inverse(gram(M1), K1);
    G2inv = small_inverse(gram(M2), K2);
  }
};
const OrbTables& orb_tables() {
  static const OrbTables t;
  return t;
}

// rho = sum_mu c_mu M_mu^T with G c = v (the member of the span of the
// invariants whose expectation values are v), symmetrised
void orb_solve(const std::vector<std::vector<double>>& M, const std::vector<double>& Ginv,
               const std::vector<double>& v, int dim, double* rho) {
  const int K = (int)M.size();
  std::vector<double> c(K, 0.0);
  for (int i = 0; i < K; ++i)
    for (int j = 0; j < K; ++j) c[i] += Ginv[(size_t)i * K + j] * v[j];
  std::vector<double> r((size_t)dim * dim, 0.0);
  for (int mu = 0; mu < K; ++mu)
    for (int i = 0; i < dim; ++i)
      for (int j = 0; j < dim; ++j) r[(size_t)i * dim + j] += c[mu] * M[mu][(size_t)j * dim + i];
  for (int i = 0; i < dim; ++i)
    for (int j = 0; j < dim; ++j)
      rho[(size_t)i * dim + j] = 0.5 * (r[(size_t)i * dim + j] + r[(size_t)j * dim + i]);
}
}  // namespace

int orbital_pair_invariant_count() { return (int)orb_pair_invariants().size(); }

void orbital_rdms_from_invariants(int n, const double* inv1, const double* inv2, double* rho1, double* rho2) {
  const OrbTables& T = orb_tables();
  const int NP = (int)orb_pair_invariants().size();
  std::vector<double> r4(16);
  for (int p = 0; p < n; ++p) {
    std::vector<double> v{1.0, inv1[2 * p], inv1[2 * p + 1]};
    orb_solve(T.M1, T.G1inv, v, 4, r4.data());
    for (int d = 0; d < 4; ++d) rho1[4 * p + d] = r4[5 * d];
  }
  std::fill(rho2, rho2 + (size_t)n * n * 256, 0.0);
  for (int p = 0; p < n; ++p)
    for (int q = p + 1; q < n; ++q) {
      std::vector<double> v{1.0, inv1[2 * p], inv1[2 * p + 1], inv1[2 * q], inv1[2 * q + 1]};
      for (int mu = 0; mu < NP; ++mu) v.push_back(inv2[((size_t)p * n + q) * NP + mu]);
      orb_solve(T.M2, T.G2inv, v, 16, rho2 + ((size_t)p * n + q) * 256);
    }
}

void Engine::orbital_invariants(std::vector<double>& inv1, std::vector<double>& inv2) {
  if (!prev_.valid) throw std::runtime_error("state: no sweep has run");
  drop_kept();
  if (n_ < 3 || prev_.bond != 1 || (int)LU_.size() < 2 || !LU_[1])
    throw std::runtime_error("state: the orbital RDMs are taken at bond 1, the end of a full sweep");
  const int n = n_;
  const auto& os = orb_strings();
  const auto& pinv = orb_pair_invariants();
  const int NP = (int)pinv.size();
  RdmAcc acc;
  acc.orb.assign((size_t)n * 2 + (size_t)n * n * NP, 0.0);
  auto t1 = [&](int p, int t) { return (size_t)p * 2 + t; };
  auto t2 = [&](int p, int q, int mu) { return (size_t)n * 2 + ((size_t)p * n + q) * NP + mu; };
  const Options saved = opt_;
  rdm_mode_ = true;
  orb_mode_ = true;
  opt_.prec_renorm = Precision::FP64;
  opt_.D = 1 << 30;  // keep the whole support when moving the state
  try {
    measurement_walk([&](int i, Block& Lb, Block& Le, Block& Re, const Block& Rp, const PsiLayout& P,
                         const double* psi) {
      RdmRequests rq;
      // <[[x (x) s]^kX (x) y]^0> with x = string xa of site xp in L(i) (xa <
      // 0: the identity), s = string sa of site i, y = string ya of the last
      // site (last bond only; < 0: the identity); kX = rank of y
      auto req = [&](int xp, int xa, int sa, int ya, size_t target) {
        std::vector<int> sd, sk;
        if (sa >= 0) sd = os[sa].dag, sk = os[sa].kl;
        auto skey = std::make_pair(sd, sk);
        auto si = rq.s_index.find(skey);
        if (si == rq.s_index.end()) {
          si = rq.s_index.emplace(skey, (int)rq.s_ops.size()).first;
          rq.s_ops.push_back(site_string(sd, sk));
        }
        std::vector<int> yd, yk;
        if (ya >= 0) yd = os[ya].dag, yk = os[ya].kl;
        auto ykey = std::make_tuple((int)yd.size(), -1, yd, yk);
        auto yi = rq.y_index.find(ykey);
        if (yi == rq.y_index.end()) {
          yi = rq.y_index.emplace(ykey, (int)rq.y_ops.size()).first;
          if (ya < 0) {
            rq.y_ops.push_back(op_id());
          } else {
            SiteOp so2 = site_string(yd, yk);
            OpKey key{K_T0 + so2.dn, (int)rq.y_temps.size(), 0, so2.k2};
            rq.y_temps.push_back({key, so2});
            rq.y_ops.push_back(op_blk(key.kind, key.i, 0, key.k2));
          }
        }
        const int kX = ya >= 0 ? orb_rank(ya) : 0;
        RdmVKey vk{yi->second, si->second, kX, xa >= 0 ? orb_key(xp, xa) : kIdentityKey, 0};
        auto vi = rq.v_index.find(vk);
        if (vi == rq.v_index.end()) {
          vi = rq.v_index.emplace(vk, (int)rq.vkeys.size()).first;
          rq.vkeys.push_back(vk);
        }
        rq.contribs.push_back({target, 3, 1.0, vi->second});
      };
      for (int t = 0; t < 2; ++t) {
        if (i == 1) req(0, kOrbScalar[t], -1, -1, t1(0, t));  // site 0 lives in L(1)
        req(-1, -1, kOrbScalar[t], -1, t1(i, t));
      }
      for (int p = 0; p < i; ++p)
        for (int mu = 0; mu < NP; ++mu) req(p, pinv[mu].first, pinv[mu].second, -1, t2(p, i, mu));
      if (i == n - 2) {
        for (int t = 0; t < 2; ++t) req(-1, -1, -1, kOrbScalar[t], t1(n - 1, t));
        for (int p = 0; p < n - 2; ++p)
          for (int mu = 0; mu < NP; ++mu) req(p, pinv[mu].first, -1, pinv[mu].second, t2(p, n - 1, mu));
        for (int mu = 0; mu < NP; ++mu) req(-1, -1, pinv[mu].first, pinv[mu].second, t2(n - 2, n - 1, mu));
      }
      rdm_eval(Lb, Le, Re, Rp, P, psi, rq, acc);
    });
  } catch (...) {
    rdm_mode_ = orb_mode_ = false;
    opt_ = saved;
    throw;
  }
  rdm_mode_ = orb_mode_ = false;
  opt_ = saved;
  inv1.assign(acc.orb.begin(), acc.orb.begin() + (size_t)n * 2);
  inv2.assign(acc.orb.begin() + (size_t)n * 2, acc.orb.end());
}

void Engine::orbital_rdms(double* rho1, double* rho2) {
  std::vector<double> inv1, inv2;
  orbital_invariants(inv1, inv2);
  orbital_rdms_from_invariants(n_, inv1.data(), inv2.data(), rho1, rho2);
}

void Engine::orbital_entanglement(double* s1, double* mutual) {
  const int n = n_;
  std::vector<double> r1((size_t)n * 4), r2((size_t)n * n * 256);
  orbital_rdms(r1.data(), r2.data());
  auto ent = [](const double* w, int m) {
    double s = 0.0;
    for (int k = 0; k < m; ++k)
      if (w[k] > 1e-14) s -= w[k] * std::log(w[k]);
    return s;
  };
  for (int p = 0; p < n; ++p) s1[p] = ent(&r1[4 * p], 4);  // rho_p is diagonal
  // eigenvalues of every rho_pq: one batched float64 eigensolver launch
  const size_t npair = (size_t)n * (n - 1) / 2;
  std::fill(mutual, mutual + (size_t)n * n, 0.0);
  if (npair == 0) return;
  struct DevBufs {
    Backend* be;
    std::vector<void*> p;
    ~DevBufs() {
      for (void* q : p) be->free(q);
    }
    double* get(size_t n) {
      p.push_back(be->alloc(n * sizeof(double)));
      return (double*)p.back();
    }
  } bufs{be_, {}};
  double* dA = bufs.get(npair * 256);
  double* dV = bufs.get(npair * 256);
  double* dw = bufs.get(npair * 16);
  std::vector<double> hA(npair * 256), hw(npair * 16);
  std::vector<EighTask> tasks;
  size_t k = 0;
  for (int p = 0; p < n; ++p)
    for (int q = p + 1; q < n; ++q, ++k) {
      std::copy(&r2[((size_t)p * n + q) * 256], &r2[((size_t)p * n + q) * 256] + 256, &hA[k * 256]);
      tasks.push_back({dA + k * 256, dw + k * 16, dV + k * 256, 16});
    }
  be_->copy_h2d(dA, hA.data(), hA.size() * sizeof(double));
  be_->eigh(tasks);
  be_->check_device_flag();
  be_->copy_d2h(hw.data(), dw, hw.size() * sizeof(double));
  be_->sync();
  k = 0;
  for (int p = 0; p < n; ++p)
    for (int q = p + 1; q < n; ++q, ++k) {
      const double I = s1[p] + s1[q] - ent(&hw[k * 16], 16);
      mutual[(size_t)p * n + q] = mutual[(size_t)q * n + p] = I;
    }
}

}  // namespace dmrg
