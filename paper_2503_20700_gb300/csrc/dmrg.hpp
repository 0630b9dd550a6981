// Spin-adapted (SU(2) x U(1)) two-site DMRG: host planner.
//
// The planner owns the quantum-number bookkeeping of Sec. II.B-C of the paper
// (MPS over SU(2) multiplet sectors, D counted in multiplets) and turns every
// step of a sweep into task lists for the device primitives of backend.hpp:
//   * blocking   (block (x) site -> enlarged block operators):   place tasks
//   * H_eff psi  (sigma = sum_t c_t O^L_t psi O^R_t^T):          grouped GEMMs
//   * decimation (rho = psi psi^T per sector, eigh, selection):  GEMM + eigh
//   * renormalisation (O' = U^T O U):                            grouped GEMMs
// The SU(2) recoupling coefficients (6j/9j) are folded into the task lists on
// the host; the device only sees scaled dense sector blocks.
//
// Operators carried by a block of sites (normal/complementary scheme of ab
// initio DMRG, with the pair operators on the side with fewer sites):
//   H            block Hamiltonian
//   C_p          a+_p spinor (rank 1/2), p in block
//   S_p          complementary three-index spinor, p outside the block
//   A^k_pq, B^k_pq   normal pair operators [a+a+]^k, [a+a~]^k, p<=q in block
//   P^k_pq, QJ_pq, QK^k_pq   complementary pair operators, p<=q outside
#pragma once
#include <cstdint>
#include <functional>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "backend.hpp"
#include "su2.hpp"

namespace dmrg {

struct PsiLayout;

struct Sector {
  int n, j, dim, off;
};

struct Basis {
  std::vector<Sector> sec;
  int total = 0;
  int find(int n, int j) const {
    for (size_t i = 0; i < sec.size(); ++i)
      if (sec[i].n == n && sec[i].j == j) return (int)i;
    return -1;
  }
};

// Component of an enlarged basis: block sector bsec coupled with site
// multiplet `site` sits in enlarged sector esec at multiplet offset eoff.
struct EnlComp {
  int bsec, site, esec, eoff;
};

struct Layout {
  int dn = 0, k2 = 0;
  struct Blk {
    int bra, ket, rows, cols;
    size_t off;
  };
  std::vector<Blk> blk;
  size_t size = 0;
  int nket = 0;
  std::vector<int> lut;  // bra * nket + ket -> block index (or -1)
  int find(int bra, int ket) const { return lut[(size_t)bra * nket + ket]; }
};

enum Kind { K_H = 0, K_C, K_S, K_A, K_B, K_P, K_QJ, K_QK,
            // temporaries of the RDM pass with particle change -2 .. 2
            K_TM2, K_TM1, K_T0, K_TP1, K_TP2 };

struct OpKey {
  int kind, i, j, k2;
  bool operator<(const OpKey& o) const {
    if (kind != o.kind) return kind < o.kind;
    if (i != o.i) return i < o.i;
    if (j != o.j) return j < o.j;
    return k2 < o.k2;
  }
};

inline int kind_dn(int kind) {
  if (kind >= K_TM2) return kind - K_T0;
  switch (kind) {
    case K_C: return 1;
    case K_S: return -1;
    case K_A: return 2;
    case K_P: return -2;
    default: return 0;
  }
}
inline int kind_parity(int kind) {
  if (kind >= K_TM2) return (kind - K_T0) & 1;
  return (kind == K_C || kind == K_S) ? 1 : 0;
}

// A set of operators on one basis, with one device allocation per layout.
struct OpSet {
  Basis basis;
  std::map<std::pair<int, int>, Layout> layouts;   // (dn, k2)
  std::map<OpKey, double*> ops;
  std::vector<void*> mem;
  Backend* be = nullptr;
  ~OpSet();
  const Layout& layout(int dn, int k2);
  double* get(const OpKey& k) const {
    auto it = ops.find(k);
    return it == ops.end() ? nullptr : it->second;
  }
  // allocate (zeroed) storage for the given keys
  void allocate(const std::vector<OpKey>& keys);
  size_t bytes() const;
  // Staging of the operator storage to pinned host memory (renormalised
  // blocks that the sweep does not need for a while, when the device budget
  // is tight): every allocation is copied out on the backend's side stream
  // and freed; stage_in brings it back and rebases the operator pointers.
  std::vector<size_t> mem_bytes;  // size of each allocation of mem
  std::vector<void*> host;        // pinned copies while staged out
  std::vector<void*> pending;     // pinned copies whose copy back may still run
  bool on_host = false;
  bool arriving = false;          // staged in; the main stream has not joined yet
  size_t device_bytes() const;
  void stage_out();
  void stage_in();
  void release_pending();
};

struct Block {
  bool left = true;
  int nsites = 0;      // left: sites 0..nsites-1; right: sites n-nsites..n-1
  bool normal = true;  // pair operators normal (own pairs) or complementary
  std::unique_ptr<OpSet> ops;
  // enlarged-block bookkeeping (set when the block was made by blocking)
  std::vector<EnlComp> comps;
  const Basis* parent = nullptr;
};

// Transformation from an enlarged block to its renormalised block (the MPS
// tensor of that bond in the block-sparse SU(2) form): for every enlarged
// sector s the kept eigenvectors are the rows of a kept[s] x dim(s) matrix.
struct SavedU {
  Basis enl;                   // enlarged basis (block (x) site or site (x) block)
  std::vector<EnlComp> comps;  // its components
  Basis parent;                // basis of the block that was enlarged
  Basis next;                  // basis of the renormalised block
  std::vector<int> kept, map;  // per enlarged sector: kept count, new sector (-1)
  std::vector<size_t> off;     // offset of each sector's rows in buf
  double* buf = nullptr;
  Backend* be = nullptr;
  ~SavedU() {
    if (be && buf) be->free(buf);
  }
  const double* ut(int s) const { return buf + off[s]; }
};

struct Options {
  int D = 64;
  int max_davidson_iter = 200;
  double davidson_tol = 1e-10;
  Precision prec = Precision::FP64;         // H_eff psi GEMMs
  Precision prec_renorm = Precision::FP64;  // renormalisation / complementary GEMMs
  int max_space = 24;
  int verbose = 0;
  uint64_t seed = 0;          // Davidson start vector where no prediction exists
  bool debug_bounds = false;  // host check of every tcgen05 plan before launch
  double trunc_target = 0.0;  // > 0: dynamic bond dimension (discarded weight bound)
  int D_min = 1;              // lower bound of the dynamic bond dimension
  bool rq64_every_bond = false;  // split runs: float64 Rayleigh quotient at every bond
  int tc_drain_terms = 1024;      // FP32 accumulation length of the tcgen05 contraction
  bool tc_autotune = false;  // time the candidate schedules of each sector histogram, keep the fastest
};

// Autotuning record of one sector histogram of the tcgen05 contraction: the
// CUDA-event time of one product under each candidate schedule (-1: not yet
// timed) and the fastest once all were timed.
struct TuneRec {
  std::vector<double> ms;
  int best = -1;
};

struct SweepStats {
  double energy = 0.0;
  double max_trunc = 0.0;
  int davidson_iters = 0;
  double hpsi_flops = 0.0;
  double hpsi_seconds = 0.0;
  int hpsi_calls = 0;
  int noconv_bonds = 0;  // Davidson solves that stopped above the tolerance
  std::vector<int> kept;  // multiplets kept at each decimation, in sweep order
  // wall time per phase of the sweep (seconds, host clock around device-synchronised steps)
  double t_enlarge = 0.0, t_plan = 0.0, t_davidson = 0.0, t_decimate = 0.0, t_renorm = 0.0,
         t_guess = 0.0;
  // inside enlarge: host term lists, host placement lists, complementary GEMMs
  double t_enl_terms = 0.0, t_enl_place_host = 0.0, t_enl_comp = 0.0, t_enl_place_run = 0.0,
         t_enl_alloc = 0.0;
  // inside plan: host item lists, task lists (tcgen05 preparation included),
  // uploads and operator splits (device-synchronised), diagonal (synchronised)
  double t_plan_items = 0.0, t_plan_tasks = 0.0, t_plan_upload = 0.0, t_plan_diag = 0.0;
};

class Engine {
 public:
  Engine(Backend* be, int n, const double* h, const double* eri, double e_core, int n_elec,
         int two_s, const Options& opt, const int* occ, const int* two_s_right);
  ~Engine();

  // One full sweep (L->R then R->L).  Returns the Davidson energy of the last
  // bond (including e_core).
  SweepStats sweep();
  // Part of a sweep: L->R over bonds 0..last (l2r), or R->L over bonds
  // n-2..last.  An L->R part starts a sweep; an R->L part needs the left
  // blocks of a completed L->R half-sweep.  Afterwards the blocks of the next
  // bond in that direction are held: bond last+1 after an L->R part, bond
  // last-1 after an R->L part.
  SweepStats sweep_part(bool l2r, int last);
  // Davidson at `bond` on the blocks the context holds (after a partial
  // sweep that stopped next to it), without decimation or any change of the
  // stored state.  Each H_eff psi is timed with CUDA events; after Davidson
  // stops, H_eff psi is applied to its vector until min_calls products ran.
  struct BondSolve {
    double energy = 0.0;       // Davidson eigenvalue (+ e_core)
    double energy_rq64 = 0.0;  // float64 Rayleigh quotient of its vector (+ e_core)
    double residual64 = 0.0;   // ||H psi - E_rq psi|| in float64, ||psi|| = 1
    double gap = 0.0;          // second minus lowest Ritz value at exit
    int iterations = 0, calls = 0;
    double flops_per_call = 0.0;
    std::vector<double> call_ms;  // CUDA-event time of every product
    double contraction_ms = 0.0;  // of which the contraction launches (kernel and chunk reduction)
    double split_ms = 0.0;        // and the psi splits of the tcgen05 path
    long contraction_launches = 0;
    size_t dim = 0;
  };
  BondSolve solve_bond(int bond, bool l2r, Precision p, int max_iter, double tol, int min_calls,
                       bool check64 = true);
  // float64 Rayleigh quotient and residual of the vector of the last
  // solve_bond (one float64 H_eff psi, timed with CUDA events: *ms)
  void check_bond64(double* energy_rq64, double* residual64, double* ms, double* flops);
  // y = H_eff x on the blocks of the last solve_bond, in precision p (host
  // vectors in the two-site layout of that bond); returns the dimension (and
  // does nothing else when x or y is null)
  size_t apply_bond(Precision p, const double* x, double* y);
  double energy() const { return energy_; }
  int n() const { return n_; }
  void set_D(int D) { opt_.D = D; }
  void set_davidson(int max_iter, double tol) {
    opt_.max_davidson_iter = max_iter;
    opt_.davidson_tol = tol;
  }
  void set_tc_autotune(bool on) { opt_.tc_autotune = on; }
  void set_precision(Precision p, Precision pr) {
    opt_.prec = p;
    opt_.prec_renorm = pr;
    drop_kept();  // complementary operators of enlarged blocks follow the precision
  }
  const std::vector<double>& bond_energies() const { return bond_e_; }
  // Multiplet count of the left block L(m) / right block R(m) (sites counted)
  int left_dim(int m) const;
  int right_dim(int m) const;
  // the same in U(1) states (each multiplet of spin S counts 2S+1): the
  // bond dimension D~ a non-spin-adapted calculation needs for this basis
  int left_dim_u1(int m) const;
  int right_dim_u1(int m) const;
  // Two-site wavefunction at the last optimised bond (for RDMs / checks)
  int last_bond() const { return last_bond_; }
  // Spin-free one- and two-particle RDMs (Eqs. onerdm, twordm) of the
  // two-site wavefunction of the last optimised bond, which must be bond 1
  // (the end of a full sweep):  gamma[p*n+q] = <sum_s a+_ps a_qs>,
  // Gamma[((p*n+q)*n+r)*n+s] = <sum_st a+_ps a+_qt a_rt a_ss>.
  void rdm12(double* gamma, double* Gamma);
  // One- and two-orbital reduced density matrices of the same state (the
  // orbital-ordering step of Sec. II "Numerical procedure"), averaged over
  // the 2S+1 states of the multiplet: rho1[4p + d] = weight of the local
  // state d of orbital p (0 empty, 1 down, 2 up, 3 doubly occupied);
  // rho2[(p n + q) 256 + 16 a + b] for p < q the 16 x 16 matrix over the
  // local states a = 4 d_p + d_q, with Tr(rho_pq X) = <X> for operators X of
  // the four modes of p and q (Jordan-Wigner order p-up, p-down, q-up,
  // q-down); entries with p >= q are zero.
  void orbital_rdms(double* rho1, double* rho2);
  // The expectation values the orbital RDMs are assembled from: inv1[2p + t]
  // = <number (t = 0) / double-occupancy (t = 1) string of p>, inv2[(p n + q)
  // P + mu] (p < q) = <[X_p (x) Y_q]^0> for the P pair invariants.
  void orbital_invariants(std::vector<double>& inv1, std::vector<double>& inv2);
  // One-orbital entropies s1[p] = -Tr rho_p ln rho_p and mutual information
  // mutual[p n + q] = s_p + s_q - s_pq (zero diagonal).
  void orbital_entanglement(double* s1, double* mutual);

  Backend* backend() const { return be_; }
  // Schedule of the last planned tcgen05 H_eff psi product: shape = {tile
  // width, item chunks per CTA, task order, CTAs per cluster}; ms[k] = time of candidate k of
  // tc_shape_candidates() for its sector histogram (-1: not timed); returns
  // false when no tcgen05 product was planned yet.
  bool tc_schedule_info(int shape[4], std::vector<double>* ms) const;
  // device and pinned-host bytes of the stored blocks, the largest one, and
  // the largest working memory of a bond beyond the stored blocks so far
  void memory_detail(size_t* dev, size_t* host, size_t* max_block, size_t* max_extra,
                     size_t* mps_bytes = nullptr) const;

 private:
  friend struct EngineAccess;
  Backend* be_;
  int n_, n_elec_, two_s_;
  double e_core_;
  Options opt_;
  std::vector<double> h_, g_;  // h_pq and g_pqrs = (ps|qr)
  std::vector<std::unique_ptr<Block>> L_, R_;  // L_[m]: sites 0..m-1, R_[m]: last m sites
  // Enlarged blocks kept for the opposite half-sweep: the enlarged L(i) (x)
  // site i built at bond i going right is the left block of bond i again on
  // the way back, and L(i) does not change in between (likewise for the
  // right side).  Kept while this context holds at most kKeepFraction of the
  // device and the device still has kKeepFreeFraction free; dropped when the
  // precision changes and before the RDM pass.
  std::vector<std::unique_ptr<Block>> keep_L_, keep_R_;
  static constexpr double kKeepFraction = 0.4, kKeepFreeFraction = 0.2;
  void drop_kept() {
    keep_L_.clear();
    keep_R_.clear();
  }
  int tL_, tR_;
  // staging policy (hbm budget): the sweep step of each block's next use and
  // the memory a bond needs beyond the stored blocks (from the last bond)
  size_t bond_extra_ = 0, max_bond_extra_ = 0;
  void stage_for_step(int step);
  int next_use(bool left, int m, int step) const;
  void resident(Block* b);  // operators on the device and joined
  bool stage_out_one();     // the stored block used farthest ahead (not by the current step)
  int cur_step_ = 0;
  double energy_ = 0.0;
  std::vector<double> bond_e_;
  int last_bond_ = -1;
  std::vector<int> occ_, path_;
  std::vector<std::unique_ptr<SavedU>> LU_, RU_;
  double* ones_ = nullptr;  // vector of ones (identity diagonals)
  size_t ones_len_ = 0;  // LU_[m]: -> L_[m], RU_[m]: -> R_[m]
  // two-site wavefunction of the last optimised bond (Davidson guess of the next one)
  struct Prev {
    bool valid = false;
    int bond = -1;
    Basis Lb, Rb;
    std::vector<EnlComp> Lc, Rc;
    std::vector<std::array<int, 5>> blk;  // (a, b, rows, cols, off)
    double* psi = nullptr;
    size_t len = 0;
  } prev_;

  double hh(int p, int q) const { return h_[(size_t)p * n_ + q]; }
  double g(int p, int q, int r, int s) const {
    return g_[(((size_t)p * n_ + q) * n_ + r) * n_ + s];
  }
  bool left_normal(int m) const { return m < tL_; }
  bool right_normal(int m) const { return m < tR_; }

  SweepStats stats_;
  bool rdm_mode_ = false;  // blocking builds only C and the normal pairs
  bool orb_mode_ = false;  // with rdm_mode_: left blocks carry the single-orbital strings of their sites
  // The measurement pass: walks bonds 1..n-2 over the state of the last
  // sweep (bond 1), calling at_bond(i, L(i), L(i) (x) site i, site i+1 (x)
  // R, R, psi layout, psi) and moving the state with its whole support.
  void measurement_walk(const std::function<void(int, Block&, Block&, Block&, const Block&,
                                                 const PsiLayout&, const double*)>& at_bond);
  struct RdmAcc;
  struct RdmRequests;
  void rdm_eval(Block& Lb, Block& Le, Block& Re, const Block& Rparent, const struct PsiLayout& P,
                const double* psi, RdmRequests& rq, RdmAcc& acc);
  void rdm_bond(int i, Block& Lb, Block& Le, Block& Re, const Block& Rparent, const struct PsiLayout& P,
                const double* psi, const std::vector<size_t>& elems, RdmAcc& acc);
  void move_lr(const Prev& from, const SavedU& U, const SavedU& V, const Block& Le, const Block& Re,
               const struct PsiLayout& P, double* psi);
  std::unique_ptr<Block> vacuum(bool left);
  std::unique_ptr<Block> enlarge(const Block& b, int site);
  void place_terms(const Block& b, const OpSet* tmp, Block& e,
                   const std::vector<std::pair<OpKey, struct Term>>& terms);
  void build_comp_from_normal(const Block& b, OpSet& dst, const std::vector<OpKey>& keys);
  std::unique_ptr<Block> renormalize(Block& enl, const SavedU& U, bool switch_to_comp);
  void tc_contract(const std::vector<HpsiBlock>& blocks, const std::vector<HpsiItem>& items, double flops);
  // tcgen05 schedules of a planned product: device lists and scratch of the
  // plan's current shape; rescheduling for another shape keeps the operands
  void tc_upload_schedule(struct HPsiPlan& plan);
  void tc_reschedule(struct HPsiPlan& plan, int candidate);
  int tc_ctas_for(int cluster) const;  // CTAs of a persistent launch in clusters of that size
  std::map<uint64_t, TuneRec> tune_cache_;
  uint64_t last_tc_key_ = 0;
  int last_tc_cand_ = -1;
  bool have_tc_plan_ = false;
  void build_initial_right();
  void plan_hpsi(Block& Le, Block& Re, struct HPsiPlan& plan);
  void apply_hpsi(struct HPsiPlan& plan);
  double davidson(struct HPsiPlan& plan, double* psi, int* iters);
  std::vector<double>* call_ms_ = nullptr;  // when set: CUDA-event ms of every H_eff psi
  // vector of the last solve_bond and where it lives
  void end_bond_solves();
  double* solve_psi_ = nullptr;
  int solve_bond_ = -1;
  bool solve_l2r_ = false;
  double last_gap_ = 0.0;                   // Ritz gap at the last Davidson exit
  int cur_i_ = -1;                          // bond the blocks are held for
  std::unique_ptr<SavedU> decimate(Block& enl, const struct HPsiPlan& plan, const double* psi,
                                   bool left, double* trunc);
  double optimize_bond(int i, bool left_to_right, double* trunc);
  int step_of(int i, bool l2r) const { return l2r ? i : (n_ - 2) + (n_ - 2 - i); }
  void guess(int bond, bool l2r, const Block& Le, const Block& Re, const struct HPsiPlan& plan,
             double* psi);
  void save_prev(int bond, const Block& Le, const Block& Re, const struct HPsiPlan& plan,
                 const double* psi);

 public:
  // ---- accounting
  double sweep_seconds = 0.0;
  double sweep_device_ms = 0.0;  // CUDA-event time of the last sweep
};

// The orbital RDMs (layout of Engine::orbital_rdms) from the invariants of
// Engine::orbital_invariants: a host computation over fixed tables.
void orbital_rdms_from_invariants(int n, const double* inv1, const double* inv2, double* rho1, double* rho2);
int orbital_pair_invariant_count();

std::string last_error();
void set_last_error(const std::string& e);

}  // namespace dmrg
