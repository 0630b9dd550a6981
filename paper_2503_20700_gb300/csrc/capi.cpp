// extern "C" entry points (include/dmrgscf.h).
#include <algorithm>
#include <cmath>
#include <numeric>
#include <atomic>
#include <cstring>
#include <exception>
#include <memory>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/dmrgscf.h"
#include "casscf.hpp"
#include "hpsi_fused.cuh"
#include "hpsi_noalloc.hpp"
#include "hpsi_tc.cuh"
#include "dmrg.hpp"

struct dmrg_ctx {
  std::unique_ptr<dmrg::Backend> be;
  std::unique_ptr<dmrg::Engine> eng;
  std::string err;
  int n = 0;
  int sweeps_done = 0;
  dmrg::SweepStats last;
  double sweep_seconds = 0.0;
  bool strict = false;
};

namespace {
// wait bound of the kernel-level entry points (dmrg_set_kernel_wait_timeout)
std::atomic<unsigned long long> g_kernel_wait_ns{2000000000ull};
std::atomic<int> g_kernel_drain_terms{dmrg::kTcDrainTerms};
// schedule shape of the kernel-level contraction (index into the candidates)
std::atomic<int> g_kernel_tc_cand{0};
thread_local std::string tl_err;
thread_local double tl_contract_ms = 0.0;

dmrg_status fail(dmrg_ctx* c, dmrg_status s, const std::string& msg) {
  if (c) c->err = msg;
  tl_err = msg;
  return s;
}

dmrg_status translate(dmrg_ctx* c, const std::exception& e) {
  std::string m = e.what();
  if (dynamic_cast<const std::invalid_argument*>(&e)) return fail(c, DMRG_EINVAL, m);
  if (dynamic_cast<const std::bad_alloc*>(&e)) return fail(c, DMRG_ENOMEM, m);
  if (m.rfind("cuda", 0) == 0 || m.rfind("CUDA", 0) == 0) return fail(c, DMRG_ECUDA, m);
  if (m.rfind("out of device memory", 0) == 0) return fail(c, DMRG_ENOMEM, m);
  if (m.rfind("timeout", 0) == 0) return fail(c, DMRG_ETIMEOUT, m);
  if (m.rfind("davidson", 0) == 0) return fail(c, DMRG_ENOCONV, m);
  if (m.rfind("state", 0) == 0) return fail(c, DMRG_ESTATE, m);
  return fail(c, DMRG_EINTERNAL, m);
}

// Makes `device` current for its lifetime and puts the caller's device back
// on every exit path (a thrown launch error included).
struct DeviceGuard {
  int prev = -1;
  DeviceGuard(int device, cudaError_t* e) {
    *e = cudaGetDevice(&prev);
    if (*e != cudaSuccess) {
      prev = -1;
      return;
    }
    *e = cudaSetDevice(device);
  }
  cudaError_t restore() {
    cudaError_t e = cudaSuccess;
    if (prev >= 0) e = cudaSetDevice(prev);
    prev = -1;
    return e;
  }
  ~DeviceGuard() { restore(); }
  DeviceGuard(const DeviceGuard&) = delete;
  DeviceGuard& operator=(const DeviceGuard&) = delete;
};

bool sweep_precision_ok(int p) {
  return p == DMRG_FP64 || p == DMRG_SPLIT_TF32 || p == DMRG_SPLIT_HPSI || p == DMRG_SPLIT_HPSI_TC ||
         p == DMRG_SPLIT_ALL_TC;
}

// dmrg_precision -> (H_eff psi kernel precision, renormalisation GEMM precision)
void map_precision(int p, dmrg::Precision* hpsi, dmrg::Precision* renorm) {
  *hpsi = p == DMRG_FP64                                   ? dmrg::Precision::FP64
          : (p == DMRG_SPLIT_HPSI_TC || p == DMRG_SPLIT_ALL_TC) ? dmrg::Precision::TC_TF32X3
                                                               : dmrg::Precision::SPLIT_TF32;
  *renorm = p == DMRG_SPLIT_TF32     ? dmrg::Precision::SPLIT_TF32
            : p == DMRG_SPLIT_ALL_TC ? dmrg::Precision::TC_TF32X3
                                     : dmrg::Precision::FP64;
}

// Default initial product state: electrons spread evenly, spins coupled from
// the right end with the smallest intermediate spins (same rule as the
// synthetic-input generator of the test suite).
bool default_state(int n, int n_elec, int two_s, std::vector<int>& occ, std::vector<int>& path) {
  occ.assign(n, 0);
  if (n_elec <= n) {
    for (int i = 0; i < n_elec; ++i) occ[i] = 1;
  } else {
    for (int i = 0; i < n; ++i) occ[i] = (i < n_elec - n) ? 2 : 1;
  }
  int single = 0;
  for (int o : occ) single += (o == 1);
  if (two_s > single) return false;
  path.assign(n + 1, 0);
  int seen = 0, cur = 0;
  for (int i = n - 1; i >= 0; --i) {
    if (occ[i] == 1) {
      ++seen;
      if (seen <= two_s) ++cur;
      else cur = (cur == two_s) ? cur + 1 : cur - 1;
    }
    path[i] = cur;
  }
  return path[0] == two_s;
}
}  // namespace

extern "C" {

void dmrg_default_opts(dmrg_opts* o) {
  if (!o) return;
  o->D = 64;
  o->max_davidson_iter = 200;
  o->davidson_tol = 1e-10;
  o->precision = DMRG_FP64;
  o->max_space = 24;
  o->verbose = 0;
  o->device = 0;
  o->strict_convergence = 0;
  o->debug_bounds = 0;
  o->seed = 0;
  o->hbm_budget_bytes = 0;
  o->wait_timeout_s = 2.0;
  o->trunc_target = 0.0;
  o->D_min = 1;
  o->rq64_every_bond = 0;
  o->tc_drain_terms = dmrg::kTcDrainTerms;
  o->tc_autotune = 0;
}

dmrg_status dmrg_init(dmrg_ctx** out, const double* h, const double* eri, const double* chol,
                      int rank, double e_core, int n, int n_elec, int two_s, const dmrg_opts* opts,
                      const int* occ, const int* two_s_right) {
  if (!out) return fail(nullptr, DMRG_EINVAL, "out is NULL");
  *out = nullptr;
  if (!h) return fail(nullptr, DMRG_EINVAL, "h is NULL");
  if (n < 2 || n > 256) return fail(nullptr, DMRG_EINVAL, "n must be in [2, 256]");
  if (!eri && !(chol && rank > 0)) return fail(nullptr, DMRG_EINVAL, "need eri or chol with rank > 0");
  if (n_elec < 0 || n_elec > 2 * n) return fail(nullptr, DMRG_EINVAL, "n_elec out of range");
  if (two_s < 0 || ((n_elec - two_s) & 1)) return fail(nullptr, DMRG_EINVAL, "two_s has the wrong parity");
  if ((occ == nullptr) != (two_s_right == nullptr))
    return fail(nullptr, DMRG_EINVAL, "occ and two_s_right must be given together");
  dmrg_opts o;
  dmrg_default_opts(&o);
  if (opts) o = *opts;
  if (o.D < 1 || o.max_space < 4 || o.davidson_tol <= 0 || o.max_davidson_iter < 1)
    return fail(nullptr, DMRG_EINVAL, "bad options");
  if (!(o.wait_timeout_s >= 0.0) || o.wait_timeout_s > 3600.0)
    return fail(nullptr, DMRG_EINVAL, "wait_timeout_s must be in [0, 3600]");
  if (o.tc_drain_terms < 0) return fail(nullptr, DMRG_EINVAL, "tc_drain_terms < 0");
  if (!(o.trunc_target >= 0.0) || o.trunc_target >= 1.0 || o.D_min < 1 || o.D_min > o.D)
    return fail(nullptr, DMRG_EINVAL, "trunc_target must be in [0, 1) and 1 <= D_min <= D");
  if (!sweep_precision_ok(o.precision)) return fail(nullptr, DMRG_EINVAL, "unsupported precision");
  auto ctx = std::make_unique<dmrg_ctx>();
  ctx->n = n;
  try {
    std::vector<int> oc, path;
    if (occ) {
      oc.assign(occ, occ + n);
      path.assign(two_s_right, two_s_right + n + 1);
      int ne = 0;
      for (int v : oc) {
        if (v < 0 || v > 2) return fail(nullptr, DMRG_EINVAL, "occupations must be 0, 1 or 2");
        ne += v;
      }
      if (ne != n_elec) return fail(nullptr, DMRG_EINVAL, "occupations do not sum to n_elec");
    } else if (!default_state(n, n_elec, two_s, oc, path)) {
      return fail(nullptr, DMRG_EINVAL, "two_s too large for this filling");
    }
    std::string err;
    ctx->be.reset(dmrg::make_cuda_backend(o.device, &err));
    if (!ctx->be) return fail(nullptr, DMRG_ECUDA, err.empty() ? "cuda: no device" : err);
    ctx->be->set_budget(o.hbm_budget_bytes);
    ctx->be->set_wait_ns((unsigned long long)(o.wait_timeout_s * 1e9));
    std::vector<double> e4;
    const double* g = eri;
    if (!g) {
      // (pq|rs) = sum_k L^k_pq L^k_rs: one (n^2 x rank)(rank x n^2) float64
      // GEMM on the device; the result enters the host task coefficients
      const size_t nn = (size_t)n * n;
      e4.assign(nn * nn, 0.0);
      double* dL = (double*)ctx->be->alloc((size_t)rank * nn * sizeof(double));
      double* dE = (double*)ctx->be->alloc(nn * nn * sizeof(double));
      ctx->be->copy_h2d(dL, chol, (size_t)rank * nn * sizeof(double));
      ctx->be->memset0(dE, nn * nn * sizeof(double));
      std::vector<dmrg::GemmGroup> gg{{dE, (int)nn, (int)nn, (int)nn, 0, 1}};
      std::vector<dmrg::GemmSeg> gs{{dL, dL, rank, (int)nn, (int)nn, 1, 0, 1.0}};
      ctx->be->gemm(gg, gs, dmrg::Precision::FP64);
      ctx->be->copy_d2h(e4.data(), dE, nn * nn * sizeof(double));
      ctx->be->sync();
      ctx->be->free(dL);
      ctx->be->free(dE);
      g = e4.data();
    }
    dmrg::Options eo;
    eo.D = o.D;
    eo.max_davidson_iter = o.max_davidson_iter;
    eo.davidson_tol = o.davidson_tol;
    map_precision(o.precision, &eo.prec, &eo.prec_renorm);
    eo.max_space = o.max_space;
    eo.verbose = o.verbose;
    eo.seed = o.seed;
    eo.debug_bounds = o.debug_bounds != 0;
    eo.trunc_target = o.trunc_target;
    eo.D_min = o.D_min;
    eo.rq64_every_bond = o.rq64_every_bond != 0;
    eo.tc_drain_terms = o.tc_drain_terms;
    eo.tc_autotune = o.tc_autotune != 0;
    ctx->strict = o.strict_convergence != 0;
    ctx->eng = std::make_unique<dmrg::Engine>(ctx->be.get(), n, h, g, e_core, n_elec, two_s, eo,
                                              oc.data(), path.data());
  } catch (const std::exception& e) {
    return translate(nullptr, e);
  }
  *out = ctx.release();
  return DMRG_OK;
}

dmrg_status dmrg_sweep(dmrg_ctx* c, int n_sweeps, double* energy, double* max_trunc) {
  if (!c || !c->eng) return fail(c, DMRG_EINVAL, "invalid context");
  if (n_sweeps < 0) return fail(c, DMRG_EINVAL, "n_sweeps < 0");
  try {
    int noconv = 0;
    for (int s = 0; s < n_sweeps; ++s) {
      c->last = c->eng->sweep();
      c->sweep_seconds = c->eng->sweep_seconds;
      ++c->sweeps_done;
      noconv += c->last.noconv_bonds;
    }
    if (energy) *energy = c->last.energy;
    if (max_trunc) *max_trunc = c->last.max_trunc;
    if (c->strict && noconv > 0)
      return fail(c, DMRG_ENOCONV, "davidson: " + std::to_string(noconv) +
                                       " bond solve(s) stopped at max_davidson_iter above davidson_tol");
  } catch (const std::exception& e) {
    return translate(c, e);
  }
  return DMRG_OK;
}

dmrg_status dmrg_sweep_part(dmrg_ctx* c, int direction, int last_bond, double* energy, double* max_trunc) {
  if (!c || !c->eng) return fail(c, DMRG_EINVAL, "invalid context");
  if (direction != 0 && direction != 1) return fail(c, DMRG_EINVAL, "direction must be 0 (L->R) or 1 (R->L)");
  try {
    c->last = c->eng->sweep_part(direction == 0, last_bond);
    c->sweep_seconds = c->eng->sweep_seconds;
    if (energy) *energy = c->last.energy;
    if (max_trunc) *max_trunc = c->last.max_trunc;
    if (c->strict && c->last.noconv_bonds > 0)
      return fail(c, DMRG_ENOCONV, "davidson: " + std::to_string(c->last.noconv_bonds) +
                                       " bond solve(s) stopped at max_davidson_iter above davidson_tol");
  } catch (const std::exception& e) {
    return translate(c, e);
  }
  return DMRG_OK;
}

dmrg_status dmrg_bond_check64(dmrg_ctx* c, double* energy_rq64, double* residual64, double* ms,
                              double* flops) {
  if (!c || !c->eng) return fail(c, DMRG_EINVAL, "invalid context");
  try {
    c->eng->check_bond64(energy_rq64, residual64, ms, flops);
  } catch (const std::exception& e) {
    return translate(c, e);
  }
  return DMRG_OK;
}

dmrg_status dmrg_bond_apply(dmrg_ctx* c, int precision, const double* x, double* y, int64_t* len) {
  if (!c || !c->eng || !len) return fail(c, DMRG_EINVAL, "invalid argument");
  if (!sweep_precision_ok(precision) || precision == DMRG_SPLIT_TF32)
    return fail(c, DMRG_EINVAL,
                "precision must be DMRG_FP64, DMRG_SPLIT_HPSI, DMRG_SPLIT_HPSI_TC or DMRG_SPLIT_ALL_TC");
  try {
    dmrg::Precision ph, pr;
    map_precision(precision, &ph, &pr);
    const size_t n = c->eng->apply_bond(ph, nullptr, nullptr);
    if (x && y && *len != (int64_t)n) {
      *len = (int64_t)n;
      return fail(c, DMRG_EINVAL, "vector length differs from the two-site dimension of the bond");
    }
    *len = (int64_t)n;
    if (x && y) c->eng->apply_bond(ph, x, y);
  } catch (const std::exception& e) {
    return translate(c, e);
  }
  return DMRG_OK;
}

dmrg_status dmrg_bond_solve(dmrg_ctx* c, int bond, int direction, int precision, int max_iter, double tol,
                            int min_calls, int check64, dmrg_bond_result* out, double* call_ms, int cap) {
  if (!c || !c->eng || !out) return fail(c, DMRG_EINVAL, "invalid argument");
  if (direction != 0 && direction != 1) return fail(c, DMRG_EINVAL, "direction must be 0 (L->R) or 1 (R->L)");
  if (!sweep_precision_ok(precision) || precision == DMRG_SPLIT_TF32)
    return fail(c, DMRG_EINVAL,
                "precision must be DMRG_FP64, DMRG_SPLIT_HPSI, DMRG_SPLIT_HPSI_TC or DMRG_SPLIT_ALL_TC");
  if (max_iter < 1 || !(tol > 0) || min_calls < 0 || cap < 0 || (cap > 0 && !call_ms))
    return fail(c, DMRG_EINVAL, "invalid argument");
  try {
    dmrg::Precision ph, pr;
    map_precision(precision, &ph, &pr);
    dmrg::Engine::BondSolve r = c->eng->solve_bond(bond, direction == 0, ph, max_iter, tol, min_calls,
                                                   check64 != 0);
    out->energy = r.energy;
    out->energy_rq64 = r.energy_rq64;
    out->residual64 = r.residual64;
    out->gap = r.gap;
    out->iterations = r.iterations;
    out->calls = r.calls;
    out->flops_per_call = r.flops_per_call;
    out->dim = (int64_t)r.dim;
    out->contraction_ms = r.contraction_ms;
    out->split_ms = r.split_ms;
    out->contraction_launches = r.contraction_launches;
    double tot = 0.0;
    for (double x : r.call_ms) tot += x;
    out->ms_total = tot;
    for (int i = 0; i < std::min(cap, (int)r.call_ms.size()); ++i) call_ms[i] = r.call_ms[i];
  } catch (const std::exception& e) {
    return translate(c, e);
  }
  return DMRG_OK;
}

dmrg_status dmrg_set_davidson(dmrg_ctx* c, int max_iter, double tol) {
  if (!c || !c->eng) return fail(c, DMRG_EINVAL, "invalid context");
  if (max_iter < 1 || !(tol > 0)) return fail(c, DMRG_EINVAL, "max_iter < 1 or tol <= 0");
  c->eng->set_davidson(max_iter, tol);
  return DMRG_OK;
}

dmrg_status dmrg_set_wait_timeout(dmrg_ctx* c, double seconds) {
  if (!c || !c->be) return fail(c, DMRG_EINVAL, "invalid context");
  if (!(seconds >= 0.0) || seconds > 3600.0) return fail(c, DMRG_EINVAL, "seconds must be in [0, 3600]");
  c->be->set_wait_ns((unsigned long long)(seconds * 1e9));
  return DMRG_OK;
}

dmrg_status dmrg_set_kernel_tc_drain_terms(int terms) {
  if (terms < 0) return fail(nullptr, DMRG_EINVAL, "terms < 0");
  g_kernel_drain_terms.store(terms);
  return DMRG_OK;
}

dmrg_status dmrg_tc_shape_candidates(int* shapes, int cap, int* count) {
  const auto c = dmrg::tc_shape_candidates();
  if (!count || (cap > 0 && !shapes)) return fail(nullptr, DMRG_EINVAL, "NULL argument");
  *count = (int)c.size();
  for (int k = 0; k < std::min(cap, (int)c.size()); ++k) {
    shapes[4 * k] = c[k].tile_n;
    shapes[4 * k + 1] = c[k].chunks_per_cta;
    shapes[4 * k + 2] = c[k].order;
    shapes[4 * k + 3] = c[k].cluster;
  }
  return DMRG_OK;
}

dmrg_status dmrg_set_kernel_tc_shape(int candidate) {
  if (candidate < 0 || candidate >= (int)dmrg::tc_shape_candidates().size())
    return fail(nullptr, DMRG_EINVAL, "schedule candidate out of range");
  g_kernel_tc_cand.store(candidate);
  return DMRG_OK;
}

dmrg_status dmrg_set_tc_autotune(dmrg_ctx* c, int on) {
  if (!c || !c->eng) return fail(c, DMRG_EINVAL, "invalid context");
  c->eng->set_tc_autotune(on != 0);
  return DMRG_OK;
}

dmrg_status dmrg_tc_schedule_info(const dmrg_ctx* c, int* shape, double* ms, int cap, int* count) {
  if (!c || !c->eng) return fail(nullptr, DMRG_EINVAL, "invalid context");
  if (!shape || !count || (cap > 0 && !ms)) return fail(nullptr, DMRG_EINVAL, "NULL argument");
  std::vector<double> t;
  if (!c->eng->tc_schedule_info(shape, &t)) return fail(nullptr, DMRG_ESTATE, "no tcgen05 product planned yet");
  *count = (int)t.size();
  for (int k = 0; k < std::min(cap, (int)t.size()); ++k) ms[k] = t[k];
  return DMRG_OK;
}

dmrg_status dmrg_set_kernel_wait_timeout(double seconds) {
  if (!(seconds >= 0.0) || seconds > 3600.0) return fail(nullptr, DMRG_EINVAL, "seconds must be in [0, 3600]");
  g_kernel_wait_ns.store((unsigned long long)(seconds * 1e9));
  return DMRG_OK;
}

dmrg_status dmrg_memory_detail(const dmrg_ctx* c, int64_t* out) {
  if (!c || !c->eng || !out) return fail(const_cast<dmrg_ctx*>(c), DMRG_EINVAL, "invalid argument");
  size_t d = 0, h = 0, mb = 0, mx = 0, mu = 0;
  c->eng->memory_detail(&d, &h, &mb, &mx, &mu);
  out[0] = (int64_t)d;
  out[1] = (int64_t)h;
  out[2] = (int64_t)c->be->staged_out_bytes;
  out[3] = (int64_t)c->be->staged_in_bytes;
  out[4] = (int64_t)mx;
  out[5] = (int64_t)mb;
  out[6] = (int64_t)mu;
  return DMRG_OK;
}

dmrg_status dmrg_set_bond_dim(dmrg_ctx* c, int D) {
  if (!c || !c->eng) return fail(c, DMRG_EINVAL, "invalid context");
  if (D < 1) return fail(c, DMRG_EINVAL, "D < 1");
  c->eng->set_D(D);
  return DMRG_OK;
}

dmrg_status dmrg_set_precision(dmrg_ctx* c, int precision) {
  if (!c || !c->eng) return fail(c, DMRG_EINVAL, "invalid context");
  if (!sweep_precision_ok(precision)) return fail(c, DMRG_EINVAL, "unsupported precision");
  dmrg::Precision ph, pr;
  map_precision(precision, &ph, &pr);
  c->eng->set_precision(ph, pr);
  return DMRG_OK;
}

dmrg_status dmrg_rdm12(dmrg_ctx* c, double* gamma, double* Gamma) {
  if (!c || !c->eng || !gamma || !Gamma) return fail(c, DMRG_EINVAL, "invalid argument");
  if (c->sweeps_done == 0) return fail(c, DMRG_ESTATE, "no sweep has run");
  try {
    c->eng->rdm12(gamma, Gamma);
  } catch (const std::exception& e) {
    return translate(c, e);
  }
  return DMRG_OK;
}

dmrg_status dmrg_orbital_rdms(dmrg_ctx* c, double* rho1, double* rho2) {
  if (!c || !c->eng || !rho1 || !rho2) return fail(c, DMRG_EINVAL, "invalid argument");
  if (c->sweeps_done == 0) return fail(c, DMRG_ESTATE, "no sweep has run");
  try {
    c->eng->orbital_rdms(rho1, rho2);
  } catch (const std::exception& e) {
    return translate(c, e);
  }
  return DMRG_OK;
}

dmrg_status dmrg_orbital_entanglement(dmrg_ctx* c, double* s1, double* mutual) {
  if (!c || !c->eng || !s1 || !mutual) return fail(c, DMRG_EINVAL, "invalid argument");
  if (c->sweeps_done == 0) return fail(c, DMRG_ESTATE, "no sweep has run");
  try {
    c->eng->orbital_entanglement(s1, mutual);
  } catch (const std::exception& e) {
    return translate(c, e);
  }
  return DMRG_OK;
}

dmrg_status dmrg_orbital_rdms_from_invariants(int n, const double* inv1, const double* inv2, double* rho1,
                                              double* rho2) {
  if (n < 1 || n > 256 || !inv1 || !inv2 || !rho1 || !rho2) return fail(nullptr, DMRG_EINVAL, "invalid argument");
  try {
    dmrg::orbital_rdms_from_invariants(n, inv1, inv2, rho1, rho2);
  } catch (const std::exception& e) {
    return translate(nullptr, e);
  }
  return DMRG_OK;
}

dmrg_status dmrg_energy(const dmrg_ctx* c, double* energy) {
  if (!c || !c->eng || !energy) return fail(const_cast<dmrg_ctx*>(c), DMRG_EINVAL, "invalid argument");
  if (c->sweeps_done == 0) return fail(const_cast<dmrg_ctx*>(c), DMRG_ESTATE, "no sweep has run");
  *energy = c->eng->energy();
  return DMRG_OK;
}

dmrg_status dmrg_last_sweep_stats(const dmrg_ctx* c, double* flops, double* secs, int* calls,
                                  int* iters, double* sweep_s) {
  if (!c || !c->eng) return fail(const_cast<dmrg_ctx*>(c), DMRG_EINVAL, "invalid context");
  if (c->sweeps_done == 0) return fail(const_cast<dmrg_ctx*>(c), DMRG_ESTATE, "no sweep has run");
  if (flops) *flops = c->last.hpsi_flops;
  if (secs) *secs = c->last.hpsi_seconds;
  if (calls) *calls = c->last.hpsi_calls;
  if (iters) *iters = c->last.davidson_iters;
  if (sweep_s) *sweep_s = c->sweep_seconds;
  return DMRG_OK;
}

dmrg_status dmrg_bond_energies(const dmrg_ctx* c, double* out, int cap, int* count) {
  if (!c || !c->eng) return fail(const_cast<dmrg_ctx*>(c), DMRG_EINVAL, "invalid context");
  const auto& v = c->eng->bond_energies();
  if (count) *count = (int)v.size();
  if (out)
    for (int i = 0; i < (int)v.size() && i < cap; ++i) out[i] = v[i];
  return DMRG_OK;
}

dmrg_status dmrg_block_dims(const dmrg_ctx* c, int* left, int* right) {
  if (!c || !c->eng) return fail(const_cast<dmrg_ctx*>(c), DMRG_EINVAL, "invalid context");
  for (int m = 0; m <= c->n; ++m) {
    if (left) left[m] = c->eng->left_dim(m);
    if (right) right[m] = c->eng->right_dim(m);
  }
  return DMRG_OK;
}

dmrg_status dmrg_block_dims_u1(const dmrg_ctx* c, int* left, int* right) {
  if (!c || !c->eng) return fail(const_cast<dmrg_ctx*>(c), DMRG_EINVAL, "invalid context");
  for (int m = 0; m <= c->n; ++m) {
    if (left) left[m] = c->eng->left_dim_u1(m);
    if (right) right[m] = c->eng->right_dim_u1(m);
  }
  return DMRG_OK;
}

dmrg_status dmrg_profile(dmrg_ctx* c, int on) {
  if (!c || !c->be) return fail(c, DMRG_EINVAL, "invalid context");
  try {
    c->be->set_profile(on != 0);
  } catch (const std::exception& e) {
    return translate(c, e);
  }
  return DMRG_OK;
}

dmrg_status dmrg_kernel_stats(dmrg_ctx* c, int which, double* ms, double* flops, int64_t* launches) {
  if (!c || !c->be) return fail(c, DMRG_EINVAL, "invalid context");
  if (which < 0 || which > 5) return fail(c, DMRG_EINVAL, "which must be 0..5");
  try {
    long l = 0;
    c->be->kernel_stats(which, ms, flops, &l);
    if (launches) *launches = l;
  } catch (const std::exception& e) {
    return translate(c, e);
  }
  return DMRG_OK;
}

dmrg_status dmrg_last_sweep_phases(const dmrg_ctx* c, double* t) {
  if (!c || !c->eng || !t) return fail(const_cast<dmrg_ctx*>(c), DMRG_EINVAL, "invalid argument");
  if (c->sweeps_done == 0) return fail(const_cast<dmrg_ctx*>(c), DMRG_ESTATE, "no sweep has run");
  const auto& s = c->last;
  t[0] = s.t_enlarge;
  t[1] = s.t_plan;
  t[2] = s.t_davidson;
  t[3] = s.t_decimate;
  t[4] = s.t_renorm;
  t[5] = s.t_guess;
  t[6] = s.t_enl_terms;
  t[7] = s.t_enl_place_host;
  t[8] = s.t_enl_comp;
  t[9] = s.t_enl_place_run;
  t[10] = s.t_enl_alloc;
  t[11] = s.t_plan_items;
  t[12] = s.t_plan_tasks;
  t[13] = s.t_plan_upload;
  t[14] = s.t_plan_diag;
  return DMRG_OK;
}

dmrg_status dmrg_last_sweep_device_ms(const dmrg_ctx* c, double* ms) {
  if (!c || !c->eng || !ms) return fail(const_cast<dmrg_ctx*>(c), DMRG_EINVAL, "invalid argument");
  if (c->sweeps_done == 0) return fail(const_cast<dmrg_ctx*>(c), DMRG_ESTATE, "no sweep has run");
  *ms = c->eng->sweep_device_ms;
  return DMRG_OK;
}

dmrg_status dmrg_memory(const dmrg_ctx* c, int64_t* in_use, int64_t* peak) {
  if (!c || !c->be) return fail(const_cast<dmrg_ctx*>(c), DMRG_EINVAL, "invalid context");
  if (in_use) *in_use = (int64_t)c->be->bytes_in_use();
  if (peak) *peak = (int64_t)c->be->peak_bytes;
  return DMRG_OK;
}

dmrg_status dmrg_launch_count(const dmrg_ctx* c, int64_t* n) {
  if (!c || !c->be || !n) return fail(const_cast<dmrg_ctx*>(c), DMRG_EINVAL, "invalid argument");
  *n = c->be->launches;
  return DMRG_OK;
}

void dmrg_free(dmrg_ctx* c) {
  if (!c) return;
  c->eng.reset();
  c->be.reset();
  delete c;
}

const char* dmrg_last_error(const dmrg_ctx* c) {
  if (c) return c->err.c_str();
  return tl_err.c_str();
}

// ---------------------------------------------------------------- kernel level
dmrg_status dmrg_grouped_gemm(const double* A, int64_t a_len, const double* B, int64_t b_len,
                              double* C, int64_t c_len, const dmrg_gemm_group* groups,
                              int n_groups, const dmrg_gemm_seg* segs, int n_segs, int precision,
                              int device) {
  if (!A || !B || !C || (!groups && n_groups) || (!segs && n_segs) || n_groups < 0 || n_segs < 0)
    return fail(nullptr, DMRG_EINVAL, "invalid argument");
  if (precision < 0 || precision > 1) return fail(nullptr, DMRG_EINVAL, "unsupported precision");
  // validate every access range on the host before any launch
  for (int g = 0; g < n_groups; ++g) {
    const auto& G = groups[g];
    if (G.m < 0 || G.n < 0 || G.ldc < G.n || G.seg_begin < 0 || G.seg_count < 0 ||
        G.seg_begin + G.seg_count > n_segs || G.c_off < 0)
      return fail(nullptr, DMRG_EINVAL, "bad group");
    if (G.m > 0 && G.n > 0 && G.c_off + (int64_t)(G.m - 1) * G.ldc + G.n > c_len)
      return fail(nullptr, DMRG_EINVAL, "C block out of range");
    for (int s = G.seg_begin; s < G.seg_begin + G.seg_count; ++s) {
      const auto& S = segs[s];
      if (S.k < 0) return fail(nullptr, DMRG_EINVAL, "bad k");
      int64_t ar = S.trans_a ? S.k : G.m, ac = S.trans_a ? G.m : S.k;
      int64_t br = S.trans_b ? G.n : S.k, bc = S.trans_b ? S.k : G.n;
      if (ar > 0 && ac > 0 && (S.lda < ac || S.a_off < 0 || S.a_off + (ar - 1) * S.lda + ac > a_len))
        return fail(nullptr, DMRG_EINVAL, "A block out of range");
      if (br > 0 && bc > 0 && (S.ldb < bc || S.b_off < 0 || S.b_off + (br - 1) * S.ldb + bc > b_len))
        return fail(nullptr, DMRG_EINVAL, "B block out of range");
    }
  }
  std::string err;
  std::unique_ptr<dmrg::Backend> be(dmrg::make_cuda_backend(device, &err));
  if (be) be->set_wait_ns(g_kernel_wait_ns.load());
  if (!be) return fail(nullptr, DMRG_ECUDA, err);
  try {
    double* dA = (double*)be->alloc(std::max<int64_t>(a_len, 1) * sizeof(double));
    double* dB = (double*)be->alloc(std::max<int64_t>(b_len, 1) * sizeof(double));
    double* dC = (double*)be->alloc(std::max<int64_t>(c_len, 1) * sizeof(double));
    be->copy_h2d(dA, A, a_len * sizeof(double));
    be->copy_h2d(dB, B, b_len * sizeof(double));
    be->copy_h2d(dC, C, c_len * sizeof(double));
    std::vector<dmrg::GemmGroup> gg(n_groups);
    std::vector<dmrg::GemmSeg> ss(n_segs);
    for (int g = 0; g < n_groups; ++g)
      gg[g] = {dC + groups[g].c_off, groups[g].m, groups[g].n, groups[g].ldc, groups[g].seg_begin,
               groups[g].seg_count};
    for (int s = 0; s < n_segs; ++s)
      ss[s] = {dA + segs[s].a_off, dB + segs[s].b_off, segs[s].k, segs[s].lda, segs[s].ldb,
               segs[s].trans_a, segs[s].trans_b, segs[s].alpha};
    be->gemm(gg, ss, (dmrg::Precision)precision);
    be->copy_d2h(C, dC, c_len * sizeof(double));
    be->free(dA);
    be->free(dB);
    be->free(dC);
    be->sync();
  } catch (const std::exception& e) {
    return translate(nullptr, e);
  }
  return DMRG_OK;
}

namespace {
// host-side validation of an H_eff psi item list against buffer lengths
const char* check_hpsi(int64_t a_len, int64_t p_len, int64_t b_len, int64_t c_len,
                       const dmrg_hpsi_block* blocks, int nb, const dmrg_hpsi_item* items, int ni) {
  auto span_ok = [](int64_t off, int64_t rows, int64_t cols, int64_t ld, int64_t len) {
    if (rows <= 0 || cols <= 0) return true;
    return off >= 0 && ld >= cols && off + (rows - 1) * ld + cols <= len;
  };
  for (int b = 0; b < nb; ++b) {
    const auto& B = blocks[b];
    if (B.m < 0 || B.n < 0 || B.item_begin < 0 || B.item_count < 0 || B.item_begin + B.item_count > ni)
      return "bad block";
    if (!span_ok(B.c_off, B.m, B.n, B.ldc, c_len)) return "C block out of range";
    for (int i = B.item_begin; i < B.item_begin + B.item_count; ++i) {
      const auto& I = items[i];
      if (I.ka < 0 || I.kb < 0) return "bad item sizes";
      if (I.a_identity && I.ka != B.m) return "identity A needs ka == m";
      if (I.b_identity && I.kb != B.n) return "identity B needs kb == n";
      if (!I.a_identity) {
        int64_t r = I.trans_a ? I.ka : B.m, c = I.trans_a ? B.m : I.ka;
        if (!span_ok(I.a_off, r, c, I.lda, a_len)) return "A block out of range";
      }
      if (!span_ok(I.p_off, I.ka, I.kb, I.ldp, p_len)) return "P block out of range";
      if (!I.b_identity) {
        int64_t r = I.trans_b ? I.kb : B.n, c = I.trans_b ? B.n : I.kb;
        if (!span_ok(I.b_off, r, c, I.ldb, b_len)) return "B block out of range";
      }
    }
  }
  return nullptr;
}

void to_device_lists(const dmrg_hpsi_block* blocks, int nb, const dmrg_hpsi_item* items, int ni,
                     const double* dA, const double* dP, const double* dB, double* dC,
                     std::vector<dmrg::HpsiBlock>& hb, std::vector<dmrg::HpsiItem>& hi, double* flops) {
  hb.resize(nb);
  hi.resize(ni);
  double fl = 0.0;
  for (int b = 0; b < nb; ++b) {
    hb[b] = {dC + blocks[b].c_off, blocks[b].m, blocks[b].n, blocks[b].ldc, blocks[b].item_begin,
             blocks[b].item_count};
    for (int i = blocks[b].item_begin; i < blocks[b].item_begin + blocks[b].item_count; ++i) {
      const auto& I = items[i];
      hi[i] = {I.a_identity ? nullptr : dA + I.a_off, dP + I.p_off, I.b_identity ? nullptr : dB + I.b_off,
               I.lda, I.ldp, I.ldb, I.trans_a, I.trans_b, I.ka, I.kb, I.alpha};
      if (!I.a_identity) fl += 2.0 * blocks[b].m * I.ka * I.kb;
      if (!I.b_identity) fl += 2.0 * blocks[b].m * blocks[b].n * I.kb;
    }
  }
  if (flops) *flops = fl;
}
}  // namespace

dmrg_status dmrg_hpsi_contract(const double* A, int64_t a_len, const double* P, int64_t p_len,
                               const double* B, int64_t b_len, double* C, int64_t c_len,
                               const dmrg_hpsi_block* blocks, int n_blocks, const dmrg_hpsi_item* items,
                               int n_items, int precision, int device) {
  if (!A || !P || !B || !C || (!blocks && n_blocks) || (!items && n_items) || n_blocks < 0 || n_items < 0)
    return fail(nullptr, DMRG_EINVAL, "invalid argument");
  if (precision != DMRG_FP64 && precision != DMRG_SPLIT_TF32 && precision != DMRG_SPLIT_HPSI_TC)
    return fail(nullptr, DMRG_EINVAL, "unsupported precision");
  if (const char* m = check_hpsi(a_len, p_len, b_len, c_len, blocks, n_blocks, items, n_items))
    return fail(nullptr, DMRG_EINVAL, m);
  std::string err;
  std::unique_ptr<dmrg::Backend> be(dmrg::make_cuda_backend(device, &err));
  if (be) be->set_wait_ns(g_kernel_wait_ns.load());
  if (!be) return fail(nullptr, DMRG_ECUDA, err);
  try {
    auto up = [&](const double* h, int64_t n) {
      double* d = (double*)be->alloc(std::max<int64_t>(n, 1) * sizeof(double));
      be->copy_h2d(d, h, n * sizeof(double));
      return d;
    };
    double* dA = up(A, a_len);
    double* dP = up(P, p_len);
    double* dB = up(B, b_len);
    double* dC = up(C, c_len);
    std::vector<dmrg::HpsiBlock> hb;
    std::vector<dmrg::HpsiItem> hi;
    double fl = 0.0;
    to_device_lists(blocks, n_blocks, items, n_items, dA, dP, dB, dC, hb, hi, &fl);
    be->sync();
    be->set_profile(true);
    const dmrg::Precision pr = precision == DMRG_FP64           ? dmrg::Precision::FP64
                               : precision == DMRG_SPLIT_HPSI_TC ? dmrg::Precision::TC_TF32X3
                                                                 : dmrg::Precision::SPLIT_TF32;
    std::vector<dmrg::HpsiTask> tasks;
    std::vector<dmrg::HpsiReduce> reds;
    const bool tc = pr == dmrg::Precision::TC_TF32X3;
    dmrg::TcPlan tp;
    void* pool = nullptr;
    size_t scr;
    if (tc) {
      const dmrg::TcShape shape = dmrg::tc_shape_candidates()[g_kernel_tc_cand.load()];
      const int tc_ctas = dmrg::hpsi_tc_max_ctas(shape.cluster);
      dmrg::hpsi_tc_prepare(hb, hi, [&](size_t bytes) { return pool = be->alloc(bytes); }, tp,
                            tc_ctas > 0 ? tc_ctas : be->sm_count() / shape.cluster * shape.cluster, shape);
      tasks = tp.tasks;
      reds = tp.reds;
      scr = tp.scratch;
    } else {
      scr = dmrg::hpsi_plan_tasks(hb, pr, tasks, reds);
    }
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    size_t ob = 0, oi = al(hb.size() * sizeof(dmrg::HpsiBlock));
    size_t oc = al(oi + hi.size() * sizeof(dmrg::HpsiItem));
    size_t ot = al(oc + tp.items.size() * sizeof(dmrg::TcItem));
    size_t orr = al(ot + tasks.size() * sizeof(dmrg::HpsiTask));
    size_t oj = al(orr + reds.size() * sizeof(dmrg::HpsiReduce));
    size_t oco = al(oj + (tp.op_jobs.size() + tp.psi_jobs.size()) * sizeof(dmrg::SplitJob));
    size_t oct = al(oco + tp.cta_off.size() * sizeof(int));
    size_t os = al(oct + tp.cta_task.size() * sizeof(dmrg::TcSlot));
    char* d = (char*)be->alloc(os + scr * sizeof(double) + 256);
    if (!hb.empty()) be->copy_h2d(d + ob, hb.data(), hb.size() * sizeof(dmrg::HpsiBlock));
    if (!hi.empty()) be->copy_h2d(d + oi, hi.data(), hi.size() * sizeof(dmrg::HpsiItem));
    if (!tp.items.empty()) be->copy_h2d(d + oc, tp.items.data(), tp.items.size() * sizeof(dmrg::TcItem));
    if (!tasks.empty()) be->copy_h2d(d + ot, tasks.data(), tasks.size() * sizeof(dmrg::HpsiTask));
    if (!reds.empty()) be->copy_h2d(d + orr, reds.data(), reds.size() * sizeof(dmrg::HpsiReduce));
    if (tc) {
      std::vector<dmrg::SplitJob> jobs = tp.op_jobs;
      jobs.insert(jobs.end(), tp.psi_jobs.begin(), tp.psi_jobs.end());
      if (!jobs.empty()) {
        be->copy_h2d(d + oj, jobs.data(), jobs.size() * sizeof(dmrg::SplitJob));
        be->split((const dmrg::SplitJob*)(d + oj), (int)jobs.size(), (float*)pool);
      }
      if (!tp.cta_off.empty()) be->copy_h2d(d + oco, tp.cta_off.data(), tp.cta_off.size() * sizeof(int));
      if (!tp.cta_task.empty()) be->copy_h2d(d + oct, tp.cta_task.data(), tp.cta_task.size() * sizeof(dmrg::TcSlot));
      dmrg::TcLaunch L;
      L.blocks = (const dmrg::HpsiBlock*)(d + ob);
      L.items = (const dmrg::TcItem*)(d + oc);
      L.tasks = (const dmrg::HpsiTask*)(d + ot);
      L.cta_off = (const int*)(d + oco);
      L.cta_task = (const dmrg::TcSlot*)(d + oct);
      L.ncta = (int)tp.cta_off.size() - 1;
      L.reds = (const dmrg::HpsiReduce*)(d + orr);
      L.nreds = (int)reds.size();
      L.scratch = (double*)(d + os);
      L.pool = pool;
      L.units = tp.units;
      L.drain_terms = g_kernel_drain_terms.load();
      L.tile_n = tp.shape.tile_n;
      L.cluster = tp.shape.cluster;
      be->hpsi_tc(L, fl);
    } else {
      be->hpsi((const dmrg::HpsiBlock*)(d + ob), (const dmrg::HpsiItem*)(d + oi),
               (const dmrg::HpsiTask*)(d + ot), (int)tasks.size(), (const dmrg::HpsiReduce*)(d + orr),
               (int)reds.size(), (double*)(d + os), pr, fl);
    }
    be->check_device_flag();
    double kms = 0.0;
    be->kernel_stats(1, &kms, nullptr, nullptr);
    tl_contract_ms = kms;
    be->copy_d2h(C, dC, c_len * sizeof(double));
    be->sync();
    for (void* q : {(void*)dA, (void*)dP, (void*)dB, (void*)dC, (void*)d}) be->free(q);
    if (pool) be->free(pool);
    be->sync();
  } catch (const std::exception& e) {
    return translate(nullptr, e);
  }
  return DMRG_OK;
}

dmrg_status dmrg_last_contract_ms(double* ms) {
  if (!ms) return fail(nullptr, DMRG_EINVAL, "invalid argument");
  *ms = tl_contract_ms;
  return DMRG_OK;
}

dmrg_status dmrg_hpsi_contract_noalloc(const double* dA, int64_t a_len, const double* dP, int64_t p_len,
                                       const double* dB, int64_t b_len, double* dC, int64_t c_len,
                                       const dmrg_hpsi_block* blocks, int n_blocks,
                                       const dmrg_hpsi_item* items, int n_items, int precision,
                                       int device, void* stream) {
  if (!dA || !dP || !dB || !dC || (!blocks && n_blocks) || (!items && n_items) || n_blocks < 0 ||
      n_items < 0)
    return fail(nullptr, DMRG_EINVAL, "invalid argument");
  if (precision != DMRG_FP64 && precision != DMRG_SPLIT_TF32)
    return fail(nullptr, DMRG_EINVAL, "unsupported precision (DMRG_FP64 or DMRG_SPLIT_TF32)");
  if (const char* m = check_hpsi(a_len, p_len, b_len, c_len, blocks, n_blocks, items, n_items))
    return fail(nullptr, DMRG_EINVAL, m);
  try {
    std::vector<dmrg::HpsiBlock> hb;
    std::vector<dmrg::HpsiItem> hi;
    to_device_lists(blocks, n_blocks, items, n_items, dA, dP, dB, dC, hb, hi, nullptr);
    const dmrg::Precision pr = precision == DMRG_FP64 ? dmrg::Precision::FP64 : dmrg::Precision::SPLIT_TF32;
    std::vector<dmrg::HpsiTask> tasks;
    std::vector<dmrg::HpsiReduce> reds;
    size_t scr = dmrg::hpsi_plan_tasks(hb, pr, tasks, reds);
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    size_t ob = 0, oi = al(hb.size() * sizeof(dmrg::HpsiBlock));
    size_t ot = al(oi + hi.size() * sizeof(dmrg::HpsiItem));
    size_t orr = al(ot + tasks.size() * sizeof(dmrg::HpsiTask));
    size_t os = al(orr + reds.size() * sizeof(dmrg::HpsiReduce));
    size_t need = os + scr * sizeof(double);
    if (need > dmrg::kNoAllocScratchBytes)
      return fail(nullptr, DMRG_EINVAL,
                  "request needs " + std::to_string(need) + " bytes of scratch; the allocation-free entry "
                  "holds " + std::to_string(dmrg::kNoAllocScratchBytes) + " (use dmrg_hpsi_contract)");
    void* base = nullptr;
    cudaError_t e = dmrg::noalloc_scratch(device, &base);
    if (e != cudaSuccess) return fail(nullptr, DMRG_ECUDA, std::string("cuda: ") + cudaGetErrorString(e));
    DeviceGuard guard(device, &e);
    if (e != cudaSuccess) return fail(nullptr, DMRG_ECUDA, std::string("cuda: ") + cudaGetErrorString(e));
    cudaStream_t st = (cudaStream_t)stream;
    char* d = (char*)base;
    auto put = [&](size_t off, const void* h, size_t bytes) {
      if (bytes && e == cudaSuccess) e = cudaMemcpyAsync(d + off, h, bytes, cudaMemcpyHostToDevice, st);
    };
    put(ob, hb.data(), hb.size() * sizeof(dmrg::HpsiBlock));
    put(oi, hi.data(), hi.size() * sizeof(dmrg::HpsiItem));
    put(ot, tasks.data(), tasks.size() * sizeof(dmrg::HpsiTask));
    put(orr, reds.data(), reds.size() * sizeof(dmrg::HpsiReduce));
    if (e == cudaSuccess)
      dmrg::hpsi_launch((const dmrg::HpsiBlock*)(d + ob), (const dmrg::HpsiItem*)(d + oi),
                        (const dmrg::HpsiTask*)(d + ot), (int)tasks.size(),
                        (const dmrg::HpsiReduce*)(d + orr), (int)reds.size(), (double*)(d + os), pr, nullptr,
                        st);
    if (e != cudaSuccess) return fail(nullptr, DMRG_ECUDA, std::string("cuda: ") + cudaGetErrorString(e));
    e = guard.restore();
    if (e != cudaSuccess) return fail(nullptr, DMRG_ECUDA, std::string("cuda: ") + cudaGetErrorString(e));
  } catch (const std::exception& ex) {
    return translate(nullptr, ex);
  }
  return DMRG_OK;
}

dmrg_status dmrg_eigh_batched(const double* mats, const int* n, int count, double* w, double* vecs,
                              int device) {
  if (!mats || !n || !w || !vecs || count < 0) return fail(nullptr, DMRG_EINVAL, "invalid argument");
  size_t tot = 0, wt = 0;
  for (int i = 0; i < count; ++i) {
    if (n[i] < 1 || n[i] > 4096) return fail(nullptr, DMRG_EINVAL, "matrix size out of range");
    tot += (size_t)n[i] * n[i];
    wt += n[i];
  }
  std::string err;
  std::unique_ptr<dmrg::Backend> be(dmrg::make_cuda_backend(device, &err));
  if (be) be->set_wait_ns(g_kernel_wait_ns.load());
  if (!be) return fail(nullptr, DMRG_ECUDA, err);
  try {
    double* dA = (double*)be->alloc(std::max<size_t>(tot, 1) * sizeof(double));
    double* dV = (double*)be->alloc(std::max<size_t>(tot, 1) * sizeof(double));
    double* dw = (double*)be->alloc(std::max<size_t>(wt, 1) * sizeof(double));
    be->copy_h2d(dA, mats, tot * sizeof(double));
    std::vector<dmrg::EighTask> t;
    size_t o = 0, ow = 0;
    for (int i = 0; i < count; ++i) {
      t.push_back({dA + o, dw + ow, dV + o, n[i]});
      o += (size_t)n[i] * n[i];
      ow += n[i];
    }
    be->eigh(t);
    be->check_device_flag();
    be->copy_d2h(w, dw, wt * sizeof(double));
    be->copy_d2h(vecs, dV, tot * sizeof(double));
    be->free(dA);
    be->free(dV);
    be->free(dw);
    be->sync();
  } catch (const std::exception& e) {
    return translate(nullptr, e);
  }
  return DMRG_OK;
}

dmrg_status dmrg_fiedler_order(const double* mutual, int n, int* order, int device) {
  if (!mutual || !order || n < 1 || n > 4096) return fail(nullptr, DMRG_EINVAL, "invalid argument");
  double scale = 0.0;
  for (size_t e = 0; e < (size_t)n * n; ++e) {
    if (!std::isfinite(mutual[e])) return fail(nullptr, DMRG_EINVAL, "mutual information not finite");
    scale = std::max(scale, std::abs(mutual[e]));
  }
  for (int p = 0; p < n; ++p)
    for (int q = 0; q < p; ++q)
      if (std::abs(mutual[(size_t)p * n + q] - mutual[(size_t)q * n + p]) > 1e-12 * std::max(scale, 1e-300))
        return fail(nullptr, DMRG_EINVAL, "mutual information not symmetric");
  if (n < 3) {
    for (int p = 0; p < n; ++p) order[p] = p;
    return DMRG_OK;
  }
  // graph Laplacian L = diag(I 1) - I (diagonal of I ignored)
  std::vector<double> L((size_t)n * n, 0.0);
  for (int p = 0; p < n; ++p)
    for (int q = 0; q < n; ++q)
      if (p != q) {
        L[(size_t)p * n + q] = -mutual[(size_t)p * n + q];
        L[(size_t)p * n + p] += mutual[(size_t)p * n + q];
      }
  std::vector<double> w(n), V((size_t)n * n);
  const int nn[1] = {n};
  const dmrg_status st = dmrg_eigh_batched(L.data(), nn, 1, w.data(), V.data(), device);
  if (st != DMRG_OK) return st;
  // eigenvalues descending: the Fiedler vector (second smallest) is row n-2;
  // orbitals sorted by it, oriented so that the first is the smaller end
  const double* f = &V[(size_t)(n - 2) * n];
  std::vector<int> o(n);
  std::iota(o.begin(), o.end(), 0);
  std::stable_sort(o.begin(), o.end(), [&](int a, int b) { return f[a] < f[b]; });
  if (o.front() > o.back()) {
    std::iota(o.begin(), o.end(), 0);
    std::stable_sort(o.begin(), o.end(), [&](int a, int b) { return f[a] > f[b]; });
  }
  std::copy(o.begin(), o.end(), order);
  return DMRG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- CAS-SCF
namespace {
thread_local double tl_casscf_ms = 0.0, tl_casscf_flops = 0.0;

template <class F>
dmrg_status with_casscf(int device, F&& f) {
  std::string err;
  std::unique_ptr<dmrg::Backend> be(dmrg::make_cuda_backend(device, &err));
  if (be) be->set_wait_ns(g_kernel_wait_ns.load());
  if (!be) return fail(nullptr, DMRG_ECUDA, err);
  tl_casscf_ms = tl_casscf_flops = 0.0;
  try {
    be->set_profile(true);
    dmrg::Casscf c(be.get());
    f(c);
    be->sync();
    be->kernel_stats(0, &tl_casscf_ms, &tl_casscf_flops, nullptr);
  } catch (const std::exception& e) {
    return translate(nullptr, e);
  }
  return DMRG_OK;
}
}  // namespace

extern "C" {

dmrg_status casscf_last_kernel_ms(double* ms, double* flops) {
  if (!ms) return fail(nullptr, DMRG_EINVAL, "invalid argument");
  *ms = tl_casscf_ms;
  if (flops) *flops = tl_casscf_flops;
  return DMRG_OK;
}

dmrg_status casscf_rotation(const double* K, int nb, double* R, int device) {
  if (!K || !R || nb < 1 || nb > 8192) return fail(nullptr, DMRG_EINVAL, "invalid argument");
  return with_casscf(device, [&](dmrg::Casscf& c) { c.rotation(K, nb, R); });
}

dmrg_status casscf_rotation_backward(const double* K, const double* G, int nb, double* dK, int device) {
  if (!K || !G || !dK || nb < 1 || nb > 4096) return fail(nullptr, DMRG_EINVAL, "invalid argument");
  return with_casscf(device, [&](dmrg::Casscf& c) { c.rotation_backward(K, G, nb, dK); });
}

dmrg_status casscf_transform(const double* R, const double* h, const double* chol, int rank, int nb,
                             double* h_out, double* chol_out, int device) {
  if (!R || !h || !chol || !h_out || !chol_out || rank < 1 || nb < 1)
    return fail(nullptr, DMRG_EINVAL, "invalid argument");
  return with_casscf(device, [&](dmrg::Casscf& c) { c.transform(R, h, chol, rank, nb, h_out, chol_out); });
}

dmrg_status casscf_active_space(const double* h, const double* chol, int rank, int nb, int ncore,
                                int ncas, double* e_core, double* h_act, double* eri_act, int device) {
  if (!h || !chol || !e_core || !h_act || !eri_act || rank < 1 || ncore < 0 || ncas < 1 ||
      ncore + ncas > nb)
    return fail(nullptr, DMRG_EINVAL, "invalid argument");
  return with_casscf(device, [&](dmrg::Casscf& c) {
    c.active_space(h, chol, rank, nb, ncore, ncas, e_core, h_act, eri_act);
  });
}

dmrg_status casscf_orbital_gradient(const double* h, const double* chol, int rank, int nb, int ncore,
                                    int ncas, const double* gamma, const double* Gamma, double* grad,
                                    double* fock, int device) {
  if (!h || !chol || !gamma || !Gamma || !grad || rank < 1 || ncore < 0 || ncas < 1 ||
      ncore + ncas > nb)
    return fail(nullptr, DMRG_EINVAL, "invalid argument");
  return with_casscf(device, [&](dmrg::Casscf& c) {
    c.gradient(h, chol, rank, nb, ncore, ncas, gamma, Gamma, grad, fock);
  });
}

dmrg_status casscf_transform_backward(const double* K, const double* R, const double* h_rot,
                                      const double* chol_rot, int rank, int nb, int ncore, int ncas,
                                      double g_core, const double* g_h, const double* g_eri, double* dK,
                                      int device) {
  if (!K || !R || !h_rot || !chol_rot || !g_h || !g_eri || !dK || rank < 1 || nb < 1 || nb > 4096 ||
      ncore < 0 || ncas < 1 || ncore + ncas > nb)
    return fail(nullptr, DMRG_EINVAL, "invalid argument");
  return with_casscf(device, [&](dmrg::Casscf& c) {
    c.transform_backward(K, R, h_rot, chol_rot, rank, nb, ncore, ncas, g_core, g_h, g_eri, dK);
  });
}

void casscf_default_scf_opts(casscf_scf_opts* o) {
  if (!o) return;
  o->max_iter = 60;
  o->e_tol = 1e-7;
  o->g_tol = 1e-3;
  o->memory = 8;
  o->max_step = 0.5;
  o->sweeps = 4;
}

dmrg_status casscf_dmrg_scf(const double* h, const double* chol, int rank, int nb, int ncore, int ncas,
                            int n_elec, int two_s, const dmrg_opts* dopts, const casscf_scf_opts* sopts,
                            double* U, double* energies, double* gmax, int* n_iter, int* converged) {
  if (!h || !chol || !U || !energies || !gmax || rank < 1 || nb < 2 || nb > 4096 || ncore < 0 || ncas < 2 ||
      ncore + ncas > nb || n_elec < 0 || n_elec > 2 * ncas || two_s < 0 || ((n_elec - two_s) & 1))
    return fail(nullptr, DMRG_EINVAL, "invalid argument");
  dmrg_opts o;
  dmrg_default_opts(&o);
  if (dopts) o = *dopts;
  casscf_scf_opts so;
  casscf_default_scf_opts(&so);
  if (sopts) so = *sopts;
  if (so.max_iter < 1 || so.sweeps < 1 || so.memory < 0 || !(so.max_step > 0) || !(so.e_tol > 0) || !(so.g_tol > 0))
    return fail(nullptr, DMRG_EINVAL, "bad SCF options");
  if (o.D < 1 || o.max_space < 4 || o.davidson_tol <= 0 || o.max_davidson_iter < 1 || !sweep_precision_ok(o.precision))
    return fail(nullptr, DMRG_EINVAL, "bad DMRG options");
  std::vector<int> occ, path;
  if (!default_state(ncas, n_elec, two_s, occ, path)) return fail(nullptr, DMRG_EINVAL, "two_s too large");
  std::string err;
  std::unique_ptr<dmrg::Backend> be(dmrg::make_cuda_backend(o.device, &err));
  if (!be) return fail(nullptr, DMRG_ECUDA, err);
  be->set_wait_ns((unsigned long long)(o.wait_timeout_s * 1e9));
  try {
    dmrg::Casscf cas(be.get());
    dmrg::ScfStepper stepper(be.get(), nb, ncore, ncas, so.memory, so.max_step);
    const size_t nn = (size_t)nb * nb, a2 = (size_t)ncas * ncas;
    std::vector<double> Ucur(nn, 0.0), h2(nn), L2(nn * rank), hact(a2), eact(a2 * a2), gam(a2), Gam(a2 * a2),
        g(nn), K(nn), R(nn), Un(nn);
    for (int p = 0; p < nb; ++p) Ucur[(size_t)p * nb + p] = 1.0;
    dmrg::Options eo;
    eo.D = o.D;
    eo.max_davidson_iter = o.max_davidson_iter;
    eo.davidson_tol = o.davidson_tol;
    map_precision(o.precision, &eo.prec, &eo.prec_renorm);
    eo.max_space = o.max_space;
    eo.seed = o.seed;
    eo.trunc_target = o.trunc_target;
    eo.D_min = o.D_min;
    int it = 0;
    bool conv = false;
    for (; it < so.max_iter; ++it) {
      cas.transform(Ucur.data(), h, chol, rank, nb, h2.data(), L2.data());
      double e_core = 0.0;
      cas.active_space(h2.data(), L2.data(), rank, nb, ncore, ncas, &e_core, hact.data(), eact.data());
      double E = 0.0;
      {
        dmrg::Engine eng(be.get(), ncas, hact.data(), eact.data(), e_core, n_elec, two_s, eo, occ.data(),
                         path.data());
        for (int sw = 0; sw < so.sweeps; ++sw) E = eng.sweep().energy;
        eng.rdm12(gam.data(), Gam.data());
      }
      cas.gradient(h2.data(), L2.data(), rank, nb, ncore, ncas, gam.data(), Gam.data(), g.data(), nullptr);
      const double gm = stepper.gradient_max(g.data());
      energies[it] = E;
      gmax[it] = gm;
      if (it > 0 && std::abs(E - energies[it - 1]) < so.e_tol && gm < so.g_tol) {
        conv = true;
        ++it;
        break;
      }
      stepper.step(cas, h2.data(), L2.data(), rank, gam.data(), Gam.data(), K.data());
      cas.rotation(K.data(), nb, R.data());
      cas.matmul(Ucur.data(), R.data(), nb, Un.data());
      Ucur.swap(Un);
    }
    std::copy(Ucur.begin(), Ucur.end(), U);
    if (n_iter) *n_iter = it;
    if (converged) *converged = conv ? 1 : 0;
  } catch (const std::exception& e) {
    return translate(nullptr, e);
  }
  return DMRG_OK;
}

}  // extern "C"
