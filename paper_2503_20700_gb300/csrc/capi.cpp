// extern "C" entry points (include/dmrgscf.h).
#include <cstring>
#include <exception>
#include <memory>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/dmrgscf.h"
#include "dmrg.hpp"

struct dmrg_ctx {
  std::unique_ptr<dmrg::Backend> be;
  std::unique_ptr<dmrg::Engine> eng;
  std::string err;
  int n = 0;
  int sweeps_done = 0;
  dmrg::SweepStats last;
  double sweep_seconds = 0.0;
};

namespace {
thread_local std::string tl_err;

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
  return fail(c, DMRG_EINTERNAL, m);
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
  if (o.precision < 0 || o.precision > 1) return fail(nullptr, DMRG_EINVAL, "unsupported precision");
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
    std::vector<double> e4;
    const double* g = eri;
    if (!g) {
      size_t nn = (size_t)n * n;
      e4.assign(nn * nn, 0.0);
      for (int k = 0; k < rank; ++k) {
        const double* L = chol + (size_t)k * nn;
        for (size_t a = 0; a < nn; ++a)
          for (size_t b = 0; b < nn; ++b) e4[a * nn + b] += L[a] * L[b];
      }
      g = e4.data();
    }
    std::string err;
    ctx->be.reset(dmrg::make_cuda_backend(o.device, &err));
    if (!ctx->be) return fail(nullptr, DMRG_ECUDA, err.empty() ? "cuda: no device" : err);
    dmrg::Options eo;
    eo.D = o.D;
    eo.max_davidson_iter = o.max_davidson_iter;
    eo.davidson_tol = o.davidson_tol;
    eo.prec = (dmrg::Precision)o.precision;
    eo.max_space = o.max_space;
    eo.verbose = o.verbose;
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
    for (int s = 0; s < n_sweeps; ++s) {
      c->last = c->eng->sweep();
      c->sweep_seconds = c->eng->sweep_seconds;
      ++c->sweeps_done;
    }
  } catch (const std::exception& e) {
    return translate(c, e);
  }
  if (energy) *energy = c->last.energy;
  if (max_trunc) *max_trunc = c->last.max_trunc;
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
  if (precision < 0 || precision > 1) return fail(c, DMRG_EINVAL, "unsupported precision");
  c->eng->set_precision((dmrg::Precision)precision);
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

}  // extern "C"
