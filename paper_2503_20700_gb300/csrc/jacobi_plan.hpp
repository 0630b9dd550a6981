// Host planning of the batched Jacobi eigensolver (the density-matrix
// sectors of a decimation): which matrices share a cooperative launch of one
// CTA per SM, and how many CTAs each matrix gets.
#pragma once
#include <algorithm>
#include <stdexcept>
#include <vector>

namespace dmrg {

constexpr int kJacSmemN = 112;  // largest matrix of the one-CTA shared-memory path

// Modelled time of an n x n matrix on g CTAs, in SM clocks (FP64 rate of 2
// operations a clock; a group barrier about 6000 clocks): the group sizes of
// a batch minimise the slowest matrix.
inline double jac_cost(int n, int g) {
  const double rounds = std::max(1, ((n + 1) & ~1) - 1);
  const double ops = 2.0 * (double)n * n;  // clocks of the FP64 work of a round on one SM
  return rounds * (g == 1 ? ops + 1000.0 : 1.15 * ops / g + 6000.0);
}

// g[k] of batch tasks (descending n) start at their minimum; spare CTAs go to
// the slowest matrix while that shortens it
inline void jac_assign_groups(const std::vector<int>& n, std::vector<int>& g, int spare) {
  while (spare > 0 && !n.empty()) {
    size_t k = 0;
    for (size_t i = 1; i < n.size(); ++i)
      if (jac_cost(n[i], g[i]) > jac_cost(n[k], g[k])) k = i;
    const int gmax = std::max(2, std::min(32, ((n[k] + 1) & ~1) / 2));
    int ng = g[k] + 1;
    while (ng <= gmax && ng - g[k] <= spare && jac_cost(n[k], ng) >= jac_cost(n[k], g[k])) ++ng;
    if (ng > gmax || ng - g[k] > spare) break;
    spare -= ng - g[k];
    g[k] = ng;
  }
}

// One cooperative launch: matrices [begin, end) of the size-sorted list and
// the CTA group size of each.
struct JacBatch {
  size_t begin = 0, end = 0;
  std::vector<int> g;
};

// Splits matrices sorted by decreasing n into launches of at most `cap`
// co-resident CTAs (a matrix above kJacSmemN needs a group of at least two)
// and sizes the groups of each launch.
inline std::vector<JacBatch> jac_plan_batches(const std::vector<int>& n_desc, int cap) {
  std::vector<JacBatch> out;
  size_t i0 = 0;
  while (i0 < n_desc.size()) {
    JacBatch b;
    b.begin = i0;
    std::vector<int> ns;
    int used = 0;
    size_t i1 = i0;
    while (i1 < n_desc.size()) {
      const int gmin = n_desc[i1] > kJacSmemN ? 2 : 1;
      if (used + gmin > cap) break;
      ns.push_back(n_desc[i1]);
      b.g.push_back(gmin);
      used += gmin;
      ++i1;
    }
    if (i1 == i0) throw std::runtime_error("eigensolver: fewer co-resident CTAs than one matrix needs");
    jac_assign_groups(ns, b.g, cap - used);
    b.end = i1;
    out.push_back(std::move(b));
    i0 = i1;
  }
  return out;
}

}  // namespace dmrg
