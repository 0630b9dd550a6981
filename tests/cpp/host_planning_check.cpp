// Checks of the host planning code on the CPU (no device calls):
//  - host_parallel_for runs every index exactly once, also when nested and
//    after an exception, and rethrows the first exception;
//  - hpsi_tc_prepare (tcgen05 H_eff psi planning) against properties any
//    correct plan has: each operand of each item refers to a split job with
//    exactly that operand's (src, trans, rows, cols, ld), identity factors to
//    one identity job per dimension; jobs are distinct and numbered in
//    first-occurrence order over (items in block order; roles A, P^T, B);
//    plane pairs are disjoint runs of 2 ceil(rows/8) ceil(cols/32) units
//    inside the pool; the chunks of every 128 x 256 tile cover its items
//    once, in order, each chunk with its own partial tile, one reduction per
//    tile names all of its chunks, and every task is in exactly one CTA list
//    of the persistent launch, whose clusters walk the same items in lockstep
//    with groups of CTAs on the same rows;
//  - jac_plan_batches (batched Jacobi eigensolver launches): every matrix in
//    exactly one launch, in order; at most `cap` CTAs per launch; group sizes
//    between the minimum (two above the shared-memory size) and the cap of
//    the cost model; extra CTAs never make the slowest matrix slower.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <map>
#include <random>
#include <set>
#include <stdexcept>
#include <tuple>
#include <vector>

#include "host_pool.hpp"
#include "hpsi_tc.cuh"
#include "jacobi_plan.hpp"

using namespace dmrg;

static int fails = 0;
#define CHECK(c)                                                   \
  do {                                                             \
    if (!(c)) {                                                    \
      std::printf("FAIL %s:%d %s\n", __FILE__, __LINE__, #c);     \
      ++fails;                                                     \
    }                                                              \
  } while (0)

static void check_pool() {
  for (int rep = 0; rep < 300; ++rep) {
    const size_t n = 1 + rep % 131;
    std::vector<int> hit(n, 0);
    host_parallel_for(n, [&](size_t i) {
      hit[i]++;
      host_parallel_for(2, [](size_t) {});  // nested: runs serially
    });
    for (size_t i = 0; i < n; ++i) CHECK(hit[i] == 1);
  }
  bool threw = false;
  try {
    host_parallel_for(64, [](size_t i) {
      if (i == 7) throw std::runtime_error("planned");
    });
  } catch (const std::runtime_error&) {
    threw = true;
  }
  CHECK(threw);
  std::vector<int> hit(500, 0);
  host_parallel_for(hit.size(), [&](size_t i) { hit[i]++; });
  for (int x : hit) CHECK(x == 1);
  CHECK(host_threads() >= 1);
}

using Key = std::tuple<const double*, int, int, int, int>;

static void check_plan(unsigned seed, const TcShape& shape) {
  std::mt19937 rng(seed);
  const int nblk = 3 + rng() % 12;
  std::vector<int> dims(nblk);
  for (auto& d : dims) d = 1 + rng() % 300;
  std::vector<HpsiBlock> blocks;
  std::vector<HpsiItem> items;
  const double* op = reinterpret_cast<const double*>(uintptr_t(1) << 32);
  const double* ps = reinterpret_cast<const double*>(uintptr_t(9) << 32);
  for (int b = 0; b < nblk; ++b) {
    HpsiBlock hb{};
    hb.m = dims[b];
    hb.n = dims[(b * 5 + 1) % nblk];
    hb.ldc = hb.n;
    hb.item_begin = (int)items.size();
    const int cnt = (b % 4 == 3) ? 0 : (int)(rng() % 700);
    for (int k = 0; k < cnt; ++k) {
      HpsiItem it{};
      const int q = rng() % nblk;
      const int ka = dims[q], kb = dims[(q * 3) % nblk];
      const int oa = rng() % 40, ob = rng() % 40;
      const bool ida = rng() % 6 == 0, idb = !ida && rng() % 6 == 0;
      it.A = ida ? nullptr : op + ((size_t)oa * 64 + q) * 4096 + b % 3;
      it.lda = ka;
      it.transA = oa % 2;
      it.P = ps + (size_t)q * 4096;
      it.ldp = kb;
      it.B = idb ? nullptr : op + ((size_t)ob * 64 + q) * 4096 + 7;
      it.ldb = kb;
      it.transB = ob % 2;
      it.ka = ida ? hb.m : ka;
      it.kb = idb ? hb.n : kb;
      it.alpha = 0.25 * (k + 1);
      items.push_back(it);
    }
    hb.item_count = cnt;
    blocks.push_back(hb);
  }
  char* const pool = reinterpret_cast<char*>(uintptr_t(0x40) << 32);
  size_t pool_bytes = 0;
  TcPlan plan;
  const int ncta = 5 + (int)(seed % 7) * 23;
  hpsi_tc_prepare(blocks, items, [&](size_t bytes) { pool_bytes = bytes; return (void*)pool; }, plan, ncta,
                  shape);
  CHECK(plan.shape == shape);
  CHECK(plan.pool_bytes == pool_bytes);
  {
    // a plan made for the default shape and rescheduled equals one made for
    // this shape directly; the operands are untouched by rescheduling
    TcPlan other;
    hpsi_tc_prepare(blocks, items, [&](size_t) { return (void*)pool; }, other, ncta);
    const size_t units0 = other.units;
    const size_t items0 = other.items.size();
    hpsi_tc_schedule(blocks, other, shape, ncta);
    CHECK(other.units == units0 && other.items.size() == items0);
    CHECK(other.tasks.size() == plan.tasks.size() && other.cta_task.size() == plan.cta_task.size());
    CHECK(other.cta_off == plan.cta_off && other.scratch == plan.scratch);
    for (size_t t = 0; t < std::min(other.tasks.size(), plan.tasks.size()); ++t)
      CHECK(other.tasks[t].block == plan.tasks[t].block && other.tasks[t].c0 == plan.tasks[t].c0 &&
            other.tasks[t].it_begin == plan.tasks[t].it_begin && other.tasks[t].part == plan.tasks[t].part);
    for (size_t e = 0; e < std::min(other.cta_task.size(), plan.cta_task.size()); ++e)
      CHECK(other.cta_task[e].task == plan.cta_task[e].task && other.cta_task[e].ghost == plan.cta_task[e].ghost);
    // the histogram key ignores the order of the blocks
    std::vector<HpsiBlock> rev(blocks.rbegin(), blocks.rend());
    CHECK(tc_histogram_key(rev, ncta) == tc_histogram_key(blocks, ncta));
    CHECK(tc_histogram_key(blocks, ncta) != tc_histogram_key(blocks, ncta + 2));
  }
  CHECK(plan.pool_bytes == plan.units * kTcUnitFloats * sizeof(float));
  // expected jobs: first occurrences in reference order; an identity factor
  // is the operand (nullptr, 0, d, d, -1)
  std::map<Key, int> first;
  std::vector<Key> order;
  std::vector<int> is_psi;
  auto note = [&](const Key& k, bool psi) {
    if (first.emplace(k, (int)order.size()).second) {
      order.push_back(k);
      is_psi.push_back(psi);
    }
  };
  auto key_a = [&](const HpsiBlock& bk, const HpsiItem& it) {
    return it.A ? Key{it.A, it.transA, bk.m, it.ka, it.lda} : Key{nullptr, 0, bk.m, bk.m, -1};
  };
  auto key_b = [&](const HpsiBlock& bk, const HpsiItem& it) {
    return it.B ? Key{it.B, it.transB, bk.n, it.kb, it.ldb} : Key{nullptr, 0, bk.n, bk.n, -1};
  };
  for (auto& bk : blocks)
    for (int i = bk.item_begin; i < bk.item_begin + bk.item_count; ++i) {
      const HpsiItem& it = items[i];
      note(key_a(bk, it), false);
      note(Key{it.P, 1, it.kb, it.ka, it.ldp}, true);
      note(key_b(bk, it), false);
    }
  std::vector<SplitJob> jobs_op, jobs_psi;
  for (size_t j = 0; j < order.size(); ++j) {
    SplitJob sj{};
    std::tie(sj.src, sj.trans, sj.rows, sj.cols, sj.ld) = order[j];
    (is_psi[j] ? jobs_psi : jobs_op).push_back(sj);
  }
  CHECK(plan.op_jobs.size() == jobs_op.size());
  CHECK(plan.psi_jobs.size() == jobs_psi.size());
  // plane pairs: 2 ceil(rows/8) ceil(cols/32) units each, disjoint, inside the pool
  std::map<int, Key> by_unit;
  std::vector<std::pair<size_t, size_t>> spans;
  auto check_jobs = [&](const std::vector<SplitJob>& got, const std::vector<SplitJob>& want) {
    for (size_t j = 0; j < std::min(got.size(), want.size()); ++j) {
      const SplitJob& g = got[j];
      CHECK(g.src == want[j].src && g.trans == want[j].trans && g.rows == want[j].rows &&
            g.cols == want[j].cols && g.ld == want[j].ld);
      const size_t units = 2 * (size_t)((g.rows + 7) / 8) * ((g.cols + 31) / 32);
      CHECK(g.unit >= 0 && (size_t)g.unit + units <= plan.units);
      spans.push_back({(size_t)g.unit, (size_t)g.unit + units});
      by_unit[g.unit] = Key{g.src, g.trans, g.rows, g.cols, g.ld};
    }
  };
  check_jobs(plan.op_jobs, jobs_op);
  check_jobs(plan.psi_jobs, jobs_psi);
  std::sort(spans.begin(), spans.end());
  for (size_t i = 1; i < spans.size(); ++i) CHECK(spans[i].first >= spans[i - 1].second);
  // items
  CHECK(plan.items.size() == items.size());
  for (auto& bk : blocks)
    for (int i = bk.item_begin; i < bk.item_begin + bk.item_count; ++i) {
      const HpsiItem& it = items[i];
      const TcItem& t = plan.items[i];
      CHECK(t.ka == (it.A ? it.ka : bk.m) && t.kb == (it.B ? it.kb : bk.n) && t.alpha == it.alpha);
      auto refers = [&](const TcMat& m, const Key& k) {
        auto f = by_unit.find(m.unit);
        return f != by_unit.end() && f->second == k && m.groups == (std::get<2>(k) + 7) / 8;
      };
      CHECK(refers(t.A, key_a(bk, it)));
      CHECK(refers(t.Pt, Key{it.P, 1, it.kb, it.ka, it.ldp}));
      CHECK(refers(t.B, key_b(bk, it)));
    }
  // persistent launch in clusters: lists of equal length per cluster, entry k
  // of each naming the same block and items; every task in exactly one list
  // (ghost entries aside); groups are contiguous ranks with the same rows and
  // distinct columns; the plan's own check agrees
  const int C = shape.cluster;
  const int G = (int)plan.cta_off.size() - 1;
  CHECK(G % C == 0);
  CHECK(plan.tasks.empty() ? G == 0 : (G >= C && G <= std::max(C, ncta / C * C)));
  std::vector<int> seen(plan.tasks.size(), 0);
  for (int k = 0; k < G / C; ++k) {
    const int len = plan.cta_off[k * C + 1] - plan.cta_off[k * C];
    CHECK(len > 0);
    for (int j = 0; j < C; ++j) CHECK(plan.cta_off[k * C + j + 1] - plan.cta_off[k * C + j] == len);
    for (int q = 0; q < len; ++q) {
      const TcSlot& s0 = plan.cta_task[plan.cta_off[k * C] + q];
      CHECK(!s0.ghost);
      for (int j = 0; j < C; ++j) {
        const TcSlot& e = plan.cta_task[plan.cta_off[k * C + j] + q];
        const HpsiTask& t = plan.tasks[e.task];
        const HpsiTask& t0 = plan.tasks[s0.task];
        CHECK(t.block == t0.block && t.it_begin == t0.it_begin && t.it_count == t0.it_count);
        if (e.ghost) {
          CHECK(e.grp0 == j && e.grpn == 1);
          continue;
        }
        seen[e.task]++;
        CHECK(e.grp0 <= j && j < e.grp0 + e.grpn && e.grp0 + e.grpn <= C);
        for (int i = e.grp0; i < e.grp0 + e.grpn; ++i) {
          const TcSlot& o = plan.cta_task[plan.cta_off[k * C + i] + q];
          CHECK(!o.ghost && o.grp0 == e.grp0 && o.grpn == e.grpn);
          CHECK(plan.tasks[o.task].r0 == t.r0 && (i == j || plan.tasks[o.task].c0 != t.c0));
        }
      }
    }
  }
  for (int x : seen) CHECK(x == 1);
  CHECK(tc_plan_check(plan, blocks).empty());
  // tiles, chunks, partial tiles, reductions
  std::map<std::tuple<int, int, int>, std::vector<const HpsiTask*>> chunks;
  std::set<long long> parts;
  for (const HpsiTask& t : plan.tasks) {
    chunks[{t.block, t.r0, t.c0}].push_back(&t);
    CHECK(t.part >= 0 && t.part % ((long long)kTcTileM * kTcTileN) == 0);
    CHECK(parts.insert(t.part).second);
    CHECK((size_t)t.part + (size_t)kTcTileM * kTcTileN <= plan.scratch);
  }
  size_t tiles = 0;
  for (int b = 0; b < nblk; ++b) {
    const HpsiBlock& bk = blocks[b];
    if (bk.item_count == 0) continue;
    for (int r0 = 0; r0 < bk.m; r0 += kTcTileM)
      for (int c0 = 0; c0 < bk.n; c0 += shape.tile_n) {
        ++tiles;
        auto& v = chunks[{b, r0, c0}];
        int next = bk.item_begin;
        for (const HpsiTask* t : v) {
          CHECK(t->it_begin == next && t->it_count > 0);
          next += t->it_count;
        }
        CHECK(next == bk.item_begin + bk.item_count);
        int nred = 0;
        for (const HpsiReduce& rd : plan.reds)
          if (rd.block == b && rd.r0 == r0 && rd.c0 == c0) {
            ++nred;
            CHECK(rd.nparts == (int)v.size());
            CHECK(!v.empty() && rd.part0 == v.front()->part);
            for (size_t k = 0; k < v.size(); ++k)
              CHECK(v[k]->part == rd.part0 + (long long)k * kTcTileM * kTcTileN);
          }
        CHECK(nred == 1);
      }
  }
  CHECK(chunks.size() == tiles && plan.reds.size() == tiles);
}

static void check_jacobi_batches(unsigned seed, int cap) {
  std::mt19937 rng(seed);
  const int count = 1 + rng() % 400;
  std::vector<int> n(count);
  for (auto& x : n) x = 1 + rng() % (seed % 2 ? 160 : 420);
  std::sort(n.begin(), n.end(), [](int a, int b) { return a > b; });
  const std::vector<JacBatch> batches = jac_plan_batches(n, cap);
  size_t next = 0;
  for (const JacBatch& b : batches) {
    CHECK(b.begin == next && b.end > b.begin && b.g.size() == b.end - b.begin);
    next = b.end;
    int sum = 0;
    double worst_min = 0.0, worst = 0.0;
    for (size_t k = b.begin; k < b.end; ++k) {
      const int g = b.g[k - b.begin];
      const int gmin = n[k] > kJacSmemN ? 2 : 1;
      const int gmax = std::max(2, std::min(32, ((n[k] + 1) & ~1) / 2));
      CHECK(g >= gmin && g <= std::max(gmin, gmax));
      sum += g;
      worst_min = std::max(worst_min, jac_cost(n[k], gmin));
      worst = std::max(worst, jac_cost(n[k], g));
    }
    CHECK(sum <= cap);
    CHECK(worst <= worst_min);
  }
  CHECK(next == n.size());
  for (int m = 2; m < 500; m += 7)
    for (int g = 2; g < 32; ++g) CHECK(jac_cost(m, g + 1) < jac_cost(m, g));
}

int main() {
  check_pool();
  for (unsigned s = 1; s <= 40; ++s) check_jacobi_batches(s, s % 3 ? 152 : 40);
  const std::vector<TcShape> cands = tc_shape_candidates();
  CHECK(!cands.empty() && cands[0] == TcShape());
  for (unsigned s = 1; s <= 12; ++s)
    for (const TcShape& sh : cands) check_plan(s, sh);
  if (fails) {
    std::printf("%d checks failed\n", fails);
    return 1;
  }
  std::printf("host planning checks passed\n");
  return 0;
}
