// Host planning of the tcgen05 H_eff psi contraction: distinct operands and
// their TF32 hi/lo plane pairs in the pool, the kernel's item descriptors,
// the 128 x 256 sigma tiles with their item chunks, and the task lists of the
// persistent launch (Sec. II.B two-site effective Hamiltonian; the kernel is
// in hpsi_tc.cu).
#include <algorithm>
#include <cstdint>
#include <numeric>
#include <queue>
#include <stdexcept>
#include <string>
#include <vector>

#include "hpsi_tc.cuh"
#include "host_pool.hpp"

namespace dmrg {
namespace {
constexpr int TM = kTcTileM, TNMAX = kTcTileN;

int ceil_div(int a, int b) { return (a + b - 1) / b; }

// tensor-pipe work of one item, in units of one k-block of 16 at MMA width
// 256 (128 x 256 x 16 in three TF32 products): stage 1 per super-chunk of 256
// columns of psi; stage 2 on a tile of width N per 16-column piece, plus a
// little for the conversion of each piece
double stage1_cost(int ka, int kb) {
  double c = 0.0;
  for (int jc = 0; jc < kb; jc += 256) c += ceil_div(ka, 16) * (((std::min(256, kb - jc) + 15) & ~15) / 256.0);
  return c;
}
double stage2_cost(int kb, int N) {
  double c = 0.0;
  for (int p = 0; p < kb; p += 16) c += N / 256.0 + 0.05;
  return c;
}
double item_cost(int ka, int kb, int N) { return stage1_cost(ka, kb) + stage2_cost(kb, N); }
}  // namespace

std::vector<TcShape> tc_shape_candidates() {
  std::vector<TcShape> c;
  c.push_back(TcShape{kTcTileN, 4, 0});  // the default
  c.push_back(TcShape{kTcTileN, 8, 0});  // finer item chunks
  c.push_back(TcShape{kTcTileN, 2, 0});  // coarser item chunks
  c.push_back(TcShape{kTcTileN, 4, 1});  // block order
  c.push_back(TcShape{128, 4, 0});       // narrow tiles
  c.push_back(TcShape{kTcTileN, 4, 0, 4});  // clusters of four: stage 1 shared by up to four tiles
  return c;
}

uint64_t tc_histogram_key(const std::vector<HpsiBlock>& blocks, int ncta) {
  std::vector<uint64_t> h;
  h.reserve(blocks.size());
  for (const HpsiBlock& b : blocks) {
    if (b.item_count <= 0 || b.m <= 0 || b.n <= 0) continue;
    int lg = 0;
    while ((1 << (lg + 1)) <= b.item_count) ++lg;
    h.push_back(((uint64_t)ceil_div(b.m, 64) << 40) | ((uint64_t)ceil_div(b.n, 64) << 16) | (uint64_t)lg);
  }
  std::sort(h.begin(), h.end());
  uint64_t k = 0x84222325cbf29ce4ull ^ (uint64_t)ncta;
  for (uint64_t x : h) {
    k ^= x + 0x9e3779b97f4a7c15ull + (k << 6) + (k >> 2);
    k *= 0x100000001b3ull;
  }
  return k;
}

void hpsi_tc_prepare(const std::vector<HpsiBlock>& blocks, const std::vector<HpsiItem>& items,
                     const std::function<void*(size_t)>& alloc, TcPlan& plan, int ncta, const TcShape& shape) {
  hpsi_tc_operands(blocks, items, alloc, plan);
  hpsi_tc_schedule(blocks, plan, shape, ncta);
}

void hpsi_tc_operands(const std::vector<HpsiBlock>& blocks, const std::vector<HpsiItem>& items,
                      const std::function<void*(size_t)>& alloc, TcPlan& plan) {
  plan = TcPlan();
  // Distinct operands (src, trans, rows, cols, ld) become split jobs, numbered
  // in first-occurrence order over the references (items in block order;
  // roles A, P^T, B).  An identity factor is the operand (nullptr, 0, d, d, -1).
  // The references are hashed into kShards tables processed in parallel; one
  // ordered scan numbers the jobs.
  struct Key {
    const double* src = nullptr;
    int trans = 0, rows = 0, cols = 0, ld = 0;
    bool operator==(const Key& o) const {
      return src == o.src && trans == o.trans && rows == o.rows && cols == o.cols && ld == o.ld;
    }
  };
  auto mix = [](uint64_t x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    return x ^ (x >> 33);
  };
  std::vector<uint32_t> iorder;
  std::vector<int> item_blk(items.size(), -1);
  iorder.reserve(items.size());
  for (size_t b = 0; b < blocks.size(); ++b)
    for (int i = blocks[b].item_begin; i < blocks[b].item_begin + blocks[b].item_count; ++i) {
      item_blk[i] = (int)b;
      iorder.push_back((uint32_t)i);
    }
  const size_t nref = 3 * iorder.size();
  auto key_of = [&](size_t r) -> Key {
    const HpsiItem& it = items[iorder[r / 3]];
    const HpsiBlock& bk = blocks[item_blk[iorder[r / 3]]];
    switch (r % 3) {
      case 0:
        return it.A ? Key{it.A, it.transA, bk.m, it.ka, it.lda} : Key{nullptr, 0, bk.m, bk.m, -1};
      case 1:
        return Key{it.P, 1, it.kb, it.ka, it.ldp};
      default:
        return it.B ? Key{it.B, it.transB, bk.n, it.kb, it.ldb} : Key{nullptr, 0, bk.n, bk.n, -1};
    }
  };
  constexpr size_t kShards = 32;
  std::vector<uint64_t> rhash(nref);
  const size_t rchunk = 4096;
  host_parallel_for((nref + rchunk - 1) / rchunk, [&](size_t c) {
    for (size_t r = c * rchunk; r < std::min(nref, (c + 1) * rchunk); ++r) {
      const Key k = key_of(r);
      rhash[r] = mix((uint64_t)(uintptr_t)k.src ^ ((uint64_t)(uint32_t)k.rows << 32) ^
                     ((uint64_t)(uint32_t)k.cols << 12) ^ ((uint64_t)(uint32_t)k.ld << 44) ^ (uint64_t)k.trans);
    }
  });
  std::vector<int> lid(nref, -1);       // shard-local operand of reference r
  std::vector<uint8_t> first(nref, 0);  // r is the first reference of its operand
  std::vector<std::vector<Key>> skeys(kShards);
  host_parallel_for(kShards, [&](size_t sh) {
    size_t mine = 0;
    for (size_t r = 0; r < nref; ++r) mine += rhash[r] % kShards == sh;
    size_t cap = 64;
    while (cap < 2 * mine + 64) cap <<= 1;
    const size_t mask = cap - 1;
    std::vector<int> slot(cap, -1);
    auto& keys = skeys[sh];
    for (size_t r = 0; r < nref; ++r) {
      if (rhash[r] % kShards != sh) continue;
      const Key k = key_of(r);
      size_t h = (rhash[r] / kShards) & mask;
      while (slot[h] >= 0 && !(keys[slot[h]] == k)) h = (h + 1) & mask;
      if (slot[h] < 0) {
        slot[h] = (int)keys.size();
        keys.push_back(k);
        first[r] = 1;
      }
      lid[r] = slot[h];
    }
  });
  std::vector<std::vector<int>> gid(kShards);
  for (size_t sh = 0; sh < kShards; ++sh) gid[sh].assign(skeys[sh].size(), -1);
  std::vector<SplitJob> jobs;
  std::vector<uint8_t> is_psi;
  size_t units = 0;
  for (size_t r = 0; r < nref; ++r) {
    if (!first[r]) continue;
    const size_t sh = rhash[r] % kShards;
    const Key& k = skeys[sh][lid[r]];
    gid[sh][lid[r]] = (int)jobs.size();
    if (units > (size_t)INT32_MAX) throw std::runtime_error("tcgen05 plan: split pool beyond 2^31 units");
    jobs.push_back(SplitJob{k.src, k.rows, k.cols, k.ld, k.trans, (int)units});
    units += 2 * (size_t)ceil_div(k.rows, 8) * (size_t)ceil_div(k.cols, 32);
    is_psi.push_back(r % 3 == 1);
  }
  if (units > (size_t)INT32_MAX) throw std::runtime_error("tcgen05 plan: split pool beyond 2^31 units");
  plan.units = units;
  plan.pool_bytes = units * kTcUnitFloats * sizeof(float);
  if (units > 0) alloc(plan.pool_bytes);
  for (size_t j = 0; j < jobs.size(); ++j) (is_psi[j] ? plan.psi_jobs : plan.op_jobs).push_back(jobs[j]);
  auto mat = [&](size_t r) {
    const SplitJob& j = jobs[gid[rhash[r] % kShards][lid[r]]];
    return TcMat{j.unit, ceil_div(j.rows, 8)};
  };
  plan.items.resize(items.size());
  const size_t ichunk = 2048;
  host_parallel_for((iorder.size() + ichunk - 1) / ichunk, [&](size_t c) {
    for (size_t q = c * ichunk; q < std::min(iorder.size(), (c + 1) * ichunk); ++q) {
      const size_t i = iorder[q];
      const HpsiItem& it = items[i];
      const HpsiBlock& bk = blocks[item_blk[i]];
      TcItem t;
      t.A = mat(3 * q);
      t.Pt = mat(3 * q + 1);
      t.B = mat(3 * q + 2);
      t.ka = it.A ? it.ka : bk.m;
      t.kb = it.B ? it.kb : bk.n;
      t.alpha = it.alpha;
      plan.items[i] = t;
    }
  });
  for (size_t i = 0; i < items.size(); ++i)
    if (item_blk[i] < 0) {  // an item of no block: never referenced by a task
      plan.items[i] = TcItem{TcMat{}, TcMat{}, TcMat{}, items[i].ka, items[i].kb, items[i].alpha};
    }
}

void hpsi_tc_schedule(const std::vector<HpsiBlock>& blocks, TcPlan& plan, const TcShape& shape, int ncta) {
  if (ncta <= 0) ncta = 152;
  const int TN = shape.tile_n;
  if (TN < 16 || TN > TNMAX || TN % 16 || shape.chunks_per_cta < 1 || shape.order < 0 || shape.order > 1 ||
      shape.cluster < 1 || shape.cluster > kTcClusterMax)
    throw std::invalid_argument("tcgen05 plan: invalid schedule shape");
  plan.shape = shape;
  plan.tasks.clear();
  plan.reds.clear();
  plan.cta_off.clear();
  plan.cta_task.clear();
  plan.scratch = 0;
  plan.cost = 0.0;
  // Tasks: 128 x TN tiles, the items of a tile cut into contiguous chunks of
  // about equal tensor work, so that the launch has a few tasks per CTA.
  double total = 0.0;
  std::vector<std::vector<double>> icost(blocks.size());
  for (size_t b = 0; b < blocks.size(); ++b) {
    const HpsiBlock& bk = blocks[b];
    if (bk.item_count == 0 || bk.m == 0 || bk.n == 0) continue;
    icost[b].resize(bk.item_count);
    for (int c0 = 0; c0 < bk.n; c0 += TN) {
      const int N = std::min(TN, (std::min(TN, bk.n - c0) + 15) & ~15);
      for (int k = 0; k < bk.item_count; ++k) {
        const TcItem& t = plan.items[bk.item_begin + k];
        const double c = item_cost(t.ka, t.kb, N);
        if (c0 == 0) icost[b][k] = c;
        total += c * ceil_div(bk.m, TM);
      }
    }
  }
  const double target = std::max(1.0, total / ((double)shape.chunks_per_cta * ncta));
  // Cluster tasks: C tasks of the same block and item chunk.  The
  // column tiles of one row tile are grouped C at a time (a group
  // shares stage 1); the remainder groups of the rows are packed first-fit
  // (largest first) into further cluster tasks, and slots left empty become
  // ghosts.
  const int C = shape.cluster;
  struct Member {
    int task, grp0, grpn;
  };
  struct CTask {
    std::vector<Member> m;  // real members in rank order (ranks 0 .. m.size()-1)
    double cost = 0.0;
  };
  std::vector<CTask> ctasks;
  std::vector<int> ct_block;     // sigma block of each cluster task
  std::vector<double> blk_cost(blocks.size(), 0.0);
  std::vector<double> s1c, s2c;  // per task: stage-1 and stage-2 cost of its items
  long long part = 0;
  const long long tile = (long long)TM * TNMAX;
  for (size_t b = 0; b < blocks.size(); ++b) {
    const HpsiBlock& bk = blocks[b];
    if (bk.item_count == 0 || bk.m == 0 || bk.n == 0) continue;
    // chunk boundaries from the first column tile's costs (the same for all
    // tiles of the block, so every tile of a block has the same chunks)
    std::vector<int> cuts{0};
    double acc = 0.0;
    for (int k = 0; k < bk.item_count; ++k) {
      acc += icost[b][k];
      if (acc >= target && k + 1 < bk.item_count) {
        cuts.push_back(k + 1);
        acc = 0.0;
      }
    }
    cuts.push_back(bk.item_count);
    const int nch = (int)cuts.size() - 1;
    const int mt = ceil_div(bk.m, TM), nt = ceil_div(bk.n, TN);
    // tasks in (tile, chunk) order: the chunks of a tile have consecutive partial tiles
    const int t_first = (int)plan.tasks.size();
    for (int r = 0; r < mt; ++r)
      for (int c = 0; c < nt; ++c) {
        const int r0 = r * TM, c0 = c * TN;
        const int N = std::min(TN, (std::min(TN, bk.n - c0) + 15) & ~15);
        plan.reds.push_back({(int)b, r0, c0, nch, part});
        for (int ch = 0; ch < nch; ++ch) {
          const int i0 = bk.item_begin + cuts[ch], cnt = cuts[ch + 1] - cuts[ch];
          plan.tasks.push_back({(int)b, r0, c0, i0, cnt, part});
          double a1 = 0.0, a2 = 0.0;
          for (int k = i0; k < i0 + cnt; ++k) {
            a1 += stage1_cost(plan.items[k].ka, plan.items[k].kb);
            a2 += stage2_cost(plan.items[k].kb, N);
          }
          s1c.push_back(a1);
          s2c.push_back(a2);
          part += tile;
        }
      }
    auto task_at = [&](int r, int c, int ch) { return t_first + (r * nt + c) * nch + ch; };
    for (int ch = 0; ch < nch; ++ch) {
      std::vector<std::vector<int>> rem;  // remainder groups (tasks of one row)
      for (int r = 0; r < mt; ++r)
        for (int c = 0; c < nt; c += C) {
          std::vector<int> g;
          for (int q = c; q < std::min(nt, c + C); ++q) g.push_back(task_at(r, q, ch));
          if ((int)g.size() == C) {
            CTask ct;
            for (int q = 0; q < C; ++q) ct.m.push_back({g[q], 0, C});
            ctasks.push_back(ct);
            ct_block.push_back((int)b);
          } else {
            rem.push_back(g);
          }
        }
      std::stable_sort(rem.begin(), rem.end(), [](const auto& x, const auto& y) { return x.size() > y.size(); });
      const size_t open0 = ctasks.size();
      for (const auto& g : rem) {
        size_t k = open0;
        while (k < ctasks.size() && ctasks[k].m.size() + g.size() > (size_t)C) ++k;
        if (k == ctasks.size()) {
          ctasks.emplace_back();
          ct_block.push_back((int)b);
        }
        const int g0 = (int)ctasks[k].m.size();
        for (int t : g) ctasks[k].m.push_back({t, g0, (int)g.size()});
      }
    }
  }
  plan.scratch = (size_t)part;
  for (CTask& ct : ctasks) {
    double w = 0.0;
    for (const Member& mb : ct.m) w = std::max(w, s1c[mb.task] / mb.grpn + s2c[mb.task]);
    ct.cost = w + 1.0;  // drain
  }
  for (size_t k = 0; k < ctasks.size(); ++k) blk_cost[ct_block[k]] += ctasks[k].cost;
  // Persistent launch, order 0: longest cluster task first onto the
  // least-loaded cluster; each cluster runs its tasks in decreasing cost.
  // Order 1: sigma blocks in decreasing total cost, the cluster tasks of a
  // block in (item chunk, row, column) order, each onto the least-loaded
  // cluster; the tasks running at one time then come from a short stretch of
  // that list and share their operand tiles.
  const int nct = (int)ctasks.size();
  const int nclu = std::max(1, std::min(std::max(1, ncta / C), nct));
  std::vector<int> order(nct);
  std::iota(order.begin(), order.end(), 0);
  if (shape.order == 0)
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return ctasks[a].cost > ctasks[b].cost; });
  else
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
      const int ba = ct_block[a], bb = ct_block[b];
      if (ba == bb) return false;
      if (blk_cost[ba] != blk_cost[bb]) return blk_cost[ba] > blk_cost[bb];
      return ba < bb;
    });
  using Load = std::pair<double, int>;
  std::priority_queue<Load, std::vector<Load>, std::greater<Load>> pq;
  for (int c = 0; c < nclu; ++c) pq.push({0.0, c});
  std::vector<std::vector<int>> lists(nclu);
  for (int t : order) {
    Load l = pq.top();
    pq.pop();
    lists[l.second].push_back(t);
    pq.push({l.first + ctasks[t].cost, l.second});
  }
  while (!pq.empty()) {
    plan.cost = std::max(plan.cost, pq.top().first);
    pq.pop();
  }
  if (nct == 0) {
    plan.cta_off.assign(1, 0);
  } else {
    plan.cta_off.assign((size_t)nclu * C + 1, 0);
    for (int k = 0; k < nclu; ++k)
      for (int j = 0; j < C; ++j) {
        const int cta = k * C + j;
        for (int t : lists[k]) {
          const CTask& ct = ctasks[t];
          if (j < (int)ct.m.size())
            plan.cta_task.push_back({ct.m[j].task, ct.m[j].grp0, ct.m[j].grpn, 0});
          else
            plan.cta_task.push_back({ct.m[0].task, j, 1, 1});
        }
        plan.cta_off[cta + 1] = (int)plan.cta_task.size();
      }
  }
}

std::string tc_plan_check(const TcPlan& plan, const std::vector<HpsiBlock>& blocks) {
  if (plan.shape.tile_n < 16 || plan.shape.tile_n > TNMAX || plan.shape.tile_n % 16)
    return "tile width not a multiple of 16 in [16, 256]";
  auto fits = [&](const TcMat& m, int rows, int cols) {
    if (m.unit < 0 || m.groups != ceil_div(rows, 8)) return false;
    return (size_t)m.unit + 2 * (size_t)m.groups * (size_t)ceil_div(cols, 32) <= plan.units;
  };
  const long long tile = (long long)TM * TNMAX;
  for (size_t t = 0; t < plan.tasks.size(); ++t) {
    const HpsiTask& tk = plan.tasks[t];
    const std::string at = "task " + std::to_string(t) + ": ";
    if (tk.block < 0 || tk.block >= (int)blocks.size()) return at + "block out of range";
    const HpsiBlock& bk = blocks[tk.block];
    if (tk.r0 < 0 || tk.r0 >= bk.m || tk.r0 % TM || tk.c0 < 0 || tk.c0 >= bk.n || tk.c0 % plan.shape.tile_n)
      return at + "tile origin out of range";
    if (tk.it_count < 1 || tk.it_begin < bk.item_begin || tk.it_begin + tk.it_count > bk.item_begin + bk.item_count ||
        tk.it_begin + tk.it_count > (int)plan.items.size())
      return at + "items out of range";
    if (tk.part < 0 || (size_t)(tk.part + tile) > plan.scratch) return at + "partial tile out of range";
    for (int i = tk.it_begin; i < tk.it_begin + tk.it_count; ++i) {
      const TcItem& it = plan.items[i];
      if (it.ka < 1 || it.kb < 1) return at + "empty item " + std::to_string(i);
      if (!fits(it.A, bk.m, it.ka) || !fits(it.Pt, it.kb, it.ka) || !fits(it.B, bk.n, it.kb))
        return at + "operand planes of item " + std::to_string(i) + " outside the pool";
    }
  }
  for (const HpsiReduce& rd : plan.reds) {
    if (rd.block < 0 || rd.block >= (int)blocks.size() || rd.nparts < 1 || rd.part0 < 0 ||
        (size_t)(rd.part0 + rd.nparts * tile) > plan.scratch)
      return "reduction out of range";
  }
  const int C = plan.shape.cluster;
  if (C < 1 || C > kTcClusterMax) return "cluster size out of range";
  if (plan.cta_off.empty() || plan.cta_off.front() != 0 || plan.cta_off.back() != (int)plan.cta_task.size())
    return "CTA lists do not cover their entries";
  const int ncta = (int)plan.cta_off.size() - 1;
  if (plan.tasks.empty() != (ncta == 0) || ncta % C) return "CTA count not a whole number of clusters";
  std::vector<int> seen(plan.tasks.size(), 0);
  for (int k = 0; k < ncta / C; ++k) {
    const int base = k * C;
    const int len = plan.cta_off[base + 1] - plan.cta_off[base];
    if (len <= 0) return "empty CTA list " + std::to_string(base);
    for (int j = 1; j < C; ++j)
      if (plan.cta_off[base + j + 1] - plan.cta_off[base + j] != len)
        return "cluster " + std::to_string(k) + ": lists of unequal length";
    for (int q = 0; q < len; ++q) {
      const TcSlot* sl[kTcClusterMax];
      for (int j = 0; j < C; ++j) {
        sl[j] = &plan.cta_task[plan.cta_off[base + j] + q];
        if (sl[j]->task < 0 || sl[j]->task >= (int)plan.tasks.size()) return "CTA entry out of range";
      }
      const HpsiTask& t0 = plan.tasks[sl[0]->task];
      for (int j = 0; j < C; ++j) {
        const TcSlot& e = *sl[j];
        const HpsiTask& t = plan.tasks[e.task];
        const std::string at = "cluster " + std::to_string(k) + " entry " + std::to_string(q) + " rank " +
                               std::to_string(j) + ": ";
        if (t.block != t0.block || t.it_begin != t0.it_begin || t.it_count != t0.it_count)
          return at + "items differ within the cluster";
        if (e.ghost) {
          if (e.grp0 != j || e.grpn != 1) return at + "ghost not alone in its group";
          continue;
        }
        if (seen[e.task]++) return at + "task listed twice";
        if (e.grpn < 1 || e.grp0 < 0 || e.grp0 > j || e.grp0 + e.grpn <= j || e.grp0 + e.grpn > C)
          return at + "group out of range";
        for (int i = e.grp0; i < e.grp0 + e.grpn; ++i) {
          const TcSlot& o = *sl[i];
          const HpsiTask& u = plan.tasks[o.task];
          if (o.ghost || o.grp0 != e.grp0 || o.grpn != e.grpn || u.r0 != t.r0 || (i != j && u.c0 == t.c0))
            return at + "inconsistent group";
        }
      }
    }
  }
  for (size_t t = 0; t < seen.size(); ++t)
    if (seen[t] != 1) return "task " + std::to_string(t) + " in no CTA list";
  if ((plan.units ? (size_t)plan.units * kTcUnitFloats * sizeof(float) : 0) != plan.pool_bytes)
    return "pool size mismatch";
  if (plan.units > (size_t)INT32_MAX) return "pool beyond 2^31 units";
  return std::string();
}

}  // namespace dmrg
