// Host planning of the tcgen05 H_eff psi contraction: distinct operands and
// their TF32 hi/lo planes, the kernel's item descriptors, and the 128 x 256
// sigma tiles with their item chunks (Sec. II.B two-site effective
// Hamiltonian; the kernel is in hpsi_tc.cu).
#include <algorithm>
#include <cstdint>
#include <vector>

#include "hpsi_tc.cuh"
#include "host_pool.hpp"

namespace dmrg {
namespace {
constexpr int TM = kTcTileM, TNMAX = kTcTileN;
}  // namespace

void hpsi_tc_prepare(const std::vector<HpsiBlock>& blocks, const std::vector<HpsiItem>& items,
                     const std::function<void*(size_t)>& alloc, TcPlan& plan) {
  plan = TcPlan();
  auto r32 = [](int x) { return (x + 31) & ~31; };
  // Distinct operands (src, trans, rows, cols, ld) become split jobs, numbered
  // in first-occurrence order over the references (items in block order;
  // roles A, P (for a non-identity A), B).  The references are hashed into
  // kShards tables processed in parallel; one ordered scan numbers the jobs.
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
  auto key_of = [&](size_t r, Key& k) -> bool {
    const HpsiItem& it = items[iorder[r / 3]];
    const HpsiBlock& bk = blocks[item_blk[iorder[r / 3]]];
    switch (r % 3) {
      case 0:
        if (!it.A) return false;
        k = Key{it.A, it.transA, bk.m, it.ka, it.lda};
        return true;
      case 1:
        if (!it.A) return false;
        k = Key{it.P, 1, it.kb, it.ka, it.ldp};
        return true;
      default:
        if (!it.B) return false;
        k = Key{it.B, it.transB, bk.n, it.kb, it.ldb};
        return true;
    }
  };
  constexpr size_t kShards = 32;
  constexpr uint64_t kNone = ~0ull;
  std::vector<uint64_t> rhash(nref);  // hash of reference r, kNone: no operand
  const size_t rchunk = 4096;
  host_parallel_for((nref + rchunk - 1) / rchunk, [&](size_t c) {
    for (size_t r = c * rchunk; r < std::min(nref, (c + 1) * rchunk); ++r) {
      Key k;
      rhash[r] = key_of(r, k) ? (mix((uint64_t)(uintptr_t)k.src ^ ((uint64_t)(uint32_t)k.rows << 32) ^
                                     ((uint64_t)(uint32_t)k.cols << 12) ^ ((uint64_t)(uint32_t)k.ld << 44) ^
                                     (uint64_t)k.trans) &
                                 (kNone >> 1))
                              : kNone;
    }
  });
  std::vector<int> lid(nref, -1);        // shard-local operand of reference r
  std::vector<uint8_t> first(nref, 0);   // r is the first reference of its operand
  std::vector<std::vector<Key>> skeys(kShards);
  host_parallel_for(kShards, [&](size_t sh) {
    size_t mine = 0;
    for (size_t r = 0; r < nref; ++r) mine += rhash[r] != kNone && rhash[r] % kShards == sh;
    size_t cap = 64;
    while (cap < 2 * mine + 64) cap <<= 1;
    const size_t mask = cap - 1;
    std::vector<int> slot(cap, -1);
    auto& keys = skeys[sh];
    for (size_t r = 0; r < nref; ++r) {
      if (rhash[r] == kNone || rhash[r] % kShards != sh) continue;
      Key k;
      key_of(r, k);
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
  size_t njobs = 0;
  for (auto& k : skeys) njobs += k.size();
  std::vector<SplitJob> jobs;
  std::vector<std::pair<size_t, size_t>> offs;
  std::vector<uint8_t> is_psi;
  jobs.reserve(njobs);
  offs.reserve(njobs);
  is_psi.reserve(njobs);
  size_t floats = 0;
  for (size_t r = 0; r < nref; ++r) {
    if (!first[r]) continue;
    const size_t sh = rhash[r] % kShards;
    const Key& k = skeys[sh][lid[r]];
    gid[sh][lid[r]] = (int)jobs.size();
    SplitJob j{k.src, k.rows, k.cols, k.ld, k.trans, nullptr, nullptr, r32(k.cols)};
    const size_t plane = (size_t)k.rows * j.ldd;
    offs.push_back({floats, floats + plane});
    floats += 2 * plane;
    floats = (floats + 3) & ~size_t(3);  // 16-byte alignment of every plane
    jobs.push_back(j);
    is_psi.push_back(r % 3 == 1);
  }
  float* pool = nullptr;
  if (floats > 0) pool = (float*)alloc(floats * sizeof(float));
  plan.pool_bytes = floats * sizeof(float);
  for (size_t j = 0; j < jobs.size(); ++j) {
    jobs[j].hi = pool + offs[j].first;
    jobs[j].lo = pool + offs[j].second;
    (is_psi[j] ? plan.psi_jobs : plan.op_jobs).push_back(jobs[j]);
  }
  auto mat = [&](size_t r) {
    TcMat m;
    if (rhash[r] != kNone) {
      const SplitJob& j = jobs[gid[rhash[r] % kShards][lid[r]]];
      m.hi = j.hi;
      m.lo = j.lo;
      m.ld = j.ldd;
    }
    return m;
  };
  plan.items.resize(items.size());
  const size_t ichunk = 2048;
  host_parallel_for((iorder.size() + ichunk - 1) / ichunk, [&](size_t c) {
    for (size_t q = c * ichunk; q < std::min(iorder.size(), (c + 1) * ichunk); ++q) {
      const size_t i = iorder[q];
      const HpsiItem& it = items[i];
      TcItem t;
      t.A = mat(3 * q);
      t.Pt = mat(3 * q + 1);
      t.P = it.P;
      t.ldp = it.ldp;
      t.B = mat(3 * q + 2);
      t.ka = it.ka;
      t.kb = it.kb;
      t.alpha = it.alpha;
      plan.items[i] = t;
    }
  });
  for (size_t i = 0; i < items.size(); ++i)
    if (item_blk[i] < 0) {  // an item of no block: no operands
      plan.items[i].P = items[i].P;
      plan.items[i].ldp = items[i].ldp;
      plan.items[i].ka = items[i].ka;
      plan.items[i].kb = items[i].kb;
      plan.items[i].alpha = items[i].alpha;
    }
  // tasks: 128 x 256 tiles, items chunked so that a launch has a few waves
  long long tile_items = 0;
  for (auto& b : blocks)
    tile_items += (long long)b.item_count * ((b.m + TM - 1) / TM) * ((b.n + TNMAX - 1) / TNMAX);
  const int max_items = (int)std::max<long long>(4, tile_items / (3 * 152) + 1);
  long long part = 0;
  for (size_t b = 0; b < blocks.size(); ++b) {
    const HpsiBlock& bk = blocks[b];
    if (bk.item_count == 0 || bk.m == 0 || bk.n == 0) continue;
    int nch = (bk.item_count + max_items - 1) / max_items;
    int per = (bk.item_count + nch - 1) / nch;
    // every chunk owns a partial tile (float pairs); the reduction adds the
    // chunks of a tile into sigma in float64
    for (int r0 = 0; r0 < bk.m; r0 += TM)
      for (int c0 = 0; c0 < bk.n; c0 += TNMAX) {
        plan.reds.push_back({(int)b, r0, c0, nch, part});
        for (int c = 0; c < nch; ++c) {
          int i0 = bk.item_begin + c * per;
          int cnt = std::min(per, bk.item_begin + bk.item_count - i0);
          plan.tasks.push_back({(int)b, r0, c0, i0, cnt, part});
          part += (long long)TM * TNMAX;
        }
      }
  }
  plan.scratch = (size_t)part;
}

}  // namespace dmrg
