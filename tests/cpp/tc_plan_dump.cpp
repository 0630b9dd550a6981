// Prints the plan of the clustered tcgen05 H_eff psi contraction for a
// problem read from a text file (CPU only, no device calls): the block
// sizes, the items' (ka, kb), the tasks and every CTA's list of entries, and
// whether the planner's own check passes.  Input: the number of blocks, then
// per block "m n items" and per item "ka kb idA idB transA transB a p b"
// (idA/idB: identity factor; a, p, b: operand numbers, equal numbers naming
// the same matrix).  Usage: tc_plan_dump problem.txt ncta [schedule candidate]
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "hpsi_tc.cuh"

using namespace dmrg;

int main(int argc, char** argv) {
  if (argc < 3) return 2;
  FILE* f = std::fopen(argv[1], "r");
  if (!f) return 2;
  const int ncta = std::atoi(argv[2]);
  const int cand = argc > 3 ? std::atoi(argv[3]) : 0;
  const std::vector<TcShape> cands = tc_shape_candidates();
  if (cand < 0 || cand >= (int)cands.size()) return 2;
  int nb = 0;
  if (std::fscanf(f, "%d", &nb) != 1) return 3;
  std::vector<HpsiBlock> blocks;
  std::vector<HpsiItem> items;
  // distinct fake addresses per operand number (never dereferenced)
  const double* base = reinterpret_cast<const double*>(uintptr_t(1) << 36);
  for (int b = 0; b < nb; ++b) {
    HpsiBlock hb{};
    int cnt = 0;
    if (std::fscanf(f, "%d %d %d", &hb.m, &hb.n, &cnt) != 3) return 3;
    hb.ldc = hb.n;
    hb.item_begin = (int)items.size();
    hb.item_count = cnt;
    for (int k = 0; k < cnt; ++k) {
      HpsiItem it{};
      int ka, kb, ida, idb, ta, tb;
      long long a, p, bb;
      if (std::fscanf(f, "%d %d %d %d %d %d %lld %lld %lld", &ka, &kb, &ida, &idb, &ta, &tb, &a, &p, &bb) != 9)
        return 3;
      it.A = ida ? nullptr : base + (a << 20);
      it.P = base + ((p + (1ll << 14)) << 20);
      it.B = idb ? nullptr : base + ((bb + (2ll << 14)) << 20);
      it.transA = ta;
      it.transB = tb;
      it.lda = ta ? hb.m : ka;
      it.ldp = kb;
      it.ldb = tb ? hb.n : kb;
      it.ka = ka;
      it.kb = kb;
      it.alpha = 1.0;
      items.push_back(it);
    }
    blocks.push_back(hb);
  }
  std::fclose(f);
  TcPlan plan;
  hpsi_tc_prepare(blocks, items, [](size_t) { return (void*)(uintptr_t(1) << 44); }, plan, ncta, cands[cand]);
  const std::string bad = tc_plan_check(plan, blocks);
  std::printf("check %s\n", bad.empty() ? "ok" : bad.c_str());
  std::printf("cluster %d\n", plan.shape.cluster);
  std::printf("tile_n %d\n", plan.shape.tile_n);
  std::printf("blocks %zu\n", blocks.size());
  for (const HpsiBlock& b : blocks) std::printf("%d %d\n", b.m, b.n);
  std::printf("items %zu\n", plan.items.size());
  for (const TcItem& t : plan.items) std::printf("%d %d\n", t.ka, t.kb);
  std::printf("tasks %zu\n", plan.tasks.size());
  for (const HpsiTask& t : plan.tasks) std::printf("%d %d %d %d %d\n", t.block, t.r0, t.c0, t.it_begin, t.it_count);
  std::printf("ctas %zu\n", plan.cta_off.empty() ? (size_t)0 : plan.cta_off.size() - 1);
  for (size_t c = 0; c + 1 < plan.cta_off.size(); ++c) {
    std::printf("%d", plan.cta_off[c + 1] - plan.cta_off[c]);
    for (int q = plan.cta_off[c]; q < plan.cta_off[c + 1]; ++q) {
      const TcSlot& s = plan.cta_task[q];
      std::printf(" %d,%d,%d,%d", s.task, s.grp0, s.grpn, s.ghost);
    }
    std::printf("\n");
  }
  return 0;
}
