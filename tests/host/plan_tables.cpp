// Host-side check of the batch plan (liblsgcpd's plan_batch): the tables every
// kernel indexes through are replayed here exactly as the kernels walk them, and
// every unit, slot, row and cell range is checked against the sizes it must
// cover.  Built and run by tests/test_plan_tables.py against the library; needs
// no GPU (without one the occupancy query falls back to one CTA per SM).
#include <cstdio>
#include <random>
#include <vector>

#include "internal.cuh"

namespace {

int failures = 0;

#define EXPECT(cond)                                                              \
  do {                                                                            \
    if (!(cond) && failures++ < 20) std::printf("failed: %s (line %d)\n", #cond, __LINE__); \
  } while (0)

void check_plan(const std::vector<long long>& N, const std::vector<long long>& M, int sms, int S,
                int seg_cap = lsg::kSegCap) {
  EXPECT(lsg::plan_fits(N, M));
  const lsg::BatchPlan plan = lsg::plan_batch(N, M, sms, S, seg_cap);
  EXPECT(plan.g.seg_cap == seg_cap);
  const lsg::Geo& g = plan.g;
  const int* t = plan.tab.data();
  const int P = g.P;
  const int* blk_off = t + g.o_blk_off;
  const int* tile_off = t + g.o_tile_off;
  const int* block_pair = t + g.o_block_pair;
  const int* unit_off = t + g.o_unit_off;
  const int* cta_slot = t + g.o_cta_slot;
  const int* cta_block = t + g.o_cta_block;
  const int* block_slot = t + g.o_block_slot;
  const int* tile_pair = t + g.o_tile_pair;

  EXPECT(g.SB % lsg::kCombineSources == 0);
  EXPECT(static_cast<int>(plan.tab.size()) == g.o_tile_pair + g.T);
  EXPECT(blk_off[P] == g.B && tile_off[P] == g.T && unit_off[g.B] == g.U);
  long long units = 0;
  for (int i = 0; i < P; ++i) {
    EXPECT(blk_off[i + 1] - blk_off[i] == (N[i] + g.SB - 1) / g.SB);
    EXPECT(tile_off[i + 1] - tile_off[i] == (M[i] + lsg::kTile - 1) / lsg::kTile);
    EXPECT(plan.off64[i + 1] - plan.off64[i] == N[i]);
    EXPECT(plan.off64[P + 2 + i] - plan.off64[P + 1 + i] == M[i]);
    for (int b = blk_off[i]; b < blk_off[i + 1]; ++b) {
      EXPECT(block_pair[b] == i);
      EXPECT(unit_off[b + 1] - unit_off[b] == tile_off[i + 1] - tile_off[i]);
    }
    for (int tt = tile_off[i]; tt < tile_off[i + 1]; ++tt) EXPECT(tile_pair[tt] == i);
    units += static_cast<long long>(blk_off[i + 1] - blk_off[i]) * (tile_off[i + 1] - tile_off[i]);
  }
  EXPECT(units == g.U);
  EXPECT(g.grid >= 1 && g.grid <= g.U);

  // the E-step kernel's walk: contiguous unit ranges per CTA, a new slot at every
  // block boundary and every seg_cap units; every unit once, every slot once
  std::vector<int> slot_block(g.total_slots, -1);
  std::vector<char> seen(g.U, 0);
  for (int c = 0; c < g.grid; ++c) {
    const long long u0 = static_cast<long long>(c) * g.U / g.grid, u1 = static_cast<long long>(c + 1) * g.U / g.grid;
    EXPECT(u1 > u0);
    int b = cta_block[c];
    EXPECT(b >= 0 && b < g.B && unit_off[b] <= u0 && u0 < unit_off[b + 1]);
    int seg = 0;
    for (long long u = u0; u < u1;) {
      while (u >= unit_off[b + 1]) ++b;
      long long e = u + g.seg_cap;
      if (e > unit_off[b + 1]) e = unit_off[b + 1];
      if (e > u1) e = u1;
      for (long long v = u; v < e; ++v) {
        const long long tile = tile_off[block_pair[b]] + (v - unit_off[b]);
        EXPECT(tile >= tile_off[block_pair[b]] && tile < tile_off[block_pair[b] + 1]);
        EXPECT(!seen[v]);
        seen[v] = 1;
      }
      const int slot = cta_slot[c] + seg;
      EXPECT(slot < cta_slot[c + 1] && slot_block[slot] == -1);
      if (slot < g.total_slots) slot_block[slot] = b;
      ++seg;
      u = e;
    }
    EXPECT(cta_slot[c] + seg == cta_slot[c + 1]);
  }
  for (long long v = 0; v < g.U; ++v) EXPECT(seen[v]);
  EXPECT(cta_slot[g.grid] == g.total_slots);
  // the combine reads each block's slots as one contiguous range
  for (int b = 0; b < g.B; ++b) {
    const int first = block_slot[2 * b], count = block_slot[2 * b + 1];
    EXPECT(count >= 1 && first >= 0 && first + count <= g.total_slots);
    for (int s = first; s < first + count && s < g.total_slots; ++s) EXPECT(slot_block[s] == b);
  }
  for (int s = 0; s < g.total_slots; ++s) EXPECT(slot_block[s] >= 0);
  EXPECT(g.combine_ctas == g.B * (g.SB / lsg::kCombineSources));
  EXPECT(lsg::estep_partial_floats(g) == static_cast<size_t>(g.total_slots) * lsg::kMom * g.SB);
  // statistics chunks cover the largest padded source range and target range of a pair
  const long long chunks = lsg::stats_chunks(g);
  EXPECT(chunks * 512 >= g.max_m && chunks * 512 >= static_cast<long long>(g.max_blocks) * g.SB);
  // grid kNN: the cell range of pair i, [4 m_off[i] + 64 i, 4 m_off[i+1] + 64 (i+1)), holds 4 M_i + 64 cells
  long long mtot = 0;
  for (long long m : M) mtot += m;
  EXPECT(lsg::knn_grid_cells(mtot, P) == 4 * plan.off64[2 * P + 1] + 64LL * P);
}

}  // namespace

int main() {
  std::mt19937_64 rng(20210000);
  int cases = 0;
  for (int sms : {152, 148, 7, 1}) {
    for (int S : {0, 1, 2, 4}) {
      for (int it = 0; it < 40; ++it) {
        const int P = 1 + static_cast<int>(rng() % (it < 15 ? 3 : 300));
        std::vector<long long> N(P), M(P);
        auto pick = [&]() -> long long {
          switch (rng() % 6) {
            case 0: return 1 + static_cast<long long>(rng() % 3);
            case 1: return 127 + static_cast<long long>(rng() % 4);
            case 2: return 1023 + static_cast<long long>(rng() % 3);
            default: return 1 + static_cast<long long>(rng() % 20000);
          }
        };
        for (int i = 0; i < P; ++i) {
          N[i] = pick();
          M[i] = pick();
        }
        check_plan(N, M, sms, S);
        ++cases;
      }
      check_plan({20000}, {20000}, sms, S);
      check_plan({1}, {1}, sms, S);
      check_plan({500000}, {500000}, sms, S);
      cases += 3;
    }
  }
  // 4 sources per thread (the tensor-core kernel's tile) with shorter segments
  for (int trial = 0; trial < 40; ++trial) {
    const int P = 1 + static_cast<int>(rng() % 300);
    std::vector<long long> N(P), M(P);
    for (int i = 0; i < P; ++i) {
      N[i] = 1 + static_cast<long long>(rng() % 30000);
      M[i] = 1 + static_cast<long long>(rng() % 30000);
    }
    check_plan(N, M, 152, 4, 16);
    ++cases;
  }
  check_plan({500000}, {500000}, 152, 4, 16);
  ++cases;
  // the size limit of the 32-bit tables: 2^30 units with one source per thread (128-source blocks)
  EXPECT(lsg::plan_fits({4000000}, {4000000}));
  EXPECT(lsg::plan_fits({4194304}, {4194304}));  // 32768 blocks x 32768 tiles = 2^30 units
  EXPECT(!lsg::plan_fits({4194305}, {4194304}));
  EXPECT(!lsg::plan_fits({4194304}, {4194305}));
  EXPECT(!lsg::plan_fits({4000000, 4000000}, {4000000, 4000000}));
  EXPECT(!lsg::plan_fits({0}, {10}));
  EXPECT(!lsg::plan_fits({10}, {0}));
  {
    const lsg::BatchPlan big = lsg::plan_batch({4194304}, {4194304}, 152, 1);
    EXPECT(big.g.U == lsg::kMaxPlanUnits);
    EXPECT(big.g.total_slots > 0 && big.g.grid == 152);
  }
  std::printf("%d plans checked, %d failures\n", cases, failures);
  return failures != 0;
}
