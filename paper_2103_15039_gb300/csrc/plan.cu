// Batch planner of the E step (host code): source blocks, target tiles, the
// stream-K split of (source block x target tile) units over the E-step grid,
// and the partial-slot tables that the E-step kernels and the combine share.
#include "internal.cuh"

namespace lsg {

bool plan_fits(const std::vector<long long>& N, const std::vector<long long>& M) {
  // the tables index (source block x target tile) units, blocks and tiles with 32-bit ints;
  // the smallest source block (one source per thread) gives the most units
  const long long SB = estep_warps(1) * 32LL;
  long long U = 0, T = 0;
  for (size_t i = 0; i < N.size(); ++i) {
    if (N[i] < 1 || M[i] < 1 || N[i] > kMaxPlanUnits * SB || M[i] > kMaxPlanUnits * kTile) return false;
    const long long tiles = (M[i] + kTile - 1) / kTile;
    U += ((N[i] + SB - 1) / SB) * tiles;
    T += tiles;
    if (U > kMaxPlanUnits || T > kMaxPlanUnits) return false;
  }
  return true;
}

BatchPlan plan_batch(const std::vector<long long>& N, const std::vector<long long>& M, int num_sms,
                     int S_override, int seg_cap) {
  BatchPlan p{};
  Geo& g = p.g;
  const int P = static_cast<int>(N.size());
  g.P = P;
  p.smem_bytes = estep_smem_bytes();
  std::vector<int> tiles(P);
  long long T = 0;
  g.max_n = 0;
  g.max_m = 0;
  g.max_tiles = 0;
  for (int i = 0; i < P; ++i) {
    tiles[i] = static_cast<int>((M[i] + kTile - 1) / kTile);
    T += tiles[i];
    if (N[i] > g.max_n) g.max_n = N[i];
    if (M[i] > g.max_m) g.max_m = M[i];
    if (tiles[i] > g.max_tiles) g.max_tiles = tiles[i];
  }
  g.T = static_cast<int>(T);
  auto units_for = [&](int S) {
    const int SB = estep_warps(S) * 32 * S;
    long long U = 0;
    for (int i = 0; i < P; ++i) U += ((N[i] + SB - 1) / SB) * static_cast<long long>(tiles[i]);
    return U;
  };
  int chosen = 1;
  if (S_override == 1 || S_override == 2 || S_override == 4) {
    chosen = S_override;
  } else {
    const int cands[3] = {4, 2, 1};
    for (int c : cands) {
      // enough units for a balanced grid, and not much padding per pair
      const int SB = estep_warps(c) * 32 * c;
      long long pad = 0, tot = 0;
      for (int i = 0; i < P; ++i) {
        pad += ((N[i] + SB - 1) / SB) * SB - N[i];
        tot += N[i];
      }
      if (units_for(c) >= 4LL * num_sms * estep_resident_ctas(c) && pad * 20 <= tot) {
        chosen = c;
        break;
      }
    }
  }
  g.S = chosen;
  g.SB = estep_warps(chosen) * 32 * chosen;
  g.seg_cap = seg_cap;
  // pair tables
  std::vector<int> blk_off(P + 1, 0), tile_off(P + 1, 0);
  g.max_blocks = 0;
  for (int i = 0; i < P; ++i) {
    const int nb = static_cast<int>((N[i] + g.SB - 1) / g.SB);
    blk_off[i + 1] = blk_off[i] + nb;
    tile_off[i + 1] = tile_off[i] + tiles[i];
    if (nb > g.max_blocks) g.max_blocks = nb;
  }
  g.B = blk_off[P];
  std::vector<int> block_pair(g.B), unit_off(g.B + 1, 0);
  for (int i = 0; i < P; ++i)
    for (int b = blk_off[i]; b < blk_off[i + 1]; ++b) {
      block_pair[b] = i;
      unit_off[b + 1] = unit_off[b] + tiles[i];
    }
  g.U = unit_off[g.B];
  const long long slots = static_cast<long long>(num_sms) * estep_resident_ctas(chosen);
  g.grid = static_cast<int>(g.U < slots ? g.U : slots);
  // slot table: replay the kernel's segmentation (same rules, host side)
  std::vector<int> cta_slot(g.grid + 1, 0), cta_block(g.grid, 0), first(g.B, -1), count(g.B, 0);
  int slot = 0;
  int b = 0;
  for (int c = 0; c < g.grid; ++c) {
    cta_slot[c] = slot;
    const long long u0 = static_cast<long long>(c) * g.U / g.grid;
    const long long u1 = static_cast<long long>(c + 1) * g.U / g.grid;
    while (u0 >= unit_off[b + 1]) ++b;
    cta_block[c] = b;
    long long u = u0;
    int bb = b;
    while (u < u1) {
      while (u >= unit_off[bb + 1]) ++bb;
      long long e = u + g.seg_cap;
      if (e > unit_off[bb + 1]) e = unit_off[bb + 1];
      if (e > u1) e = u1;
      if (first[bb] < 0) first[bb] = slot;
      ++count[bb];
      ++slot;
      u = e;
    }
  }
  cta_slot[g.grid] = slot;
  g.total_slots = slot;
  g.combine_ctas = g.B * (g.SB / kCombineSources);
  // pack the device table
  auto& t = p.tab;
  t.clear();
  auto put = [&](const std::vector<int>& v) {
    const int o = static_cast<int>(t.size());
    t.insert(t.end(), v.begin(), v.end());
    return o;
  };
  g.o_blk_off = put(blk_off);
  g.o_tile_off = put(tile_off);
  g.o_block_pair = put(block_pair);
  g.o_unit_off = put(unit_off);
  g.o_cta_slot = put(cta_slot);
  g.o_cta_block = put(cta_block);
  std::vector<int> bs(2 * static_cast<size_t>(g.B));
  for (int q = 0; q < g.B; ++q) {
    bs[2 * q] = first[q];
    bs[2 * q + 1] = count[q];
  }
  g.o_block_slot = put(bs);
  std::vector<int> tile_pair(g.T);
  for (int i = 0; i < P; ++i)
    for (int t = tile_off[i]; t < tile_off[i + 1]; ++t) tile_pair[t] = i;
  g.o_tile_pair = put(tile_pair);
  p.off64.assign(2 * static_cast<size_t>(P) + 2, 0);
  for (int i = 0; i < P; ++i) {
    p.off64[i + 1] = p.off64[i] + N[i];
    p.off64[P + 1 + i + 1] = p.off64[P + 1 + i] + M[i];
  }
  return p;
}

size_t estep_partial_floats(const Geo& g) { return static_cast<size_t>(g.total_slots) * kMom * g.SB; }

}  // namespace lsg
