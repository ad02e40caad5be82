// Exhaustive host check of the tile layouts and exchange barriers in csrc/tile_layout.cuh,
// for every layout configuration the sweep and batch kernels instantiate and a few more.
// A move between layouts F and T writes each thread's values at the slots of its local
// indices in layout F and reads them back at the slots of its indices in layout T, with one
// barrier between (kind 0 = warp, 1 = block, 2 = named barrier).  Checked here:
//  * every layout is a bijection of (thread, register) onto the 2^B local indices, and the
//    slot map phys is a bijection of the local indices;
//  * every value a thread reads was written by a thread of the same barrier set;
//  * every named barrier id lies in 1..15 and joins, in every move that uses it, the same
//    warps with a count of 32 times their number.
// Exit 0 = all good.
#include <cstdio>
#include <map>
#include <set>
#include <vector>

#include "tile_layout.cuh"

using namespace qaoa;

static int fails = 0;

template <class CF>
static void check(const char* name) {
  const int NT = CF::NT, R = CF::R, N = 1 << CF::B;
  // owner[k][i] = thread holding local index i in layout k
  std::vector<std::vector<int>> owner(CF::NR, std::vector<int>(N, -1));
  for (int k = 0; k < CF::NR; ++k) {
    for (int t = 0; t < NT; ++t)
      for (int r = 0; r < R; ++r) {
        const uint32_t i = CF::idx(k, (uint32_t)t, r);
        if (i >= (uint32_t)N || owner[k][i] != -1) {
          if (fails++ < 10) printf("%s: layout %d is not a bijection\n", name, k);
          return;
        }
        owner[k][i] = t;
      }
  }
  std::vector<int> seen(N, 0);
  for (int i = 0; i < N; ++i) {
    const uint32_t p = CF::phys((uint32_t)i);
    if (p >= (uint32_t)N || seen[p]++) {
      if (fails++ < 10) printf("%s: phys is not a bijection\n", name);
      return;
    }
  }
  // id -> (warp set, count) over all moves
  std::map<uint32_t, std::pair<std::set<int>, uint32_t>> ids;
  for (int F = 0; F < CF::NR; ++F)
    for (int T = 0; T < CF::NR; ++T) {
      if (F == T) continue;
      const int kind = CF::move_sync(F, T);
      std::map<uint32_t, std::set<int>> members;  // this move's named barriers
      for (int i = 0; i < N; ++i) {
        const int wr = owner[F][i], rd = owner[T][i];
        bool ok = true;
        if (kind == 0) ok = (wr >> 5) == (rd >> 5);
        if (kind == 2) ok = CF::bar_id(F, T, (uint32_t)(wr >> 5)) == CF::bar_id(F, T, (uint32_t)(rd >> 5));
        if (!ok && fails++ < 10) printf("%s: move %d -> %d crosses its barrier set at index %d\n", name, F, T, i);
      }
      if (kind != 2) continue;
      for (int w = 0; w < NT / 32; ++w) members[CF::bar_id(F, T, (uint32_t)w)].insert(w);
      for (auto& m : members) {
        const uint32_t id = m.first, cnt = CF::bar_count(F, T);
        if (id < 1 || id > 15 || cnt != 32u * m.second.size()) {
          if (fails++ < 10) printf("%s: move %d -> %d barrier %u count %u for %zu warps\n", name, F, T, id, cnt,
                                   m.second.size());
        }
        auto it = ids.find(id);
        if (it == ids.end()) {
          ids[id] = {m.second, cnt};
        } else if (it->second.first != m.second || it->second.second != cnt) {
          if (fails++ < 10) printf("%s: barrier %u joins different warps in different moves\n", name, id);
        }
      }
    }
  printf("%s: %d layouts, %zu named barriers\n", name, CF::NR, ids.size());
}

int main() {
  // the kernels' configurations, as the test harness reads them from the sources
#if __has_include("exchange_cfgs.inc")
#include "exchange_cfgs.inc"
#endif
  check<Cfg<13, 5, 5, 4, 2>>("complex64 single buffer");
  check<Cfg<13, 4, 4, 4, 1>>("complex64 two buffers");
  check<Cfg<13, 5, 5, 4, 1>>("8192-amplitude tiles, 5 register bits, one block");
  check<Cfg<12, 4, 4, 3, 2>>("complex128 single buffer");
  check<Cfg<12, 3, 3, 3, 1>>("complex128 two buffers");
  check<Cfg<10, 3, 3, 3, 2>>("batched complex128, 2^10 tiles");
  check<Cfg<12, 4, 4, 4, 2>>("batched complex64");
  check<Cfg<10, 3, 3, 4, 2>>("batched complex64, 2^10 tiles");
  check<Cfg<13, 3, 3, 3, 1>>("1024 threads, 3 register bits");
  check<Cfg<11, 2, 2, 2, 1>>("512 threads, 2 register bits");
  check<Cfg<9, 4, 4, 4, 1>>("one warp");
  printf(fails ? "FAIL %d\n" : "OK\n", fails);
  return fails ? 1 : 0;
}
