// Host check of the windowed XY-mixer passes (paper_2407_13012_gb300/csrc/xy_window.cuh):
//  * the multiply-high division of the tile index arithmetic is exact;
//  * the windows' pairs plus the closing pair are the ring pairs, each exactly once, and
//    every odd pair comes after the even pairs it shares a qubit with;
//  * for every (n, k) with n <= 16, every tile element's rank is in range, is visited once,
//    and is the state whose bits below / inside / above the window are the column's L, the
//    row's pattern and the column's H; exactly the states whose window popcount lies in
//    1 .. w - 1 are visited (every state, for the pass that carries the cost unitary);
//  * a pair's partner row is the row of the pattern with that set bit moved up by one;
//  * for n up to 40 the class tables count the right states and sampled tiles address
//    states of the right shape; every size stays inside the kernel's fixed arrays.
// The states of F_k are enumerated here by brute force (small n) or unranked by a plain
// search (large n), independently of the header's functions.  Exit 0 = all good.
#include <cstdio>
#include <cstdlib>
#include <set>
#include <vector>

#include "xy_window.cuh"

using namespace qaoa::xyw;

static int fails = 0;
#define CHECK(c, ...)                   \
  do {                                  \
    if (!(c)) {                         \
      if (fails < 20) {                 \
        std::printf("FAIL: " __VA_ARGS__); \
        std::printf("\n");              \
      }                                 \
      ++fails;                          \
    }                                   \
  } while (0)

static u64 Bt[kBN][kBN];

static u64 binom(int c, int i) {
  if (i < 0 || i > c) return 0;
  u64 v = 1;
  for (int j = 1; j <= i; ++j) v = v * (u64)(c - i + j) / (u64)j;
  return v;
}

// z of rank r in F_k by walking bits from the top: bit c is set when the states below it
// (binom(c, i) of them with i bits left) do not reach r
static u64 unrank_search(u64 r, int n, int k) {
  u64 z = 0;
  int i = k;
  for (int c = n - 1; c >= 0 && i > 0; --c) {
    const u64 below = binom(c, i);
    if (r >= below) {
      z |= 1ull << c;
      r -= below;
      --i;
    }
  }
  return z;
}

static int popc(u64 x) { return __builtin_popcountll(x); }

// rank of the low `lo` bits of z among the lo-bit patterns of the same popcount
static u64 low_rank(u64 z, int lo) {
  const u64 L = lo >= 64 ? z : (z & ((1ull << lo) - 1));
  u64 r = 0;
  int i = 0;
  for (int c = 0; c < lo; ++c)
    if ((L >> c) & 1) r += binom(c, ++i);
  return r;
}

static void check_windows(int n) {
  int lo[kMaxWindows + 1], w[kMaxWindows + 1];
  const int nw = plan_ring_windows(n, lo, w);
  CHECK(nw >= 1 && nw <= kMaxWindows, "n=%d windows %d", n, nw);
  CHECK(lo[0] == 0 && lo[nw - 1] + w[nw - 1] == n, "n=%d window cover", n);
  for (int i = 0; i < nw; ++i) {
    CHECK(w[i] >= 2 && w[i] <= kMaxW, "n=%d window %d width %d", n, i, w[i]);
    if (i > 0) CHECK(lo[i] == lo[i - 1] + w[i - 1] - 1, "n=%d window %d overlap", n, i);
    if (i + 1 < nw) CHECK(((lo[i] + w[i]) & 1) == 0, "n=%d window %d ends at odd bit", n, i);
  }
  // application position of every pair (a, a + 1): window index, then index in the window
  std::vector<int> pos(n, -1);
  int order = 0;
  for (int i = 0; i < nw; ++i) {
    Window W;
    plan_window(W, n, n / 2, lo[i], w[i], 2048, Bt);
    CHECK(W.ngates <= kMaxGates, "n=%d gates", n);
    int prev_par = 0;
    for (int g = 0; g < W.ngates; ++g) {
      const int a = lo[i] + W.ga[g];
      CHECK(W.ga[g] >= 0 && W.ga[g] + 1 < w[i], "n=%d pair out of window", n);
      CHECK(a + 1 < n, "n=%d pair past n", n);
      CHECK(pos[a] < 0, "n=%d pair %d twice", n, a);
      CHECK((a & 1) >= prev_par, "n=%d odd pair before even pair in a window", n);
      prev_par = a & 1;
      pos[a] = order++;
    }
  }
  for (int a = 0; a + 1 < n; ++a) CHECK(pos[a] >= 0, "n=%d pair %d missing", n, a);
  // ring parity order: odd pair (a, a+1) after the even pairs (a-1, a) and (a+1, a+2)
  for (int a = 1; a + 1 < n; a += 2) {
    if (a - 1 >= 0) CHECK(pos[a - 1] < pos[a], "n=%d pair %d before %d", n, a, a - 1);
    if (a + 2 < n) CHECK(pos[a + 1] < pos[a], "n=%d pair %d before %d", n, a, a + 1);
  }
}

// every element of every tile of window [lo, lo + w) for (n, k), against brute force
static void check_tiles_exhaustive(int n, int k, int lo, int w, int target, bool every) {
  Window W;
  plan_window(W, n, k, lo, w, target, Bt, every);
  std::vector<u64> states;
  for (u64 z = 0; z < (1ull << n); ++z)
    if (popc(z) == k) states.push_back(z);
  const u64 D = states.size();
  std::vector<int> seen(D, 0);
  CHECK(W.ncls <= kMaxClasses, "classes");
  u64 elems = 0;
  for (u64 tile = 0; tile < W.tiles; ++tile) {
    const int ci = find_class(W, tile);
    const Class& C = W.cls[ci];
    CHECK(tile >= C.first_tile && (ci + 1 == W.ncls || tile < W.cls[ci + 1].first_tile), "find_class");
    CHECK(C.rows <= kMaxRows && C.m <= kMaxCols && C.m >= 1, "class sizes");
    CHECK(C.rows * C.m <= W.tile_elems, "tile_elems");
    const u64 col0 = (tile - C.first_tile) * (u64)C.m;
    CHECK(col0 < C.ncols, "col0");
    const int ncol = (int)((u64)C.m < C.ncols - col0 ? (u64)C.m : C.ncols - col0);
    std::vector<unsigned> pat(C.rows);
    for (int r = 0; r < C.rows; ++r) {
      pat[r] = (unsigned)unrank_bits(r, w, C.kw, Bt);
      CHECK(popc(pat[r]) == C.kw && (pat[r] >> w) == 0, "row pattern");
      if (r > 0) CHECK(pat[r] > pat[r - 1], "row order");
    }
    for (int c = 0; c < ncol; ++c) {
      const u64 col = col0 + c;
      const u64 base = col_base(W, C, col, Bt);
      const u64 hidx = col / C.len, l = col % C.len;
      for (int r = 0; r < C.rows; ++r) {
        const u64 rank = rank_part(pat[r], lo, C.kL, Bt) + base;
        CHECK(rank < D, "rank %llu >= D %llu", rank, D);
        if (rank >= D) continue;
        ++seen[rank];
        ++elems;
        const u64 z = states[rank];
        CHECK(((z >> lo) & ((1ull << w) - 1)) == pat[r], "n=%d k=%d lo=%d: window bits", n, k, lo);
        CHECK(popc(z >> (lo + w)) == C.h, "H popcount");
        CHECK(low_rank(z, lo) == l, "L rank");
        CHECK(popc(lo ? (z & ((1ull << lo) - 1)) : 0) == C.kL, "L popcount");
        // H index: rank of the high pattern among nh-bit patterns of popcount h
        const u64 H = z >> (lo + w);
        u64 hr = 0;
        int i = 0;
        for (int b = 0; b < W.nh; ++b)
          if ((H >> b) & 1) hr += binom(b, ++i);
        CHECK(hr == hidx, "H index");
      }
    }
    // pairs of every gate
    for (int g = 0; g < W.ngates; ++g) {
      const int ga = W.ga[g];
      int np = 0;
      for (int r = 0; r < C.rows; ++r) {
        if (((pat[r] >> ga) & 3u) != 1u) continue;
        ++np;
        const int r2 = partner_row(r, pat[r], ga, Bt);
        CHECK(r2 > r && r2 < C.rows, "partner range");
        if (r2 < C.rows) CHECK(pat[r2] == (pat[r] ^ (3u << ga)), "partner pattern");
      }
      CHECK((C.rows == 1 ? np == 0 : np >= 1) && np <= kMaxPairs, "pairs per gate %d", np);
    }
  }
  CHECK(elems == W.elems, "elems count");
  for (u64 rk = 0; rk < D; ++rk) {
    const int kw = popc((states[rk] >> lo) & ((1ull << w) - 1));
    const int want = (every || (kw >= 1 && kw <= w - 1)) ? 1 : 0;
    CHECK(seen[rk] == want, "n=%d k=%d lo=%d w=%d: rank %llu seen %d want %d", n, k, lo, w, rk, seen[rk], want);
  }
}

// class-table totals and sampled tiles for large n
static void check_tables_large(int n, int k, int target) {
  int lo[kMaxWindows + 1], w[kMaxWindows + 1];
  const int nw = plan_ring_windows(n, lo, w);
  const u64 D = binom(n, k);
  for (int i = 0; i < nw; ++i) {
    Window W;
    plan_window(W, n, k, lo[i], w[i], target, Bt, i == 0);  // the first window carries the cost unitary
    CHECK(W.ncls <= kMaxClasses, "classes");
    CHECK(W.tile_elems <= target, "tile larger than the target");
    u64 want = 0;
    for (int kw = (i == 0 ? 0 : 1); kw <= w[i] - (i == 0 ? 0 : 1); ++kw) want += binom(w[i], kw) * binom(n - w[i], k - kw);
    if (i == 0) CHECK(want == D, "every state");
    CHECK(W.elems == want, "n=%d k=%d window %d: elems %llu want %llu", n, k, i, W.elems, want);
    if (W.tiles == 0) continue;
    const u64 samples[4] = {0, W.tiles / 3, (W.tiles * 2) / 3, W.tiles - 1};
    for (u64 tile : samples) {
      const Class& C = W.cls[find_class(W, tile)];
      CHECK(C.rows <= kMaxRows && C.m <= kMaxCols && C.rows * C.m <= W.tile_elems, "sizes");
      const u64 col0 = (tile - C.first_tile) * (u64)C.m;
      const int ncol = (int)((u64)C.m < C.ncols - col0 ? (u64)C.m : C.ncols - col0);
      for (int c = 0; c < ncol; c += (ncol > 7 ? ncol / 7 : 1)) {
        const u64 base = col_base(W, C, col0 + c, Bt);
        for (int r = 0; r < C.rows; r += (C.rows > 5 ? C.rows / 5 : 1)) {
          const unsigned P = (unsigned)unrank_bits(r, w[i], C.kw, Bt);
          const u64 rank = rank_part(P, lo[i], C.kL, Bt) + base;
          CHECK(rank < D, "large rank");
          if (rank >= D) continue;
          const u64 z = unrank_search(rank, n, k);
          CHECK(popc(z) == k, "large popcount");
          CHECK(((z >> lo[i]) & ((1ull << w[i]) - 1)) == P, "n=%d k=%d: large window bits", n, k);
          CHECK(popc(z >> (lo[i] + w[i])) == C.h, "large H popcount");
          CHECK(low_rank(z, lo[i]) == (col0 + c) % C.len, "large L rank");
        }
      }
    }
  }
}

int main() {
  for (int c = 0; c < kBN; ++c) binom_row(Bt, c);
  for (int c = 0; c < kBN; ++c)
    for (int i = 0; i < kBN; ++i) CHECK(Bt[c][i] == binom(c, i), "binomial table %d %d", c, i);
  for (unsigned d = 1; d < (1u << 16); d += (d < 600 ? 1 : 97))
    for (unsigned x = 0; x < (1u << 16); x += (x < 5000 ? 1 : 31))
      CHECK(div_small(x, div_magic(d)) == x / d, "division %u / %u", x, d);
  for (int n = 2; n <= kMaxN; ++n) check_windows(n);
  for (int n = 2; n <= 16; ++n) {
    int lo[kMaxWindows + 1], w[kMaxWindows + 1];
    const int nw = plan_ring_windows(n, lo, w);
    for (int k = 1; k <= n - 1; ++k)
      for (int i = 0; i < nw; ++i)
        for (int target : {2048, 4096, 40})  // the kernels' tile sizes and a small one (ragged tiles)
          for (bool every : {false, true}) check_tiles_exhaustive(n, k, lo[i], w[i], target, every);
  }
  for (int n : {20, 24, 28, 31, 32, 36, 40})
    for (int k = 1; k <= n - 1; ++k)
      for (int target : {2048, 4096}) check_tables_large(n, k, target);
  if (fails) {
    std::printf("%d failures\n", fails);
    return 1;
  }
  std::printf("OK\n");
  return 0;
}
