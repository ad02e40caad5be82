// Windowed passes of the ring XY mixer on the Hamming-weight subspace F_k (states in rank
// order, as in xy.cu).  Everything here compiles for the device and for the host, so the
// tile addressing can be checked exhaustively on the CPU (tests/xy_window_check.cpp).
//
// A window is a run of w consecutive qubits [lo, lo + w).  A state z of F_k splits into the
// bits below the window (L, popcount kL), in it (P, popcount kw) and above it (H, popcount
// h).  The rank of z is the sum over its set bits c_1 < ... < c_k of binom(c_i, i), so
//   rank(z) = rank(L) + sum_j binom(lo + p_j, kL + j) + sum_j binom(lo + w + q_j, kL + kw + j)
// with p_j, q_j the positions (inside P and H) of their j-th set bit, j = 1, 2, ..., and
// rank(L) running over 0 .. binom(lo, kL) - 1 in the order of L.  A pair gate on two qubits
// of the window keeps L, H and popcount(P).  So for a class (h, kw) every column (H, L)
// holds the binom(w, kw) patterns P of popcount kw ("rows"), every gate of the window acts
// inside columns, and element (row r, column c) sits at rank rowoff[r] + colbase[c]:
//   rowoff[r]  = sum_j binom(lo + p_j, kL + j), P the r-th pattern of popcount kw,
//   colbase[c] = rank(L) + sum_j binom(lo + w + q_j, kL + kw + j).
// Columns are ordered H-major (H by its rank among the patterns of nh = n - lo - w bits with
// popcount h) and rank(L)-minor, so a row of a tile reads runs of consecutive ranks.  A tile
// is up to m consecutive columns of one class.  Classes with kw = 0 or kw = w have a single
// row that no gate of the window changes; only a pass that also applies the cost unitary
// (to every amplitude) visits them.
//
// The ring mixer applies the pairs (a, a + 1) with a even, then those with a odd, then the
// closing pair (0, n - 1).  The windows [0, e_0), [e_0 - 1, e_1), [e_1 - 1, e_2), ... (every
// e_i even except the last, e_last = n) share one qubit with their neighbour, so every pair
// (a, a + 1) lies in exactly one window.  A window applies its even pairs, then its odd
// pairs; pairs of different windows either commute or come in the order of the sets (an odd
// pair that crosses e_i - 1 needs the even pair (e_i, e_i + 1), which its own window applies
// first).  The closing pair is a pass of its own.
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define XYW_HD __host__ __device__ __forceinline__
#else
#define XYW_HD inline
#endif

namespace qaoa {
namespace xyw {

constexpr int kMaxN = 40;                                // qubits (QAOA_XY_MAX_N)
constexpr int kBN = kMaxN + 1;                           // binomial table side
constexpr int kMaxW = 9;                                 // qubits per window
constexpr int kMaxRows = 126;                            // binom(9, 4)
constexpr int kMaxPairs = 35;                            // binom(7, 3): rows one gate moves
constexpr int kMaxCols = 512;                            // columns per tile
constexpr int kMaxGates = kMaxW - 1;                     // pairs inside one window
constexpr int kMaxClasses = (kMaxN - 1) * (kMaxW + 1);  // h = 0..nh <= n - 2, kw = 0..w
constexpr int kMaxWindows = (kMaxN + 6) / 8 + 1;         // [0, 8), then 8 new qubits per window

typedef unsigned long long u64;

struct Class {
  u64 first_tile;  // tiles of the classes before this one
  u64 ncols;       // binom(nh, h) * len
  u64 len;         // binom(lo, kL): ranks per row run of one H
  int h, kw, kL;   // popcounts above, inside and below the window
  int rows, m;     // binom(w, kw); columns per tile
};

struct Window {
  int n, k, lo, w, nh;
  int ngates;
  int ga[kMaxGates];  // window-relative low qubit of each pair (lo + ga, lo + ga + 1), in order
  int ncls;
  int tile_elems;     // largest rows * m over the classes
  u64 tiles;
  u64 elems;          // amplitudes visited by one pass
  Class cls[kMaxClasses];
};

XYW_HD int ctz64(u64 x) {
#ifdef __CUDA_ARCH__
  return __ffsll((long long)x) - 1;
#else
  return __builtin_ctzll(x);
#endif
}
XYW_HD int popc32(unsigned x) {
#ifdef __CUDA_ARCH__
  return __popc(x);
#else
  return __builtin_popcount(x);
#endif
}

// the pattern of nb bits with popcount kk whose rank among those patterns (increasing order)
// is r, r < binom(nb, kk): the i-th set bit is the largest c with binom(c, i) <= r
XYW_HD u64 unrank_bits(u64 r, int nb, int kk, const u64 (*B)[kBN]) {
  u64 z = 0;
  int c = nb - 1;
  for (int i = kk; i >= 1; --i) {
    while (B[c][i] > r) --c;
    z |= 1ull << c;
    r -= B[c][i];
    --c;
  }
  return z;
}

// sum over the set bits of x (j = 1, 2, ... in increasing order) of binom(base + pos, first + j)
XYW_HD u64 rank_part(u64 x, int base, int first, const u64 (*B)[kBN]) {
  u64 s = 0;
  for (int j = first + 1; x != 0; ++j) {
    s += B[base + ctz64(x)][j];
    x &= x - 1;
  }
  return s;
}

// rank of the first element of column `col` of class C, without the row's part
XYW_HD u64 col_base(const Window& W, const Class& C, u64 col, const u64 (*B)[kBN]) {
  const u64 hi = col / C.len, l = col - hi * C.len;
  const u64 H = unrank_bits(hi, W.nh, C.h, B);
  return l + rank_part(H, W.lo + W.w, C.kL + C.kw, B);
}

// the row of pattern P moved by the pair at window bits (ga, ga + 1): P has bit ga set and
// bit ga + 1 clear, and moving its (j + 1)-th set bit up by one adds binom(ga, j) to its rank
XYW_HD int partner_row(int r, unsigned P, int ga, const u64 (*B)[kBN]) {
  return r + (int)B[ga][popc32(P & ((1u << ga) - 1u))];
}

// x / d for x, d < 2^16 as a multiply-high by m = floor(2^32 / d) + 1 (d >= 2): exact,
// because x (m d - 2^32) <= x d < 2^32; m = 0 stands for d = 1
XYW_HD unsigned div_magic(unsigned d) { return d < 2 ? 0u : (unsigned)((1ull << 32) / d + 1); }
XYW_HD unsigned div_small(unsigned x, unsigned m) {
  if (m == 0) return x;
#ifdef __CUDA_ARCH__
  return __umulhi(x, m);
#else
  return (unsigned)(((u64)x * m) >> 32);
#endif
}

XYW_HD int find_class(const Window& W, u64 tile) {
  int a = 0, b = W.ncls - 1;
  while (a < b) {
    const int mid = (a + b + 1) / 2;
    if (W.cls[mid].first_tile <= tile) a = mid;
    else b = mid - 1;
  }
  return a;
}

// Pascal's triangle up to kMaxN
XYW_HD void binom_row(u64 (*B)[kBN], int c) {
  u64 v = 1;
  for (int i = 0; i < kBN; ++i) {
    B[c][i] = i <= c ? v : 0;
    v = i < c ? v * (u64)(c - i) / (u64)(i + 1) : 0;  // binom(c, i + 1), exact
  }
}

// ---------------------------------------------------------------- host planning

// The windows of the ring mixer on n qubits (n >= 2): their [lo, lo + w) ranges.
inline int plan_ring_windows(int n, int* lo, int* w) {
  if (n < 2) return 0;
  int nw = 0;
  int e = n <= kMaxW ? n : kMaxW - 1;  // the first window ends at an even bit unless it is the last
  lo[nw] = 0;
  w[nw++] = e;
  while (e < n) {
    const int s = e - 1;
    e = s + kMaxW < n ? s + kMaxW : n;  // s is odd, so s + kMaxW is even
    lo[nw] = s;
    w[nw++] = e - s;
  }
  return nw;
}

// Window [lo, lo + w) of the ring mixer on n qubits: its pairs and its tile classes.
// `target` = amplitudes per tile (per buffer); `every_state` also visits the single-row
// classes (kw = 0, kw = w), for a pass that applies the cost unitary to every amplitude.
inline void plan_window(Window& W, int n, int k, int lo, int w, int target, const u64 (*B)[kBN],
                        bool every_state = false) {
  W.n = n;
  W.k = k;
  W.lo = lo;
  W.w = w;
  W.nh = n - lo - w;
  W.ngates = 0;
  for (int par = 0; par < 2; ++par)  // even pairs, then odd pairs
    for (int a = lo; a + 1 < lo + w; ++a)
      if ((a & 1) == par) W.ga[W.ngates++] = a - lo;
  W.ncls = 0;
  W.tiles = 0;
  W.elems = 0;
  W.tile_elems = 0;
  for (int h = 0; h <= W.nh; ++h) {
    for (int kw = every_state ? 0 : 1; kw <= (every_state ? w : w - 1); ++kw) {
      const int kL = k - h - kw;
      if (kL < 0 || kL > lo) continue;
      Class& C = W.cls[W.ncls++];
      C.h = h;
      C.kw = kw;
      C.kL = kL;
      C.rows = (int)B[w][kw];
      C.len = B[lo][kL];
      C.ncols = B[W.nh][h] * C.len;
      u64 m = (u64)(target / C.rows);
      if (m < 1) m = 1;
      if (m > (u64)kMaxCols) m = kMaxCols;
      if (m > C.ncols) m = C.ncols;
      C.m = (int)m;
      C.first_tile = W.tiles;
      W.tiles += (C.ncols + m - 1) / m;
      W.elems += C.ncols * (u64)C.rows;
      if (C.rows * C.m > W.tile_elems) W.tile_elems = C.rows * C.m;
    }
  }
}

}  // namespace xyw
}  // namespace qaoa
