// Register/shared-memory tile layouts of the layer sweeps (host-compilable, so the CPU
// tests can check the exchange groups exhaustively).
//
// A tile holds 2^B local amplitudes; each thread holds 2^RB of them in registers.  Layout k
// gives the thread the local bits [lo(k), lo(k) + RB) in its registers, its thread index the
// rest; a qubit is processed while its local bit is a register bit, and the tile moves
// between layouts through a shared exchange area.
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define QAOA_HDC __host__ __device__
#else
#define QAOA_HDC
#endif

namespace qaoa {

template <int B_, int RB_, int SW_, int SWW_, int MINB_>
struct Cfg {
  static constexpr int MINB = MINB_;        // blocks per SM the register budget is sized for
  static constexpr int B = B_;              // tile bits
  static constexpr int RB = RB_;            // register bits per layout
  static constexpr int R = 1 << RB_;        // amplitudes per thread (per buffer)
  static constexpr int NT = 1 << (B_ - RB_);  // threads per block
  static constexpr int NR = (B_ + RB_ - 1) / RB_;  // layouts (rounds)
  QAOA_HDC static constexpr int lo(int k) {
    const int v = B - RB * (k + 1);
    return v < 0 ? 0 : v;
  }
  // first local bit of round k that no earlier round covers: round k processes
  // [lo(k), newhi(k)) where newhi(0) = B and newhi(k) = lo(k - 1)
  QAOA_HDC static constexpr int newhi(int k) { return k == 0 ? B : lo(k - 1); }
  QAOA_HDC static constexpr uint32_t idx(int k, uint32_t tid, int r) {
    const int l = lo(k);
    return (tid & ((1u << l) - 1)) | ((uint32_t)r << l) | ((tid >> l) << (l + RB));
  }
  // shared-memory slot of local index i: XOR-fold higher bits into the bank bits
  QAOA_HDC static constexpr uint32_t phys(uint32_t i) { return i ^ ((i >> SW_) & ((1u << SWW_) - 1)); }

  // Exchange groups.  Thread bit b stands for local bit b in a layout with lo(k) > b and for
  // bit b + RB otherwise, so in a move between layouts F and T a thread's values go only to
  // threads that differ from it in the thread bits [min(lo F, lo T), max(lo F, lo T)); such
  // a group holds the same local indices (hence the same exchange slots) in both layouts,
  // and one barrier over the group orders the move.  A group inside a warp takes a warp
  // barrier; a move between adjacent layouts k, k + 1 whose groups span some but not all
  // warps takes one named barrier per warp group, ids [bar_base(k), bar_base(k) + groups)
  // disjoint between moves, so each id always joins the same warps with the same count.
  static constexpr int NWB = B_ - RB_ - 5;  // log2 of the warps per block
  QAOA_HDC static constexpr int wlo(int m) { return m > 5 ? m - 5 : 0; }
  // warp groups of the move k <-> k + 1 that need named barriers (0: warp or block barrier)
  QAOA_HDC static constexpr int move_groups(int k) {
    return lo(k) <= 5 ? 0
                      : (wlo(lo(k + 1)) == 0 && lo(k) - 5 >= NWB ? 0 : 1 << (NWB - (lo(k) - 5 - wlo(lo(k + 1)))));
  }
  QAOA_HDC static constexpr int bar_base(int k) { return k == 0 ? 1 : bar_base(k - 1) + move_groups(k - 1); }
  // barrier of the move F <-> T: 0 = warp, 1 = block, 2 = named barrier of the warp's group
  QAOA_HDC static constexpr int mlo(int F, int T) { return lo(F) < lo(T) ? lo(F) : lo(T); }
  QAOA_HDC static constexpr int mhi(int F, int T) { return lo(F) < lo(T) ? lo(T) : lo(F); }
  QAOA_HDC static constexpr int move_sync(int F, int T) {
    return mhi(F, T) <= 5 ? 0 : ((F - T != 1 && T - F != 1) || move_groups(F < T ? F : T) == 0) ? 1 : 2;
  }
  QAOA_HDC static constexpr uint32_t bar_id(int F, int T, uint32_t warp) {
    return (uint32_t)bar_base(F < T ? F : T) +
           ((warp & ((1u << wlo(mlo(F, T))) - 1)) | ((warp >> (mhi(F, T) - 5)) << wlo(mlo(F, T))));
  }
  QAOA_HDC static constexpr uint32_t bar_count(int F, int T) {
    return 32u << (mhi(F, T) - 5 - wlo(mlo(F, T)));
  }
  static_assert(NWB >= 0, "a block holds whole warps");
  static_assert(bar_base(NR - 1) <= 16, "named barrier ids 1..15");
};

}  // namespace qaoa
