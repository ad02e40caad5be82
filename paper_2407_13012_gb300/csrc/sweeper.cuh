// Tile machinery shared by the layer sweeps and the batched kernel: tile layouts, the
// per-tile state (Sweeper) with its phase, mixer, lambda and reduction operations.
//
// A sweep streams every tile of the state once.  A tile holds the 2^t combinations of
// one group of qubits (local bits [c, c + t)) together with the 2^c lowest index bits
// (local bits [0, c), kept for coalesced access); the other index bits are fixed per
// tile.  Each thread holds R = 2^RB amplitudes of the tile in registers.  In "layout" k
// the register index is the local bit range [lo(k), lo(k) + RB) and the thread index
// is the rest, so butterflies on the qubits of that range run in registers; moving
// to the next layout is one swizzled shared-memory exchange.  A sweep runs a short
// program of operations on each tile (phase, mixer, lambda init, reductions) and
// writes the tile back.  The grid is persistent over tiles and every reduction has a
// fixed order, so results are deterministic for a given device.
//
// Arithmetic.
//  * complex64: float32 throughout; the mixer applies RX(2 beta) = cos(b) I - i sin(b) X
//    as one butterfly per qubit.
//  * complex128: the state lives in int64 fixed point with scale 2^S inside a call
//    (GB300 retires ~1.75 float64 FMA per SM clock, 1/73 of its float32 rate, so
//    float64 butterflies would cost ~20x the sweep's memory time).  The mixer on a
//    group of t qubits uses RX(2b)^{(x)t} = H^{(x)t} D H^{(x)t} = 2^-t W D W, where W is
//    the unnormalised Walsh-Hadamard transform on the group (exact integer add/sub
//    butterflies) and D = diag(exp(-i b (t - 2 popcount(g)))) is one complex multiply
//    per amplitude, rounded once.  Phase factors are Q62 fixed point.  Reductions
//    accumulate exact int128 products per thread and per tile and are converted to
//    float64 once per tile.
#pragma once

#include "internal.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>
#include <type_traits>

#include "fixedpoint.cuh"
#include "tile_layout.cuh"

namespace qaoa {
namespace {


// Kernel attributes (the dynamic shared-memory limit) belong to a device: setup() runs once
// per device for each call site, under the site's lock, before that device's first launch.
template <class F>
inline void once_per_device(std::mutex& mu, uint64_t& done, F&& setup) {
  int dev = 0;
  cudaGetDevice(&dev);
  const uint64_t bit = 1ull << (dev & 63);
  std::lock_guard<std::mutex> lk(mu);
  if (!(done & bit)) {
    setup();
    done |= bit;
  }
}

// complex64 single buffer: 8192-amplitude tiles, 32 per thread, 256 threads
using CfgF1 = Cfg<13, 5, 5, 4, 2>;
// complex64 two buffers (gradient) with 8192-amplitude tiles: 16 amplitudes per thread per
// buffer, 512 threads, one block per SM; at n = 32 this keeps >= 3 carried low bits (64-byte
// rows)
using CfgF3 = Cfg<13, 4, 4, 4, 1>;
// complex128 fixed point single buffer: 4096-amplitude tiles, 16 per thread
using CfgX1 = Cfg<12, 4, 4, 3, 2>;
// complex128 fixed point two buffers: 4096-amplitude tiles, 8 per thread per buffer, 512 threads
using CfgX2 = Cfg<12, 3, 3, 3, 1>;

// cost-tile slot of local index i; the XOR leaves the bits inside a 16-byte chunk alone so
// the tile can be fetched with 16-byte asynchronous copies
__device__ __forceinline__ uint32_t phys_cost(uint32_t i, bool f64) {
  return f64 ? (i ^ ((i >> 3) & 14)) : (i ^ ((i >> 3) & 28));
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// all but the newest N committed groups of this thread are complete
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ uint64_t tile_base(const SweepGeom& g, int64_t tile) {
  const int lowrest_bits = g.j0 - g.c;
  const uint64_t lowrest = (uint64_t)tile & ((1ull << lowrest_bits) - 1);
  const uint64_t highrest = (uint64_t)tile >> lowrest_bits;
  return (lowrest << g.c) | (highrest << (g.j0 + g.t));
}

__device__ __forceinline__ uint64_t local_to_z(const SweepGeom& g, uint64_t base, uint32_t i) {
  const uint32_t l = i & ((1u << g.c) - 1);
  const uint64_t q = i >> g.c;
  return base | l | (q << g.j0);
}

// ------------------------------------------------------------------ fixed point helpers

using i128 = __int128;
using fx::round_shift;

// (x * e) / 2^(62 + extra) for a state value x (|re|, |im| < 2^61) and a Q62 unit complex e
__device__ __forceinline__ longlong2 cmul_fx(longlong2 x, longlong2 e, int extra) {
  const fx::C64 o = fx::cmul_q62(x.x, x.y, e.x, e.y, extra);
  return make_longlong2(o.x, o.y);
}
// the same with 128-bit products, for operands up to 2^63 (products of two Q62 factors)
__device__ __forceinline__ longlong2 cmul_fx_wide(longlong2 x, longlong2 e, int extra) {
  const fx::C64 o = fx::cmul_q62_exact(x.x, x.y, e.x, e.y, extra);
  return make_longlong2(o.x, o.y);
}
__device__ __forceinline__ double fx_to_double(long long x, int s) { return fx::to_double(x, s); }
__device__ __forceinline__ double i128_to_double(i128 v, int s) { return fx::i128_to_double(v, s); }
__device__ __forceinline__ long long double_to_fx(double d, int s) { return fx::from_double(d, s); }
__device__ __forceinline__ unsigned long long frac_turns(double d) { return fx::frac_turns(d); }

// exp(-2 pi i th) in float32 for a turn count th (the rare path of float costs or costs
// outside the table); kept out of line so it does not raise the register budget of the
// common path
__device__ __noinline__ float2 phase_f32_direct(double th) {
  const float f = (float)(th - rint(th));
  float s, c;
  sincospif(2.0f * f, &s, &c);
  return make_float2(c, -s);
}

__device__ __forceinline__ longlong2 turn_phase(unsigned long long t, const longlong2* __restrict__ tt);

// exp(-2 pi i th) in Q62 for a turn count th (out of line, like phase_f32_direct)
__device__ __noinline__ longlong2 phase_fx_direct(double th, const longlong2* __restrict__ tt) {
  return turn_phase(frac_turns(th), tt);
}

// exp(-2 pi i t / 2^64) in Q62 from three 1024-entry tables and a first-order residual
__device__ __forceinline__ longlong2 turn_phase(unsigned long long t, const longlong2* __restrict__ tt) {
  const longlong2 e1 = tt[t >> 54];
  const longlong2 e2 = tt[1024 + ((t >> 44) & 1023)];
  const longlong2 e3 = tt[2048 + ((t >> 34) & 1023)];
  longlong2 e = cmul_fx_wide(e1, e2, 0);
  e = cmul_fx_wide(e, e3, 0);
  // residual angle rho = 2 pi r 2^-64 < 2 pi 2^-30; exp(-i rho) = 1 - i rho to 2e-17
  const unsigned long long r = t & ((1ull << 34) - 1);
  const long long rho = (long long)(((r >> 2) * 3373259426ull) >> 29);  // rho * 2^62, 3373259426 = round(pi/2 2^31)
  const long long dre = round_shift((i128)rho * e.y, 62);
  const long long dim = round_shift((i128)rho * e.x, 62);
  return make_longlong2(e.x + dre, e.y - dim);
}

// ------------------------------------------------------------------ kernel

// per-layer angle terms: kernel parameters, or device memory ([g2pi p | cos p | sin p],
// written by angle_prep_kernel) when the angles live on the device
__device__ __forceinline__ double arg_g2pi(const SweepArgs& a, const double* trig, int l) {
  return trig ? trig[l] : a.g2pi[l];
}
__device__ __forceinline__ double arg_cosb(const SweepArgs& a, const double* trig, int l) {
  return trig ? trig[a.np + l] : a.cosb[l];
}
__device__ __forceinline__ double arg_sinb(const SweepArgs& a, const double* trig, int l) {
  return trig ? trig[2 * a.np + l] : a.sinb[l];
}

__device__ __forceinline__ double cost_f(const void* Cs, bool f64, uint32_t i) {
  return f64 ? ((const double*)Cs)[phys_cost(i, true)] : (double)((const int*)Cs)[phys_cost(i, false)];
}
__device__ __forceinline__ int cost_i(const void* Cs, uint32_t i) { return ((const int*)Cs)[phys_cost(i, false)]; }

template <class CF, bool FX, bool TWO>
struct Sweeper {
  using V = typename std::conditional<FX, longlong2, float2>::type;
  static constexpr int R = CF::R;

  const SweepArgs& a;
  V v[R];        // register tile of psi (layout cur)
  V w[R];        // register tile of lambda (two-buffer sweeps)
  V* X;          // exchange buffer, 2^B slots (2 x 2^B for two-buffer sweeps: psi, then lambda)
  V* Ps = nullptr;  // lean two-buffer sweeps: psi of the next tile, 2^B slots (or nullptr)
  void* Cs;      // cost tile, 2^B slots
  const V* Ts;   // shared-memory copy of one layer's phase table (or nullptr); float32 states
  const fx::Factor* Tf;  // the same for fixed-point states, as prepared factors
  fx::Factor* Ds;  // shared-memory mixer diagonal of the current fixed-point mixer (<= 14 entries)
  int ts_layer;  // layer whose table Ts holds (-1: none)
  double* blk;   // block accumulators
  double* wacc = nullptr;  // per-warp accumulators [kLeanAcc][NT / 32], if set (lean sweeps)
  double* red;   // reduction scratch [2][NT/32]
  int cur;       // current layout
  int lam_shift;  // lambda scale exponent (fixed point)
  int in_shift;   // extra input scale exponent of a user state (fixed point)
  uint32_t evalid;
  uint64_t base;
  const uint32_t tid;
  // the graph's data: a's, or one graph's of a grouped sweep (lean kernels)
  int64_t zoff;          // element offset of psi, lambda and C
  const void* ptab;      // phase tables
  int64_t pcmin, pspan;  // their integer cost range
  const double* trig;    // per-layer angle terms in device memory, or nullptr (kernel parameters)
  const void* dtab;      // fixed point: mixer diagonals

  __device__ Sweeper(const SweepArgs& a_, V* X_, void* Cs_, double* blk_, double* red_)
      : a(a_), X(X_), Cs(Cs_), Ts(nullptr), Tf(nullptr), Ds(nullptr), ts_layer(-1), blk(blk_), red(red_), cur(0),
        lam_shift(0),
        in_shift(0), evalid(0), base(0), tid(threadIdx.x), zoff(0), ptab(a_.phase_table), pcmin(a_.cmin),
        pspan(a_.span), trig(a_.dev_trig), dtab(a_.d_table) {}

  __device__ __forceinline__ uint32_t idx(int r) const { return CF::idx(cur, tid, r); }

  // barrier over the exchange group of a move between layouts F and T (Cfg: exchange groups).
  // Only exchanges use the exchange area, every tile starts and ends in layout 0, and each
  // move starts in the layout the previous one ended in: the slots a thread writes are the
  // slots of its own local indices, which it alone read in the previous move.  So a move
  // needs one barrier, between its writes and its reads, over its exchange group.
  template <int F, int T>
  __device__ __forceinline__ void xsync() const {
    constexpr int kind = CF::move_sync(F, T);
    if constexpr (kind == 0) {
      __syncwarp();
    } else if constexpr (kind == 1) {
      __syncthreads();
    } else {
      asm volatile("bar.sync %0, %1;" ::"r"(CF::bar_id(F, T, tid >> 5)), "r"(CF::bar_count(F, T)) : "memory");
    }
  }

  // move u from layout F to layout T through the shared exchange buffer; layouts known at
  // compile time so each slot address is one base plus an immediate
  // The swizzle is linear over GF(2) and idx(k, tid, r) = idx(k, tid, 0) | (r << lo(k)) with
  // disjoint bits, so a slot is the thread's base slot XOR a compile-time constant.
  template <int F, int T>
  __device__ __forceinline__ void ex(V (&u)[R]) {
    const uint32_t pf = CF::phys(CF::idx(F, tid, 0)), pt = CF::phys(CF::idx(T, tid, 0));
#pragma unroll
    for (int r = 0; r < R; ++r) X[pf ^ CF::phys((uint32_t)r << CF::lo(F))] = u[r];
    xsync<F, T>();
#pragma unroll
    for (int r = 0; r < R; ++r) u[r] = X[pt ^ CF::phys((uint32_t)r << CF::lo(T))];
  }
  template <int F>
  __device__ __forceinline__ void ex_from(V (&u)[R], int to) {
    switch (to) {
      case 0: ex<F, 0>(u); break;
      case 1: if constexpr (CF::NR > 1) ex<F, (CF::NR > 1 ? 1 : 0)>(u); break;
      case 2: if constexpr (CF::NR > 2) ex<F, (CF::NR > 2 ? 2 : 0)>(u); break;
      default: if constexpr (CF::NR > 3) ex<F, (CF::NR > 3 ? 3 : 0)>(u); break;
    }
  }
  __device__ __forceinline__ void exchange_one(V (&u)[R], int to) {
    switch (cur) {
      case 0: ex_from<0>(u, to); break;
      case 1: if constexpr (CF::NR > 1) ex_from<(CF::NR > 1 ? 1 : 0)>(u, to); break;
      case 2: if constexpr (CF::NR > 2) ex_from<(CF::NR > 2 ? 2 : 0)>(u, to); break;
      default: if constexpr (CF::NR > 3) ex_from<(CF::NR > 3 ? 3 : 0)>(u, to); break;
    }
  }
  // both buffers at once: psi through X, lambda through the second half X + 2^B, so one
  // barrier serves the two
  template <int F, int T>
  __device__ __forceinline__ void ex2() {
    const uint32_t pf = CF::phys(CF::idx(F, tid, 0)), pt = CF::phys(CF::idx(T, tid, 0));
    V* X2 = X + (1u << CF::B);
#pragma unroll
    for (int r = 0; r < R; ++r) X[pf ^ CF::phys((uint32_t)r << CF::lo(F))] = v[r];
#pragma unroll
    for (int r = 0; r < R; ++r) X2[pf ^ CF::phys((uint32_t)r << CF::lo(F))] = w[r];
    xsync<F, T>();
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = X[pt ^ CF::phys((uint32_t)r << CF::lo(T))];
#pragma unroll
    for (int r = 0; r < R; ++r) w[r] = X2[pt ^ CF::phys((uint32_t)r << CF::lo(T))];
  }
  template <int F>
  __device__ __forceinline__ void ex2_from(int to) {
    switch (to) {
      case 0: ex2<F, 0>(); break;
      case 1: if constexpr (CF::NR > 1) ex2<F, (CF::NR > 1 ? 1 : 0)>(); break;
      case 2: if constexpr (CF::NR > 2) ex2<F, (CF::NR > 2 ? 2 : 0)>(); break;
      default: if constexpr (CF::NR > 3) ex2<F, (CF::NR > 3 ? 3 : 0)>(); break;
    }
  }
  __device__ __forceinline__ void exchange_both(int to) {
    switch (cur) {
      case 0: ex2_from<0>(to); break;
      case 1: if constexpr (CF::NR > 1) ex2_from<(CF::NR > 1 ? 1 : 0)>(to); break;
      case 2: if constexpr (CF::NR > 2) ex2_from<(CF::NR > 2 ? 2 : 0)>(to); break;
      default: if constexpr (CF::NR > 3) ex2_from<(CF::NR > 3 ? 3 : 0)>(to); break;
    }
  }
  // both buffers always share one layout; two-buffer kernels own an exchange area of 2 x 2^B
  // slots
  __device__ __forceinline__ void go(int to) {
    if (to == cur) return;
    if constexpr (TWO) exchange_both(to);
    else exchange_one(v, to);
    cur = to;
  }

  // block-reduce and add to blk[r] (and blk[r + 1])
  // (with per-warp accumulators: lane 0 adds the warp's sum to the warp's own slot, no
  // barrier; the slots are summed in warp order once, at the end of the launch)
  __device__ __forceinline__ void block_add(int r, double v0, double v1, bool pair) {
    const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v0 += __shfl_down_sync(0xffffffffu, v0, o);
      v1 += __shfl_down_sync(0xffffffffu, v1, o);
    }
    if (wacc != nullptr) {
      if (lane == 0) {
        wacc[r * (CF::NT / 32) + warp] += v0;
        if (pair) wacc[(r + 1) * (CF::NT / 32) + warp] += v1;
      }
      return;
    }
    __syncthreads();
    if (lane == 0) {
      red[warp] = v0;
      red[CF::NT / 32 + warp] = v1;
    }
    __syncthreads();
    if (tid == 0) {
      double s0 = 0.0, s1 = 0.0;
      for (int k = 0; k < CF::NT / 32; ++k) {
        s0 += red[k];
        s1 += red[CF::NT / 32 + k];
      }
      blk[r] += s0;
      if (pair) blk[r + 1] += s1;
    }
  }

  // ---------------------------------------------------------------- phase
  __device__ __forceinline__ static V vmul(V x, V e) {
    if constexpr (FX) {
      return cmul_fx(x, e, 0);
    } else {
      return make_float2(x.x * e.x - x.y * e.y, x.x * e.y + x.y * e.x);
    }
  }
  // phase factor of cost c computed directly (out of line: only costs outside the table and
  // float costs take it)
  __device__ __forceinline__ V phase_direct(int layer, double c) const {
    if constexpr (FX) return phase_fx_direct(arg_g2pi(a, trig, layer) * c, (const longlong2*)a.turn_table);
    else return phase_f32_direct(arg_g2pi(a, trig, layer) * c);
  }
  // psi (or lambda) *= exp(-i s gamma_l C): table lookups first, the rest out of line
  template <bool INV>
  __device__ __forceinline__ void phase_apply(V (&u)[R], int layer) {
    const bool f64 = a.cost_dtype == QAOA_COST_F64;
    unsigned miss = 0;
    if (FX && !f64 && layer == ts_layer && Tf != nullptr) {  // prepared factors in shared memory
#pragma unroll
      for (int r = 0; r < R; ++r) {
        // table index in 32-bit arithmetic (the host keeps table bounds inside int32, so an
        // entry outside [cmin, cmax] can never wrap into the table)
        const uint32_t k = (uint32_t)cost_i(Cs, idx(r)) - (uint32_t)pcmin;
        if (k < (uint32_t)pspan) {
          if constexpr (FX) {
            const fx::C64 o = fx::cmul_factor<false, INV>(u[r].x, u[r].y, Tf[k], 0);
            u[r] = make_longlong2(o.x, o.y);
          }
        } else {
          miss |= 1u << r;
        }
      }
    } else if (!f64 && ptab != nullptr) {
      const V* tab = (layer == ts_layer && Ts != nullptr) ? Ts : (const V*)ptab + (long long)layer * pspan;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        // table index in 32-bit arithmetic (the host keeps table bounds inside int32, so an
        // entry outside [cmin, cmax] can never wrap into the table)
        const uint32_t k = (uint32_t)cost_i(Cs, idx(r)) - (uint32_t)pcmin;
        if (k < (uint32_t)pspan) {
          V e = tab[k];
          if constexpr (INV) e.y = -e.y;
          u[r] = vmul(u[r], e);
        } else {
          miss |= 1u << r;
        }
      }
    } else {
      miss = R == 32 ? 0xffffffffu : ((1u << R) - 1);
    }
    if (miss) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (!((miss >> r) & 1u)) continue;
        V e = phase_direct(layer, cost_f(Cs, f64, idx(r)));
        if constexpr (INV) e.y = -e.y;
        u[r] = vmul(u[r], e);
      }
    }
  }

  // the same factors on psi and lambda: looked up (or computed) once per amplitude
  template <bool INV>
  __device__ __forceinline__ void phase_apply2(int layer) {
    const bool f64 = a.cost_dtype == QAOA_COST_F64;
    unsigned miss = 0;
    if (FX && !f64 && layer == ts_layer && Tf != nullptr) {  // prepared factors in shared memory
#pragma unroll
      for (int r = 0; r < R; ++r) {
        // table index in 32-bit arithmetic (the host keeps table bounds inside int32, so an
        // entry outside [cmin, cmax] can never wrap into the table)
        const uint32_t k = (uint32_t)cost_i(Cs, idx(r)) - (uint32_t)pcmin;
        if (k < (uint32_t)pspan) {
          if constexpr (FX) {
            const fx::Factor& f = Tf[k];
            const fx::C64 o = fx::cmul_factor<false, INV>(v[r].x, v[r].y, f, 0);
            const fx::C64 q = fx::cmul_factor<false, INV>(w[r].x, w[r].y, f, 0);
            v[r] = make_longlong2(o.x, o.y);
            w[r] = make_longlong2(q.x, q.y);
          }
        } else {
          miss |= 1u << r;
        }
      }
    } else if (!f64 && ptab != nullptr) {
      const V* tab = (layer == ts_layer && Ts != nullptr) ? Ts : (const V*)ptab + (long long)layer * pspan;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        // table index in 32-bit arithmetic (the host keeps table bounds inside int32, so an
        // entry outside [cmin, cmax] can never wrap into the table)
        const uint32_t k = (uint32_t)cost_i(Cs, idx(r)) - (uint32_t)pcmin;
        if (k < (uint32_t)pspan) {
          V e = tab[k];
          if constexpr (INV) e.y = -e.y;
          v[r] = vmul(v[r], e);
          w[r] = vmul(w[r], e);
        } else {
          miss |= 1u << r;
        }
      }
    } else {
      miss = R == 32 ? 0xffffffffu : ((1u << R) - 1);
    }
    if (miss) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (!((miss >> r) & 1u)) continue;
        V e = phase_direct(layer, cost_f(Cs, f64, idx(r)));
        if constexpr (INV) e.y = -e.y;
        v[r] = vmul(v[r], e);
        w[r] = vmul(w[r], e);
      }
    }
  }

  __device__ __forceinline__ void op_phase(int layer, bool inverse, bool on_psi, bool on_lam) {
    if constexpr (TWO) {
      if (on_psi && on_lam) {
        if (inverse) phase_apply2<true>(layer);
        else phase_apply2<false>(layer);
        return;
      }
    }
    if (inverse) {
      if (on_psi) phase_apply<true>(v, layer);
      if (TWO && on_lam) phase_apply<true>(w, layer);
    } else {
      if (on_psi) phase_apply<false>(v, layer);
      if (TWO && on_lam) phase_apply<false>(w, layer);
    }
  }

  // ---------------------------------------------------------------- mixer, float32: RX butterflies
  // RX(2b) = cos(b) (I - i tan(b) X) = -i sin(b) (X + i cot(b) I).  For |tan b| <= 1 a pair
  // (x, y) goes to (x - i t y, y - i t x) with t = tan b and the factor cos b; otherwise to
  // (y + i u x, x + i u y) with u = cot b and the factor -i sin b.  Either way a butterfly
  // is 4 FMAs with |t|, |u| <= 1; the per-qubit factors of a round are applied once at its end.
  __device__ __forceinline__ void bf_tan(float2& x, float2& y, float t) {
    const float2 p = x, q = y;
    x = make_float2(fmaf(t, q.y, p.x), fmaf(-t, q.x, p.y));
    y = make_float2(fmaf(t, p.y, q.x), fmaf(-t, p.x, q.y));
  }
  __device__ __forceinline__ void bf_cot(float2& x, float2& y, float u) {
    const float2 p = x, q = y;
    x = make_float2(fmaf(-u, p.y, q.x), fmaf(u, p.x, q.y));
    y = make_float2(fmaf(-u, q.y, p.x), fmaf(u, q.x, p.y));
  }
  // butterflies on the register bits set in todo, branch-free inside the pair loops
  template <bool TAN>
  __device__ __forceinline__ void bf_round(V (&u)[R], unsigned todo, float tu) {
#pragma unroll
    for (int rb = 0; rb < CF::RB; ++rb) {
      if (!((todo >> rb) & 1u)) continue;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (r & (1 << rb)) continue;
        const int q = r | (1 << rb);
        if constexpr (TAN) bf_tan(u[r], u[q], tu);
        else bf_cot(u[r], u[q], tu);
      }
    }
  }

  // multiply every amplitude of u by the complex factor f
  __device__ __forceinline__ void scale_f32(V (&u)[R], float2 f) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float2 z = u[r];
      u[r] = make_float2(z.x * f.x - z.y * f.y, z.x * f.y + z.y * f.x);
    }
  }
  // (m)^nb (tangent form) or (-i m)^nb (cotangent form)
  __device__ __forceinline__ static float2 round_factor(bool tanf, float m, int nb) {
    float f = 1.f;
    for (int j = 0; j < nb; ++j) f *= m;
    if (tanf) return make_float2(f, 0.f);
    switch (nb & 3) {
      case 0: return make_float2(f, 0.f);
      case 1: return make_float2(0.f, -f);
      case 2: return make_float2(-f, 0.f);
      default: return make_float2(0.f, f);
    }
  }

  __device__ __forceinline__ void mix_f32(int layer, bool inverse, bool on_psi, bool on_lam, int xacc) {
    const double cbd = arg_cosb(a, trig, layer), sbd = inverse ? -arg_sinb(a, trig, layer) : arg_sinb(a, trig, layer);
    const bool tanf = fabs(cbd) >= fabs(sbd);
    const float tu = tanf ? (float)(sbd / cbd) : (float)(cbd / sbd);
    const float m = tanf ? (float)cbd : (float)sbd;
    const int gl = a.g.c, gh = a.g.c + a.g.t;
    const bool rev = (cur == CF::NR - 1) && CF::NR > 1;
    const bool xt = TWO && xacc >= 0;
    float xs = 0.f;
    int pending = 0;  // qubits whose factor is not applied yet
    for (int s = 0; s < CF::NR; ++s) {
      const int k = rev ? CF::NR - 1 - s : s;
      const int l0 = CF::lo(k), l1 = CF::newhi(k);
      if (l1 <= gl || l0 >= gh) continue;  // no group qubit in this round
      go(k);
      if (xt) {  // sum over this round's qubits of Im(conj(la) pb + conj(lb) pa); state exact here
#pragma unroll
        for (int rb = 0; rb < CF::RB; ++rb) {
          const int b = l0 + rb;
          if (!(b < l1 && b >= gl && b < gh)) continue;
#pragma unroll
          for (int r = 0; r < R; ++r) {
            if (r & (1 << rb)) continue;
            const int q = r | (1 << rb);
            xs += w[r].x * v[q].y - w[r].y * v[q].x + w[q].x * v[r].y - w[q].y * v[r].x;
          }
        }
      }
      // which of this round's register bits are group qubits (uniform)
      unsigned todo = 0;
#pragma unroll
      for (int rb = 0; rb < CF::RB; ++rb) {
        const int b = l0 + rb;
        if (b < l1 && b >= gl && b < gh) todo |= 1u << rb;
      }
      pending += __popc(todo);
      if (tanf) {
        if (on_psi) bf_round<true>(v, todo, tu);
        if (TWO && on_lam) bf_round<true>(w, todo, tu);
      } else {
        if (on_psi) bf_round<false>(v, todo, tu);
        if (TWO && on_lam) bf_round<false>(w, todo, tu);
      }
      if (xt && pending) {  // the X-terms of the next round need the exact state
        const float2 f = round_factor(tanf, m, pending);
        if (on_psi) scale_f32(v, f);
        if (on_lam) scale_f32(w, f);
        pending = 0;
      }
    }
    if (pending) {
      const float2 f = round_factor(tanf, m, pending);
      if (on_psi) scale_f32(v, f);
      if (TWO && on_lam) scale_f32(w, f);
    }
    if (xt) block_add(xacc, 2.0 * (double)xs, 0.0, false);
  }

  // ---------------------------------------------------------------- mixer, fixed point: W D W
  template <int RBc>
  __device__ __forceinline__ void wht_bit(V (&u)[R]) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (r & (1 << RBc)) continue;
      const int q = r | (1 << RBc);
      const longlong2 x = u[r], y = u[q];
      u[r] = make_longlong2(x.x + y.x, x.y + y.y);
      u[q] = make_longlong2(x.x - y.x, x.y - y.y);
    }
  }
  __device__ __forceinline__ void wht_round(int k, bool on_psi, bool on_lam) {
    const int l0 = CF::lo(k), l1 = CF::newhi(k);
    const int gl = a.g.c, gh = a.g.c + a.g.t;
#pragma unroll
    for (int rb = 0; rb < CF::RB; ++rb) {
      const int b = l0 + rb;
      if (b < l1 && b >= gl && b < gh) {
        if (on_psi) {
          if constexpr (FX) {
            if (rb == 0) wht_bit<0>(v);
            if (CF::RB > 1 && rb == 1) wht_bit<(CF::RB > 1 ? 1 : 0)>(v);
            if (CF::RB > 2 && rb == 2) wht_bit<(CF::RB > 2 ? 2 : 0)>(v);
            if (CF::RB > 3 && rb == 3) wht_bit<(CF::RB > 3 ? 3 : 0)>(v);
            if (CF::RB > 4 && rb == 4) wht_bit<(CF::RB > 4 ? 4 : 0)>(v);
          }
        }
        if (TWO && on_lam) {
          if constexpr (FX) {
            if (rb == 0) wht_bit<0>(w);
            if (CF::RB > 1 && rb == 1) wht_bit<(CF::RB > 1 ? 1 : 0)>(w);
            if (CF::RB > 2 && rb == 2) wht_bit<(CF::RB > 2 ? 2 : 0)>(w);
            if (CF::RB > 3 && rb == 3) wht_bit<(CF::RB > 3 ? 3 : 0)>(w);
            if (CF::RB > 4 && rb == 4) wht_bit<(CF::RB > 4 ? 4 : 0)>(w);
          }
        }
      }
    }
  }

  // D multiply on the register tile: u[r] *= Ds[popcount] / 2^t; E = t >= 3 selects the
  // shift form of the limb multiply at compile time
  template <bool BIG>
  __device__ __forceinline__ void d_mul(V (&u)[R], const fx::Factor* Ds, int gl, int t) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const fx::Factor& f = Ds[__popc((idx(r) >> gl) & ((1u << t) - 1))];
      const fx::C64 o = fx::cmul_factor<!BIG, false>(u[r].x, u[r].y, f, t);
      u[r] = make_longlong2(o.x, o.y);
    }
  }
  // this mixer's diagonal exp(-i s b (t - 2k)), k = 0..t, as prepared factors in shared memory
  // (sign applied); the caller synchronises before and after
  __device__ __forceinline__ void load_diagonal(int layer, bool inverse, int t) {
    if (tid <= (uint32_t)t) {
      const longlong2 e = __ldg((const longlong2*)dtab + ((long long)layer * 14 + t) * 14 + tid);
      Ds[tid] = fx::factor(e.x, inverse ? -e.y : e.y);
    }
  }

  __device__ __forceinline__ void mix_fx(int layer, bool inverse, bool on_psi, bool on_lam, int xacc) {
    const int gl = a.g.c, gh = a.g.c + a.g.t, t = a.g.t;
    // rounds that hold group qubits, walked from the current layout outwards
    int ks[8], nk = 0;
    const bool rev = (cur == CF::NR - 1) && CF::NR > 1;
    for (int s = 0; s < CF::NR; ++s) {
      const int k = rev ? CF::NR - 1 - s : s;
      if (CF::newhi(k) <= gl || CF::lo(k) >= gh) continue;
      ks[nk++] = k;
    }
    __syncthreads();
    load_diagonal(layer, inverse, t);
    for (int j = 0; j < nk; ++j) {
      go(ks[j]);
      wht_round(ks[j], on_psi, on_lam);
    }
    __syncthreads();
    if (TWO && xacc >= 0) {  // 2 Im <lam|sum_j X_j|psi> = 2 Im sum conj(lam~) (t - 2 popcount) psi~ 2^-t
      i128 xs = 0;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int pc = __popc((idx(r) >> gl) & ((1u << t) - 1));
        const i128 pr = fx::dot2_exact(w[r].x, v[r].y, w[r].y, v[r].x);  // Im(conj(lam~) psi~)
        xs += (pr >> 32) * (t - 2 * pc);
      }
      // value = 2 * xs * 2^32 * 2^-t * 2^-2S (lambda carries the scale 2^lam_shift)
      block_add(xacc, 2.0 * i128_to_double(xs, 2 * a.fx_shift + t - 32 - lam_shift), 0.0, false);
    }
    if (t >= 3) {
      if (on_psi) d_mul<true>(v, Ds, gl, t);
      if (TWO && on_lam) d_mul<true>(w, Ds, gl, t);
    } else {
      if (on_psi) d_mul<false>(v, Ds, gl, t);
      if (TWO && on_lam) d_mul<false>(w, Ds, gl, t);
    }
    for (int j = nk - 1; j >= 0; --j) {
      go(ks[j]);
      wht_round(ks[j], on_psi, on_lam);
    }
  }

  // ---------------------------------------------------------------- elementwise ops
  // lambda := C psi; fixed point stores lambda / 2^lam_shift (2^lam_shift >= max |C|) so
  // that lambda keeps the norm bound of the state
  __device__ __forceinline__ void op_lambda() {
    const bool f64 = a.cost_dtype == QAOA_COST_F64;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const uint32_t i = idx(r);
      if constexpr (FX) {
        if (!f64) {
          const long long c = cost_i(Cs, i);
          w[r] = make_longlong2(round_shift(fx::mul_wide32(v[r].x, (int)c), lam_shift),
                                round_shift(fx::mul_wide32(v[r].y, (int)c), lam_shift));
        } else {
          const long long cq = double_to_fx(cost_f(Cs, true, i), 62 - lam_shift);
          w[r] = make_longlong2(round_shift((i128)v[r].x * cq, 62), round_shift((i128)v[r].y * cq, 62));
        }
      } else {
        const float c = (float)cost_f(Cs, f64, i);
        w[r] = make_float2(c * v[r].x, c * v[r].y);
      }
    }
  }

  __device__ __forceinline__ void op_expect(int acc) {
    const bool f64 = a.cost_dtype == QAOA_COST_F64;
    double e0 = 0.0, e1 = 0.0;
    if constexpr (FX) {
      i128 sc = 0, sn = 0;
      double sf = 0.0;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const uint32_t i = idx(r);
        if (i >= evalid) continue;
        const i128 p2 = fx::dot2_exact(v[r].x, v[r].x, -v[r].y, v[r].y);  // |psi|^2, exact
        sn += p2 >> 16;
        if (!f64) sc += (p2 >> 32) * cost_i(Cs, i);
        else sf += cost_f(Cs, true, i) * i128_to_double(p2, 2 * a.fx_shift);
      }
      e1 = i128_to_double(sn, 2 * (a.fx_shift - in_shift) - 16);
      e0 = f64 ? ldexp(sf, 2 * in_shift) : i128_to_double(sc, 2 * (a.fx_shift - in_shift) - 32);
    } else {
      float s0[4] = {0.f, 0.f, 0.f, 0.f}, s1[4] = {0.f, 0.f, 0.f, 0.f};  // independent partial sums
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const uint32_t i = idx(r);
        if (i >= evalid) continue;
        const float p2 = v[r].x * v[r].x + v[r].y * v[r].y;
        s0[r & 3] += (float)cost_f(Cs, f64, i) * p2;
        s1[r & 3] += p2;
      }
      e0 = (double)((s0[0] + s0[1]) + (s0[2] + s0[3]));
      e1 = (double)((s1[0] + s1[1]) + (s1[2] + s1[3]));
    }
    block_add(acc, e0, e1, true);
  }

  __device__ __forceinline__ void op_cterm(int acc) {
    const bool f64 = a.cost_dtype == QAOA_COST_F64;
    double e0 = 0.0;
    if constexpr (FX) {
      i128 sc = 0;
      double sf = 0.0;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const uint32_t i = idx(r);
        if (i >= evalid) continue;
        const i128 pr = fx::dot2_exact(w[r].x, v[r].y, w[r].y, v[r].x);
        if (!f64) sc += (pr >> 32) * cost_i(Cs, i);
        else sf += cost_f(Cs, true, i) * i128_to_double(pr, 2 * a.fx_shift - lam_shift);
      }
      e0 = f64 ? sf : i128_to_double(sc, 2 * a.fx_shift - 32 - lam_shift);
    } else {
      float s[4] = {0.f, 0.f, 0.f, 0.f};  // independent partial sums
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const uint32_t i = idx(r);
        if (i >= evalid) continue;
        s[r & 3] += (float)cost_f(Cs, f64, i) * (w[r].x * v[r].y - w[r].y * v[r].x);
      }
      e0 = (double)((s[0] + s[1]) + (s[2] + s[3]));
    }
    block_add(acc, 2.0 * e0, 0.0, false);
  }
};

// ------------------------------------------------------------------ table entries
//
// Integer-cost phase tables hold exp(-i gamma c); fixed-point mixer diagonals hold
// exp(-i beta (t - 2k)) at [(l * 14 + t) * 14 + k] for t = 1..13, k = 0..t (zero past t);
// the turn tables hold exp(-2 pi i k / 2^(10 (level + 1))) for level 0..2, k < 1024.
__device__ __forceinline__ long long q62(double x) { return llrint(ldexp(x, 62)); }
__device__ __forceinline__ longlong2 unit_q62(double th) {
  double sn, cs;
  sincos(th, &sn, &cs);
  return make_longlong2(q62(cs), q62(-sn));
}
__device__ __forceinline__ float2 unit_f32(double th) {
  double sn, cs;
  sincos(th, &sn, &cs);
  return make_float2((float)cs, (float)(-sn));
}
// entry j = t * 14 + k of one layer's mixer diagonals
__device__ __forceinline__ longlong2 d_entry(double beta, int j) {
  const int t = j / 14, k = j % 14;
  return k <= t ? unit_q62(beta * (double)(t - 2 * k)) : make_longlong2(0, 0);
}
__device__ __forceinline__ longlong2 turn_entry(int j) {
  const int level = j / 1024, k = j % 1024;
  return unit_q62(2.0 * 3.141592653589793238 * (double)k * ldexp(1.0, -10 * (level + 1)));
}

// state loads: through the read-only path, or (COHERENT) through L2 for state that the same
// launch wrote earlier
template <bool COHERENT, class T>
__device__ __forceinline__ T ld_state(const T* p) {
  if constexpr (COHERENT) return __ldcg(p);
  else return __ldg(p);
}

// One tile of a generic sweep: stage the cost tile, load (or create) the state in layout 0,
// run the op program, store in layout 0.
template <class CF, bool FX, bool TWO, bool COHERENT>
__device__ __forceinline__ void sweep_tile(Sweeper<CF, FX, TWO>& s, const SweepArgs& a, int64_t tile, void* Cs) {
  using V = typename Sweeper<CF, FX, TWO>::V;
  constexpr int R = CF::R;
  V (&v)[R] = s.v;
  V (&w)[R] = s.w;
  const SweepGeom& g = a.g;
  const bool cf64 = a.cost_dtype == QAOA_COST_F64;
  const uint32_t tid = threadIdx.x;
  const uint64_t base = tile_base(g, tile);
  s.base = base;
  s.cur = 0;
  // cost tile: 16-byte asynchronous copies when every chunk is contiguous in memory
  // (the first group, or at least one chunk of carried low bits), element copies otherwise
  if (a.needs_cost) {
    __syncthreads();  // the previous tile's ops are done with Cs
    const int per = cf64 ? 2 : 4;  // elements per 16-byte chunk
    const bool chunky = (g.j0 == 0) || ((1 << g.c) >= per);
    if (chunky && s.evalid >= (uint32_t)per) {
      const uint32_t nch = s.evalid / per;
      for (uint32_t ch = tid; ch < nch; ch += CF::NT) {
        const uint32_t i = ch * per;
        const uint64_t z = local_to_z(g, base, i);
        const char* src = (const char*)a.C + z * (cf64 ? 8 : 4);
        char* dst = (char*)Cs + (size_t)phys_cost(i, cf64) * (cf64 ? 8 : 4);
        cp_async16(dst, src);
      }
    } else {
      for (uint32_t i = tid; i < s.evalid; i += CF::NT) {
        const uint64_t z = local_to_z(g, base, i);
        if (cf64) ((double*)Cs)[phys_cost(i, true)] = __ldg((const double*)a.C + z);
        else ((int*)Cs)[phys_cost(i, false)] = __ldg((const int*)a.C + z);
      }
    }
    // slots past the tile's valid range hold cost 0 (phase 1) so their zero amplitudes
    // stay zero
    for (uint32_t i = s.evalid + tid; i < (1u << CF::B); i += CF::NT) {
      if (cf64) ((double*)Cs)[phys_cost(i, true)] = 0.0;
      else ((int*)Cs)[phys_cost(i, false)] = 0;
    }
  }
  // state (layout 0): register r holds local index tb0 + (r << lo(0)), i.e. global index
  // z0 + r * zs, since the register bits of layout 0 are group bits
  // (when the carried low bits reach into the register bits, the general map is used)
  {
  const uint32_t tb0 = CF::idx(0, tid, 0);
  const uint64_t z0 = local_to_z(g, base, tb0);
  const bool affine = g.c <= CF::lo(0);
  const uint64_t zs = affine ? (1ull << (CF::lo(0) - g.c + g.j0)) : 0ull;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const uint32_t i = tb0 + ((uint32_t)r << CF::lo(0));
    const bool ok = i < s.evalid;
    const uint64_t z = affine ? z0 + (uint64_t)r * zs : local_to_z(g, base, i);
    if constexpr (FX) {
      if (!ok) v[r] = make_longlong2(0, 0);
      else if (a.load_fmt == 2) v[r] = make_longlong2(a.init_fx, 0);
      else if (a.load_fmt == 1) {
        const double2 d = ld_state<COHERENT>((const double2*)a.psi + z);
        v[r] = make_longlong2(double_to_fx(d.x, a.fx_shift - s.in_shift), double_to_fx(d.y, a.fx_shift - s.in_shift));
      } else v[r] = ld_state<COHERENT>((const longlong2*)a.psi + z);
      if (TWO) w[r] = (ok && a.load_lam) ? ld_state<COHERENT>((const longlong2*)a.lam + z) : make_longlong2(0, 0);
    } else {
      if (!ok) v[r] = make_float2(0.f, 0.f);
      else if (a.load_fmt == 2) v[r] = make_float2(a.init_f32, 0.f);
      else v[r] = ld_state<COHERENT>((const float2*)a.psi + z);
      if (TWO) w[r] = (ok && a.load_lam) ? ld_state<COHERENT>((const float2*)a.lam + z) : make_float2(0.f, 0.f);
    }
  }
  }

  if (a.needs_cost) {
    cp_async_wait_all();
    __syncthreads();
  }
  for (int k = 0; k < a.nops; ++k) {
    const uint32_t op = a.ops[k];
    const uint32_t kind = op & 0xff;
    const int layer = (op >> 16) & 0xff;
    const int acc = (int)((op >> 24) & 0xff);
    const bool on_psi = op & F_PSI, on_lam = op & F_LAM, inv = op & F_SIGN;
    const bool has_x = op & F_XTERM;
    if (kind == OP_PHASE) {
      s.op_phase(layer, inv, on_psi, on_lam);
    } else if (kind == OP_MIX) {
      if constexpr (FX) s.mix_fx(layer, inv, on_psi, on_lam, has_x ? acc : -1);
      else s.mix_f32(layer, inv, on_psi, on_lam, has_x ? acc : -1);
    } else if (kind == OP_LAMBDA) {
      if constexpr (TWO) s.op_lambda();
    } else if (kind == OP_RED_EXPECT) {
      s.op_expect(acc);
    } else if (kind == OP_RED_CTERM) {
      if constexpr (TWO) s.op_cterm(acc);
    }
  }

  // store (layout 0); addresses recomputed rather than kept live through the ops
  s.go(0);
  {
  const uint32_t tb0 = CF::idx(0, tid, 0);
  const uint64_t z0 = local_to_z(g, base, tb0);
  const bool affine = g.c <= CF::lo(0);
  const uint64_t zs = affine ? (1ull << (CF::lo(0) - g.c + g.j0)) : 0ull;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const uint32_t i = tb0 + ((uint32_t)r << CF::lo(0));
    if (i >= s.evalid) continue;
    const uint64_t z = affine ? z0 + (uint64_t)r * zs : local_to_z(g, base, i);
    if constexpr (FX) {
      if (a.store_fmt == 1) {
        ((double2*)a.psi)[z] = make_double2(fx_to_double(v[r].x, a.fx_shift - s.in_shift),
                                            fx_to_double(v[r].y, a.fx_shift - s.in_shift));
      } else if (a.store_fmt == 0) {
        ((longlong2*)a.psi)[z] = v[r];
      }
      if (TWO && a.store_lam) ((longlong2*)a.lam)[z] = w[r];
    } else {
      if (a.store_fmt >= 0) ((float2*)a.psi)[z] = v[r];
      if (TWO && a.store_lam) ((float2*)a.lam)[z] = w[r];
    }
  }
  }
}

// ------------------------------------------------------------------ lean sweeps
//
// Sweeps on full tiles run in kernels whose layout sequence is fixed at compile time, so
// each instance holds only the code it runs: a plain mixer sweep, and a sweep that runs its
// op program (mixers, phases, lambda and reductions) with the same mixer code.  The host
// checks the tile shape, the formats and the affine layout-0 addresses before choosing
// them.

template <class CF, bool FX, bool TWO>
struct Lean : Sweeper<CF, FX, TWO> {
  using B = Sweeper<CF, FX, TWO>;
  using V = typename B::V;
  static constexpr int R = CF::R, NR = CF::NR;
  using B::B;
  // mixer diagonals of the launch's mixers, staged once in shared memory ([kLeanMix][16]),
  // or nullptr: each mixer then stages its own between block barriers
  const fx::Factor* dpre = nullptr;

  // group-qubit register bits of round K (relative to lo(K)), uniform
  template <int K>
  __device__ __forceinline__ unsigned gmask() const {
    const int gl = this->a.g.c, gh = this->a.g.c + this->a.g.t;
    unsigned m = 0;
#pragma unroll
    for (int rb = 0; rb < CF::RB; ++rb) {
      const int b = CF::lo(K) + rb;
      if (b < CF::newhi(K) && b >= gl && b < gh) m |= 1u << rb;
    }
    return m;
  }
  template <int F, int T>
  __device__ __forceinline__ void exb() {
    if constexpr (TWO) this->template ex2<F, T>();
    else this->template ex<F, T>(this->v);
    this->cur = T;
  }
  template <int K>
  __device__ __forceinline__ uint32_t ix(int r) const { return CF::idx(K, this->tid, r); }

  // ---- fixed point: W rounds, D multiply (and X-term) at layout L
  // two Walsh-Hadamard rounds on register bits B0 and B1 at once: for each quadruple
  // (x0, x1, x2, x3) = u[r], u[r | b0], u[r | b1], u[r | b0 | b1] the outputs are
  // (x0 + x1) +- (x2 + x3) and (x0 - x1) +- (x2 - x3), written as three-input sums
  template <int B0, int B1>
  __device__ __forceinline__ void wht_bit2(V (&u)[R]) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (r & ((1 << B0) | (1 << B1))) continue;
      const int q1 = r | (1 << B0), q2 = r | (1 << B1), q3 = q1 | q2;
      const longlong2 x0 = u[r], x1 = u[q1], x2 = u[q2], x3 = u[q3];
      const long long a0x = x0.x + x1.x, a0y = x0.y + x1.y, a1x = x0.x - x1.x, a1y = x0.y - x1.y;
      u[r] = make_longlong2(a0x + x2.x + x3.x, a0y + x2.y + x3.y);
      u[q2] = make_longlong2(a0x - x2.x - x3.x, a0y - x2.y - x3.y);
      u[q1] = make_longlong2(a1x + x2.x - x3.x, a1y + x2.y - x3.y);
      u[q3] = make_longlong2(a1x - x2.x + x3.x, a1y - x2.y + x3.y);
    }
  }
  __device__ __forceinline__ void wht_mask(V (&u)[R], unsigned m) {
    if constexpr (FX) {
      if (CF::RB > 1 && (m & 3u) == 3u) {
        this->template wht_bit2<0, (CF::RB > 1 ? 1 : 0)>(u);
      } else {
        if (m & 1u) this->template wht_bit<0>(u);
        if constexpr (CF::RB > 1) if (m & 2u) this->template wht_bit<(CF::RB > 1 ? 1 : 0)>(u);
      }
      if constexpr (CF::RB > 3) {
        if ((m & 12u) == 12u) {
          this->template wht_bit2<(CF::RB > 3 ? 2 : 0), (CF::RB > 3 ? 3 : 0)>(u);
        } else {
          if (m & 4u) this->template wht_bit<(CF::RB > 2 ? 2 : 0)>(u);
          if (m & 8u) this->template wht_bit<(CF::RB > 3 ? 3 : 0)>(u);
        }
      } else if constexpr (CF::RB > 2) {
        if (m & 4u) this->template wht_bit<(CF::RB > 2 ? 2 : 0)>(u);
      }
      if constexpr (CF::RB > 4) if (m & 16u) this->template wht_bit<(CF::RB > 4 ? 4 : 0)>(u);
    }
  }
  template <int K>
  __device__ __forceinline__ void wht_k(bool lam) {
    const unsigned m = gmask<K>();
    wht_mask(this->v, m);
    if constexpr (TWO) if (lam) wht_mask(this->w, m);
  }
  template <int K, int L>
  __device__ __forceinline__ void fx_fwd(bool lam) {
    if constexpr (K > 0) exb<K - 1, K>();
    wht_k<K>(lam);
    if constexpr (K < L) fx_fwd<K + 1, L>(lam);
  }
  template <int K>
  __device__ __forceinline__ void fx_back(bool lam) {
    wht_k<K>(lam);
    if constexpr (K > 0) {
      exb<K, K - 1>();
      fx_back<K - 1>(lam);
    }
  }
  template <int L, bool BIG>
  __device__ __forceinline__ void dmul_l(V (&u)[R], const fx::Factor* Ds, int gl, int t) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const fx::Factor& f = Ds[__popc((ix<L>(r) >> gl) & ((1u << t) - 1))];
      const fx::C64 o = fx::cmul_factor<!BIG, false>(u[r].x, u[r].y, f, t);
      u[r] = make_longlong2(o.x, o.y);
    }
  }
  // W D W from layout 0 back to layout 0; D at layout L (the last round with group qubits)
  template <int L>
  __device__ __forceinline__ void fx_mixer(int layer, bool inverse, bool lam, int xacc, int mix) {
    const int gl = this->a.g.c, t = this->a.g.t;
    const fx::Factor* Ds = dpre != nullptr ? dpre + 16 * mix : this->Ds;
    if (dpre == nullptr) {
      __syncthreads();
      this->load_diagonal(layer, inverse, t);
    }
    fx_fwd<0, L>(lam);
    if (dpre == nullptr) __syncthreads();
    if constexpr (TWO) {
      if (xacc >= 0) {
        // sum_r pr_r (t - 2 popcount(group bits of index r)); the index is the thread's
        // bits OR r << lo(L), so the popcount is the thread's part pt plus popcount(r & gm),
        // gm = the register bits that are group bits, and the sum is
        // (t - 2 pt) S - 2 sum_{b in gm} U_b with S = sum_r pr_r, U_b = sum_{r: bit b} pr_r
        // (exact int128 sums of products below 2^123, shifted once before the weighting)
        const uint32_t gmask = (1u << t) - 1;
        const int pt = __popc((ix<L>(0) >> gl) & gmask);
        const uint32_t gm = (((uint32_t)gmask << gl) >> CF::lo(L)) & (uint32_t)(R - 1);
        i128 S = 0, U[CF::RB];
#pragma unroll
        for (int b = 0; b < CF::RB; ++b) U[b] = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const i128 pr = fx::dot2_exact(this->w[r].x, this->v[r].y, this->w[r].y, this->v[r].x);
          S += pr;
#pragma unroll
          for (int b = 0; b < CF::RB; ++b)
            if (r & (1 << b)) U[b] += pr;
        }
        i128 xs = (S >> 32) * (t - 2 * pt);
#pragma unroll
        for (int b = 0; b < CF::RB; ++b)
          if (gm & (1u << b)) xs -= (U[b] >> 32) * 2;
        this->block_add(xacc, 2.0 * i128_to_double(xs, 2 * this->a.fx_shift + t - 32 - this->lam_shift), 0.0, false);
      }
    }
    // lean sweeps run only on groups of >= 3 qubits, so the shift form of the multiply
    // applies; the two-buffer kernels keep the branch (it schedules better there)
    if constexpr (TWO) {
      if (t >= 3) {
        dmul_l<L, true>(this->v, Ds, gl, t);
        if (lam) dmul_l<L, true>(this->w, Ds, gl, t);
      } else {
        dmul_l<L, false>(this->v, Ds, gl, t);
        if (lam) dmul_l<L, false>(this->w, Ds, gl, t);
      }
    } else {
      dmul_l<L, true>(this->v, Ds, gl, t);
    }
    fx_back<L>(lam);
  }

  // ---- float32: RX(2 beta) = m (I - i u X) per qubit in tangent or cotangent form, as
  // unit-free butterflies round by round through layouts 0..L; the factors m (or -i m) of
  // all t qubits are applied once at the end, then one exchange returns to layout 0.
  // X-terms (adjoint pass): psi and lambda carry the same factor c of the qubits already
  // done, so Im conj(lambda) X_j psi of the unscaled buffers is |c|^2 = m^(2 done) times the
  // true value; X_j commutes with every RX_i, so each round's terms may be taken just before
  // its butterflies.
  template <int K>
  __device__ __forceinline__ void f32_round(bool tanf, float tu, float m2, bool xt, float& xs, float& w2) {
    if constexpr (!FX) {
      const unsigned msk = gmask<K>();
      if (xt) {
        // four independent partial sums (pairs by r mod 4) keep the FMA chains short
        float pa[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int rb = 0; rb < CF::RB; ++rb) {
          if (!((msk >> rb) & 1u)) continue;
#pragma unroll
          for (int r = 0; r < R; ++r) {
            if (r & (1 << rb)) continue;
            const int q = r | (1 << rb);
            pa[r & 3] += this->w[r].x * this->v[q].y - this->w[r].y * this->v[q].x + this->w[q].x * this->v[r].y -
                         this->w[q].y * this->v[r].x;
          }
        }
        xs = fmaf((pa[0] + pa[1]) + (pa[2] + pa[3]), w2, xs);
        for (unsigned b = msk; b; b &= b - 1) w2 *= m2;
      }
      if (tanf) {
        this->template bf_round<true>(this->v, msk, tu);
        if constexpr (TWO) this->template bf_round<true>(this->w, msk, tu);
      } else {
        this->template bf_round<false>(this->v, msk, tu);
        if constexpr (TWO) this->template bf_round<false>(this->w, msk, tu);
      }
    }
  }
  template <int K, int L>
  __device__ __forceinline__ void f32_fwd(bool tanf, float tu, float m2, bool xt, float& xs, float& w2) {
    if constexpr (K > 0) exb<K - 1, K>();
    f32_round<K>(tanf, tu, m2, xt, xs, w2);
    if constexpr (K < L) f32_fwd<K + 1, L>(tanf, tu, m2, xt, xs, w2);
  }
  template <int L>
  __device__ __forceinline__ void f32_mixer(int layer, bool inverse, int xacc) {
    if constexpr (!FX) {
      const double cbd = arg_cosb(this->a, this->trig, layer);
      const double sbd = inverse ? -arg_sinb(this->a, this->trig, layer) : arg_sinb(this->a, this->trig, layer);
      const bool tanf = fabs(cbd) >= fabs(sbd);
      const float tu = tanf ? (float)(sbd / cbd) : (float)(cbd / sbd);
      const float m = tanf ? (float)cbd : (float)sbd;
      const bool xt = TWO && xacc >= 0;
      float xs = 0.f, w2 = 1.f;
      f32_fwd<0, L>(tanf, tu, m * m, xt, xs, w2);
      const float2 f = B::round_factor(tanf, m, this->a.g.t);
      this->scale_f32(this->v, f);
      if constexpr (TWO) this->scale_f32(this->w, f);
      if (xt) this->block_add(xacc, 2.0 * (double)xs, 0.0, false);
      if constexpr (L > 0) exb<L, 0>();
    }
  }
  template <int L>
  __device__ __forceinline__ void mixer(int layer, bool inverse, int xacc, int mix) {
    if constexpr (FX) fx_mixer<L>(layer, inverse, TWO, xacc, mix);
    else f32_mixer<L>(layer, inverse, xacc);
  }

  // ---- the sweep: one mixer (OPS = false), or the sweep's op program (OPS = true) with
  // every mixer on the compile-time layout sequence and the elementwise ops in layout 0;
  // L = last round with group qubits
  template <int L, bool OPS>
  __device__ __forceinline__ void run() {
    const uint32_t* ops = this->a.ops;
    if constexpr (!OPS) {
      const uint32_t o = ops[0];
      mixer<L>((o >> 16) & 0xff, o & F_SIGN, (o & F_XTERM) ? (int)((o >> 24) & 0xff) : -1, 0);
    } else {
      // one copy of the mixer code for every mixer of the program keeps the kernel within
      // the instruction cache.  Two-buffer kernels apply mixers and phases to both buffers:
      // an op on psi alone only occurs while lambda is still zero (the host checks that).
      int mix = 0;
#pragma unroll 1
      for (int k = 0; k < this->a.nops; ++k) {
        const uint32_t op = ops[k];
        const uint32_t kind = op & 0xff;
        const int layer = (op >> 16) & 0xff, acc = (int)((op >> 24) & 0xff);
        const bool inv = op & F_SIGN;
        // every mixer returns to layout 0, where the elementwise ops run: restating cur = 0
        // before each lets the compiler fold their register-to-index maps to constants
        if (kind == OP_MIX) {
          mixer<L>(layer, inv, (op & F_XTERM) ? acc : -1, mix++);
        } else if (kind == OP_PHASE) {
          this->cur = 0;
          this->op_phase(layer, inv, true, TWO);
        } else if (kind == OP_LAMBDA) {
          this->cur = 0;
          if constexpr (TWO) this->op_lambda();
        } else if (kind == OP_RED_EXPECT) {
          this->cur = 0;
          this->op_expect(acc);
        } else if (kind == OP_RED_CTERM) {
          this->cur = 0;
          if constexpr (TWO) this->op_cterm(acc);
        }
      }
    }
  }
};

// One tile of a lean sweep: stage the cost tile (op programs), load or create the state in
// layout 0, run the mixer or the op program, store.  COHERENT loads read state written
// earlier in the same launch.  With a staging area (two-buffer sweeps, s.Ps), psi of the
// block's next tile `next` travels into it by asynchronous copies while this tile computes;
// `have` says that this tile's psi is there.  Each thread copies and reads back only its own
// layout-0 slots, so the staging needs no barrier, only waits for the thread's own copy
// groups; the cost tile's group is committed after the prefetch of this tile's psi and before
// the prefetch of the next one.
template <class CF, bool FX, bool TWO, bool OPS, int LAST, bool COHERENT>
__device__ __forceinline__ void lean_tile(Lean<CF, FX, TWO>& s, const SweepArgs& a, int64_t tile, void* Cs,
                                          int64_t next = -1, bool have = false) {
  using V = typename Lean<CF, FX, TWO>::V;
  constexpr int R = CF::R;
  V (&v)[R] = s.v;
  V (&w)[R] = s.w;
  const SweepGeom& g = a.g;
  const uint32_t tid = threadIdx.x;
  const bool cf64 = a.cost_dtype == QAOA_COST_F64;
  const bool cost = OPS && a.needs_cost;
  const uint32_t tb0 = CF::idx(0, tid, 0);
  const uint64_t zs = 1ull << (CF::lo(0) - g.c + g.j0);
  const bool init = OPS && a.load_fmt == 2;
  const bool ld_lam = TWO && (!OPS || a.load_lam), st_lam = TWO && (!OPS || a.store_lam);
  const int st_fmt = OPS ? a.store_fmt : 0;
  const bool stage = TWO && s.Ps != nullptr && !init;
  const bool staged = stage && have;
  const uint64_t base = tile_base(g, tile);
  s.base = base;
  s.cur = 0;
  if (cost) {  // cost tile, 16-byte asynchronous copies
    __syncthreads();
    const int per = cf64 ? 2 : 4;
    const uint32_t nch = (1u << CF::B) / per;
    for (uint32_t ch = tid; ch < nch; ch += CF::NT) {
      const uint32_t i = ch * per;
      const uint64_t z = local_to_z(g, base, i);
      cp_async16((char*)Cs + (size_t)phys_cost(i, cf64) * (cf64 ? 8 : 4), (const char*)a.C + (s.zoff + z) * (cf64 ? 8 : 4));
    }
    if (stage) cp_async_commit();
  }
  if (staged) {  // this tile's psi (the group before the cost tile's) is in
    if (cost) cp_async_wait<1>();
    else cp_async_wait<0>();
  }
  const uint64_t z0 = local_to_z(g, base, tb0);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const uint64_t z = z0 + (uint64_t)r * zs;
    const uint32_t ps = tb0 + ((uint32_t)r << CF::lo(0));
    if constexpr (FX) v[r] = init ? make_longlong2(a.init_fx, 0) : staged ? s.Ps[ps] : ld_state<COHERENT>((const V*)a.psi + s.zoff + z);
    else v[r] = init ? make_float2(a.init_f32, 0.f) : staged ? s.Ps[ps] : ld_state<COHERENT>((const V*)a.psi + s.zoff + z);
    if constexpr (TWO) w[r] = ld_lam ? ld_state<COHERENT>((const V*)a.lam + s.zoff + z) : V{};
  }
  if (stage && next >= 0) {
    const uint64_t zn = local_to_z(g, tile_base(g, next), tb0);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      V* dst = s.Ps + tb0 + ((uint32_t)r << CF::lo(0));
      const V* src = (const V*)a.psi + s.zoff + zn + (uint64_t)r * zs;
      if constexpr (sizeof(V) == 16) cp_async16(dst, src);
      else cp_async8(dst, src);
    }
    cp_async_commit();
  }
  if (cost) {
    if (stage) {  // all but the newest group (the prefetch, if any): the cost tile is in
      if (next >= 0) cp_async_wait<1>();
      else cp_async_wait<0>();
    } else {
      cp_async_wait_all();
    }
    __syncthreads();
  }
  s.template run<LAST, OPS>();
  const uint64_t z1 = local_to_z(g, base, tb0);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const uint64_t z = s.zoff + z1 + (uint64_t)r * zs;
    if constexpr (FX) {
      if (st_fmt == 0) ((V*)a.psi)[z] = v[r];
      else if (st_fmt == 1)
        ((double2*)a.psi)[z] = make_double2(fx_to_double(v[r].x, a.fx_shift), fx_to_double(v[r].y, a.fx_shift));
    } else {
      if (st_fmt >= 0) ((V*)a.psi)[z] = v[r];
    }
    if (st_lam) ((V*)a.lam)[z] = w[r];
  }
}

}  // namespace
}  // namespace qaoa
