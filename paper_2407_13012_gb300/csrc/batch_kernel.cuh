// Persistent kernel of the batched gradients (shared by the translation units that
// instantiate it): one CTA per graph at a time, the graph's whole sweep plan, tile after
// tile, with CTA barriers between sweeps; complex128 sweeps on full 2^12 tiles may use the
// lean tile code.
#pragma once

#include "sweeper.cuh"

namespace qaoa {
namespace {

// complex128 (fixed point) and complex64 tiles for two buffers
using CfgXB = Cfg<12, 3, 3, 3, 1>;
using CfgXS = Cfg<10, 3, 3, 3, 2>;
using CfgFB = Cfg<12, 4, 4, 4, 2>;
using CfgFS = Cfg<10, 3, 3, 4, 2>;

// the sweep's tiles with the lean tile code of layout sequence 0..L
template <class CF, bool FX, bool TWO>
__device__ __forceinline__ void lean_tiles(Lean<CF, FX, TWO>& s, const SweepArgs& a, int last, void* Cs) {
  const int64_t tiles = a.g.tiles;
  switch (last) {
    case 0:
      for (int64_t t = 0; t < tiles; ++t) lean_tile<CF, FX, TWO, true, 0, true>(s, a, t, Cs);
      break;
    case 1:
      if constexpr (CF::NR > 1)
        for (int64_t t = 0; t < tiles; ++t) lean_tile<CF, FX, TWO, true, (CF::NR > 1 ? 1 : 0), true>(s, a, t, Cs);
      break;
    case 2:
      if constexpr (CF::NR > 2)
        for (int64_t t = 0; t < tiles; ++t) lean_tile<CF, FX, TWO, true, (CF::NR > 2 ? 2 : 0), true>(s, a, t, Cs);
      break;
    default:
      if constexpr (CF::NR > 3)
        for (int64_t t = 0; t < tiles; ++t) lean_tile<CF, FX, TWO, true, (CF::NR > 3 ? 3 : 0), true>(s, a, t, Cs);
      break;
  }
}

template <class CF, bool FX, bool LEAN>
__global__ void __launch_bounds__(CF::NT, CF::MINB) batch_kernel(const __grid_constant__ BatchArgs b, int first,
                                                                int count, int* queue) {
  using S = Lean<CF, FX, true>;
  using V = typename S::V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* X = (V*)smem_raw;  // exchange area for two buffers: 2 x 2^B slots
  void* Cs = smem_raw + ((sizeof(V) << CF::B) << 1);
  __shared__ SweepArgs sa;
  __shared__ double blk[kMaxAcc];
  __shared__ double red[2 * (CF::NT / 32)];
  __shared__ fx::Factor dsm[16];
  __shared__ int cur;
  // lean sweeps: per-warp accumulators (summed with blk at the end of the graph) and every
  // mixer diagonal of the sweep staged once
  constexpr int NW = CF::NT / 32;
  __shared__ double wacc[LEAN ? kMaxAcc * NW : 1];
  __shared__ fx::Factor dpre[LEAN && FX ? kLeanMix * 16 : 1];
  const int tid = threadIdx.x;
  const int p = b.p;
  const int nout = 2 * p + 2;
  for (;;) {
    __syncthreads();  // the previous graph is finished with cur, blk and sa
    if (tid == 0) cur = atomicAdd(queue, 1);
    for (int r = tid; r < nout; r += CF::NT) blk[r] = 0.0;
    if constexpr (LEAN)
      for (int r = tid; r < nout * NW; r += CF::NT) wacc[r] = 0.0;
    __syncthreads();
    const int gi = cur;
    if (gi >= count) break;
    const int64_t gidx = first + gi;
    const BatchGraph G = b.graphs[gidx];
    const BatchPlan& P = b.plans[G.plan];
    const size_t vs = sizeof(V);
    for (int si = 0; si < P.nsweeps; ++si) {
      const BatchSweep& bs = P.sw[si];
      __syncthreads();  // the previous sweep's stores and its use of sa are complete
      if (tid == 0) {
        sa.kind = SWEEP_GENERIC;
        sa.psi = (char*)b.psi + G.state * vs;
        sa.lam = (char*)b.lam + G.state * vs;
        sa.C = (const char*)b.C + G.cost * (b.cost_f64 ? 8 : 4);
        sa.cost_dtype = b.cost_f64 ? QAOA_COST_F64 : QAOA_COST_I32;
        sa.needs_cost = bs.needs_cost;
        sa.g = bs.g;
        sa.tile_bits = CF::B;
        sa.load_fmt = bs.load_fmt;
        sa.store_fmt = bs.store_fmt;
        sa.load_lam = bs.load_lam;
        sa.store_lam = bs.store_lam;
        sa.init_fx = P.init_fx;
        sa.init_f32 = P.init_f32;
        sa.fx_shift = P.fx_shift;
        sa.norm2_dev = nullptr;
        sa.cmax_dev = nullptr;
        sa.nops = bs.nops;
        sa.dev_trig = b.trig + gidx * 3 * p;
        sa.np = p;
        sa.phase_table = G.span > 0 ? (const char*)b.phase + G.table * vs : nullptr;
        sa.cmin = G.cmin;
        sa.span = G.span;
        sa.smem_table_layer = -1;
        sa.d_table = FX ? (const char*)b.dtab + gidx * p * 196 * sizeof(longlong2) : nullptr;
        sa.turn_table = b.turn;
        sa.nred = 0;
        sa.partials = nullptr;
        sa.grid = 0;
      }
      for (int k = tid; k < bs.nops; k += CF::NT) sa.ops[k] = bs.ops[k];
      __syncthreads();
      const bool lean = LEAN && bs.lean_last >= 0;
      bool staged = false;
      if constexpr (LEAN && FX) {
        if (lean) {  // exp(-i beta (t - 2k)), k = 0..t, of each mixer, as prepared factors
          const int t = bs.g.t;
          int m = 0;
          for (int k = 0; k < bs.nops; ++k) m += (bs.ops[k] & 0xff) == OP_MIX;
          if (m <= kLeanMix) {
            m = 0;
            for (int k = 0; k < bs.nops; ++k) {
              const uint32_t op = bs.ops[k];
              if ((op & 0xff) != OP_MIX) continue;
              if (tid <= t) {
                const longlong2 e =
                    __ldg((const longlong2*)sa.d_table + ((long long)((op >> 16) & 0xff) * 14 + t) * 14 + tid);
                dpre[16 * m + tid] = fx::factor(e.x, (op & F_SIGN) ? -e.y : e.y);
              }
              ++m;
            }
            staged = true;
            __syncthreads();
          }
        }
      }
      if (lean && !bs.two) {  // forward sweep: psi alone
        Lean<CF, FX, false> s1(sa, X, Cs, blk, red);
        s1.Ds = dsm;
        s1.evalid = 1u << CF::B;
        s1.wacc = wacc;
        if (staged) s1.dpre = dpre;
        lean_tiles<CF, FX, false>(s1, sa, bs.lean_last, Cs);
      } else {
        S s(sa, X, Cs, blk, red);
        s.Ds = dsm;
        s.evalid = 1u << (bs.g.t + bs.g.c);
        if constexpr (FX) s.lam_shift = G.lam_shift;
        if (lean) {
          s.wacc = wacc;
          if (staged) s.dpre = dpre;
          lean_tiles<CF, FX, true>(s, sa, bs.lean_last, Cs);
        } else {
          for (int64_t tile = 0; tile < bs.g.tiles; ++tile) sweep_tile<CF, FX, true, true>(s, sa, tile, Cs);
        }
      }
    }
    __syncthreads();  // block_add results are in blk and wacc
    for (int r = tid; r < nout; r += CF::NT) {
      double v = blk[r];
      if constexpr (LEAN)
        for (int w = 0; w < NW; ++w) v += wacc[r * NW + w];
      b.out[(int64_t)G.out * nout + r] = v;
    }
  }
}

template <class CF, bool FX, bool LEAN>
cudaError_t launch_batch_cfg(const BatchArgs& b, int first, int count, int* queue, cudaStream_t s) {
  const size_t xb = (sizeof(typename Sweeper<CF, FX, true>::V) << CF::B) << 1;  // two-buffer exchange area
  const size_t smem = xb + ((size_t)(b.cost_f64 ? 8 : 4) << CF::B);
  const size_t smem_max = xb + ((size_t)8 << CF::B);
  static std::mutex mu;
  static uint64_t done = 0;
  static int per_sm = 1, sms = 1;
  once_per_device(mu, done, [&] {
    cudaFuncSetAttribute(batch_kernel<CF, FX, LEAN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<CF, FX, LEAN>, CF::NT, smem_max);
    if (per_sm < 1) per_sm = 1;
  });
  const int grid = std::max(1, std::min(count, sms * per_sm));
  batch_kernel<CF, FX, LEAN><<<grid, CF::NT, smem, s>>>(b, first, count, queue);
  return cudaGetLastError();
}

}  // namespace
}  // namespace qaoa
