// Layer sweeps: phase separator, RX mixer, lambda = C psi and the fused reductions of
// <C>, the norm and the adjoint-gradient terms (Eq. 1; Sec. II-B, IV-B, IV-C, IV-D).
//
// One kernel runs one sweep: a persistent grid walks the tiles of the state; each
// tile is staged in shared memory, the sweep's operation program runs on it, and
// the tile is written back.  Reductions accumulate per thread across tiles and are
// folded per block into a partials array, so the order of every floating-point sum
// is fixed for a given grid (deterministic results).
#include "internal.h"

#include <cuda_runtime.h>

namespace qaoa {
namespace {

constexpr int kThreads = 256;
constexpr int kTileBits = 11;  // 2^11 amplitudes per buffer per tile

template <typename R> struct Cplx;
template <> struct Cplx<double> { using T = double2; };
template <> struct Cplx<float> { using T = float2; };

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

__device__ __forceinline__ double cost_at(const void* C, int cost_dtype, uint64_t z) {
  if (cost_dtype == QAOA_COST_I32) return (double)__ldg((const int*)C + z);
  return __ldg((const double*)C + z);
}

template <typename R>
__device__ __forceinline__ typename Cplx<R>::T cmul(typename Cplx<R>::T a, typename Cplx<R>::T e) {
  typename Cplx<R>::T r;
  r.x = a.x * e.x - a.y * e.y;
  r.y = a.x * e.y + a.y * e.x;
  return r;
}

// exp(-i s gamma_l C(z)) as (re, im)
template <typename R>
__device__ __forceinline__ typename Cplx<R>::T phase_at(const SweepArgs& a, int layer, bool inverse,
                                                         uint64_t z) {
  typename Cplx<R>::T e;
  const int64_t k = a.phase_table != nullptr ? (int64_t)__ldg((const int*)a.C + z) - a.cmin : -1;
  if (k >= 0 && k < a.span) {  // entries outside the descriptor's bounds take the direct path
    const typename Cplx<R>::T* tab = (const typename Cplx<R>::T*)a.phase_table;
    e = tab[(int64_t)layer * a.span + k];
  } else {
    const double th = a.gamma[layer] * cost_at(a.C, a.cost_dtype, z);
    double sn, cs;
    sincos(th, &sn, &cs);
    e.x = (R)cs;
    e.y = (R)(-sn);
  }
  if (inverse) e.y = -e.y;
  return e;
}

template <typename R>
__global__ void __launch_bounds__(kThreads) sweep_kernel(const __grid_constant__ SweepArgs a) {
  using T = typename Cplx<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SweepGeom& g = a.g;
  const int bits = g.t + g.c;
  const uint32_t E = 1u << bits;
  T* sp = (T*)smem_raw;
  T* sl = sp + E;
  const bool two = (a.lam != nullptr);
  T* gpsi = (T*)a.psi;
  T* glam = (T*)a.lam;
  __shared__ double blk_acc[kMaxAcc];
  __shared__ double red_tmp[2][kThreads / 32];
  for (int r = threadIdx.x; r < kMaxAcc; r += kThreads) blk_acc[r] = 0.0;
  // block-reduce (v0, v1) and add to blk_acc[r] (and blk_acc[r + 1] when two)
  auto block_add = [&](int r, double v0, double v1, bool two_vals) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int o = 16; o > 0; o >>= 1) {
      v0 += __shfl_down_sync(0xffffffffu, v0, o);
      v1 += __shfl_down_sync(0xffffffffu, v1, o);
    }
    if (lane == 0) {
      red_tmp[0][warp] = v0;
      red_tmp[1][warp] = v1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double s0 = 0.0, s1 = 0.0;
      for (int w = 0; w < kThreads / 32; ++w) {
        s0 += red_tmp[0][w];
        s1 += red_tmp[1][w];
      }
      blk_acc[r] += s0;
      if (two_vals) blk_acc[r + 1] += s1;
    }
    __syncthreads();
  };
  const R amp0 = (R)rsqrt((double)(1ull << g.n));

  for (int64_t tile = blockIdx.x; tile < g.tiles; tile += gridDim.x) {
    const uint64_t base = tile_base(g, tile);
    for (uint32_t i = threadIdx.x; i < E; i += kThreads) {
      const uint64_t z = local_to_z(g, base, i);
      if (a.init_plus) {
        sp[i] = T{amp0, (R)0};
      } else if (a.load_psi) {
        sp[i] = gpsi[z];
      }
      if (two && a.load_lam) sl[i] = glam[z];
    }
    __syncthreads();

    for (int k = 0; k < a.nops; ++k) {
      const uint32_t op = a.ops[k];
      const uint32_t kind = op & 0xff;
      const uint32_t arg = op >> 16;
      const bool on_psi = op & F_PSI, on_lam = op & F_LAM, inv = op & F_SIGN;
      if (kind == OP_PHASE) {
        for (uint32_t i = threadIdx.x; i < E; i += kThreads) {
          const uint64_t z = local_to_z(g, base, i);
          const T e = phase_at<R>(a, arg, inv, z);
          if (on_psi) sp[i] = cmul<R>(sp[i], e);
          if (on_lam) sl[i] = cmul<R>(sl[i], e);
        }
      } else if (kind == OP_MIX) {
        const R cb = (R)a.cosb[arg];
        const R sb = (R)(inv ? -a.sinb[arg] : a.sinb[arg]);
        for (int q = 0; q < g.t; ++q) {
          const int bit = g.c + q;
          const uint32_t lowmask = (1u << bit) - 1;
          for (uint32_t pi = threadIdx.x; pi < (E >> 1); pi += kThreads) {
            const uint32_t ia = ((pi & ~lowmask) << 1) | (pi & lowmask);
            const uint32_t ib = ia | (1u << bit);
            if (on_psi) {
              const T x = sp[ia], y = sp[ib];
              sp[ia] = T{cb * x.x + sb * y.y, cb * x.y - sb * y.x};
              sp[ib] = T{cb * y.x + sb * x.y, cb * y.y - sb * x.x};
            }
            if (on_lam) {
              const T x = sl[ia], y = sl[ib];
              sl[ia] = T{cb * x.x + sb * y.y, cb * x.y - sb * y.x};
              sl[ib] = T{cb * y.x + sb * x.y, cb * y.y - sb * x.x};
            }
          }
          __syncthreads();
        }
      } else if (kind == OP_LAMBDA) {
        for (uint32_t i = threadIdx.x; i < E; i += kThreads) {
          const uint64_t z = local_to_z(g, base, i);
          const R cz = (R)cost_at(a.C, a.cost_dtype, z);
          sl[i] = T{cz * sp[i].x, cz * sp[i].y};
        }
      } else if (kind == OP_RED_EXPECT) {
        double e0 = 0.0, e1 = 0.0;
        for (uint32_t i = threadIdx.x; i < E; i += kThreads) {
          const uint64_t z = local_to_z(g, base, i);
          const double pr = (double)sp[i].x * sp[i].x + (double)sp[i].y * sp[i].y;
          e0 += cost_at(a.C, a.cost_dtype, z) * pr;
          e1 += pr;
        }
        block_add(arg, e0, e1, true);
      } else if (kind == OP_RED_XTERM) {
        double e0 = 0.0;
        for (int q = 0; q < g.t; ++q) {
          const int bit = g.c + q;
          const uint32_t lowmask = (1u << bit) - 1;
          for (uint32_t pi = threadIdx.x; pi < (E >> 1); pi += kThreads) {
            const uint32_t ia = ((pi & ~lowmask) << 1) | (pi & lowmask);
            const uint32_t ib = ia | (1u << bit);
            const T la = sl[ia], lb = sl[ib], pa = sp[ia], pb = sp[ib];
            // Im(conj(la) pb + conj(lb) pa)
            e0 += (double)la.x * pb.y - (double)la.y * pb.x + (double)lb.x * pa.y - (double)lb.y * pa.x;
          }
        }
        block_add(arg, 2.0 * e0, 0.0, false);
      } else if (kind == OP_RED_CTERM) {
        double e0 = 0.0;
        for (uint32_t i = threadIdx.x; i < E; i += kThreads) {
          const uint64_t z = local_to_z(g, base, i);
          const T l = sl[i], p = sp[i];
          e0 += cost_at(a.C, a.cost_dtype, z) * ((double)l.x * p.y - (double)l.y * p.x);
        }
        block_add(arg, 2.0 * e0, 0.0, false);
      }
      __syncthreads();
    }

    for (uint32_t i = threadIdx.x; i < E; i += kThreads) {
      const uint64_t z = local_to_z(g, base, i);
      if (a.store_psi) gpsi[z] = sp[i];
      if (two && a.store_lam) glam[z] = sl[i];
    }
    __syncthreads();
  }

  // write this block's accumulators
  __syncthreads();
  for (int r = threadIdx.x; r < a.nred; r += kThreads)
    a.partials[(int64_t)a.red_slot[r] * a.grid + blockIdx.x] = blk_acc[r];
}

__global__ void reduce_kernel(const __grid_constant__ ReducePlan r, const double* __restrict__ partials,
                              double* __restrict__ out) {
  const int o = blockIdx.x;
  __shared__ double sh[256];
  double v = 0.0;
  const int64_t n = (int64_t)r.ncontrib[o] * r.grid;
  const double* base = partials + (int64_t)o * kMaxContrib * r.grid;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) v += base[i];
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[o] = sh[0];
}

template <typename T>
__global__ void phase_table_kernel(const __grid_constant__ SweepArgs a, int p, T* __restrict__ table) {
  const int64_t total = (int64_t)p * a.span;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int l = (int)(i / a.span);
    const int64_t c = a.cmin + (i - (int64_t)l * a.span);
    const double th = a.gamma[l] * (double)c;
    double sn, cs;
    sincos(th, &sn, &cs);
    table[i] = T{(decltype(T::x))cs, (decltype(T::x))(-sn)};
  }
}

template <typename R>
int max_blocks_per_sm() {
  static int cached = 0;
  if (!cached) {
    int dev = 0;
    cudaGetDevice(&dev);
    const size_t smem = 2 * sizeof(typename Cplx<R>::T) << kTileBits;
    cudaFuncSetAttribute(sweep_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel<R>, kThreads, smem);
    cached = nb > 0 ? nb : 1;
  }
  return cached;
}

int num_sms() {
  static int cached = 0;
  if (!cached) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&cached, cudaDevAttrMultiProcessorCount, dev);
    if (cached <= 0) cached = 1;
  }
  return cached;
}

}  // namespace

int sweep_tile_bits(int /*dtype*/) { return kTileBits; }

int sweep_grid(int dtype, int64_t tiles) {
  const int per_sm = dtype == QAOA_C128 ? max_blocks_per_sm<double>() : max_blocks_per_sm<float>();
  const int64_t cap = (int64_t)num_sms() * per_sm;
  return (int)(tiles < cap ? tiles : cap);
}

cudaError_t launch_sweep(int dtype, const SweepArgs& a, cudaStream_t s) {
  const int bits = a.g.t + a.g.c;
  const bool two = a.lam != nullptr;
  note_launch(0, s, true);
  if (dtype == QAOA_C128) {
    max_blocks_per_sm<double>();
    const size_t smem = (two ? 2 : 1) * sizeof(double2) << bits;
    sweep_kernel<double><<<a.grid, kThreads, smem, s>>>(a);
  } else {
    max_blocks_per_sm<float>();
    const size_t smem = (two ? 2 : 1) * sizeof(float2) << bits;
    sweep_kernel<float><<<a.grid, kThreads, smem, s>>>(a);
  }
  note_launch(0, s, false, a.algo_bytes);
  return cudaGetLastError();
}

cudaError_t launch_reduce(const ReducePlan& r, const double* partials, double* out, cudaStream_t s) {
  note_launch(3, s, true);
  reduce_kernel<<<r.nout, 256, 0, s>>>(r, partials, out);
  note_launch(3, s, false);
  return cudaGetLastError();
}

cudaError_t launch_phase_table(int dtype, const double* gamma, int p, int64_t cmin, int64_t span,
                               void* table, cudaStream_t s) {
  SweepArgs a{};
  for (int l = 0; l < p; ++l) a.gamma[l] = gamma[l];
  a.cmin = cmin;
  a.span = span;
  const int64_t total = (int64_t)p * span;
  const int blocks = (int)((total + 255) / 256 < 1024 ? (total + 255) / 256 : 1024);
  note_launch(3, s, true);
  if (dtype == QAOA_C128)
    phase_table_kernel<double2><<<blocks > 0 ? blocks : 1, 256, 0, s>>>(a, p, (double2*)table);
  else
    phase_table_kernel<float2><<<blocks > 0 ? blocks : 1, 256, 0, s>>>(a, p, (float2*)table);
  note_launch(3, s, false);
  return cudaGetLastError();
}

}  // namespace qaoa
