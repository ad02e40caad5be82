// S1 — cost vector C(z) of a weighted MaxCut instance over all 2^n bitstrings
// ("precomputation of the cost Hamiltonian", Sec. I and Sec. IV-A; bit order of Eq. 3).
//
// Split z into its low L bits x and high bits h.  Every edge is low-low, high-high
// or low-high, and for a low-high edge (u low, v high)
//   w [x_u != h_v] = w h_v + x_u w (1 - 2 h_v),
// so C(z) = A[x] + K(h) + sum_{u < L} x_u a_u(h) with
//   A[x]   = sum over low-low edges of w [x_u != x_v]        (one table per block),
//   K(h)   = sum over high-high edges of w [h_u != h_v] + sum over low-high edges of w h_v,
//   a_u(h) = sum over high neighbours v of u of w_uv (1 - 2 h_v).
// A block builds A once in shared memory, then walks its high parts h; per element
// the work is four shared-memory reads and three adds (details at the kernel).  Integer weights accumulate
// exactly in int64 (stored as int32 or float64).  Float weights are quantised once to
// a common fixed point (int64, value * 2^shift), summed exactly, and rounded once to
// float64 at the store.
#include "internal.h"

namespace qaoa {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxLowBits = 12;

// A block stages the weights in shared memory, builds the low-low table A and the sums
// b_v = sum_{u < L} w_uv of every high vertex once, then per high part h: a_u(h) for the L
// low vertices, K(h) by one warp (a lane per high vertex), and sum_u x_u a_u(h) as two
// 64-entry tables over the low six and the next six low bits; an element is then four
// shared-memory reads and three adds, and the block writes 2^L consecutive costs.
__global__ void __launch_bounds__(kThreads) cost_kernel(const __grid_constant__ CostArgs a) {
  __shared__ long long A[1 << kMaxLowBits];
  __shared__ long long W[QAOA_MAX_N][QAOA_MAX_N];
  __shared__ long long bsum[QAOA_MAX_N];
  __shared__ long long au[kMaxLowBits];
  __shared__ long long S0[64], S1[64];
  __shared__ long long Kh;
  const int n = a.n, L = a.lo_bits, tid = threadIdx.x;
  const uint32_t X = 1u << L;
  for (int i = tid; i < n * n; i += kThreads) W[i / n][i % n] = a.wi[i / n][i % n];
  __syncthreads();
  for (uint32_t x = tid; x < X; x += kThreads) {  // low-low table
    long long s = 0;
    for (int u = 0; u < L; ++u)
      for (int v = u + 1; v < L; ++v)
        if (((x >> u) ^ (x >> v)) & 1) s += W[u][v];
    A[x] = s;
  }
  for (int v = L + tid; v < n; v += kThreads) {
    long long s = 0;
    for (int u = 0; u < L; ++u) s += W[u][v];
    bsum[v] = s;
  }
  const int64_t H = 1ll << (n - L);
  for (int64_t h = blockIdx.x; h < H; h += gridDim.x) {
    __syncthreads();  // the previous h is done with au, S0, S1 and Kh
    if (tid < L) {
      long long s = 0;
      for (int v = L; v < n; ++v) s += ((h >> (v - L)) & 1) ? -W[tid][v] : W[tid][v];
      au[tid] = s;
    } else if (tid >= 32 && tid < 64) {  // K(h): lane k handles high vertex L + k (n - L <= 32)
      const int u = L + (tid - 32);
      long long s = 0;
      if (u < n) {
        const int hu = (h >> (u - L)) & 1;
        if (hu) s = bsum[u];
        for (int v = u + 1; v < n; ++v)
          if (hu ^ ((h >> (v - L)) & 1)) s += W[u][v];
      }
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (tid == 32) Kh = s;
    }
    __syncthreads();
    if (tid < 128) {  // sum_u x_u a_u(h) over bits [0, 6) and [6, 12)
      const int idx = tid & 63, b0 = (tid >> 6) * 6;
      long long s = 0;
      for (int k = 0; k < 6; ++k)
        if (b0 + k < L && ((idx >> k) & 1)) s += au[b0 + k];
      if (tid < 64) S0[idx] = s;
      else S1[idx] = s;
    }
    __syncthreads();
    const uint64_t zbase = (uint64_t)h << L;
    const long long kh = Kh;
    for (uint32_t x = tid; x < X; x += kThreads) {
      const long long c = A[x] + kh + S0[x & 63] + S1[x >> 6];
      const uint64_t z = zbase | x;
      if (a.cost_dtype == QAOA_COST_I32) {
        ((int*)a.C)[z] = (int)c;
      } else if (a.integer) {
        ((double*)a.C)[z] = (double)c;
      } else {
        ((double*)a.C)[z] = ldexp((double)c, -a.fixed_shift);
      }
    }
  }
}

// General PUBO cost (Eq. 3): C(z) = sum_t w_t [z AND mask_t == mask_t] over one chunk of
// terms held in the kernel parameters.  A block owns 2^L consecutive z (fixed high part h)
// and walks the terms in order; a term whose high mask h does not cover is skipped by the
// whole block at once.  Weights are integers or one common fixed point, so the sum is
// exact in int64 and independent of the term order; float64 costs are rounded once per
// chunk.
constexpr int kPuboPer = 16;  // z per thread: 2^12 per block

__global__ void __launch_bounds__(kThreads) pubo_kernel(const __grid_constant__ PuboArgs a) {
  const int L = a.n < 12 ? a.n : 12;
  const uint32_t X = 1u << L;
  const int64_t H = 1ll << (a.n - L);
  for (int64_t h = blockIdx.x; h < H; h += gridDim.x) {
    long long c[kPuboPer];
#pragma unroll
    for (int j = 0; j < kPuboPer; ++j) c[j] = 0;
    for (int t = 0; t < a.nterms; ++t) {
      const uint32_t m = a.mask[t];
      const uint64_t mh = (uint64_t)(m >> L);
      if (((uint64_t)h & mh) != mh) continue;  // uniform over the block
      const uint32_t ml = m & (X - 1);
      const long long q = a.q[t];
#pragma unroll
      for (int j = 0; j < kPuboPer; ++j) {
        const uint32_t x = threadIdx.x + j * kThreads;
        if ((x & ml) == ml) c[j] += q;
      }
    }
    const uint64_t zbase = (uint64_t)h << L;
#pragma unroll
    for (int j = 0; j < kPuboPer; ++j) {
      const uint32_t x = threadIdx.x + j * kThreads;
      if (x >= X) continue;
      const uint64_t z = zbase | x;
      if (a.cost_dtype == QAOA_COST_I32) {
        ((int*)a.C)[z] = (int)(c[j] + (a.accumulate ? ((int*)a.C)[z] : 0));
      } else {
        const double v = a.integer ? (double)c[j] : ldexp((double)c[j], -a.fixed_shift);
        ((double*)a.C)[z] = a.accumulate ? ((double*)a.C)[z] + v : v;
      }
    }
  }
}

}  // namespace

cudaError_t launch_cost(const CostArgs& a, cudaStream_t s) {
  const int64_t H = 1ll << (a.n - a.lo_bits);
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t cap = (int64_t)sms * 4;
  const int grid = (int)(H < cap ? H : cap);
  note_launch(1, s, true);
  cost_kernel<<<grid, kThreads, 0, s>>>(a);
  note_launch(1, s, false, (double)(1ull << a.n) * (a.cost_dtype == QAOA_COST_I32 ? 4.0 : 8.0));
  return cudaGetLastError();
}

cudaError_t launch_pubo(const PuboArgs& a, cudaStream_t s) {
  const int L = a.n < 12 ? a.n : 12;
  const int64_t H = 1ll << (a.n - L);
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t cap = (int64_t)sms * 8;
  const int grid = (int)(H < cap ? H : cap);
  const double cb = a.cost_dtype == QAOA_COST_I32 ? 4.0 : 8.0;
  note_launch(1, s, true);
  pubo_kernel<<<grid, kThreads, 0, s>>>(a);
  note_launch(1, s, false, (double)(1ull << a.n) * cb * (a.accumulate ? 2.0 : 1.0));
  return cudaGetLastError();
}

}  // namespace qaoa
