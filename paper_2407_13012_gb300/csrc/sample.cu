// S5 + S6 — sampling bitstrings from |psi_z|^2 on the device, each returned with its
// objective value (Sec. IV-D).
//
// The state is cut into leaves of 2^leaf_bits amplitudes.  (1) one read sweep sums
// |psi|^2 per leaf; (2) an exclusive scan turns the leaf sums into a prefix array
// whose last entry is the total; (3) one warp per shot draws u_i from the SplitMix64
// counter stream, finds the leaf holding u_i * total by binary search in the prefix,
// and scans that leaf with a warp prefix sum to find
//   z_i = min{z : P(z) > u_i * P_total}.
// Every sum runs in float64 in a fixed order, so a given seed always yields the same
// samples on a given device.
#include "internal.h"

namespace qaoa {
namespace {

constexpr int kThreads = 256;
constexpr int kChunk = kThreads * 16;  // leaves per scan block

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double prob_at(const void* psi, int dtype, uint64_t z) {
  if (dtype == QAOA_C128) {
    const double2 v = __ldg((const double2*)psi + z);
    return v.x * v.x + v.y * v.y;
  }
  const float2 v = __ldg((const float2*)psi + z);
  return (double)v.x * v.x + (double)v.y * v.y;
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Double-float accumulation in float32 (the float64 pipe retires ~1.75 FMA per SM clock, so
// a float64 product per amplitude would bound the complex64 leaf sums): x^2 = p + e exactly
// (one FMA gives e), and (s, c) absorbs p by Knuth's two-sum, so s + c carries the exact
// sum to ~2^-44 relative.
struct F2Sum {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add_sq(float x) {
    const float p = x * x;
    const float e = fmaf(x, x, -p);
    const float t = s + p;
    const float bp = t - s;
    const float err = (s - (t - bp)) + (p - bp);
    s = t;
    c += err + e;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// (1) one warp per leaf; a.len entries (the last leaf may be partly past the end).  Full
// leaves of an aligned vector take 16-byte loads, all issued before the sums (complex128:
// one amplitude per load, two independent float64 FMA chains; complex64: two amplitudes
// per load, double-float sums in float32); other leaves go amplitude by amplitude.
__global__ void leaf_sum_kernel(const __grid_constant__ SampleArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const uint32_t L = 1u << a.leaf_bits;
  const int64_t nleaf = (int64_t)((a.len + L - 1) >> a.leaf_bits);
  const bool vec = a.leaf_bits == 10 && ((uintptr_t)a.psi & 15) == 0;
  for (int64_t li = warp; li < nleaf; li += nwarps) {
    const uint64_t base = (uint64_t)li << a.leaf_bits;
    double s = 0.0;
    if (vec && base + L <= a.len) {
      if (a.dtype == QAOA_C128) {
        const double2* q = (const double2*)a.psi + base + lane;
        double s0 = 0.0, s1 = 0.0;
#pragma unroll
        for (int m0 = 0; m0 < 32; m0 += 8) {
          double2 v[8];
#pragma unroll
          for (int m = 0; m < 8; ++m) v[m] = __ldg(q + 32 * (m0 + m));
#pragma unroll
          for (int m = 0; m < 8; ++m) {
            s0 = fma(v[m].x, v[m].x, s0);
            s1 = fma(v[m].y, v[m].y, s1);
          }
        }
        s = s0 + s1;
      } else {
        const float4* q = (const float4*)a.psi + (base >> 1) + lane;
        F2Sum f0, f1;
#pragma unroll
        for (int m0 = 0; m0 < 16; m0 += 8) {
          float4 v[8];
#pragma unroll
          for (int m = 0; m < 8; ++m) v[m] = __ldg(q + 32 * (m0 + m));
#pragma unroll
          for (int m = 0; m < 8; ++m) {
            f0.add_sq(v[m].x);
            f1.add_sq(v[m].y);
            f0.add_sq(v[m].z);
            f1.add_sq(v[m].w);
          }
        }
        s = f0.value() + f1.value();
      }
    } else {
      for (uint32_t k = lane; k < L && base + k < a.len; k += 32) s += prob_at(a.psi, a.dtype, base + k);
    }
    s = warp_sum(s);
    if (lane == 0) a.leaf[li] = s;
  }
}

// (2a) per chunk totals
__global__ void chunk_sum_kernel(const double* __restrict__ leaf, int64_t nleaf, double* __restrict__ bsum) {
  __shared__ double sh[kThreads];
  const int64_t base = (int64_t)blockIdx.x * kChunk;
  double s = 0.0;
  for (int k = 0; k < 16; ++k) {
    const int64_t i = base + (int64_t)threadIdx.x * 16 + k;
    if (i < nleaf) s += leaf[i];
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int st = kThreads / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) bsum[blockIdx.x] = sh[0];
}

// (2b) exclusive scan of the chunk totals, one thread (a few thousand entries at most)
__global__ void chunk_scan_kernel(double* bsum, int64_t nchunks) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double run = 0.0;
    for (int64_t i = 0; i < nchunks; ++i) {
      const double v = bsum[i];
      bsum[i] = run;
      run += v;
    }
    bsum[nchunks] = run;
  }
}

// (2c) exclusive scan inside each chunk; prefix[nleaf] = total
__global__ void leaf_scan_kernel(const double* __restrict__ leaf, int64_t nleaf, const double* __restrict__ bsum,
                                 double* __restrict__ prefix, int64_t nchunks) {
  __shared__ double sh[kThreads];
  const int64_t base = (int64_t)blockIdx.x * kChunk + (int64_t)threadIdx.x * 16;
  double v[16];
  double s = 0.0;
  for (int k = 0; k < 16; ++k) {
    v[k] = (base + k < nleaf) ? leaf[base + k] : 0.0;
    s += v[k];
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {  // sequential exclusive scan of 256 thread totals
    double run = 0.0;
    for (int t = 0; t < kThreads; ++t) {
      const double x = sh[t];
      sh[t] = run;
      run += x;
    }
  }
  __syncthreads();
  double run = bsum[blockIdx.x] + sh[threadIdx.x];
  for (int k = 0; k < 16; ++k) {
    if (base + k < nleaf) prefix[base + k] = run;
    run += v[k];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) prefix[nleaf] = bsum[nchunks];
}

// (3) one warp per shot
__global__ void draw_kernel(const __grid_constant__ SampleArgs a, const double* __restrict__ prefix) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const uint32_t L = 1u << a.leaf_bits;
  const int64_t nleaf = (int64_t)((a.len + L - 1) >> a.leaf_bits);
  const double total = prefix[nleaf];
  const uint64_t sbase = mix64(mix64(a.seed) ^ 0x5f5f656c706d6173ull);
  for (int64_t i = warp; i < a.shots; i += nwarps) {
    const uint64_t x = mix64(sbase + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull);
    const double u = (double)(x >> 11) * 0x1.0p-53;
    const double target = u * total;
    // largest leaf li with prefix[li] <= target and positive mass; all lanes agree
    int64_t lo = 0, hi = nleaf;  // invariant: prefix[lo] <= target, answer in [lo, hi)
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) >> 1;
      if (prefix[mid] <= target) lo = mid; else hi = mid;
    }
    int64_t li = lo;
    bool past_end = !(target < total);
    if (past_end) {  // the last leaf with positive mass (the last leaf if there is none)
      li = nleaf - 1;
      if (total > 0.0)
        while (li > 0 && !(prefix[li + 1] > prefix[li])) --li;
    }
    const uint64_t base = (uint64_t)li << a.leaf_bits;
    const uint32_t Lh = a.len - base < L ? (uint32_t)(a.len - base) : L;  // entries in this leaf
    const double rem = target - prefix[li];
    double run = 0.0;
    int64_t found = -1, last_nz = -1;
    for (uint32_t k0 = 0; k0 < Lh && found < 0; k0 += 32) {
      const uint32_t k = k0 + lane;
      const double pk = (k < Lh) ? prob_at(a.psi, a.dtype, base + k) : 0.0;
      double incl = pk;
      for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const unsigned hit = __ballot_sync(0xffffffffu, !past_end && (run + incl > rem) && pk > 0.0);
      const unsigned nzm = __ballot_sync(0xffffffffu, pk > 0.0);
      if (nzm) last_nz = k0 + 31 - __clz(nzm);
      if (hit) found = k0 + __ffs(hit) - 1;
      run += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (found < 0) found = (last_nz >= 0 && total > 0.0) ? last_nz : (int64_t)Lh - 1;
    if (lane == 0) {
      const uint64_t z = base + (uint64_t)found;
      a.z[i] = z;
      a.cost[i] = (a.cost_dtype == QAOA_COST_I32) ? (double)((const int*)a.C)[z] : ((const double*)a.C)[z];
    }
  }
}

// leaves of 2^10 entries, or one leaf of 2^ceil(log2 len) for shorter vectors (2^n: min(n, 10))
int leaf_bits_for_len(uint64_t len) {
  int lb = 0;
  while (lb < 10 && (1ull << lb) < len) ++lb;
  return lb;
}

}  // namespace

size_t sample_ws_bytes_len(uint64_t len) {
  const int lb = leaf_bits_for_len(len);
  const int64_t nleaf = (int64_t)((len + (1ull << lb) - 1) >> lb);
  const int64_t nchunks = (nleaf + kChunk - 1) / kChunk;
  return (size_t)(nleaf + (nleaf + 1) + (nchunks + 1)) * sizeof(double) + 3 * 256;
}

size_t sample_ws_bytes(int n, int /*dtype*/) { return sample_ws_bytes_len(1ull << n); }

cudaError_t launch_sample(const SampleArgs& a0, cudaStream_t s) {
  SampleArgs a = a0;
  if (a.len == 0) a.len = 1ull << a.n;
  a.leaf_bits = leaf_bits_for_len(a.len);
  const int64_t nleaf = (int64_t)((a.len + (1ull << a.leaf_bits) - 1) >> a.leaf_bits);
  const int64_t nchunks = (nleaf + kChunk - 1) / kChunk;
  // carve the workspace: leaf sums, prefix, chunk sums (256-byte aligned pieces)
  char* p = (char*)a.leaf;
  auto carve = [&](size_t bytes) {
    char* r = p;
    p += (bytes + 255) & ~(size_t)255;
    return r;
  };
  double* leaf = (double*)carve(nleaf * sizeof(double));
  double* prefix = (double*)carve((nleaf + 1) * sizeof(double));
  double* bsum = (double*)carve((nchunks + 1) * sizeof(double));
  a.leaf = leaf;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);

  note_launch(2, s, true);
  {
    const int64_t warps = nleaf;
    int64_t blocks = (warps * 32 + kThreads - 1) / kThreads;
    if (blocks > (int64_t)sms * 16) blocks = (int64_t)sms * 16;
    leaf_sum_kernel<<<(int)blocks, kThreads, 0, s>>>(a);
  }
  note_launch(2, s, false, (double)a.len * (a.dtype == QAOA_C128 ? 16.0 : 8.0));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  note_launch(3, s, true);
  chunk_sum_kernel<<<(int)nchunks, kThreads, 0, s>>>(leaf, nleaf, bsum);
  note_launch(3, s, false);
  note_launch(3, s, true);
  chunk_scan_kernel<<<1, 32, 0, s>>>(bsum, nchunks);
  note_launch(3, s, false);
  note_launch(3, s, true);
  leaf_scan_kernel<<<(int)nchunks, kThreads, 0, s>>>(leaf, nleaf, bsum, prefix, nchunks);
  note_launch(3, s, false);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (a.shots > 0) {
    int64_t blocks = (a.shots * 32 + kThreads - 1) / kThreads;
    if (blocks > (int64_t)sms * 16) blocks = (int64_t)sms * 16;
    note_launch(2, s, true);
    draw_kernel<<<(int)blocks, kThreads, 0, s>>>(a, prefix);
    note_launch(2, s, false);
  }
  return cudaGetLastError();
}

}  // namespace qaoa
