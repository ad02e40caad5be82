// Constraint-preserving QAOA: the state lives on the feasible states only (the direction
// the paper names for future work in Sec. VI — reduce the search space the simulator
// carries for a constrained problem).  The constraint is a Hamming weight,
//   F_k = {z in [0, 2^n) : popcount(z) = k}   (for MaxCut with k = n/2: graph bisection),
// and the mixer is the ring XY mixer of the quantum alternating operator ansatz
// (Hadfield et al., Algorithms 12(2):34, 2019), which keeps popcount(z):
//   G_ab(beta) = exp(-i beta (X_a X_b + Y_a Y_b) / 2)
// on the ring pairs (j, j+1 mod n), applied as parity sets: even j (j < n-1), then odd j
// (j < n-1), then the closing pair (n-1, 0) alone when n is odd (with the odd set when n
// is even); n = 2 has the single pair (0, 1).  The start state is the uniform
// superposition over F_k (Dicke state), the cost unitary is Eq. 1's, restricted to F_k.
//
// Layout: binom(n, k) amplitudes in rank order, the rank of z being its position among
// the states of F_k in increasing integer order (combinatorial number system:
// rank(z) = sum_i binom(c_i, i) over the set bits c_1 < ... < c_k of z).  A thread walks a
// chunk of consecutive ranks: it unranks the first (O(n)) and steps to the next state of
// F_k with Gosper's rule (the next larger integer of equal popcount, O(1)).
//
// A pair gate on (a, b), a < b, pairs z (z_a = 1, z_b = 0) with z' = z ^ 2^a ^ 2^b, the
// same state with that set bit moved from a up to b (z' > z); states with z_a = z_b are
// unchanged.  The thread owning z updates both amplitudes, so a launch touches every
// amplitude at most once.  For adjacent qubits (b = a + 1) the moved bit keeps its index
// j + 1 among the set bits (j = set bits below a), so
//   rank(z') - rank(z) = binom(a + 1, j + 1) - binom(a, j + 1) = binom(a, j);
// the closing pair (0, n-1) ranks z' directly.
#include "fixedpoint.cuh"
#include "internal.h"
#include "xy_window.cuh"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <type_traits>

namespace qaoa {
namespace {

constexpr int kXYThreads = 256;
constexpr int kXYChunk = 16;       // consecutive ranks per thread
constexpr int kXYRedBlocks = 1024;  // expectation partials (fixed grid: fixed reduction order)
constexpr int kBN = QAOA_XY_MAX_N + 1;

struct XYShape {
  int n, k;
  unsigned long long D;                 // binom(n, k)
  unsigned long long binom[kBN][kBN];  // binom[c][i] = binom(c, i), 0 for i > c
};

struct XYCostArgs {
  XYShape s;
  int m;
  int cost_dtype;
  int integer;
  int fixed_shift;
  void* C;
  unsigned char eu[QAOA_XY_MAX_EDGES], ev[QAOA_XY_MAX_EDGES];
  long long ew[QAOA_XY_MAX_EDGES];  // integer or fixed-point weights
};

__device__ __forceinline__ void load_binom(unsigned long long (*B)[kBN], const XYShape& s) {
  for (int i = threadIdx.x; i < kBN * kBN; i += blockDim.x) B[i / kBN][i % kBN] = s.binom[i / kBN][i % kBN];
  __syncthreads();
}

// the state of F_k with rank r (r < binom(n, k)): the largest c with binom(c, i) <= r is
// the i-th set bit, from i = k down to 1 (binom(i - 1, i) = 0 stops the search at c >= i - 1)
__device__ __forceinline__ unsigned long long xy_unrank(unsigned long long r, int n, int k,
                                                        const unsigned long long (*B)[kBN]) {
  unsigned long long z = 0;
  int c = n - 1;
  for (int i = k; i >= 1; --i) {
    while (B[c][i] > r) --c;
    z |= 1ull << c;
    r -= B[c][i];
    --c;
  }
  return z;
}

__device__ __forceinline__ unsigned long long xy_rank(unsigned long long z, const unsigned long long (*B)[kBN]) {
  unsigned long long r = 0;
  for (int i = 1; z != 0; ++i) {
    r += B[__ffsll((long long)z) - 1][i];
    z &= z - 1;
  }
  return r;
}

// next larger integer with the same popcount (Gosper); z != 0
__device__ __forceinline__ unsigned long long xy_next(unsigned long long z) {
  const unsigned long long t = z | (z - 1);
  return (t + 1) | (((~t & (t + 1)) - 1) >> __ffsll((long long)z));
}

template <typename T>
struct Real;
template <>
struct Real<double2> {
  using type = double;
};
template <>
struct Real<float2> {
  using type = float;
};

template <typename T>
__global__ void __launch_bounds__(kXYThreads)
    xy_gate_kernel(const __grid_constant__ XYShape s, T* __restrict__ psi, int qa, int qb,
                   typename Real<T>::type cb, typename Real<T>::type sb) {
  __shared__ unsigned long long B[kBN][kBN];
  load_binom(B, s);
  const unsigned long long D = s.D, nch = (D + kXYChunk - 1) / kXYChunk;
  const unsigned long long ma = 1ull << qa, mb = 1ull << qb, below = ma - 1;
  const bool adjacent = qb == qa + 1;
  for (unsigned long long ch = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; ch < nch;
       ch += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long r0 = ch * kXYChunk, r1 = r0 + kXYChunk < D ? r0 + kXYChunk : D;
    unsigned long long z = xy_unrank(r0, s.n, s.k, B);
    for (unsigned long long r = r0; r < r1; ++r) {
      if ((z & ma) && !(z & mb)) {
        const unsigned long long rp = adjacent ? r + B[qa][__popcll(z & below)] : xy_rank(z ^ ma ^ mb, B);
        if (rp < D) {
          const T x = psi[r], y = psi[rp];
          T u, v;
          u.x = cb * x.x + sb * y.y;  // cos(beta) x - i sin(beta) y
          u.y = cb * x.y - sb * y.x;
          v.x = cb * y.x + sb * x.y;  // cos(beta) y - i sin(beta) x
          v.y = cb * y.y - sb * x.x;
          psi[r] = u;
          psi[rp] = v;
        }
      }
      if (r + 1 < r1) z = xy_next(z);
    }
  }
}

__global__ void __launch_bounds__(kXYThreads) xy_cost_kernel(const __grid_constant__ XYCostArgs a) {
  __shared__ unsigned long long B[kBN][kBN];
  __shared__ unsigned char eu[QAOA_XY_MAX_EDGES], ev[QAOA_XY_MAX_EDGES];
  __shared__ long long ew[QAOA_XY_MAX_EDGES];
  for (int e = threadIdx.x; e < a.m; e += blockDim.x) {
    eu[e] = a.eu[e];
    ev[e] = a.ev[e];
    ew[e] = a.ew[e];
  }
  load_binom(B, a.s);
  const unsigned long long D = a.s.D, nch = (D + kXYChunk - 1) / kXYChunk;
  for (unsigned long long ch = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; ch < nch;
       ch += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long r0 = ch * kXYChunk, r1 = r0 + kXYChunk < D ? r0 + kXYChunk : D;
    unsigned long long z = xy_unrank(r0, a.s.n, a.s.k, B);
    for (unsigned long long r = r0; r < r1; ++r) {
      long long c = 0;  // exact: integer weights, or one common fixed point
      for (int e = 0; e < a.m; ++e)
        if (((z >> eu[e]) ^ (z >> ev[e])) & 1) c += ew[e];
      if (a.cost_dtype == QAOA_COST_I32) {
        ((int*)a.C)[r] = (int)c;
      } else if (a.integer) {
        ((double*)a.C)[r] = (double)c;
      } else {
        ((double*)a.C)[r] = ldexp((double)c, -a.fixed_shift);
      }
      if (r + 1 < r1) z = xy_next(z);
    }
  }
}

template <typename T>
__global__ void xy_init_kernel(T* __restrict__ psi, unsigned long long D, double amp) {
  for (unsigned long long r = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; r < D;
       r += (unsigned long long)gridDim.x * blockDim.x) {
    T v;
    v.x = (typename Real<T>::type)amp;
    v.y = 0;
    psi[r] = v;
  }
}

// exp(-i theta) in the state's precision; float states reduce theta mod 2 pi in float64 first
__device__ __forceinline__ double2 phase_of(double theta, double2*) {
  double sn, cs;
  sincos(theta, &sn, &cs);
  return make_double2(cs, -sn);
}
__device__ __forceinline__ float2 phase_of(double theta, float2*) {
  const double two_pi = 6.283185307179586476925286766559;
  const double red = theta - two_pi * rint(theta / two_pi);
  float sn, cs;
  sincosf((float)red, &sn, &cs);
  return make_float2(cs, -sn);
}

template <typename T>
__global__ void xy_phase_kernel(T* __restrict__ psi, const void* __restrict__ C, int cost_dtype, unsigned long long D,
                                const T* __restrict__ tab, long long cmin, long long span, double gamma) {
  for (unsigned long long r = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; r < D;
       r += (unsigned long long)gridDim.x * blockDim.x) {
    T f;
    if (cost_dtype == QAOA_COST_I32) {
      const long long c = ((const int*)C)[r];
      const long long i = c - cmin;
      f = (tab != nullptr && i >= 0 && i < span) ? tab[i] : phase_of(gamma * (double)c, (T*)nullptr);
    } else {
      f = phase_of(gamma * ((const double*)C)[r], (T*)nullptr);
    }
    const T x = psi[r];
    T y;
    y.x = x.x * f.x - x.y * f.y;
    y.y = x.x * f.y + x.y * f.x;
    psi[r] = y;
  }
}

// sampled ranks -> the states of F_k they index (in place)
__global__ void __launch_bounds__(kXYThreads) xy_unrank_kernel(const __grid_constant__ XYShape s,
                                                                unsigned long long* __restrict__ z, long long shots) {
  __shared__ unsigned long long B[kBN][kBN];
  load_binom(B, s);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < shots; i += (long long)gridDim.x * blockDim.x)
    z[i] = xy_unrank(z[i], s.n, s.k, B);
}

// ------------------------------------------------------------------ adjoint gradient on F_k
//
// The circuit is a sequence of gates exp(-i theta H_g): per layer the cost unitary
// (H = diag(C), theta = gamma_l), then the ring pair gates (H = K_ab, the swap of a state
// with z_a = 1, z_b = 0 and its partner; theta = beta_l).  With psi_g the state right after
// gate g and lambda_g = (gates after g)^dagger C psi_final, dE/dtheta_g = 2 Im <lambda_g|H_g|psi_g>
// (Sec. II-B, IV-C); a parameter's derivative is the sum over its gates.  The pass walks the
// gates backwards from lambda = C psi_final, undoing each on psi and lambda after taking its
// term, so it needs the two subspace buffers only.  Every term is summed in float64 per
// thread and per block, one partial per block in a fixed grid (deterministic).

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kXYThreads / 32; ++w) t += red[w];
  return t;  // valid in thread 0
}

// lambda = C psi, with block partials of [sum C |psi|^2, sum |psi|^2] (E = Re <psi|lambda>)
template <typename T>
__global__ void __launch_bounds__(kXYThreads)
    xy_lambda_kernel(const T* __restrict__ psi, T* __restrict__ lam, const void* __restrict__ C, int cost_dtype,
                     unsigned long long D, double* __restrict__ pe, double* __restrict__ pn) {
  __shared__ double red[kXYThreads / 32];
  double e = 0.0, nn = 0.0;
  for (unsigned long long r = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; r < D;
       r += (unsigned long long)gridDim.x * blockDim.x) {
    const T x = psi[r];
    const double c = cost_dtype == QAOA_COST_I32 ? (double)((const int*)C)[r] : ((const double*)C)[r];
    T y;
    y.x = (typename Real<T>::type)c * x.x;
    y.y = (typename Real<T>::type)c * x.y;
    lam[r] = y;
    const double pr = (double)x.x * (double)x.x + (double)x.y * (double)x.y;
    e += c * pr;
    nn += pr;
  }
  const double se = block_sum(e, red);
  __syncthreads();
  const double sn = block_sum(nn, red);
  if (threadIdx.x == 0) {
    pe[blockIdx.x] = se;
    pn[blockIdx.x] = sn;
  }
}

// one pair gate backwards: the block partial of 2 Im <lambda|K_ab|psi>, then G_ab(-beta) on
// both buffers (cb = cos beta, sb = -sin beta in the forward gate's formula)
template <typename T>
__global__ void __launch_bounds__(kXYThreads)
    xy_gate_adjoint_kernel(const __grid_constant__ XYShape s, T* __restrict__ psi, T* __restrict__ lam, int qa,
                           int qb, typename Real<T>::type cb, typename Real<T>::type sb, double* __restrict__ part) {
  __shared__ unsigned long long B[kBN][kBN];
  __shared__ double red[kXYThreads / 32];
  load_binom(B, s);
  const unsigned long long D = s.D, nch = (D + kXYChunk - 1) / kXYChunk;
  const unsigned long long ma = 1ull << qa, mb = 1ull << qb, below = ma - 1;
  const bool adjacent = qb == qa + 1;
  double acc = 0.0;
  for (unsigned long long ch = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; ch < nch;
       ch += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long r0 = ch * kXYChunk, r1 = r0 + kXYChunk < D ? r0 + kXYChunk : D;
    unsigned long long z = xy_unrank(r0, s.n, s.k, B);
    for (unsigned long long r = r0; r < r1; ++r) {
      if ((z & ma) && !(z & mb)) {
        const unsigned long long rp = adjacent ? r + B[qa][__popcll(z & below)] : xy_rank(z ^ ma ^ mb, B);
        if (rp < D) {
          const T x = psi[r], y = psi[rp], lx = lam[r], ly = lam[rp];
          // Im(conj(lam_z) psi_z' + conj(lam_z') psi_z)
          acc += (double)lx.x * y.y - (double)lx.y * y.x + (double)ly.x * x.y - (double)ly.y * x.x;
          T u, v;
          u.x = cb * x.x + sb * y.y;
          u.y = cb * x.y - sb * y.x;
          v.x = cb * y.x + sb * x.y;
          v.y = cb * y.y - sb * x.x;
          psi[r] = u;
          psi[rp] = v;
          u.x = cb * lx.x + sb * ly.y;
          u.y = cb * lx.y - sb * ly.x;
          v.x = cb * ly.x + sb * lx.y;
          v.y = cb * ly.y - sb * lx.x;
          lam[r] = u;
          lam[rp] = v;
        }
      }
      if (r + 1 < r1) z = xy_next(z);
    }
  }
  const double t = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = 2.0 * t;
}

// the cost unitary backwards: the block partial of 2 Im <lambda|C|psi>, then both buffers
// times exp(+i gamma C) (the conjugate of the forward table entry, or computed directly)
template <typename T>
__global__ void __launch_bounds__(kXYThreads)
    xy_cost_adjoint_kernel(T* __restrict__ psi, T* __restrict__ lam, const void* __restrict__ C, int cost_dtype,
                           unsigned long long D, const T* __restrict__ tab, long long cmin, long long span,
                           double gamma, double* __restrict__ part) {
  __shared__ double red[kXYThreads / 32];
  double acc = 0.0;
  for (unsigned long long r = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; r < D;
       r += (unsigned long long)gridDim.x * blockDim.x) {
    T f;
    double c;
    if (cost_dtype == QAOA_COST_I32) {
      const long long ci = ((const int*)C)[r];
      const long long i = ci - cmin;
      c = (double)ci;
      f = (tab != nullptr && i >= 0 && i < span) ? tab[i] : phase_of(gamma * c, (T*)nullptr);
    } else {
      c = ((const double*)C)[r];
      f = phase_of(gamma * c, (T*)nullptr);
    }
    f.y = -f.y;  // exp(+i gamma c)
    const T x = psi[r], l = lam[r];
    acc += c * ((double)l.x * x.y - (double)l.y * x.x);
    T y;
    y.x = x.x * f.x - x.y * f.y;
    y.y = x.x * f.y + x.y * f.x;
    psi[r] = y;
    y.x = l.x * f.x - l.y * f.y;
    y.y = l.x * f.y + l.y * f.x;
    lam[r] = y;
  }
  const double t = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = 2.0 * t;
}

// ------------------------------------------------------------------ windowed mixer passes
//
// One launch applies every pair gate of a window [lo, lo + w) of the ring mixer (its even
// pairs, then its odd pairs; xy_window.cuh derives the tile addressing and why the order is
// the ring's).  A tile is up to m columns of one class: its binom(w, kw) rows x m columns of
// amplitudes are gathered into shared memory, each gate in turn rotates its pairs of rows in
// every column (the pairs of one gate are disjoint), and the tile is written back.  Backwards (TWO: psi and lambda) the gates run in reverse order; before
// undoing a gate the owner of each pair adds Im(conj(lambda_z) psi_z' + conj(lambda_z') psi_z),
// the gate's term at the state right after it.  All gates of a window share the layer's beta,
// so one partial per block suffices.  complex128 tiles hold psi (and lambda) as int64 fixed
// point and rotate with 32-bit limb products (fixedpoint.cuh): GB300's float64 pipe would
// otherwise bound the pass.  Each buffer's scale is the tile's own: with every component
// below 2^E, value = integer x 2^-(56 - E).  The gates keep each column's 2-norm, which is
// below sqrt(2 rows) 2^E < 2^(E + 4) for rows <= 126, so every value stays below 2^(E + 4),
// i.e. below 2^60 integer units, as the limb products require (any norm is accepted); the
// gradient terms are exact 128-bit products, converted to float64 once per tile.
static_assert(xyw::kMaxN == QAOA_XY_MAX_N, "window tables sized for QAOA_XY_MAX_N");
static_assert(xyw::kMaxRows <= 128, "tile scale headroom assumes columns of <= 128 rows");

template <typename T>
__device__ __forceinline__ void xy_rotate(T& x, T& y, typename Real<T>::type cb, typename Real<T>::type sb) {
  T u, v;
  u.x = cb * x.x + sb * y.y;  // cos(beta) x - i sin(beta) y
  u.y = cb * x.y - sb * y.x;
  v.x = cb * y.x + sb * x.y;  // cos(beta) y - i sin(beta) x
  v.y = cb * y.y - sb * x.x;
  x = u;
  y = v;
}

// Q62 of |d| <= 1 (from a 2^-61 rounding, so that d = +-1 stays inside from_double's range)
__device__ __forceinline__ long long xy_q62(double d) { return fx::from_double(d, 61) * 2; }

// the same rotation in fixed point: cb, sb as Q62 limbs (nsb = -sb); each part from six limb
// products (the two low x low ones dropped: within three units of exact rounding)
__device__ __forceinline__ void xy_rotate_fx(longlong2& x, longlong2& y, fx::Limbs cb, fx::Limbs sb, fx::Limbs nsb) {
  const fx::Limbs xr = fx::split(x.x), xi = fx::split(x.y), yr = fx::split(y.x), yi = fx::split(y.y);
  x = make_longlong2(fx::dot2_q62_hi(xr, cb, yi, sb, 0), fx::dot2_q62_hi(xi, cb, yr, nsb, 0));
  y = make_longlong2(fx::dot2_q62_hi(yr, cb, xi, sb, 0), fx::dot2_q62_hi(yi, cb, xr, nsb, 0));
}

// The layer's cost unitary fused into the first window's pass (PH): forward, each amplitude
// is multiplied by exp(-i gamma C) as it is loaded; backward, after the window's gates are
// undone, the owner adds c Im(conj(lambda) psi) (the gamma term at the state right after the
// cost unitary) to `cpart` and multiplies both buffers by exp(+i gamma C) before the store.
template <typename T>
struct XYPhaseArgs {
  const void* C;
  int cost_dtype;
  const T* tab;  // exp(-i gamma c) for c in [cmin, cmin + span), or nullptr
  long long cmin, span;
  double gamma;
  double* cpart;  // backward: the block partials of the gamma term
};

template <typename T>
__device__ __forceinline__ T xy_phase_factor(const XYPhaseArgs<T>& ph, unsigned long long r, double& c) {
  if (ph.cost_dtype == QAOA_COST_I32) {
    const long long ci = ((const int*)ph.C)[r];
    const long long i = ci - ph.cmin;
    c = (double)ci;
    return (ph.tab != nullptr && i >= 0 && i < ph.span) ? ph.tab[i] : phase_of(ph.gamma * c, (T*)nullptr);
  }
  c = ((const double*)ph.C)[r];
  return phase_of(ph.gamma * c, (T*)nullptr);
}

template <typename T>
__device__ __forceinline__ T xy_cmul(T x, T f) {
  T y;
  y.x = x.x * f.x - x.y * f.y;
  y.y = x.x * f.y + x.y * f.x;
  return y;
}

// float64 components of a fixed-point tile slot (raw bits while the tile's scale is open)
__device__ __forceinline__ longlong2 xy_fx_load(const longlong2 raw, int fs) {
  return make_longlong2(fx::from_double(fx::bits_to_double((unsigned long long)raw.x), fs),
                        fx::from_double(fx::bits_to_double((unsigned long long)raw.y), fs));
}
__device__ __forceinline__ unsigned xy_exp_bits(double2 v) {
  const unsigned long long bx = fx::double_to_bits(v.x), by = fx::double_to_bits(v.y);
  return max((unsigned)(bx >> 52) & 0x7FFu, (unsigned)(by >> 52) & 0x7FFu);
}
// x * f (conj(f) when CONJ) for a fixed-point x and a unit float64 factor f, as Q62 limbs
template <bool CONJ>
__device__ __forceinline__ longlong2 xy_fx_phase(longlong2 x, double2 f) {
  const long long fre = xy_q62(f.x), fim = xy_q62(CONJ ? -f.y : f.y);
  const fx::Limbs fr = fx::split(fre), fi = fx::split(fim), nfi = fx::split(-fim);
  const fx::Limbs xr = fx::split(x.x), xi = fx::split(x.y);
  return make_longlong2(fx::dot2_q62_hi(xr, fr, xi, nfi, 0), fx::dot2_q62_hi(xr, fi, xi, fr, 0));
}

template <typename T, bool TWO, bool PH>
__global__ void __launch_bounds__(kXYThreads)
    xy_window_kernel(const __grid_constant__ xyw::Window W, T* __restrict__ psi, T* __restrict__ lam,
                     typename Real<T>::type cb, typename Real<T>::type sb, double* __restrict__ part,
                     const __grid_constant__ XYPhaseArgs<T> ph) {
  constexpr bool FXR = std::is_same<T, double2>::value;  // complex128: fixed-point tiles
  using S = typename std::conditional<FXR, longlong2, T>::type;
  __shared__ unsigned long long B[xyw::kBN][xyw::kBN];
  __shared__ unsigned long long rowoff[xyw::kMaxRows];
  __shared__ unsigned long long colbase[xyw::kMaxCols];
  __shared__ unsigned short rowpat[xyw::kMaxRows];
  __shared__ unsigned char pr0[xyw::kMaxGates][xyw::kMaxPairs], pr1[xyw::kMaxGates][xyw::kMaxPairs];
  __shared__ int npr[xyw::kMaxGates];
  __shared__ double red[kXYThreads / 32];
  __shared__ unsigned tile_ex[2];  // fixed-point tiles: largest biased float64 exponent of psi, lambda
  extern __shared__ __align__(16) unsigned char xy_win_smem[];
  S* tp = (S*)xy_win_smem;     // psi tile
  S* tl = tp + W.tile_elems;   // lambda tile (TWO)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int c = tid; c < xyw::kBN; c += kXYThreads) xyw::binom_row(B, c);
  fx::Limbs qc = {0, 0}, qs = {0, 0}, qns = {0, 0};
  if constexpr (FXR) {
    qc = fx::split(xy_q62((double)cb));
    qs = fx::split(xy_q62((double)sb));
    qns = fx::split(-xy_q62((double)sb));
  }
  double acc = 0.0, cacc = 0.0;
  int cur = -1;  // class whose row tables are in shared memory (the same in every thread)
  for (unsigned long long tile = blockIdx.x; tile < W.tiles; tile += gridDim.x) {
    const int ci = xyw::find_class(W, tile);
    const xyw::Class& C = W.cls[ci];
    const int rows = C.rows;
    const unsigned long long col0 = (tile - C.first_tile) * (unsigned long long)C.m;
    const int ncol = (int)(C.ncols - col0 < (unsigned long long)C.m ? C.ncols - col0 : (unsigned long long)C.m);
    __syncthreads();  // Pascal's triangle is ready; the previous tile is stored
    if (ci != cur) {  // row patterns, their rank parts, and each gate's moved rows
      for (int r = tid; r < rows; r += kXYThreads) {
        const unsigned long long P = xyw::unrank_bits((unsigned long long)r, W.w, C.kw, B);
        rowpat[r] = (unsigned short)P;
        rowoff[r] = xyw::rank_part(P, W.lo, C.kL, B);
      }
      __syncthreads();
      for (int g = warp; g < W.ngates; g += kXYThreads / 32) {
        const int ga = W.ga[g];
        int cnt = 0;
        for (int base = 0; base < rows; base += 32) {
          const int r = base + lane;
          const unsigned P = r < rows ? rowpat[r] : 0u;
          const bool mv = r < rows && ((P >> ga) & 3u) == 1u;
          const unsigned bal = __ballot_sync(0xffffffffu, mv);
          if (mv) {
            const int q = cnt + __popc(bal & ((1u << lane) - 1u));
            pr0[g][q] = (unsigned char)r;
            pr1[g][q] = (unsigned char)xyw::partner_row(r, P, ga, B);
          }
          cnt += __popc(bal);
        }
        if (lane == 0) npr[g] = cnt;
      }
      cur = ci;
    }
    for (int c = tid; c < ncol; c += kXYThreads) colbase[c] = xyw::col_base(W, C, col0 + c, B);
    if (FXR && tid == 0) tile_ex[0] = tile_ex[1] = 0;
    __syncthreads();
    // element e of the tile: column-major when a column's rows are consecutive ranks (len = 1),
    // otherwise row-major, so consecutive threads touch consecutive ranks
    const bool cm = C.len == 1;
    const unsigned inner = cm ? (unsigned)rows : (unsigned)ncol;  // < 2^16
    const unsigned mg = xyw::div_magic(inner);
    const int ne = rows * ncol;
    unsigned exp_psi = 0, exp_lam = 0;
    for (int e = tid; e < ne; e += kXYThreads) {
      const unsigned o = xyw::div_small((unsigned)e, mg), i = (unsigned)e - o * inner;
      const int r = cm ? (int)i : (int)o, c = cm ? (int)o : (int)i;
      const unsigned long long rk = rowoff[r] + colbase[c];
      const T x = psi[rk];
      if constexpr (FXR) {  // raw bits for now; the exponents give the tile's scales
        exp_psi = max(exp_psi, xy_exp_bits(x));
        tp[e] = make_longlong2((long long)fx::double_to_bits(x.x), (long long)fx::double_to_bits(x.y));
        if constexpr (TWO) {
          const T l = lam[rk];
          exp_lam = max(exp_lam, xy_exp_bits(l));
          tl[e] = make_longlong2((long long)fx::double_to_bits(l.x), (long long)fx::double_to_bits(l.y));
        }
      } else {
        T v = x;
        if constexpr (PH && !TWO) {
          double cv;
          v = xy_cmul(v, xy_phase_factor(ph, rk, cv));
        }
        tp[e] = v;
        if constexpr (TWO) tl[e] = lam[rk];
      }
    }
    int fs = 0, fl = 0;  // fixed-point tiles: psi value = integer x 2^-fs, lambda 2^-fl
    if constexpr (FXR) {
      exp_psi = __reduce_max_sync(0xffffffffu, exp_psi);
      if (lane == 0) atomicMax(&tile_ex[0], exp_psi);
      if constexpr (TWO) {
        exp_lam = __reduce_max_sync(0xffffffffu, exp_lam);
        if (lane == 0) atomicMax(&tile_ex[1], exp_lam);
      }
      __syncthreads();
      fs = 56 - ((int)tile_ex[0] - 1022);  // every component is below 2^(tile_ex - 1022)
      fl = 56 - ((int)tile_ex[1] - 1022);
      for (int e = tid; e < ne; e += kXYThreads) {  // the slots this thread loaded
        longlong2 X = xy_fx_load(tp[e], fs);
        if constexpr (PH && !TWO) {  // the layer's cost unitary; a unit factor keeps the bound
          const unsigned o = xyw::div_small((unsigned)e, mg), i = (unsigned)e - o * inner;
          const int r = cm ? (int)i : (int)o, c = cm ? (int)o : (int)i;
          double cv;
          X = xy_fx_phase<false>(X, xy_phase_factor(ph, rowoff[r] + colbase[c], cv));
        }
        tp[e] = X;
        if constexpr (TWO) tl[e] = xy_fx_load(tl[e], fl);
      }
    }
    __syncthreads();
    // gates one after another, each gate's (pair, column) items spread over the block:
    // consecutive threads take consecutive columns (row-major tiles) or consecutive pairs of
    // one column (column-major tiles), so shared-memory accesses stay conflict-free
    fx::i128 tacc = 0;  // fixed point: this thread's gate terms of the tile, x 2^-(fs + fl - 4)
    for (int gi = 0; gi < W.ngates; ++gi) {
      const int g = TWO ? W.ngates - 1 - gi : gi;
      const int np = npr[g];
      const int items = np * ncol;
      const unsigned in2 = cm ? (unsigned)np : (unsigned)ncol;
      const unsigned m2 = xyw::div_magic(in2);
      for (int it = tid; it < items; it += kXYThreads) {
        const unsigned o = xyw::div_small((unsigned)it, m2), i = (unsigned)it - o * in2;
        const int q = cm ? (int)i : (int)o, c = cm ? (int)o : (int)i;
        const int r0 = pr0[g][q], r1 = pr1[g][q];
        const int s0 = cm ? c * rows + r0 : r0 * ncol + c;
        const int s1 = cm ? c * rows + r1 : r1 * ncol + c;
        S x = tp[s0], y = tp[s1];
        if constexpr (TWO) {
          S lx = tl[s0], ly = tl[s1];
          if constexpr (FXR) {  // exact products (each below 2^121), summed with 4 bits to spare
            tacc += (fx::dot2_exact(lx.x, y.y, lx.y, y.x) + fx::dot2_exact(ly.x, x.y, ly.y, x.x)) >> 4;
            xy_rotate_fx(lx, ly, qc, qs, qns);
          } else {
            acc += (double)lx.x * y.y - (double)lx.y * y.x + (double)ly.x * x.y - (double)ly.y * x.x;
            xy_rotate(lx, ly, cb, sb);
          }
          tl[s0] = lx;
          tl[s1] = ly;
        }
        if constexpr (FXR) xy_rotate_fx(x, y, qc, qs, qns);
        else xy_rotate(x, y, cb, sb);
        tp[s0] = x;
        tp[s1] = y;
      }
      __syncthreads();
    }
    if constexpr (FXR && TWO) acc += fx::i128_to_double(tacc, fs + fl - 4);
    fx::i128 cacc_i = 0;  // fixed point, integer costs: sum of c (conj(lambda) psi products >> 32)
    for (int e = tid; e < ne; e += kXYThreads) {
      const unsigned o = xyw::div_small((unsigned)e, mg), i = (unsigned)e - o * inner;
      const int r = cm ? (int)i : (int)o, c = cm ? (int)o : (int)i;
      const unsigned long long rk = rowoff[r] + colbase[c];
      if constexpr (FXR) {
        longlong2 X = tp[e];
        if constexpr (TWO) {
          longlong2 L = tl[e];
          if constexpr (PH) {  // the gamma term at the state right after the cost unitary, then undo it
            double cv;
            const T f = xy_phase_factor(ph, rk, cv);
            const fx::i128 pr = fx::dot2_exact(L.x, X.y, L.y, X.x);  // Im(conj(lambda) psi)
            if (ph.cost_dtype == QAOA_COST_I32) cacc_i += (pr >> 32) * (long long)cv;
            else cacc += cv * fx::i128_to_double(pr, fs + fl);
            X = xy_fx_phase<true>(X, f);
            L = xy_fx_phase<true>(L, f);
          }
          lam[rk] = make_double2(fx::to_double(L.x, fl), fx::to_double(L.y, fl));
        }
        psi[rk] = make_double2(fx::to_double(X.x, fs), fx::to_double(X.y, fs));
      } else if constexpr (TWO) {
        T x = tp[e], l = tl[e];
        if constexpr (PH) {
          double cv;
          T f = xy_phase_factor(ph, rk, cv);
          cacc += cv * ((double)l.x * x.y - (double)l.y * x.x);
          f.y = -f.y;  // exp(+i gamma c)
          x = xy_cmul(x, f);
          l = xy_cmul(l, f);
        }
        psi[rk] = x;
        lam[rk] = l;
      } else {
        psi[rk] = tp[e];
      }
    }
    if constexpr (FXR && TWO && PH) cacc += fx::i128_to_double(cacc_i, fs + fl - 32);
  }
  if constexpr (TWO) {
    const double t = block_sum(acc, red);
    if (tid == 0) part[blockIdx.x] = 2.0 * t;
    if constexpr (PH) {
      __syncthreads();
      const double tc = block_sum(cacc, red);
      if (tid == 0) ph.cpart[blockIdx.x] = 2.0 * tc;
    }
  }
}

// out[o] = sum of nparts[o] consecutive partial rows (stride kXYPartStride) from row first[o]
struct XYReducePlan {
  int nout;
  int first[2 * QAOA_MAX_P + 2];
  int rows[2 * QAOA_MAX_P + 2];
  int cols[2 * QAOA_MAX_P + 2];  // blocks per row
};
constexpr int kXYPartStride = 2048;  // partial slots per launch (>= any grid used here)

__global__ void __launch_bounds__(kXYThreads) xy_grad_reduce_kernel(const __grid_constant__ XYReducePlan rp,
                                                                    const double* __restrict__ part,
                                                                    double* __restrict__ out) {
  __shared__ double red[kXYThreads / 32];
  const int o = blockIdx.x;
  double acc = 0.0;
  for (int row = 0; row < rp.rows[o]; ++row) {
    const double* src = part + (size_t)(rp.first[o] + row) * kXYPartStride;
    for (int b = threadIdx.x; b < rp.cols[o]; b += kXYThreads) acc += src[b];
  }
  const double t = block_sum(acc, red);
  if (threadIdx.x == 0) out[o] = t;
}

// block partials of [sum C |psi|^2, sum |psi|^2] in float64, fixed order for a fixed grid
template <typename T>
__global__ void __launch_bounds__(kXYThreads)
    xy_expect_kernel(const T* __restrict__ psi, const void* __restrict__ C, int cost_dtype, unsigned long long D,
                     double* __restrict__ part) {
  __shared__ double se[kXYThreads], sn[kXYThreads];
  double e = 0.0, nn = 0.0;
  if (std::is_same<T, float2>::value && cost_dtype == QAOA_COST_I32) {
    // complex64 with integer costs: float32 sums of 32 consecutive terms of a thread, added in
    // float64 (GB300's float64 rate would otherwise bound this pass)
    float ef = 0.f, nf = 0.f;
    int cnt = 0;
    for (unsigned long long r = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; r < D;
         r += (unsigned long long)gridDim.x * blockDim.x) {
      const T x = psi[r];
      const float pr = (float)x.x * (float)x.x + (float)x.y * (float)x.y;
      ef = fmaf((float)((const int*)C)[r], pr, ef);
      nf += pr;
      if (++cnt == 32) {
        e += ef;
        nn += nf;
        ef = nf = 0.f;
        cnt = 0;
      }
    }
    e += ef;
    nn += nf;
  } else {
    for (unsigned long long r = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; r < D;
         r += (unsigned long long)gridDim.x * blockDim.x) {
      const T x = psi[r];
      const double pr = (double)x.x * (double)x.x + (double)x.y * (double)x.y;
      const double c = cost_dtype == QAOA_COST_I32 ? (double)((const int*)C)[r] : ((const double*)C)[r];
      e += c * pr;
      nn += pr;
    }
  }
  se[threadIdx.x] = e;
  sn[threadIdx.x] = nn;
  __syncthreads();
  for (int h = kXYThreads / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      se[threadIdx.x] += se[threadIdx.x + h];
      sn[threadIdx.x] += sn[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = se[0];
    part[2 * blockIdx.x + 1] = sn[0];
  }
}

__global__ void __launch_bounds__(kXYThreads) xy_finish_kernel(const double* __restrict__ part, int nb,
                                                               double* __restrict__ out) {
  __shared__ double se[kXYThreads], sn[kXYThreads];
  double e = 0.0, nn = 0.0;
  for (int b = threadIdx.x; b < nb; b += kXYThreads) {
    e += part[2 * b];
    nn += part[2 * b + 1];
  }
  se[threadIdx.x] = e;
  sn[threadIdx.x] = nn;
  __syncthreads();
  for (int h = kXYThreads / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      se[threadIdx.x] += se[threadIdx.x + h];
      sn[threadIdx.x] += sn[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = se[0];
    out[1] = sn[0];
  }
}

struct XYTableArgs {
  double gam[QAOA_MAX_P];
  int p;
  long long cmin, span;
  void* tab;
};

template <typename T>
__global__ void xy_tables_kernel(const __grid_constant__ XYTableArgs a) {
  const long long total = (long long)a.p * a.span;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int l = (int)(i / a.span);
    ((T*)a.tab)[i] = phase_of(a.gam[l] * (double)(a.cmin + i % a.span), (T*)nullptr);
  }
}

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

int sm_count() {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

unsigned grid_for(unsigned long long work, int sms) {
  const unsigned long long cap = (unsigned long long)sms * 8;
  const unsigned long long b = (work + kXYThreads - 1) / kXYThreads;
  return (unsigned)(b < 1 ? 1 : (b < cap ? b : cap));
}

void fill_shape(XYShape& s, int n, int k) {
  std::memset(&s, 0, sizeof(s));
  s.n = n;
  s.k = k;
  for (int c = 0; c < kBN; ++c) {
    s.binom[c][0] = 1;
    for (int i = 1; i <= c; ++i) s.binom[c][i] = s.binom[c - 1][i - 1] + s.binom[c - 1][i];
  }
  s.D = s.binom[n][k];
}

bool shape_ok(int n, int k) { return n >= 1 && n <= QAOA_XY_MAX_N && k >= 0 && k <= n; }
bool dtype_ok(int dtype) { return dtype == QAOA_C128 || dtype == QAOA_C64; }
size_t elem_bytes(int dtype) { return dtype == QAOA_C128 ? 16 : 8; }
size_t cost_bytes(int cost_dtype) { return cost_dtype == QAOA_COST_I32 ? 4 : 8; }
int status_of(cudaError_t e) { return e == cudaSuccess ? QAOA_OK : QAOA_ERR_CUDA; }

// phase-table span of an integer cost descriptor, 0 when the phases are computed directly
long long table_span(const qaoa_cost_t* c) {
  if (c == nullptr || c->dtype != QAOA_COST_I32 || c->cmax < c->cmin) return 0;
  const long long span = c->cmax - c->cmin + 1;
  return span <= QAOA_MAX_TABLE_SPAN ? span : 0;
}

size_t ws_bytes_for(int dtype, int p, long long span) {
  size_t b = round256(2 * (size_t)kXYRedBlocks * sizeof(double));
  if (span > 0 && p > 0) b += round256((size_t)p * span * elem_bytes(dtype));
  return b;
}

// the ring pairs (a < b) in application order: even set, odd set, closing pair
int ring_pairs(int n, int (*pr)[2]) {
  int np = 0;
  if (n < 2) return 0;
  if (n == 2) {
    pr[0][0] = 0;
    pr[0][1] = 1;
    return 1;
  }
  for (int j = 0; j < n - 1; j += 2, ++np) pr[np][0] = j, pr[np][1] = j + 1;
  for (int j = 1; j < n - 1; j += 2, ++np) pr[np][0] = j, pr[np][1] = j + 1;
  pr[np][0] = 0;
  pr[np][1] = n - 1;
  return np + 1;
}

int graph_check(const qaoa_graph_t* g, long long* neg, long long* pos, double* sum_abs) {
  if (g == nullptr || g->n < 1 || g->n > QAOA_XY_MAX_N || g->m < 0 || g->m > QAOA_XY_MAX_EDGES)
    return QAOA_ERR_INVALID_ARG;
  if (g->m > 0 && g->uv == nullptr) return QAOA_ERR_INVALID_ARG;
  if (g->weight_kind != QAOA_WEIGHT_INT && g->weight_kind != QAOA_WEIGHT_F64) return QAOA_ERR_INVALID_ARG;
  bool seen[QAOA_XY_MAX_N][QAOA_XY_MAX_N] = {};
  *neg = *pos = 0;
  *sum_abs = 0.0;
  for (int64_t e = 0; e < g->m; ++e) {
    const int u = g->uv[2 * e], v = g->uv[2 * e + 1];
    if (u < 0 || v < 0 || u >= g->n || v >= g->n || u == v) return QAOA_ERR_INVALID_ARG;
    if (seen[u][v]) return QAOA_ERR_INVALID_ARG;
    seen[u][v] = seen[v][u] = true;
    const double w = g->w ? g->w[e] : 1.0;
    if (!std::isfinite(w)) return QAOA_ERR_INVALID_ARG;
    *sum_abs += std::fabs(w);
    if (g->weight_kind == QAOA_WEIGHT_INT) {
      if (w != std::floor(w) || std::fabs(w) >= 2147483648.0) return QAOA_ERR_INVALID_ARG;
      if (w < 0) *neg += (long long)w; else *pos += (long long)w;
    }
  }
  if (g->weight_kind == QAOA_WEIGHT_INT && *sum_abs >= 2147483648.0) return QAOA_ERR_INVALID_ARG;
  if (g->weight_kind == QAOA_WEIGHT_F64 && !(*sum_abs < 1e300)) return QAOA_ERR_INVALID_ARG;
  return QAOA_OK;
}

bool cost_ok(const qaoa_cost_t* c) {
  return c != nullptr && c->C_dev != nullptr && (c->dtype == QAOA_COST_I32 || c->dtype == QAOA_COST_F64);
}

template <typename T>
int expectation_t(const XYShape& s, const T* psi, const qaoa_cost_t* cost, double* out, double* part,
                  cudaStream_t st) {
  const int nb = (int)(s.D < (unsigned long long)kXYRedBlocks * kXYThreads ? (s.D + kXYThreads - 1) / kXYThreads
                                                                         : kXYRedBlocks);
  note_launch(3, st, true);
  xy_expect_kernel<T><<<nb, kXYThreads, 0, st>>>(psi, cost->C_dev, cost->dtype, s.D, part);
  note_launch(3, st, false, (double)s.D * (sizeof(T) + cost_bytes(cost->dtype)));
  note_launch(3, st, true);
  xy_finish_kernel<<<1, kXYThreads, 0, st>>>(part, nb, out);
  note_launch(3, st, false);
  return status_of(cudaGetLastError());
}

// The windows of the ring mixer for (n, k), 0 < k < n, n >= 2: tiles of 32 KB of amplitudes
// per buffer; the first window visits every amplitude, since the layer's cost unitary rides
// on its pass; the closing pair (0, n - 1) (n >= 3) is a per-gate pass after the windows.
struct XYMixPlan {
  int nwin;
  bool closing;
  xyw::Window win[xyw::kMaxWindows];
};

template <typename T>
XYMixPlan* make_mix_plan(const XYShape& s) {
  XYMixPlan* mp = new XYMixPlan;
  int lo[xyw::kMaxWindows + 1], w[xyw::kMaxWindows + 1];
  mp->nwin = xyw::plan_ring_windows(s.n, lo, w);
  for (int i = 0; i < mp->nwin; ++i)
    xyw::plan_window(mp->win[i], s.n, s.k, lo[i], w[i], (int)(32768 / sizeof(T)), s.binom, i == 0);
  mp->closing = s.n >= 3;
  return mp;
}

template <typename T, bool TWO>
size_t window_smem(const xyw::Window& W) {
  return (size_t)W.tile_elems * sizeof(T) * (TWO ? 2 : 1);
}

// one windowed pass; grid = 0 takes every SM's resident blocks (forward), the gradient passes
// its partial-row grid
template <typename T, bool TWO, bool PH>
cudaError_t launch_window(const xyw::Window& W, T* psi, T* lam, typename Real<T>::type cb,
                          typename Real<T>::type sb, double* part, const XYPhaseArgs<T>& ph, unsigned grid,
                          cudaStream_t st) {
  static std::mutex mu;
  static unsigned long long done = 0;
  static int per_sm = 1;
  const size_t max_smem = (size_t)32768 * (TWO ? 2 : 1);  // tiles hold <= 32 KB of amplitudes per buffer
  {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    if (!(done & (1ull << (dev & 63)))) {
      cudaFuncSetAttribute(xy_window_kernel<T, TWO, PH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_smem);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, xy_window_kernel<T, TWO, PH>, kXYThreads, max_smem);
      if (per_sm < 1) per_sm = 1;
      done |= 1ull << (dev & 63);
    }
  }
  if (W.tiles == 0) return cudaSuccess;
  if (window_smem<T, TWO>(W) > max_smem) return cudaErrorInvalidValue;
  if (grid == 0) {
    const unsigned long long g = (unsigned long long)sm_count() * per_sm;
    grid = (unsigned)(W.tiles < g ? W.tiles : g);
  }
  const double cb_bytes = PH ? (double)W.elems * cost_bytes(ph.cost_dtype) : 0.0;
  const double bytes = (double)W.elems * sizeof(T) * 2 * (TWO ? 2 : 1) + cb_bytes;
  note_launch(0, st, true);
  xy_window_kernel<T, TWO, PH><<<grid, kXYThreads, window_smem<T, TWO>(W), st>>>(W, psi, lam, cb, sb, part, ph);
  note_launch(0, st, false, bytes);
  return cudaGetLastError();
}

template <typename T>
int layers_t(const XYShape& s, T* psi, const qaoa_cost_t* cost, const double* gamma, const double* beta, int p,
             int init, double* expect_dev, char* ws, cudaStream_t st) {
  using R = typename Real<T>::type;
  const int sms = sm_count();
  const size_t sb = sizeof(T);
  double* part = (double*)ws;
  const long long span = p > 0 ? table_span(cost) : 0;
  T* tab = span > 0 ? (T*)(ws + round256(2 * (size_t)kXYRedBlocks * sizeof(double))) : nullptr;
  if (init) {
    note_launch(3, st, true);
    xy_init_kernel<T><<<grid_for(s.D, sms), kXYThreads, 0, st>>>(psi, s.D, 1.0 / std::sqrt((double)s.D));
    note_launch(3, st, false, (double)s.D * sb);
  }
  if (tab != nullptr) {
    XYTableArgs ta;
    std::memset(&ta, 0, sizeof(ta));
    for (int l = 0; l < p; ++l) ta.gam[l] = gamma[l];
    ta.p = p;
    ta.cmin = cost->cmin;
    ta.span = span;
    ta.tab = tab;
    note_launch(3, st, true);
    xy_tables_kernel<T><<<grid_for((unsigned long long)p * span, sms), kXYThreads, 0, st>>>(ta);
    note_launch(3, st, false);
  }
  const bool mixes = s.k > 0 && s.k < s.n && s.n >= 2;
  XYMixPlan* mp = mixes && p > 0 ? make_mix_plan<T>(s) : nullptr;
  const unsigned long long moved = s.n >= 2 && s.k >= 1 && s.k <= s.n - 1 ? 2 * s.binom[s.n - 2][s.k - 1] : 0;
  const unsigned long long nch = (s.D + kXYChunk - 1) / kXYChunk;
  for (int l = 0; l < p; ++l) {
    const XYPhaseArgs<T> ph = {cost->C_dev, cost->dtype, tab ? tab + (size_t)l * span : nullptr, cost->cmin, span,
                               gamma[l], nullptr};
    if (mp == nullptr) {  // no mixer (k = 0 or k = n): the cost unitary alone
      note_launch(0, st, true);
      xy_phase_kernel<T><<<grid_for(s.D, sms), kXYThreads, 0, st>>>(psi, cost->C_dev, cost->dtype, s.D, ph.tab,
                                                                    cost->cmin, span, gamma[l]);
      note_launch(0, st, false, (double)s.D * (2 * sb + cost_bytes(cost->dtype)));
    }
    const R cb = (R)std::cos(beta[l]), snb = (R)std::sin(beta[l]);
    if (mp != nullptr) {  // the cost unitary on the first window's pass, the ring mixer, the closing pair
      for (int i = 0; i < mp->nwin; ++i) {
        const cudaError_t e =
            i == 0 ? launch_window<T, false, true>(mp->win[i], psi, nullptr, cb, snb, nullptr, ph, 0, st)
                   : launch_window<T, false, false>(mp->win[i], psi, nullptr, cb, snb, nullptr, ph, 0, st);
        if (e != cudaSuccess) {
          delete mp;
          return QAOA_ERR_CUDA;
        }
      }
      if (mp->closing) {
        note_launch(0, st, true);
        xy_gate_kernel<T><<<grid_for(nch, sms), kXYThreads, 0, st>>>(s, psi, 0, s.n - 1, cb, snb);
        note_launch(0, st, false, (double)moved * 2 * sb);
      }
    }
    const int rc = status_of(cudaGetLastError());
    if (rc) {
      delete mp;
      return rc;
    }
  }
  delete mp;
  if (expect_dev != nullptr) return expectation_t<T>(s, psi, cost, expect_dev, part, st);
  return status_of(cudaGetLastError());
}

// partial rows of the gradient: E, norm, dE/dgamma_l (p rows), dE/dbeta_l (p x pairs rows, of
// which a layer uses one per mixer window and one for the closing pair)
size_t xy_grad_part_bytes(int n, int k, int p) {
  int pr[QAOA_XY_MAX_N][2];
  const int np = (k > 0 && k < n) ? ring_pairs(n, pr) : 0;
  return round256((size_t)(2 + p + (size_t)p * np) * kXYPartStride * sizeof(double));
}

template <typename T>
int gradient_t(const XYShape& s, T* psi, T* lam, const qaoa_cost_t* cost, const double* gamma, const double* beta,
               int p, double* out, char* ws, cudaStream_t st) {
  using R = typename Real<T>::type;
  const int sms = sm_count();
  const size_t sb = sizeof(T);
  // forward pass (Dicke start, p layers) with the layer workspace at the front
  int rc = layers_t<T>(s, psi, cost, gamma, beta, p, 1, nullptr, ws, st);
  if (rc) return rc;
  const long long span = p > 0 ? table_span(cost) : 0;
  const T* tab = span > 0 ? (const T*)(ws + round256(2 * (size_t)kXYRedBlocks * sizeof(double))) : nullptr;
  double* part = (double*)(ws + ws_bytes_for(sizeof(T) == 16 ? QAOA_C128 : QAOA_C64, p, span));
  int pr[QAOA_XY_MAX_N][2];
  const int np = (s.k > 0 && s.k < s.n) ? ring_pairs(s.n, pr) : 0;
  const unsigned gr = std::min<unsigned>(grid_for(s.D, sms), kXYPartStride);  // one partial slot per block
  const unsigned long long nch = (s.D + kXYChunk - 1) / kXYChunk;
  const unsigned gg = std::min<unsigned>(grid_for(nch, sms), kXYPartStride);
  const unsigned long long moved = s.n >= 2 && s.k >= 1 && s.k <= s.n - 1 ? 2 * s.binom[s.n - 2][s.k - 1] : 0;
  note_launch(0, st, true);
  xy_lambda_kernel<T><<<gr, kXYThreads, 0, st>>>(psi, lam, cost->C_dev, cost->dtype, s.D, part, part + kXYPartStride);
  note_launch(0, st, false, (double)s.D * (2 * sb + cost_bytes(cost->dtype)));
  // beta rows of layer l: one per window and one for the closing pair (at most np of them),
  // every row written by a launch of gg blocks
  XYMixPlan* mp = np > 0 && p > 0 ? make_mix_plan<T>(s) : nullptr;
  const int brows = mp != nullptr ? mp->nwin + (mp->closing ? 1 : 0) : 0;
  const bool fused = mp != nullptr;  // gamma terms from the first window's pass (gg blocks)
  for (int l = p - 1; l >= 0; --l) {
    const R cb = (R)std::cos(beta[l]), snb = (R)(-std::sin(beta[l]));
    double* rows = part + (size_t)(2 + p + (size_t)l * np) * kXYPartStride;
    if (mp != nullptr) {
      if (mp->closing) {  // applied last in the layer, undone first
        note_launch(0, st, true);
        xy_gate_adjoint_kernel<T><<<gg, kXYThreads, 0, st>>>(s, psi, lam, 0, s.n - 1, cb, snb,
                                                              rows + (size_t)mp->nwin * kXYPartStride);
        note_launch(0, st, false, (double)moved * 4 * sb);
      }
      // the first window's pass also takes the gamma term and undoes the cost unitary
      const XYPhaseArgs<T> ph = {cost->C_dev, cost->dtype, tab ? tab + (size_t)l * span : nullptr, cost->cmin,
                                 span, gamma[l], part + (size_t)(2 + l) * kXYPartStride};
      for (int i = mp->nwin - 1; i >= 0; --i) {
        double* row = rows + (size_t)i * kXYPartStride;
        const cudaError_t e = i == 0 ? launch_window<T, true, true>(mp->win[i], psi, lam, cb, snb, row, ph, gg, st)
                                     : launch_window<T, true, false>(mp->win[i], psi, lam, cb, snb, row, ph, gg, st);
        if (e != cudaSuccess) {
          delete mp;
          return QAOA_ERR_CUDA;
        }
      }
    } else {
      note_launch(0, st, true);
      xy_cost_adjoint_kernel<T><<<gr, kXYThreads, 0, st>>>(psi, lam, cost->C_dev, cost->dtype, s.D,
                                                           tab ? tab + (size_t)l * span : nullptr, cost->cmin, span,
                                                           gamma[l], part + (size_t)(2 + l) * kXYPartStride);
      note_launch(0, st, false, (double)s.D * (4 * sb + cost_bytes(cost->dtype)));
    }
    rc = status_of(cudaGetLastError());
    if (rc) {
      delete mp;
      return rc;
    }
  }
  delete mp;
  XYReducePlan rp;
  std::memset(&rp, 0, sizeof(rp));
  rp.nout = 2 + 2 * p;
  for (int o = 0; o < 2; ++o) rp.first[o] = o, rp.rows[o] = 1, rp.cols[o] = (int)gr;
  for (int l = 0; l < p; ++l) {
    rp.first[2 + l] = 2 + l, rp.rows[2 + l] = 1, rp.cols[2 + l] = (int)(fused ? gg : gr);
    rp.first[2 + p + l] = 2 + p + l * np, rp.rows[2 + p + l] = brows, rp.cols[2 + p + l] = (int)gg;
  }
  note_launch(3, st, true);
  xy_grad_reduce_kernel<<<rp.nout, kXYThreads, 0, st>>>(rp, part, out);
  note_launch(3, st, false);
  return status_of(cudaGetLastError());
}

}  // namespace
}  // namespace qaoa

using namespace qaoa;

extern "C" {

int qaoa_xy_dim(int n, int k, int64_t* dim) {
  if (dim == nullptr || !shape_ok(n, k)) return QAOA_ERR_INVALID_ARG;
  XYShape s;
  fill_shape(s, n, k);
  *dim = (int64_t)s.D;
  return QAOA_OK;
}

int qaoa_xy_workspace_size(int n, int k, int dtype, int p, int64_t cost_span, size_t* bytes) {
  if (bytes == nullptr || !shape_ok(n, k) || !dtype_ok(dtype) || p < 0 || p > QAOA_MAX_P || cost_span < 0)
    return QAOA_ERR_INVALID_ARG;
  *bytes = ws_bytes_for(dtype, p, cost_span <= QAOA_MAX_TABLE_SPAN ? cost_span : 0);
  return QAOA_OK;
}

int qaoa_xy_cost_vector(const qaoa_graph_t* g, int k, void* C_dev, int cost_dtype, qaoa_cost_t* desc, void* stream) {
  long long neg = 0, pos = 0;
  double sum_abs = 0.0;
  int rc = graph_check(g, &neg, &pos, &sum_abs);
  if (rc) return rc;
  if (k < 0 || k > g->n || C_dev == nullptr) return QAOA_ERR_INVALID_ARG;
  if (cost_dtype != QAOA_COST_I32 && cost_dtype != QAOA_COST_F64) return QAOA_ERR_INVALID_ARG;
  if (cost_dtype == QAOA_COST_I32 && g->weight_kind != QAOA_WEIGHT_INT) return QAOA_ERR_INVALID_ARG;
  XYCostArgs* a = new XYCostArgs;
  std::memset(a, 0, sizeof(*a));
  fill_shape(a->s, g->n, k);
  a->m = (int)g->m;
  a->cost_dtype = cost_dtype;
  a->integer = g->weight_kind == QAOA_WEIGHT_INT;
  a->C = C_dev;
  if (!a->integer) {  // one common fixed point; every partial sum stays below 2^62
    int e2 = 0;
    std::frexp(sum_abs > 0.0 ? sum_abs : 1.0, &e2);  // sum_abs < 2^e2, so the scale follows the weights
    a->fixed_shift = 62 - e2;
  }
  for (int e = 0; e < a->m; ++e) {
    const double w = g->w ? g->w[e] : 1.0;
    a->eu[e] = (unsigned char)g->uv[2 * e];
    a->ev[e] = (unsigned char)g->uv[2 * e + 1];
    a->ew[e] = a->integer ? (long long)w : (long long)std::llrint(std::ldexp(w, a->fixed_shift));
  }
  const cudaStream_t st = (cudaStream_t)stream;
  const unsigned long long nch = (a->s.D + kXYChunk - 1) / kXYChunk;
  note_launch(1, st, true);
  xy_cost_kernel<<<grid_for(nch, sm_count()), kXYThreads, 0, st>>>(*a);
  note_launch(1, st, false, (double)a->s.D * cost_bytes(cost_dtype));
  rc = status_of(cudaGetLastError());
  delete a;
  if (rc) return rc;
  if (desc) {
    desc->C_dev = C_dev;
    desc->dtype = cost_dtype;
    desc->cmin = g->weight_kind == QAOA_WEIGHT_INT ? neg : 1;
    desc->cmax = g->weight_kind == QAOA_WEIGHT_INT ? pos : 0;
  }
  return QAOA_OK;
}

int qaoa_xy_apply_layers(int n, int k, int dtype, void* psi_dev, const qaoa_cost_t* cost, const double* gamma,
                         const double* beta, int p, int init, double* expect_dev, void* ws_dev, size_t ws_bytes,
                         void* stream) {
  if (!shape_ok(n, k) || !dtype_ok(dtype) || psi_dev == nullptr || p < 0 || p > QAOA_MAX_P) return QAOA_ERR_INVALID_ARG;
  if ((p > 0 || expect_dev != nullptr) && !cost_ok(cost)) return QAOA_ERR_INVALID_ARG;
  if (p > 0 && (gamma == nullptr || beta == nullptr)) return QAOA_ERR_INVALID_ARG;
  for (int l = 0; l < p; ++l)
    if (!std::isfinite(gamma[l]) || !std::isfinite(beta[l])) return QAOA_ERR_INVALID_ARG;
  if (ws_dev == nullptr || ((uintptr_t)ws_dev & 255) != 0) return QAOA_ERR_INVALID_ARG;
  if (ws_bytes < ws_bytes_for(dtype, p, p > 0 ? table_span(cost) : 0)) return QAOA_ERR_WORKSPACE;
  XYShape* s = new XYShape;
  fill_shape(*s, n, k);
  const cudaStream_t st = (cudaStream_t)stream;
  const int rc = dtype == QAOA_C128
                     ? layers_t<double2>(*s, (double2*)psi_dev, cost, gamma, beta, p, init, expect_dev, (char*)ws_dev, st)
                     : layers_t<float2>(*s, (float2*)psi_dev, cost, gamma, beta, p, init, expect_dev, (char*)ws_dev, st);
  delete s;
  return rc;
}

int qaoa_xy_gradient_workspace_size(int n, int k, int dtype, int p, int64_t cost_span, size_t* bytes) {
  if (bytes == nullptr || !shape_ok(n, k) || !dtype_ok(dtype) || p < 0 || p > QAOA_MAX_P || cost_span < 0)
    return QAOA_ERR_INVALID_ARG;
  *bytes = ws_bytes_for(dtype, p, cost_span <= QAOA_MAX_TABLE_SPAN ? cost_span : 0) + xy_grad_part_bytes(n, k, p);
  return QAOA_OK;
}

int qaoa_xy_gradient(int n, int k, int dtype, void* psi_dev, void* lam_dev, const qaoa_cost_t* cost,
                     const double* gamma, const double* beta, int p, double* out_dev, void* ws_dev, size_t ws_bytes,
                     void* stream) {
  if (!shape_ok(n, k) || !dtype_ok(dtype) || psi_dev == nullptr || lam_dev == nullptr || psi_dev == lam_dev ||
      out_dev == nullptr || p < 0 || p > QAOA_MAX_P || !cost_ok(cost))
    return QAOA_ERR_INVALID_ARG;
  if (p > 0 && (gamma == nullptr || beta == nullptr)) return QAOA_ERR_INVALID_ARG;
  for (int l = 0; l < p; ++l)
    if (!std::isfinite(gamma[l]) || !std::isfinite(beta[l])) return QAOA_ERR_INVALID_ARG;
  if (ws_dev == nullptr || ((uintptr_t)ws_dev & 255) != 0) return QAOA_ERR_INVALID_ARG;
  size_t need = 0;
  qaoa_xy_gradient_workspace_size(n, k, dtype, p, p > 0 ? table_span(cost) : 0, &need);
  if (ws_bytes < need) return QAOA_ERR_WORKSPACE;
  XYShape* s = new XYShape;
  fill_shape(*s, n, k);
  const cudaStream_t st = (cudaStream_t)stream;
  const int rc = dtype == QAOA_C128
                     ? gradient_t<double2>(*s, (double2*)psi_dev, (double2*)lam_dev, cost, gamma, beta, p, out_dev,
                                           (char*)ws_dev, st)
                     : gradient_t<float2>(*s, (float2*)psi_dev, (float2*)lam_dev, cost, gamma, beta, p, out_dev,
                                          (char*)ws_dev, st);
  delete s;
  return rc;
}

int qaoa_xy_sample_workspace_size(int n, int k, size_t* bytes) {
  if (bytes == nullptr || !shape_ok(n, k)) return QAOA_ERR_INVALID_ARG;
  XYShape s;
  fill_shape(s, n, k);
  *bytes = round256(sample_ws_bytes_len(s.D));
  return QAOA_OK;
}

int qaoa_xy_sample(int n, int k, int dtype, const void* psi_dev, const qaoa_cost_t* cost, int64_t shots,
                   uint64_t seed, uint64_t* z_dev, double* cost_dev, void* ws_dev, size_t ws_bytes, void* stream) {
  if (!shape_ok(n, k) || !dtype_ok(dtype) || psi_dev == nullptr || !cost_ok(cost) || shots < 0)
    return QAOA_ERR_INVALID_ARG;
  if (shots > 0 && (z_dev == nullptr || cost_dev == nullptr)) return QAOA_ERR_INVALID_ARG;
  if (ws_dev == nullptr || ((uintptr_t)ws_dev & 255) != 0) return QAOA_ERR_INVALID_ARG;
  size_t need = 0;
  qaoa_xy_sample_workspace_size(n, k, &need);
  if (ws_bytes < need) return QAOA_ERR_WORKSPACE;
  XYShape* s = new XYShape;
  fill_shape(*s, n, k);
  SampleArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n = n;
  a.len = s->D;  // the sampler walks the subspace vector in rank order and returns ranks
  a.dtype = dtype;
  a.psi = psi_dev;
  a.C = cost->C_dev;
  a.cost_dtype = cost->dtype;
  a.shots = shots;
  a.seed = seed;
  a.z = z_dev;
  a.cost = cost_dev;
  a.leaf = (double*)ws_dev;
  const cudaStream_t st = (cudaStream_t)stream;
  int rc = status_of(launch_sample(a, st));
  if (rc == QAOA_OK && shots > 0) {
    note_launch(3, st, true);
    xy_unrank_kernel<<<grid_for((unsigned long long)shots, sm_count()), kXYThreads, 0, st>>>(
        *s, (unsigned long long*)z_dev, shots);
    note_launch(3, st, false);
    rc = status_of(cudaGetLastError());
  }
  delete s;
  return rc;
}

int qaoa_xy_expectation(int n, int k, int dtype, const void* psi_dev, const qaoa_cost_t* cost, double* out_dev,
                        void* ws_dev, size_t ws_bytes, void* stream) {
  if (!shape_ok(n, k) || !dtype_ok(dtype) || psi_dev == nullptr || out_dev == nullptr || !cost_ok(cost))
    return QAOA_ERR_INVALID_ARG;
  if (ws_dev == nullptr || ((uintptr_t)ws_dev & 255) != 0) return QAOA_ERR_INVALID_ARG;
  if (ws_bytes < ws_bytes_for(dtype, 0, 0)) return QAOA_ERR_WORKSPACE;
  XYShape* s = new XYShape;
  fill_shape(*s, n, k);
  const cudaStream_t st = (cudaStream_t)stream;
  const int rc = dtype == QAOA_C128
                     ? expectation_t<double2>(*s, (const double2*)psi_dev, cost, out_dev, (double*)ws_dev, st)
                     : expectation_t<float2>(*s, (const float2*)psi_dev, cost, out_dev, (double*)ws_dev, st);
  delete s;
  return rc;
}

}  // extern "C"
