// Layer sweeps: phase separator, mixer, lambda = C psi and the fused reductions of <C>,
// the norm and the adjoint-gradient terms (Eq. 1; Sec. II-B, IV-B, IV-C, IV-D); the tile
// machinery and the arithmetic are described in sweeper.cuh.
#include "sweeper.cuh"

namespace qaoa {
namespace {


// One layer's phase table (the sweeper's graph's) in shared memory: float32 factors as they
// are, fixed-point factors prepared for the limb multiply (fx::Factor, 24 bytes per entry).
// Callers synchronise.
template <bool FX, class S>
__device__ __forceinline__ void stage_table(S& s, const SweepArgs& a, void* dst, int nt) {
  using V = typename S::V;
  const V* src = (const V*)s.ptab + (long long)a.smem_table_layer * s.pspan;
  if constexpr (FX) {
    fx::Factor* tf = (fx::Factor*)dst;
    for (int k = threadIdx.x; k < s.pspan; k += nt) {
      const longlong2 e = __ldg((const longlong2*)src + k);
      tf[k] = fx::factor(e.x, e.y);
    }
    s.Tf = tf;
  } else {
    V* ts = (V*)dst;
    for (int k = threadIdx.x; k < s.pspan; k += nt) ts[k] = __ldg(src + k);
    s.Ts = ts;
  }
  s.ts_layer = a.smem_table_layer;
}

// Lean sweeps: full tiles, affine layout-0 addresses, state loaded in the internal format
// or created as |+>, stored in the internal or the caller's format (complex64: the same).
template <class CF, bool FX, bool TWO, bool OPS, int LAST>
__global__ void __launch_bounds__(CF::NT, CF::MINB) lean_kernel(const __grid_constant__ SweepArgs a) {
  using S = Lean<CF, FX, TWO>;
  using V = typename S::V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* X = (V*)smem_raw;  // exchange area: 2^B slots, twice that for two-buffer sweeps
  void* Cs = smem_raw + ((sizeof(V) << CF::B) << (TWO ? 1 : 0));
  const bool cost = OPS && a.needs_cost;
  V* Tsm = (V*)((unsigned char*)Cs + (cost ? ((a.cost_dtype == QAOA_COST_F64 ? 8 : 4) << CF::B) : 0));
  constexpr int NW = CF::NT / 32;
  __shared__ double wacc[kLeanAcc * NW];
  __shared__ fx::Factor dpre[FX ? kLeanMix * 16 : 1];
  for (int r = threadIdx.x; r < kLeanAcc * NW; r += CF::NT) wacc[r] = 0.0;
  S s(a, X, Cs, nullptr, nullptr);
  s.wacc = wacc;
  // grouped sweeps: this block's graph and its share of the graph's tiles
  int64_t t0 = blockIdx.x, tstep = gridDim.x;
  if (a.gslot != nullptr) {
    const GroupSlot& gsl = a.gslot[blockIdx.x / a.gbpg];
    s.zoff = gsl.zoff;
    s.ptab = gsl.phase_table;
    s.pcmin = gsl.cmin;
    s.pspan = gsl.span;
    s.trig = gsl.trig;
    s.dtab = gsl.d_table;
    t0 = blockIdx.x % a.gbpg;
    tstep = a.gbpg;
  }
  if constexpr (FX) {  // every mixer's diagonal exp(-i beta (t - 2k)), k = 0..t, as prepared factors
    const int t = a.g.t;
    int m = 0;
    for (int k = 0; k < (OPS ? a.nops : 1) && m < kLeanMix; ++k) {
      const uint32_t op = a.ops[k];
      if ((op & 0xff) != OP_MIX) continue;
      if (threadIdx.x <= (uint32_t)t) {
        const longlong2 e = __ldg((const longlong2*)s.dtab + ((long long)((op >> 16) & 0xff) * 14 + t) * 14 + threadIdx.x);
        dpre[16 * m + threadIdx.x] = fx::factor(e.x, (op & F_SIGN) ? -e.y : e.y);
      }
      ++m;
    }
    s.dpre = dpre;
  }
  if (OPS && a.smem_table_layer >= 0) {
    stage_table<FX>(s, a, Tsm, CF::NT);
  }
  if (TWO && a.stage) {  // staging area after the phase table, 16-byte aligned
    const size_t tb = FX ? sizeof(fx::Factor) : sizeof(V);
    const size_t off = (size_t)((unsigned char*)Tsm - smem_raw) + (OPS && a.smem_table_layer >= 0 ? tb * a.span : 0);
    s.Ps = (V*)(smem_raw + ((off + 15) & ~(size_t)15));
  }
  s.evalid = 1u << CF::B;
  if constexpr (FX && TWO) {
    if (a.gslot != nullptr) {
      s.lam_shift = a.gslot[blockIdx.x / a.gbpg].lam_shift;
    } else if (a.cmax_dev != nullptr) {
      const unsigned long long b = *a.cmax_dev;
      const int ex = (int)((b >> 52) & 0x7FF);
      const int k = ex == 0 ? 0 : ex - 1023 + ((b & ((1ull << 52) - 1)) != 0 ? 1 : 0);
      s.lam_shift = k < 0 ? 0 : k;
    }
  }
  __syncthreads();
  bool have = false;  // this tile's psi is in the staging area
  for (int64_t tile = t0; tile < a.g.tiles; tile += tstep) {
    const int64_t next = tile + tstep < a.g.tiles ? tile + tstep : -1;
    lean_tile<CF, FX, TWO, OPS, LAST, false>(s, a, tile, Cs, next, have);
    have = s.Ps != nullptr && next >= 0;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < a.nred; r += CF::NT) {
    double v = 0.0;
    for (int w = 0; w < NW; ++w) v += wacc[r * NW + w];
    a.partials[(int64_t)a.red_slot[r] * a.grid + blockIdx.x] = v;
  }
}

template <class CF, bool FX, bool TWO>
__global__ void __launch_bounds__(CF::NT, CF::MINB) sweep_kernel(const __grid_constant__ SweepArgs a) {
  using S = Sweeper<CF, FX, TWO>;
  using V = typename S::V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* X = (V*)smem_raw;  // exchange area: 2^B slots, twice that for two-buffer sweeps
  void* Cs = smem_raw + ((sizeof(V) << CF::B) << (TWO ? 1 : 0));
  V* Tsm = (V*)((unsigned char*)Cs + (a.needs_cost ? ((a.cost_dtype == QAOA_COST_F64 ? 8 : 4) << CF::B) : 0));
  __shared__ double blk[kMaxAcc];
  __shared__ double red[2 * (CF::NT / 32)];
  __shared__ fx::Factor dsm[16];
  for (int r = threadIdx.x; r < kMaxAcc; r += CF::NT) blk[r] = 0.0;

  S s(a, X, Cs, blk, red);
  s.Ds = dsm;
  if (a.smem_table_layer >= 0) {  // one layer's phase table in shared memory
    stage_table<FX>(s, a, Tsm, CF::NT);
    __syncthreads();
  }
  const SweepGeom& g = a.g;
  s.evalid = 1u << (g.t + g.c);
  if constexpr (FX) {
    if (a.cmax_dev != nullptr) {  // smallest k >= 0 with 2^k >= max |C|
      const unsigned long long b = *a.cmax_dev;
      const int ex = (int)((b >> 52) & 0x7FF);
      int k = ex == 0 ? 0 : ex - 1023 + ((b & ((1ull << 52) - 1)) != 0 ? 1 : 0);
      s.lam_shift = k < 0 ? 0 : k;
    }
    if (a.norm2_dev != nullptr) {  // 2^k with |psi| / 2^k in [1, 2)
      const unsigned long long b = (unsigned long long)__double_as_longlong(*a.norm2_dev);
      const int ex = (int)((b >> 52) & 0x7FF);
      s.in_shift = ex == 0 ? 0 : ((ex - 1023) >= 0 ? (ex - 1023) / 2 : -((1023 - ex + 1) / 2));
    }
  }
  for (int64_t tile = blockIdx.x; tile < g.tiles; tile += gridDim.x) sweep_tile<CF, FX, TWO, false>(s, a, tile, Cs);

  __syncthreads();
  for (int r = threadIdx.x; r < a.nred; r += CF::NT)
    a.partials[(int64_t)a.red_slot[r] * a.grid + blockIdx.x] = blk[r];
}

// ------------------------------------------------------------------ small kernels

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
  if (threadIdx.x == 0) out[o] = sh[0] * r.scale[o];
}

// grouped sweeps: one warp per (graph, output), summing the graph's contributions and blocks
// in a fixed order
__global__ void group_reduce_kernel(const __grid_constant__ ReducePlan r, int ngraphs, int bpg,
                                    const int* __restrict__ out_row, const double* __restrict__ partials,
                                    double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t item = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (item >= (int64_t)ngraphs * r.nout) return;
  const int g = (int)(item / r.nout), o = (int)(item % r.nout);
  double v = 0.0;
  for (int i = lane; i < r.ncontrib[o] * bpg; i += 32) {
    const int k = i / bpg, j = i - k * bpg;
    v += partials[((int64_t)o * kMaxContrib + k) * r.grid + (int64_t)g * bpg + j];
  }
  for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
  if (lane == 0) out[(int64_t)out_row[g] * r.nout + o] = v * r.scale[o];
}

// integer-cost phase tables exp(-i gamma_l c), c = cmin + k; then (fixed point) the
// mixer diagonals exp(-i beta_l (t - 2k)) for t = 1..13, k = 0..t, and the turn tables
__global__ void tables_kernel(const __grid_constant__ TableArgs ta) {
  const int64_t nphase = (int64_t)ta.p * ta.span;
  const int64_t nd = ta.fx ? (int64_t)ta.p * 14 * 14 : 0;
  const int64_t nt = ta.fx ? 3 * 1024 : 0;
  const int64_t total = nphase + nd + nt;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < nphase) {
      const int l = (int)(i / ta.span);
      const int64_t c = ta.cmin + (i - (int64_t)l * ta.span);
      const double th = (ta.dev_angles ? ta.dev_angles[l] : ta.gamma[l]) * (double)c;
      if (ta.fx) ((longlong2*)ta.phase)[i] = unit_q62(th);
      else ((float2*)ta.phase)[i] = unit_f32(th);
    } else if (i < nphase + nd) {
      const int64_t j = i - nphase;
      const int l = (int)(j / 196);
      ((longlong2*)ta.dtab)[j] = d_entry(ta.dev_angles ? ta.dev_angles[ta.p + l] : ta.beta[l], (int)(j % 196));
    } else {
      ((longlong2*)ta.turn)[i - nphase - nd] = turn_entry((int)(i - nphase - nd));
    }
  }
}

// [g2pi p | cos(beta) p | sin(beta) p] from device angles [gamma p | beta p]
__global__ void angle_prep_kernel(const double* __restrict__ ang, int p, double* __restrict__ trig) {
  const int l = threadIdx.x;
  if (l < p) {
    trig[l] = ang[l] / (2.0 * 3.141592653589793238);
    double sn, cs;
    sincos(ang[p + l], &sn, &cs);
    trig[p + l] = cs;
    trig[2 * p + l] = sn;
  }
}

// One Adam ascent step on the angles from the gradient output g = [E, norm, dE/dgamma,
// dE/dbeta]; state = [m (2p) | v (2p)]; *step counts completed steps.  The record of this
// step (the 2p + 2 gradient outputs followed by the 2p angles it was evaluated at) goes to
// history[step * (4p + 2)] when history is non-null.
__global__ void adam_kernel(double* __restrict__ ang, const double* __restrict__ g, double* __restrict__ state,
                            long long* __restrict__ step, int p, double lr, double b1, double b2, double eps,
                            double* __restrict__ history, long long row0, long long max_rows) {
  const int i = threadIdx.x;
  const long long t = *step;  // completed steps before this one
  const int np2 = 2 * p;
  if (history != nullptr && t >= row0 && t - row0 < max_rows) {
    double* h = history + (t - row0) * (2 * np2 + 2);
    for (int k = i; k < np2 + 2; k += blockDim.x) h[k] = g[k];
    for (int k = i; k < np2; k += blockDim.x) h[np2 + 2 + k] = ang[k];
  }
  __syncthreads();
  const double c1 = 1.0 - pow(b1, (double)(t + 1)), c2 = 1.0 - pow(b2, (double)(t + 1));
  for (int k = i; k < np2; k += blockDim.x) {
    const double gk = g[2 + k];  // ascent on <C>
    double m = state[k], v = state[np2 + k];
    m = b1 * m + (1.0 - b1) * gk;
    v = b2 * v + (1.0 - b2) * gk * gk;
    state[k] = m;
    state[np2 + k] = v;
    ang[k] += lr * (m / c1) / (sqrt(v / c2) + eps);
  }
  __syncthreads();
  if (i == 0) *step = t + 1;
}

// max |C(z)| over the cost vector -> lam_shift = smallest k with 2^k >= max|C| (device scalar)
__global__ void cost_bound_kernel(const void* __restrict__ C, int f64, int64_t count, unsigned long long* out) {
  unsigned long long mx = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    double c = f64 ? __ldg((const double*)C + i) : (double)__ldg((const int*)C + i);
    c = fabs(c);
    const unsigned long long b = (unsigned long long)__double_as_longlong(c);  // monotone for c >= 0
    mx = b > mx ? b : mx;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_down_sync(0xffffffffu, mx, o);
    mx = y > mx ? y : mx;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(out, mx);
}

// state norm^2 of a user (float64 / float32) state, for the fixed-point input scale
__global__ void norm_kernel(const void* __restrict__ psi, int dtype, int64_t count, double* __restrict__ partials) {
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    if (dtype == QAOA_C128) {
      const double2 d = __ldg((const double2*)psi + i);
      s += d.x * d.x + d.y * d.y;
    } else {
      const float2 f = __ldg((const float2*)psi + i);
      s += (double)f.x * f.x + (double)f.y * f.y;
    }
  }
  __shared__ double sh[256];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

// ------------------------------------------------------------------ launch plumbing

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

template <class CF, bool FX, bool TWO>
size_t smem_bytes(int cost_bytes, int table_entries = 0) {
  const size_t vb = FX ? sizeof(longlong2) : sizeof(float2);
  const size_t tb = FX ? sizeof(fx::Factor) : sizeof(float2);  // staged phase-table entry
  return ((vb << CF::B) << (TWO ? 1 : 0)) + ((size_t)cost_bytes << CF::B) + tb * table_entries;
}

// blocks per SM for a configuration with a cost tile of cost_bytes per amplitude (0, 4, 8)
template <class CF, bool FX, bool TWO>
int blocks_per_sm(int cost_bytes) {
  static int cached[3] = {0, 0, 0};
  static std::mutex mu;
  static uint64_t done = 0;
  const int slot = cost_bytes == 0 ? 0 : (cost_bytes == 4 ? 1 : 2);
  once_per_device(mu, done, [] {
    cudaFuncSetAttribute(sweep_kernel<CF, FX, TWO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem_bytes<CF, FX, TWO>(8, kSmemTable));
  });
  if (!cached[slot]) {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel<CF, FX, TWO>, CF::NT,
                                                  smem_bytes<CF, FX, TWO>(cost_bytes, kSmemTable));
    cached[slot] = nb > 0 ? nb : 1;
  }
  return cached[slot];
}

// dynamic shared memory a lean kernel may take on this device: the opt-in limit less its
// static shared memory (two-buffer kernels, which may add the psi staging area), else the
// largest exchange + cost + table layout
template <class CF, bool FX, bool TWO>
size_t lean_smem_cap() {
  static size_t cached[64] = {};
  static std::mutex mu;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  size_t& c = cached[dev & 63];
  if (c == 0) {
    c = smem_bytes<CF, FX, TWO>(8, kSmemTable);
    if (TWO) {
      int optin = 0;
      cudaFuncAttributes fa;
      if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
          cudaFuncGetAttributes(&fa, lean_kernel<CF, FX, TWO, true, 0>) == cudaSuccess &&
          (size_t)optin > fa.sharedSizeBytes + 1024)
        c = std::max(c, (size_t)optin - fa.sharedSizeBytes - 1024);
    }
  }
  return c;
}

template <class CF, bool FX, bool TWO, bool OPS, int LAST>
void lean_launch_l(const SweepArgs& a, size_t sm, cudaStream_t s) {
  static std::mutex mu;
  static uint64_t done = 0;
  once_per_device(mu, done, [] {
    cudaFuncSetAttribute(lean_kernel<CF, FX, TWO, OPS, LAST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)lean_smem_cap<CF, FX, TWO>());
  });
  lean_kernel<CF, FX, TWO, OPS, LAST><<<a.grid, CF::NT, sm, s>>>(a);
}
template <class CF, bool FX, bool TWO, bool OPS>
void lean_launch(const SweepArgs& a, int last, size_t sm, cudaStream_t s) {
  switch (last) {
    case 0: lean_launch_l<CF, FX, TWO, OPS, 0>(a, sm, s); break;
    case 1: lean_launch_l<CF, FX, TWO, OPS, 1>(a, sm, s); break;
    case 2: lean_launch_l<CF, FX, TWO, OPS, 2>(a, sm, s); break;
    default: lean_launch_l<CF, FX, TWO, OPS, (CF::NR > 3 ? 3 : 2)>(a, sm, s); break;
  }
}

template <class CF, bool FX, bool TWO>
void launch_t(const SweepArgs& a, cudaStream_t s) {
  blocks_per_sm<CF, FX, TWO>(8);
  const int cb = a.needs_cost ? (a.cost_dtype == QAOA_COST_F64 ? 8 : 4) : 0;
  const int te = a.smem_table_layer >= 0 ? (int)a.span : 0;
  const size_t sm = smem_bytes<CF, FX, TWO>(cb, te);
  if (a.kind == SWEEP_LEAN_MIX || a.kind == SWEEP_LEAN_OPS) {
    // last round holding group qubits selects the instance
    int last = 0;
    for (int k = 0; k < CF::NR; ++k) {
      const int lo = std::max(0, CF::B - CF::RB * (k + 1)), hi = k == 0 ? CF::B : std::max(0, CF::B - CF::RB * k);
      if (hi > a.g.c && lo < a.g.c + a.g.t) last = k;
    }
    // complex128 two-buffer sweeps that load psi stage the next tile's psi when shared
    // memory allows (complex64: measured no gain)
    SweepArgs b = a;
    b.stage = 0;
    if (TWO && FX && !(a.kind == SWEEP_LEAN_OPS && a.load_fmt == 2)) {
      const size_t st = ((sm + 15) & ~(size_t)15) + ((FX ? sizeof(longlong2) : sizeof(float2)) << CF::B);
      if (st <= lean_smem_cap<CF, FX, TWO>()) {
        b.stage = 1;
        if (a.kind == SWEEP_LEAN_OPS) lean_launch<CF, FX, TWO, true>(b, last, st, s);
        else lean_launch<CF, FX, TWO, false>(b, last, st, s);
        return;
      }
    }
    if (a.kind == SWEEP_LEAN_OPS) lean_launch<CF, FX, TWO, true>(b, last, sm, s);
    else lean_launch<CF, FX, TWO, false>(b, last, sm, s);
    return;
  }
  sweep_kernel<CF, FX, TWO><<<a.grid, CF::NT, sm, s>>>(a);
}

// <C> and the norm of a user-format state, one pass (stand-alone expectation)
template <bool C128>
__global__ void expect_kernel(const void* __restrict__ psi, const void* __restrict__ C, int cost_f64, int64_t count,
                              double* __restrict__ partials, int grid) {
  double e0 = 0.0, e1 = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < count; i0 += 32 * stride) {
    float f0 = 0.f, f1 = 0.f;
    for (int k = 0; k < 32; ++k) {
      const int64_t i = i0 + k * stride;
      if (i >= count) break;
      const double c = cost_f64 ? __ldg((const double*)C + i) : (double)__ldg((const int*)C + i);
      if (C128) {
        const double2 d = __ldg((const double2*)psi + i);
        const double pr = d.x * d.x + d.y * d.y;
        e0 += c * pr;
        e1 += pr;
      } else {
        const float2 f = __ldg((const float2*)psi + i);
        const float pr = f.x * f.x + f.y * f.y;
        f0 += (float)c * pr;
        f1 += pr;
      }
    }
    if (!C128) {
      e0 += f0;
      e1 += f1;
    }
  }
  __shared__ double sh[2][256];
  sh[0][threadIdx.x] = e0;
  sh[1][threadIdx.x] = e1;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + st];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + st];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = sh[0][0];
    partials[(int64_t)kMaxContrib * grid + blockIdx.x] = sh[1][0];
  }
}

}  // namespace

int sweep_tile_bits(int dtype, bool /*two*/) {
  return dtype == QAOA_C128 ? 12 : 13;
}

// values stay below 2^61 through a group's Walsh-Hadamard transform (growth 2^(t/2)) for
// states of norm < 2, as the limb multiply requires
int fx_shift_for(int tmax) { return 62 - (tmax + 1) / 2 - 2; }

int sweep_grid(int dtype, bool two, int tile_bits, int cost_bytes, int64_t tiles) {
  int per_sm;
  if (dtype == QAOA_C128) {
    per_sm = two ? blocks_per_sm<CfgX2, true, true>(cost_bytes) : blocks_per_sm<CfgX1, true, false>(cost_bytes);
  } else if (two) {
    per_sm = blocks_per_sm<CfgF3, false, true>(cost_bytes);
  } else {
    per_sm = blocks_per_sm<CfgF1, false, false>(cost_bytes);
  }
  const int64_t cap = (int64_t)num_sms() * per_sm;
  return (int)(tiles < cap ? tiles : cap);
}

cudaError_t launch_sweep(int dtype, bool two, const SweepArgs& a, cudaStream_t s) {
  note_launch(0, s, true);
  if (dtype == QAOA_C128) {
    if (two) launch_t<CfgX2, true, true>(a, s);
    else launch_t<CfgX1, true, false>(a, s);
  } else {
    if (two) launch_t<CfgF3, false, true>(a, s);
    else launch_t<CfgF1, false, false>(a, s);
  }
  note_launch(0, s, false, a.algo_bytes);
  return cudaGetLastError();
}

cudaError_t launch_expect(int dtype, const void* psi, const void* C, int cost_dtype, int n, double* partials,
                          int grid, cudaStream_t s) {
  const int64_t count = 1ll << n;
  const double bytes = (double)count * ((dtype == QAOA_C128 ? 16.0 : 8.0) + (cost_dtype == QAOA_COST_F64 ? 8.0 : 4.0));
  note_launch(0, s, true);
  if (dtype == QAOA_C128)
    expect_kernel<true><<<grid, 256, 0, s>>>(psi, C, cost_dtype == QAOA_COST_F64, count, partials, grid);
  else
    expect_kernel<false><<<grid, 256, 0, s>>>(psi, C, cost_dtype == QAOA_COST_F64, count, partials, grid);
  note_launch(0, s, false, bytes);
  return cudaGetLastError();
}

cudaError_t launch_reduce(const ReducePlan& r, const double* partials, double* out, cudaStream_t s) {
  note_launch(3, s, true);
  reduce_kernel<<<r.nout, 256, 0, s>>>(r, partials, out);
  note_launch(3, s, false);
  return cudaGetLastError();
}

cudaError_t launch_group_reduce(const ReducePlan& r, int ngraphs, int bpg, const int* out_row,
                                const double* partials, double* out, cudaStream_t s) {
  const int64_t items = (int64_t)ngraphs * r.nout;
  if (items == 0) return cudaSuccess;
  note_launch(3, s, true);
  group_reduce_kernel<<<(unsigned)((items + 7) / 8), 256, 0, s>>>(r, ngraphs, bpg, out_row, partials, out);
  note_launch(3, s, false);
  return cudaGetLastError();
}

cudaError_t launch_tables(const TableArgs& t, cudaStream_t s) {
  const int64_t total = (int64_t)t.p * t.span + (t.fx ? (int64_t)t.p * 196 + 3072 : 0);
  if (total <= 0) return cudaSuccess;
  const int blocks = (int)((total + 255) / 256 < 1024 ? (total + 255) / 256 : 1024);
  note_launch(3, s, true);
  tables_kernel<<<blocks, 256, 0, s>>>(t);
  note_launch(3, s, false);
  return cudaGetLastError();
}

cudaError_t launch_cost_bound(const void* C, int f64, int n, unsigned long long* out, cudaStream_t s) {
  note_launch(3, s, true, (double)(1ull << n) * (f64 ? 8.0 : 4.0));
  cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
  const int64_t count = 1ll << n;
  int64_t blocks = (count + 255) / 256;
  if (blocks > (int64_t)num_sms() * 8) blocks = (int64_t)num_sms() * 8;
  cost_bound_kernel<<<(int)blocks, 256, 0, s>>>(C, f64, count, out);
  note_launch(3, s, false, (double)(1ull << n) * (f64 ? 8.0 : 4.0));
  return cudaGetLastError();
}

cudaError_t launch_angle_prep(const double* ang, int p, double* trig, cudaStream_t s) {
  note_launch(3, s, true);
  angle_prep_kernel<<<1, 64, 0, s>>>(ang, p, trig);
  note_launch(3, s, false);
  return cudaGetLastError();
}

cudaError_t launch_adam(double* ang, const double* g, double* state, long long* step, int p, double lr, double b1,
                        double b2, double eps, double* history, long long row0, long long max_rows, cudaStream_t s) {
  note_launch(3, s, true);
  adam_kernel<<<1, 128, 0, s>>>(ang, g, state, step, p, lr, b1, b2, eps, history, row0, max_rows);
  note_launch(3, s, false);
  return cudaGetLastError();
}

cudaError_t launch_norm(const void* psi, int dtype, int n, double* partials, int* nblocks, cudaStream_t s) {
  const int64_t count = 1ll << n;
  int64_t blocks = (count + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  *nblocks = (int)blocks;
  note_launch(3, s, true);
  norm_kernel<<<(int)blocks, 256, 0, s>>>(psi, dtype, count, partials);
  note_launch(3, s, false, (double)count * (dtype == QAOA_C128 ? 16.0 : 8.0));
  return cudaGetLastError();
}

}  // namespace qaoa
