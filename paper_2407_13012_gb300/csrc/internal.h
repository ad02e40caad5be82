// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "qaoa_gb300.h"

namespace qaoa {

// ---------------------------------------------------------------- sweeps
//
// A "sweep" reads (or creates) the state in tiles, runs a short program of
// operations on each tile, and writes it back.  A tile holds every
// combination of the group qubits [j0, j0 + t) together with the 2^c lowest
// index bits (kept for coalesced access); the other index bits are fixed per
// tile.  Elementwise operations (phase, lambda = C psi, reductions) can run
// at any point of the program; RX mixers act on the group qubits only.

enum OpKind : uint32_t {
  OP_PHASE = 1,        // psi_z *= exp(-i s gamma_l C(z))           arg = layer, flag SIGN = inverse
  OP_MIX = 2,          // RX(2 s beta_l) on every group qubit        arg = layer, flag SIGN = inverse
  OP_LAMBDA = 3,       // lam := C psi
  OP_RED_EXPECT = 4,   // partial += [sum C|psi|^2, sum |psi|^2]     arg = output index (two outputs)
  OP_RED_XTERM = 5,    // partial += 2 Im sum_{j in group} <lam|X_j|psi>   arg = output index
  OP_RED_CTERM = 6,    // partial += 2 Im <lam|C|psi>                arg = output index
};
enum OpFlags : uint32_t { F_PSI = 1u << 8, F_LAM = 1u << 9, F_SIGN = 1u << 10 };

inline uint32_t make_op(uint32_t kind, uint32_t flags, uint32_t arg) {
  return kind | flags | (arg << 16);
}

constexpr int kMaxOps = 200;
constexpr int kMaxAcc = 2 * QAOA_MAX_P + 2;  // reduction accumulators per sweep (double each)
constexpr int kMaxContrib = 8;               // partial slots per output

struct SweepGeom {
  int n;      // qubits
  int j0;     // first group qubit
  int t;      // group qubits in the tile (j0 + t <= n), may be < tile bits for tiny n
  int c;      // low index bits carried in the tile (c <= j0), 0 for the first group
  int64_t tiles;  // number of tiles = 2^(n - t - c)
};

struct SweepArgs {
  void* psi;
  void* lam;
  const void* C;
  int cost_dtype;
  SweepGeom g;
  int init_plus;   // create |+> instead of loading psi
  int load_psi, store_psi, load_lam, store_lam;
  int nops;
  uint32_t ops[kMaxOps];
  // per layer angles, indexed by the op's layer argument
  double gamma[QAOA_MAX_P];
  double cosb[QAOA_MAX_P];
  double sinb[QAOA_MAX_P];
  // integer-cost phase tables: table + l * span holds exp(-i gamma_l c) for c = cmin + k
  const void* phase_table;  // double2 (C128) or float2 (C64), NULL = compute sincos
  int64_t cmin;
  int64_t span;
  // reductions: accumulator r (the argument of a reduction op; OP_RED_EXPECT uses r and
  // r + 1) is written to partials[red_slot[r] * grid + block], with
  // red_slot = out * kMaxContrib + contrib
  int nred;
  int red_slot[kMaxAcc];
  double* partials;
  int grid;
  double algo_bytes;  // HBM bytes this sweep must move (for timing reports)
};

// A reduction plan: out[o] = sum over contributions k < ncontrib[o] and blocks b of
// partials[(o * kMaxContrib + k) * grid + b].
struct ReducePlan {
  int nout;
  int grid;
  int ncontrib[2 * QAOA_MAX_P + 2];
};

// launchers (return a CUDA error code)
cudaError_t launch_sweep(int dtype, const SweepArgs& a, cudaStream_t s);
cudaError_t launch_reduce(const ReducePlan& r, const double* partials, double* out, cudaStream_t s);
cudaError_t launch_phase_table(int dtype, const double* gamma, int p, int64_t cmin, int64_t span,
                               void* table, cudaStream_t s);
int sweep_tile_bits(int dtype);   // max t + c per tile
int sweep_grid(int dtype, int64_t tiles);  // persistent grid size for a sweep

// cost vector
struct CostArgs {
  int n;
  int lo_bits;           // low bits handled by the per-CTA table
  int cost_dtype;
  int integer;           // integer weights (int32 exact) vs fixed-point float weights
  int fixed_shift;       // float weights: value = fixed * 2^-fixed_shift
  void* C;
  int64_t wi[QAOA_MAX_N][QAOA_MAX_N];  // symmetric adjacency weights (integer or fixed point)
};
cudaError_t launch_cost(const CostArgs& a, cudaStream_t s);

// sampling
struct SampleArgs {
  int n;
  int dtype;
  const void* psi;
  const void* C;
  int cost_dtype;
  int64_t shots;
  uint64_t seed;
  uint64_t* z;
  double* cost;
  double* leaf;     // 2^n / leaf_size leaf sums, then exclusive prefix (+1 total)
  double* blocksum; // scan scratch
  int leaf_bits;
};
cudaError_t launch_sample(const SampleArgs& a, cudaStream_t s);
size_t sample_ws_bytes(int n, int dtype);

// bookkeeping for benchmarks: call with begin = true before a launch and begin = false
// after it; `bytes` (algorithmic HBM bytes of the launch) is read on the second call
void note_launch(int kind, cudaStream_t s, bool begin, double bytes = 0.0);

}  // namespace qaoa
