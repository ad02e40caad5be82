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
  OP_PHASE = 1,       // psi_z *= exp(-i s gamma_l C(z))                 flag SIGN = inverse
  OP_MIX = 2,         // RX(2 s beta_l) on every group qubit              flag SIGN = inverse; flag XTERM:
                      //   also accumulate 2 Im sum_{j in group} <lam|X_j|psi> into accumulator acc
  OP_LAMBDA = 3,      // lam := C psi
  OP_RED_EXPECT = 4,  // accumulators acc, acc + 1 += [sum C|psi|^2, sum |psi|^2]
  OP_RED_CTERM = 6,   // accumulator acc += 2 Im <lam|C|psi>
};
enum OpFlags : uint32_t { F_PSI = 1u << 8, F_LAM = 1u << 9, F_SIGN = 1u << 10, F_XTERM = 1u << 11 };

// op word: kind (bits 0-7) | flags (8-15) | layer (16-23) | accumulator (24-31)
inline uint32_t make_op(uint32_t kind, uint32_t flags, uint32_t layer, uint32_t acc = 0) {
  return kind | flags | (layer << 16) | (acc << 24);
}

constexpr int kMaxOps = 200;
constexpr int kMaxAcc = 2 * QAOA_MAX_P + 2;  // reduction accumulators per sweep (double each)
constexpr int kMaxContrib = 8;               // partial slots per output
constexpr int kLeanAcc = 8;   // reduction accumulators of a lean sweep (per-warp slots)
constexpr int kLeanMix = 4;   // mixers of a lean sweep (diagonals staged once per launch)
constexpr int kGridCap = 2048;               // most blocks a reduction writes partials for
// qaoa_expectation's workspace: partials of its 2 outputs (kMaxContrib slots x kGridCap
// blocks each); the size qaoa_workspace_size reports adds kHostResultBytes, the slot where
// qaoa_expectation_host lets the device write the result before copying it out
constexpr size_t kExpectPartialBytes = 2 * (size_t)kMaxContrib * kGridCap * sizeof(double);
constexpr size_t kHostResultBytes = 256;
constexpr int kSmemTable = 1024;             // phase-table entries a sweep may keep in shared memory

struct SweepGeom {
  int n;      // qubits
  int j0;     // first group qubit
  int t;      // group qubits in the tile (j0 + t <= n)
  int c;      // low index bits carried in the tile (c <= j0), 0 for the first group
  int64_t tiles;  // number of tiles = 2^(n - t - c)
};

enum SweepKind : int { SWEEP_GENERIC = 0, SWEEP_LEAN_MIX = 1, SWEEP_LEAN_OPS = 2 };

// One graph of a grouped sweep (batched gradients): the lean kernel runs the same sweep for
// many graphs of one size, blocks [g * gbpg, (g + 1) * gbpg) on graph g, whose state, lambda
// and cost vector start zoff elements into the arenas and whose tables and angles are its own.
struct GroupSlot {
  int64_t zoff;
  const void* phase_table;  // p * span entries, or nullptr
  int64_t cmin, span;
  const void* d_table;      // fixed point: p * 14 * 14 mixer-diagonal entries
  const double* trig;       // [g2pi p | cos p | sin p]
  int lam_shift;            // fixed point: 2^lam_shift >= max |C|
};

struct SweepArgs {
  int kind;  // SweepKind: generic op program or one of the lean shapes
  void* psi;
  void* lam;
  const void* C;
  int cost_dtype;
  int needs_cost;  // stage the cost tile in shared memory
  SweepGeom g;
  int tile_bits;   // B of the kernel configuration
  // state formats: load 0 = internal, 1 = user (complex128 / complex64), 2 = create |+>;
  // store 0 = internal, 1 = user, -1 = none.  complex64 internal == user.
  int load_fmt, store_fmt;
  int load_lam, store_lam;
  int stage;          // lean two-buffer sweeps: psi of the block's next tile staged in shared memory
  long long init_fx;  // |+> amplitude in fixed point
  float init_f32;     // |+> amplitude in float32
  int fx_shift;       // fixed-point scale S (value = integer * 2^-S)
  const double* norm2_dev;             // optional: |psi|^2 of a user state (input scale)
  const unsigned long long* cmax_dev;  // optional: bits of max |C| (lambda scale)
  int nops;
  uint32_t ops[kMaxOps];
  // per layer angles, indexed by the op's layer field (dev_trig overrides them when the
  // angles live in device memory: [g2pi np | cos np | sin np])
  const double* dev_trig;
  int np;
  double g2pi[QAOA_MAX_P];  // gamma / (2 pi)
  double cosb[QAOA_MAX_P];
  double sinb[QAOA_MAX_P];
  // tables (workspace): integer-cost phases exp(-i gamma_l c) at [l * span + (c - cmin)];
  // fixed point also mixer diagonals [(l * 14 + t) * 14 + k] and turn tables [3 * 1024]
  const void* phase_table;
  int64_t cmin;
  int64_t span;
  int smem_table_layer;  // layer whose table the kernel copies to shared memory (-1: none)
  const void* d_table;
  const void* turn_table;
  // reductions: accumulator r is written to partials[red_slot[r] * grid + block],
  // red_slot = out * kMaxContrib + contrib
  int nred;
  int red_slot[kMaxAcc];
  double* partials;
  int grid;
  double algo_bytes;  // HBM bytes this sweep must move (for timing reports)
  // grouped sweeps (lean kernels only): per-graph data, blocks per graph; nullptr = one graph
  const GroupSlot* gslot;
  int gbpg;
};

// A reduction plan: out[o] = scale[o] * sum over contributions k < ncontrib[o] and
// blocks b of partials[(o * kMaxContrib + k) * grid + b].
struct ReducePlan {
  int nout;
  int grid;
  int ncontrib[2 * QAOA_MAX_P + 2];
  double scale[2 * QAOA_MAX_P + 2];
};

struct TableArgs {
  int fx;        // fixed point tables (complex128) or float32 (complex64)
  int p;
  const double* dev_angles;  // device [gamma p | beta p], overrides gamma/beta when set
  int64_t cmin, span;  // integer-cost phase table (span 0 = none)
  double gamma[QAOA_MAX_P];
  double beta[QAOA_MAX_P];
  void* phase;   // p * span entries
  void* dtab;    // fixed point: p * 14 * 14 entries
  void* turn;    // fixed point: 3 * 1024 entries
};

// launchers (return a CUDA error code)
cudaError_t launch_sweep(int dtype, bool two, const SweepArgs& a, cudaStream_t s);
cudaError_t launch_reduce(const ReducePlan& r, const double* partials, double* out, cudaStream_t s);
// out[out_row[g] * nout + o] = sum over contributions k < ncontrib[o] and the blocks j < bpg of
// graph g of partials[(o * kMaxContrib + k) * grid + g * bpg + j], for graphs g < ngraphs
cudaError_t launch_group_reduce(const ReducePlan& r, int ngraphs, int bpg, const int* out_row,
                                const double* partials, double* out, cudaStream_t s);
cudaError_t launch_tables(const TableArgs& t, cudaStream_t s);
cudaError_t launch_cost_bound(const void* C, int f64, int n, unsigned long long* out, cudaStream_t s);
cudaError_t launch_norm(const void* psi, int dtype, int n, double* partials, int* nblocks, cudaStream_t s);
cudaError_t launch_angle_prep(const double* ang, int p, double* trig, cudaStream_t s);
cudaError_t launch_adam(double* ang, const double* g, double* state, long long* step, int p, double lr, double b1,
                        double b2, double eps, double* history, long long row0, long long max_rows, cudaStream_t s);
size_t lbfgs_state_doubles(int p, int m);
cudaError_t launch_lbfgs(double* ang, const double* gout, double* st, int p, int m, double gtol, double c1,
                         double* history, long long row0, long long max_rows, cudaStream_t s);
cudaError_t launch_lbfgs_resume(double* ang, const double* st, int p, cudaStream_t s);
cudaError_t launch_lbfgs_finish(double* ang, const double* st, int p, double* info, cudaStream_t s);
cudaError_t launch_expect(int dtype, const void* psi, const void* C, int cost_dtype, int n, double* partials,
                          int grid, cudaStream_t s);
int sweep_tile_bits(int dtype, bool two);     // B of the kernel a sweep uses
// persistent grid size for a sweep (cost_bytes: 0, 4 or 8 bytes of cost tile per amplitude)
int sweep_grid(int dtype, bool two, int tile_bits, int cost_bytes, int64_t tiles);
int fx_shift_for(int tmax);                   // fixed-point scale for groups of <= tmax qubits

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

// general PUBO cost, one chunk of terms per launch (parameters stay below 32 KB)
constexpr int kPuboChunk = 2048;
struct PuboArgs {
  int n;
  int nterms;       // terms in this chunk
  int accumulate;   // add to C (later chunks) instead of overwriting it
  int cost_dtype;
  int integer;      // integer weights (q = w) or fixed point (q = w 2^fixed_shift)
  int fixed_shift;
  void* C;
  uint32_t mask[kPuboChunk];
  long long q[kPuboChunk];
};
cudaError_t launch_pubo(const PuboArgs& a, cudaStream_t s);

// sampling
struct SampleArgs {
  int n;
  uint64_t len;     // entries of the sampled vector (0: 2^n); the returned z are indices into it
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
size_t sample_ws_bytes_len(uint64_t len);  // workspace for a vector of len entries

// bookkeeping for benchmarks: call with begin = true before a launch and begin = false
// after it; `bytes` (algorithmic HBM bytes of the launch) is read on the second call
void note_launch(int kind, cudaStream_t s, bool begin, double bytes = 0.0);

// ---------------------------------------------------------------- batched gradients
//
// Many small graphs in one persistent launch: each CTA takes the next graph from a work
// counter (graphs sorted by n, largest first) and runs that graph's whole sweep plan
// (forward layers, lambda, adjoint pass) over its own state, synchronising only within
// the CTA; its reductions go straight to the graph's output row.

constexpr int kBatchMaxOps = 64;     // ops per sweep of a batched plan
constexpr int kBatchMaxSweeps = 32;  // sweeps per batched plan

struct BatchSweep {
  SweepGeom g;
  int load_fmt, store_fmt, load_lam, store_lam, needs_cost, nops;
  int two;        // the sweep carries lambda
  int lean_last;  // >= 0: last layout with group qubits, for the lean tile code (2^12 tiles); -1: generic
  uint32_t ops[kBatchMaxOps];  // accumulator field = output index
};

// sweep plan of one qubit count on one tile configuration
struct BatchPlan {
  int n;
  int fx_shift;
  long long init_fx;
  float init_f32;
  int nsweeps;
  BatchSweep sw[kBatchMaxSweeps];
};

struct BatchGraph {
  int n, m;
  int plan;        // index into the plans
  int out;         // output row (the caller's graph index)
  int lam_shift;   // fixed point: 2^lam_shift >= max |C|
  int cmin, span;  // integer cost range covered by the phase table (span 0: no table)
  int64_t state;   // element offset of psi and lambda in the state arenas
  int64_t cost;    // element offset of C in the cost arena
  int64_t table;   // entry offset of the p * span phase-table entries
  int64_t edge;    // index of the graph's first edge in the edge arrays
};

struct BatchArgs {
  int ngraphs;               // graphs in processing order
  int p;
  int dtype;
  const BatchGraph* graphs;
  const BatchPlan* plans;
  const int* edges;          // (u, v) pairs
  const double* ew;          // edge weights
  int cost_f64;              // float64 costs (float weights in the batch) instead of int32
  const int64_t* blk_off;    // cost kernel: first block of each graph (ngraphs + 1)
  const double* angles;      // [gamma p | beta p] per graph, processing order
  void* psi;                 // state arenas (internal format)
  void* lam;
  void* C;                   // cost arena (int32 or float64)
  void* phase;               // phase tables
  void* dtab;                // fixed point: p * 196 mixer diagonals per graph
  void* turn;                // fixed point: shared turn tables
  double* trig;              // [g2pi p | cos p | sin p] per graph
  double* out;               // (2p + 2) per graph, rows in the caller's order
};

constexpr int kBatchCostBits = 12;  // cost-kernel entries per block: 2^12

cudaError_t launch_batch_prep(const BatchArgs& b, int64_t cost_blocks, cudaStream_t s);
// tile: 0 = small tiles (2^10 amplitudes), 1 = large tiles (2^12)
cudaError_t launch_batch(const BatchArgs& b, int tile, int first, int count, int* queue, cudaStream_t s);
cudaError_t launch_batch_c128_large(const BatchArgs& b, int first, int count, int* queue, cudaStream_t s);
int batch_tile_bits(int tile);
int batch_register_bits(int dtype, int tile);  // RB of the batched tile configuration

// learned angle proposer (fused network inference, one CTA per graph)
struct ProposeArgs {
  int p;
  const int* n;              // per graph
  const int64_t* edge_off;   // ngraphs + 1
  const int* uv;             // (u, v) pairs
  const double* w;           // edge weights
  const float* params;       // packed network parameters
  double* angles;            // ngraphs x 2p
};
int64_t proposer_param_count(int p);
cudaError_t launch_propose(const ProposeArgs& a, int ngraphs, cudaStream_t s);

}  // namespace qaoa
