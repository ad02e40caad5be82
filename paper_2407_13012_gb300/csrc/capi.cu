// C ABI entry points: argument checks, sweep planning, workspace carving, launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <set>
#include <utility>
#include <vector>

#include "internal.h"

namespace qaoa {

// ------------------------------------------------------------ launch accounting

namespace {
std::atomic<int64_t> g_launches{0};
std::mutex g_timing_mu;
bool g_timing_on = false;
constexpr int kMaxTimed = 65536;
struct TimedLaunch {
  cudaEvent_t e0, e1;
  int kind;
  double bytes;
};
std::vector<TimedLaunch> g_timed;
std::vector<cudaEvent_t> g_event_pool;
int64_t g_dropped = 0;
cudaEvent_t g_pending_begin = nullptr;

cudaEvent_t pool_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

void note_launch(int kind, cudaStream_t s, bool begin, double bytes) {
  if (begin) g_launches.fetch_add(1, std::memory_order_relaxed);
  if (!g_timing_on) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) return;  // graph capture
  std::lock_guard<std::mutex> lk(g_timing_mu);
  if (begin) {
    if ((int)g_timed.size() >= kMaxTimed) {
      ++g_dropped;
      g_pending_begin = nullptr;
      return;
    }
    g_pending_begin = pool_event();
    cudaEventRecord(g_pending_begin, s);
  } else if (g_pending_begin != nullptr) {
    cudaEvent_t e1 = pool_event();
    cudaEventRecord(e1, s);
    g_timed.push_back({g_pending_begin, e1, kind, bytes});
    g_pending_begin = nullptr;
  }
}

// ------------------------------------------------------------ planning

struct Group {
  int j0, t, c;
};

// Cover the qubits with groups: the first holds bits [0, min(n, B)); the rest carry
// c low bits for coalescing and as many group qubits as the tile allows, using the
// fewest groups and then the most carried bits.
static std::vector<Group> plan_groups(int n, int B) {
  std::vector<Group> gs;
  const int t0 = std::min(n, B);
  gs.push_back({0, t0, 0});
  int rem = n - t0;
  if (rem <= 0) return gs;
  int best_c = 0, best_k = 1 << 30;
  for (int c = 0; c <= 3; ++c) {
    const int per = B - c;
    const int k = (rem + per - 1) / per;
    if (k < best_k || (k == best_k && c > best_c)) {
      best_k = k;
      best_c = c;
    }
  }
  int j = t0;
  for (int i = 0; i < best_k; ++i) {
    const int left = best_k - i;
    const int t = (n - j + left - 1) / left;  // balanced split
    gs.push_back({j, t, std::min(j, B - t)});  // carry as many low bits as fill the tile
    j += t;
  }
  return gs;
}

struct Sweep {
  int group;
  bool two = false;        // lambda buffer present (gradient backward part)
  bool init = false;       // create |+> instead of loading
  bool load_user = false;  // load psi in the caller's format
  bool store_psi = true, store_user = false, load_lam = false, store_lam = false;
  std::vector<uint32_t> ops;
  std::vector<int> red_slot;  // per accumulator
};

static int64_t tiles_of(const Group& g, int n) { return 1ll << (n - g.t - g.c); }

constexpr size_t kScalarBytes = 256;                     // norm^2 (double), max|C| bits (u64)
constexpr size_t kNormPartialBytes = 1024 * sizeof(double);
constexpr size_t kTrigBytes = 3 * QAOA_MAX_P * sizeof(double);  // per-layer terms of device angles

static size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }
static size_t partial_bytes(int nout) { return round256((size_t)nout * kMaxContrib * kGridCap * sizeof(double)); }
static size_t phase_table_bytes(int dtype, int p, int64_t span) {
  if (span <= 0 || span > QAOA_MAX_TABLE_SPAN || p <= 0) return 0;
  return round256((size_t)p * span * (dtype == QAOA_C128 ? 16 : 8));
}
static size_t fx_table_bytes(int dtype, int p) {
  if (dtype != QAOA_C128) return 0;
  return round256((size_t)p * 196 * 16) + round256(3072 * 16);
}
// workspace of the optimiser beyond the gradient's: Adam moments (4p), step counter,
// gradient output (2p + 2)
static size_t adam_extra_bytes(int p) {
  return round256((4 * p + 1) * sizeof(double)) + round256((2 * p + 2) * sizeof(double));
}
// L-BFGS state (history of QAOA_LBFGS_MAX_M pairs) and the gradient output
static size_t lbfgs_extra_bytes(int p) {
  return round256(lbfgs_state_doubles(p, QAOA_LBFGS_MAX_M) * sizeof(double)) + round256((2 * p + 2) * sizeof(double));
}
static size_t layer_ws_bytes(int dtype, int p, int64_t span, int nout) {
  return kScalarBytes + kNormPartialBytes + kTrigBytes + partial_bytes(nout) + phase_table_bytes(dtype, p, span) +
         fx_table_bytes(dtype, p);
}

struct Ctx {
  int n, dtype;
  const qaoa_cost_t* cost;
  cudaStream_t s;
  char* ws;
  size_t ws_bytes;
};

static int cuda_status(cudaError_t e) { return e == cudaSuccess ? QAOA_OK : QAOA_ERR_CUDA; }

// Whether a sweep runs in a lean kernel: full tiles with affine layout-0 addresses
// (t + c = B, c <= B - RB), groups of >= 3 qubits, the state loaded in the internal format
// (complex64: also the caller's, which is the same) or created as |+>.  A single mixer on
// internal formats is the plain shape; any other program runs as an op program (its cost
// tile by 16-byte copies, which need whole 16-byte chunks per row).
static int lean_kind(const Sweep& s, const Group& g, int tile_bits, int dtype, bool cost_f64) {
  const bool fx = dtype == QAOA_C128;
  const int rb = fx ? (s.two ? 3 : 4) : (s.two ? 4 : 5);
  if (g.t + g.c != tile_bits || g.c > tile_bits - rb || g.t < 3) return SWEEP_GENERIC;
  if (fx && s.load_user) return SWEEP_GENERIC;
  if ((int)s.red_slot.size() > kLeanAcc) return SWEEP_GENERIC;
  int mixers = 0;
  for (uint32_t op : s.ops) mixers += (op & 0xff) == OP_MIX;
  if (mixers > kLeanMix) return SWEEP_GENERIC;
  const uint32_t want_mix = s.two ? (F_PSI | F_LAM | F_XTERM) : F_PSI;
  const std::vector<uint32_t>& o = s.ops;
  const bool plain_formats = !s.init && !s.load_user && !s.store_user && s.store_psi &&
                             (!s.two || (s.load_lam && s.store_lam));
  if (plain_formats && o.size() == 1 && (o[0] & 0xff) == OP_MIX && ((o[0] & 0xff00) & ~(uint32_t)F_SIGN) == want_mix)
    return SWEEP_LEAN_MIX;
  bool reads_c = false, lam_live = s.two && s.load_lam;
  for (uint32_t op : o) {
    const uint32_t kind = op & 0xff;
    reads_c |= (kind == OP_PHASE || kind == OP_LAMBDA || kind == OP_RED_EXPECT || kind == OP_RED_CTERM);
    // the two-buffer lean kernel applies every mixer and phase to both buffers, which is
    // exact for an op on psi alone only while lambda is still zero
    if (s.two && (kind == OP_MIX || kind == OP_PHASE) && !(op & F_LAM) && lam_live) return SWEEP_GENERIC;
    if (kind == OP_LAMBDA) lam_live = true;
  }
  const bool chunky = g.j0 == 0 || (1 << g.c) >= (cost_f64 ? 2 : 4);
  if (reads_c && !chunky) return SWEEP_GENERIC;
  return SWEEP_LEAN_OPS;
}

// Run a list of sweeps with one shared grid, then reduce the partials into out[0..nout).
// Fixed-point (complex128) calls also get: the input scale from the norm of a loaded
// user state, the lambda scale from max |C| (gradient), and the mixer/turn tables.
static int run_sweeps(const Ctx& c, std::vector<Sweep>& sw, const std::vector<Group>& gs, int tile_bits, void* psi,
                      void* lam, const double* gamma, const double* beta, const double* ang_dev, int p, int nout,
                      const std::vector<int>& ncontrib, double* out) {
  const bool fx = c.dtype == QAOA_C128;
  bool any_two = false, any_user_load = false;
  int64_t max_tiles = 1;
  int tmax = 1;
  for (const Sweep& s : sw) {
    max_tiles = std::max(max_tiles, tiles_of(gs[s.group], c.n));
    any_two |= s.two;
    any_user_load |= s.load_user;
  }
  for (const Group& g : gs) tmax = std::max(tmax, g.t);
  const int cost_bytes = c.cost->C_dev == nullptr ? 0 : (c.cost->dtype == QAOA_COST_I32 ? 4 : 8);
  // one grid (the partials' stride) for all sweeps: sized for the single-buffer kernels;
  // two-buffer kernels with fewer resident blocks per SM run it in waves
  int grid = sweep_grid(c.dtype, false, tile_bits, cost_bytes, max_tiles);
  if (any_two) grid = std::max(grid, sweep_grid(c.dtype, true, tile_bits, cost_bytes, max_tiles));
  grid = std::min(grid, kGridCap);
  // workspace carving
  char* p_ws = c.ws;
  double* norm2 = (double*)p_ws;
  unsigned long long* cmax_bits = (unsigned long long*)(p_ws + 8);
  p_ws += kScalarBytes;
  double* norm_part = (double*)p_ws;
  p_ws += kNormPartialBytes;
  double* trig = (double*)p_ws;
  p_ws += kTrigBytes;
  double* partials = (double*)p_ws;
  p_ws += partial_bytes(nout);
  const bool int_cost = c.cost->dtype == QAOA_COST_I32;
  int64_t cmin = 0, span = 0;
  // a phase table over [cmin, cmax]: only for bounds inside int32 (the kernels index it in 32-bit
  // arithmetic; int32 costs outside such bounds take the direct phase)
  if (int_cost && c.cost->cmax >= c.cost->cmin && p > 0 && c.cost->cmax - c.cost->cmin + 1 <= QAOA_MAX_TABLE_SPAN &&
      c.cost->cmin >= INT32_MIN && c.cost->cmax <= INT32_MAX) {
    span = c.cost->cmax - c.cost->cmin + 1;
    cmin = c.cost->cmin;
  }
  void* phase_table = span > 0 ? p_ws : nullptr;
  p_ws += phase_table_bytes(c.dtype, p, span);
  void* d_table = fx ? p_ws : nullptr;
  void* turn_table = fx ? p_ws + round256((size_t)p * 196 * 16) : nullptr;
  p_ws += fx_table_bytes(c.dtype, p);
  if ((size_t)(p_ws - c.ws) > c.ws_bytes) return QAOA_ERR_WORKSPACE;

  if (p > 0 && (span > 0 || fx)) {
    TableArgs t;
    std::memset(&t, 0, sizeof(t));
    t.fx = fx;
    t.p = p;
    t.cmin = cmin;
    t.span = span;
    if (ang_dev != nullptr) {
      t.dev_angles = ang_dev;
    } else {
      for (int l = 0; l < p; ++l) {
        t.gamma[l] = gamma[l];
        t.beta[l] = beta[l];
      }
    }
    t.phase = phase_table;
    t.dtab = d_table;
    t.turn = turn_table;
    int rc = cuda_status(launch_tables(t, c.s));
    if (rc) return rc;
  }
  if (fx && any_user_load) {  // input scale from |psi|^2 of the caller's state
    int nb = 0;
    int rc = cuda_status(launch_norm(psi, c.dtype, c.n, norm_part, &nb, c.s));
    if (rc) return rc;
    ReducePlan r;
    std::memset(&r, 0, sizeof(r));
    r.nout = 1;
    r.grid = nb;
    r.ncontrib[0] = 1;
    r.scale[0] = 1.0;
    rc = cuda_status(launch_reduce(r, norm_part, norm2, c.s));
    if (rc) return rc;
  }
  if (fx && any_two) {  // lambda scale from max |C|
    int rc = cuda_status(launch_cost_bound(c.cost->C_dev, c.cost->dtype == QAOA_COST_F64, c.n, cmax_bits, c.s));
    if (rc) return rc;
  }

  if (ang_dev != nullptr && p > 0) {
    int rc = cuda_status(launch_angle_prep(ang_dev, p, trig, c.s));
    if (rc) return rc;
  }
  const double amp0 = std::pow(2.0, -0.5 * c.n);
  const int S = fx_shift_for(tmax);
  for (const Sweep& s : sw) {
    SweepArgs a;
    std::memset(&a, 0, sizeof(a));
    a.psi = psi;
    a.lam = s.two ? lam : nullptr;
    a.C = c.cost->C_dev;
    a.cost_dtype = c.cost->dtype;
    const Group& g = gs[s.group];
    a.g = {c.n, g.j0, g.t, g.c, tiles_of(g, c.n)};
    a.tile_bits = tile_bits;
    a.load_fmt = s.init ? 2 : (s.load_user ? 1 : 0);
    a.store_fmt = !s.store_psi ? -1 : (s.store_user ? 1 : 0);
    a.load_lam = s.load_lam;
    a.store_lam = s.store_lam;
    a.fx_shift = S;
    a.init_fx = (long long)std::llrint(std::ldexp(amp0, S));
    a.init_f32 = (float)amp0;
    a.norm2_dev = (fx && any_user_load) ? norm2 : nullptr;
    a.cmax_dev = (fx && any_two) ? cmax_bits : nullptr;
    if ((int)s.ops.size() > kMaxOps) return QAOA_ERR_UNSUPPORTED;
    a.nops = (int)s.ops.size();
    bool reads_c = false;
    for (size_t k = 0; k < s.ops.size(); ++k) {
      a.ops[k] = s.ops[k];
      const uint32_t kind = s.ops[k] & 0xff;
      reads_c |= (kind == OP_PHASE || kind == OP_LAMBDA || kind == OP_RED_EXPECT || kind == OP_RED_CTERM);
    }
    a.needs_cost = reads_c;
    a.np = p;
    a.dev_trig = ang_dev != nullptr ? trig : nullptr;
    if (ang_dev == nullptr) {
      for (int l = 0; l < p; ++l) {
        a.g2pi[l] = gamma[l] / (2.0 * 3.14159265358979323846);
        a.cosb[l] = std::cos(beta[l]);
        a.sinb[l] = std::sin(beta[l]);
      }
    }
    a.phase_table = phase_table;
    a.cmin = cmin;
    a.span = span;
    a.smem_table_layer = -1;
    if (phase_table != nullptr && span <= kSmemTable) {
      for (uint32_t op : s.ops)
        if ((op & 0xff) == OP_PHASE) {
          a.smem_table_layer = (int)((op >> 16) & 0xff);
          break;
        }
    }
    a.d_table = d_table;
    a.turn_table = turn_table;
    a.nred = (int)s.red_slot.size();
    if (a.nred > kMaxAcc) return QAOA_ERR_UNSUPPORTED;
    for (int r = 0; r < a.nred; ++r) a.red_slot[r] = s.red_slot[r];
    a.partials = partials;
    a.grid = grid;
    {
      const double S_b = c.dtype == QAOA_C128 ? 16.0 : 8.0;
      const double cb = c.cost->dtype == QAOA_COST_I32 ? 4.0 : 8.0;
      const double per = S_b * ((s.init ? 0 : 1) + (s.store_psi ? 1 : 0) + (s.two && s.load_lam ? 1 : 0) +
                                (s.two && s.store_lam ? 1 : 0)) +
                         (reads_c ? cb : 0.0);
      a.algo_bytes = per * (double)(1ull << c.n);
    }
    a.kind = lean_kind(s, g, tile_bits, c.dtype, c.cost->dtype == QAOA_COST_F64);
    int rc = cuda_status(launch_sweep(c.dtype, s.two, a, c.s));
    if (rc) return rc;
  }
  if (nout > 0) {
    ReducePlan r;
    std::memset(&r, 0, sizeof(r));
    r.nout = nout;
    r.grid = grid;
    for (int o = 0; o < nout; ++o) {
      r.ncontrib[o] = ncontrib[o];
      r.scale[o] = 1.0;
    }
    int rc = cuda_status(launch_reduce(r, partials, out, c.s));
    if (rc) return rc;
  }
  return QAOA_OK;
}

// Sweep schedule of p forward layers.  Layer l visits the groups in increasing
// order for even l and decreasing order for odd l, so the last group of one layer
// is the first of the next and the two share a sweep (phase applied in between).
static void plan_forward(int k, int p, bool init, std::vector<Sweep>& sw) {
  for (int l = 0; l < p; ++l) {
    for (int idx = 0; idx < k; ++idx) {
      const int gi = (l % 2 == 0) ? idx : k - 1 - idx;
      if (idx == 0 && l > 0) {
        sw.back().ops.push_back(make_op(OP_PHASE, F_PSI, l));
        sw.back().ops.push_back(make_op(OP_MIX, F_PSI, l));
        continue;
      }
      Sweep s;
      s.group = gi;
      if (l == 0 && idx == 0) {
        s.init = init;
        s.load_user = !init;
        s.ops.push_back(make_op(OP_PHASE, F_PSI, 0));
      }
      s.ops.push_back(make_op(OP_MIX, F_PSI, l));
      sw.push_back(s);
    }
  }
}

// Gradient schedule (Sec. IV-D): the p forward layers from |+>; in the last forward sweep
// lambda = C psi and <C>; then the adjoint pass, layer by layer in reverse, visiting the
// groups so that consecutive layers share a sweep.  new_acc(sweep, out0, outs) returns the
// accumulator for `outs` consecutive outputs from out0 (0 = E, 1 = norm, 2 + l = dE/dgamma_l,
// 2 + p + l = dE/dbeta_l).  The last sweep stores psi (uncomputed) and drops lambda.
template <class F>
static void plan_gradient(int k, int p, std::vector<Sweep>& sw, F new_acc) {
  plan_forward(k, p, true, sw);
  Sweep* cur = &sw.back();
  cur->two = true;
  cur->store_lam = true;
  cur->ops.push_back(make_op(OP_LAMBDA, 0, 0));
  cur->ops.push_back(make_op(OP_RED_EXPECT, F_PSI, 0, new_acc(*cur, 0, 2)));
  for (int l = p - 1; l >= 0; --l) {
    const int first = cur->group;
    for (int idx = 0; idx < k; ++idx) {
      const int gi = (first == 0) ? idx : k - 1 - idx;
      if (idx > 0) {
        Sweep s;
        s.group = gi;
        s.two = true;
        s.load_lam = true;
        s.store_lam = true;
        sw.push_back(s);
        cur = &sw.back();
      }
      cur->ops.push_back(make_op(OP_MIX, F_PSI | F_LAM | F_SIGN | F_XTERM, l, new_acc(*cur, 2 + p + l, 1)));
    }
    cur->ops.push_back(make_op(OP_RED_CTERM, F_PSI | F_LAM, l, new_acc(*cur, 2 + l, 1)));
    cur->ops.push_back(make_op(OP_PHASE, F_PSI | F_LAM | F_SIGN, l));
  }
  cur->store_lam = false;
}

static bool valid_dtype(int d) { return d == QAOA_C128 || d == QAOA_C64; }
static bool valid_cost(const qaoa_cost_t* c) {
  return c != nullptr && c->C_dev != nullptr && (c->dtype == QAOA_COST_I32 || c->dtype == QAOA_COST_F64);
}
static bool angles_ok(const double* g, const double* b, int p) {
  if (p < 0 || p > QAOA_MAX_P) return false;
  if (p > 0 && (g == nullptr || b == nullptr)) return false;
  for (int l = 0; l < p; ++l)
    if (!std::isfinite(g[l]) || !std::isfinite(b[l])) return false;
  return true;
}

}  // namespace qaoa

using namespace qaoa;

// Run `steps` iterations of a fixed launch sequence on the caller's stream: the first one
// directly (it also settles every per-kernel setting), the rest by replaying a CUDA graph of
// one iteration, with no host round trip inside.  When done_flag is set, the host reads that
// device double every `poll` replays and stops once it is non-zero.  The legacy default
// stream cannot be captured: then the graph runs on a private blocking stream, which is
// ordered after (and before) work on the legacy stream.  Synchronises before returning.
template <class F>
static int replay_steps(cudaStream_t s, int64_t steps, F&& iteration, const double* done_flag, int poll) {
  if (steps <= 0) return QAOA_OK;
  int rc = iteration(s);
  if (rc) return rc;
  if (steps == 1) return cuda_status(cudaStreamSynchronize(s));
  cudaStream_t cur = s;
  bool own = false;
  if (s == nullptr) {
    if (cudaStreamCreate(&cur) != cudaSuccess) return QAOA_ERR_CUDA;
    own = true;
  }
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int out = QAOA_OK;
  if (cudaStreamBeginCapture(cur, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    out = QAOA_ERR_CUDA;
  } else {
    const int rc_cap = iteration(cur);
    const cudaError_t ec = cudaStreamEndCapture(cur, &graph);
    if (rc_cap != QAOA_OK || ec != cudaSuccess) out = rc_cap != QAOA_OK ? rc_cap : QAOA_ERR_CUDA;
    else if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) out = QAOA_ERR_CUDA;
  }
  int64_t k = 1;
  while (out == QAOA_OK && k < steps) {
    const int64_t chunk = done_flag ? std::min<int64_t>(poll, steps - k) : steps - k;
    for (int64_t j = 0; j < chunk && out == QAOA_OK; ++j)
      if (cudaGraphLaunch(exec, cur) != cudaSuccess) out = QAOA_ERR_CUDA;
    k += chunk;
    if (done_flag && out == QAOA_OK && k < steps) {
      double flag = 0.0;
      if (cudaMemcpyAsync(&flag, done_flag, sizeof(double), cudaMemcpyDeviceToHost, cur) != cudaSuccess ||
          cudaStreamSynchronize(cur) != cudaSuccess)
        out = QAOA_ERR_CUDA;
      else if (flag != 0.0)
        break;
    }
  }
  if (cudaStreamSynchronize(cur) != cudaSuccess && out == QAOA_OK) out = QAOA_ERR_CUDA;
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (own) cudaStreamDestroy(cur);
  return out;
}

extern "C" {

int qaoa_version(void) { return 100; }

const char* qaoa_strerror(int status) {
  switch (status) {
    case QAOA_OK: return "ok";
    case QAOA_ERR_INVALID_ARG: return "invalid argument";
    case QAOA_ERR_UNSUPPORTED: return "unsupported size or option";
    case QAOA_ERR_CUDA: return "CUDA error";
    case QAOA_ERR_TIMEOUT: return "device-side wait timed out";
    case QAOA_ERR_WORKSPACE: return "workspace too small";
    default: return "unknown status";
  }
}

int qaoa_graph_check(const qaoa_graph_t* g, int64_t* cmin, int64_t* cmax) {
  if (g == nullptr || g->n < 1 || g->n > QAOA_MAX_N || g->m < 0) return QAOA_ERR_INVALID_ARG;
  if (g->m > 0 && g->uv == nullptr) return QAOA_ERR_INVALID_ARG;
  if (g->weight_kind != QAOA_WEIGHT_INT && g->weight_kind != QAOA_WEIGHT_F64) return QAOA_ERR_INVALID_ARG;
  if (g->m > (int64_t)g->n * (g->n - 1) / 2) return QAOA_ERR_INVALID_ARG;
  static_assert(QAOA_MAX_N <= 32, "adjacency rows are 32-bit masks");
  uint32_t adj[QAOA_MAX_N] = {};  // edges seen so far, one bit per neighbour
  double sum_abs = 0.0;
  int64_t neg = 0, pos = 0;
  for (int64_t e = 0; e < g->m; ++e) {
    const int u = g->uv[2 * e], v = g->uv[2 * e + 1];
    if (u < 0 || v < 0 || u >= g->n || v >= g->n || u == v) return QAOA_ERR_INVALID_ARG;
    if (adj[u] & (1u << v)) return QAOA_ERR_INVALID_ARG;  // a repeated edge (either orientation)
    adj[u] |= 1u << v;
    adj[v] |= 1u << u;
    const double w = g->w ? g->w[e] : 1.0;
    if (!std::isfinite(w)) return QAOA_ERR_INVALID_ARG;
    sum_abs += std::fabs(w);
    if (g->weight_kind == QAOA_WEIGHT_INT) {
      if (w != std::floor(w) || std::fabs(w) >= 2147483648.0) return QAOA_ERR_INVALID_ARG;
      if (w < 0) neg += (int64_t)w; else pos += (int64_t)w;
    }
  }
  if (g->weight_kind == QAOA_WEIGHT_INT && sum_abs >= 2147483648.0) return QAOA_ERR_INVALID_ARG;
  if (g->weight_kind == QAOA_WEIGHT_F64 && !(sum_abs < 1e300)) return QAOA_ERR_INVALID_ARG;
  if (cmin) *cmin = g->weight_kind == QAOA_WEIGHT_INT ? neg : 1;
  if (cmax) *cmax = g->weight_kind == QAOA_WEIGHT_INT ? pos : 0;
  return QAOA_OK;
}

int qaoa_workspace_size(int n, int dtype, int op, int p, int64_t shots, int64_t cost_span, size_t* bytes) {
  if (bytes == nullptr || n < 1 || n > QAOA_MAX_N || !valid_dtype(dtype)) return QAOA_ERR_INVALID_ARG;
  if (p < 0 || p > QAOA_MAX_P || shots < 0 || cost_span < 0) return QAOA_ERR_INVALID_ARG;
  size_t b = 0;
  switch (op) {
    case QAOA_OP_COST: b = 0; break;
    case QAOA_OP_LAYERS: b = layer_ws_bytes(dtype, p, cost_span, 2); break;
    case QAOA_OP_EXPECTATION: b = kExpectPartialBytes + kHostResultBytes; break;
    case QAOA_OP_SAMPLE: b = round256(sample_ws_bytes(n, dtype)); break;
    case QAOA_OP_GRADIENT: b = layer_ws_bytes(dtype, p, cost_span, 2 * p + 2); break;
    case QAOA_OP_OPTIMIZE: b = layer_ws_bytes(dtype, p, cost_span, 2 * p + 2) + adam_extra_bytes(p); break;
    case QAOA_OP_LBFGS: b = layer_ws_bytes(dtype, p, cost_span, 2 * p + 2) + lbfgs_extra_bytes(p); break;
    default: return QAOA_ERR_INVALID_ARG;
  }
  *bytes = b;
  return QAOA_OK;
}

int qaoa_cost_vector(const qaoa_graph_t* g, void* C_dev, int cost_dtype, qaoa_cost_t* desc, void* stream) {
  int64_t cmin = 0, cmax = 0;
  int rc = qaoa_graph_check(g, &cmin, &cmax);
  if (rc) return rc;
  if (C_dev == nullptr || (cost_dtype != QAOA_COST_I32 && cost_dtype != QAOA_COST_F64)) return QAOA_ERR_INVALID_ARG;
  if (cost_dtype == QAOA_COST_I32 && g->weight_kind != QAOA_WEIGHT_INT) return QAOA_ERR_INVALID_ARG;
  CostArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n = g->n;
  a.lo_bits = std::min(g->n, 12);
  a.cost_dtype = cost_dtype;
  a.integer = g->weight_kind == QAOA_WEIGHT_INT;
  a.C = C_dev;
  double sum_abs = 0.0;
  for (int64_t e = 0; e < g->m; ++e) sum_abs += std::fabs(g->w ? g->w[e] : 1.0);
  if (!a.integer) {
    // fixed point: every partial sum is bounded by sum|w|, keep it below 2^62
    int e2 = 0;
    std::frexp(sum_abs > 0.0 ? sum_abs : 1.0, &e2);  // sum_abs < 2^e2, so the scale follows the weights
    a.fixed_shift = 62 - e2;
  }
  for (int64_t e = 0; e < g->m; ++e) {
    const int u = g->uv[2 * e], v = g->uv[2 * e + 1];
    const double w = g->w ? g->w[e] : 1.0;
    const int64_t q = a.integer ? (int64_t)w : (int64_t)std::llrint(std::ldexp(w, a.fixed_shift));
    a.wi[u][v] = q;
    a.wi[v][u] = q;
  }
  rc = cuda_status(launch_cost(a, (cudaStream_t)stream));
  if (rc) return rc;
  if (desc) {
    desc->C_dev = C_dev;
    desc->dtype = cost_dtype;
    desc->cmin = a.integer ? cmin : 1;
    desc->cmax = a.integer ? cmax : 0;
  }
  return QAOA_OK;
}

int qaoa_cost_vector_pubo(int n, int64_t nterms, const uint32_t* masks, const double* w, int weight_kind,
                          void* C_dev, int cost_dtype, qaoa_cost_t* desc, void* stream) {
  if (n < 1 || n > QAOA_MAX_N || nterms < 0 || nterms > QAOA_MAX_PUBO_TERMS || C_dev == nullptr)
    return QAOA_ERR_INVALID_ARG;
  if (nterms > 0 && (masks == nullptr || w == nullptr)) return QAOA_ERR_INVALID_ARG;
  if (weight_kind != QAOA_WEIGHT_INT && weight_kind != QAOA_WEIGHT_F64) return QAOA_ERR_INVALID_ARG;
  if (cost_dtype != QAOA_COST_I32 && cost_dtype != QAOA_COST_F64) return QAOA_ERR_INVALID_ARG;
  if (cost_dtype == QAOA_COST_I32 && weight_kind != QAOA_WEIGHT_INT) return QAOA_ERR_INVALID_ARG;
  const bool integer = weight_kind == QAOA_WEIGHT_INT;
  double sum_abs = 0.0;
  int64_t neg = 0, pos = 0;
  for (int64_t t = 0; t < nterms; ++t) {
    if (n < 32 && (masks[t] >> n) != 0) return QAOA_ERR_INVALID_ARG;  // a variable outside [0, n)
    if (!std::isfinite(w[t])) return QAOA_ERR_INVALID_ARG;
    if (integer && (w[t] != std::floor(w[t]) || std::fabs(w[t]) >= 2147483648.0)) return QAOA_ERR_INVALID_ARG;
    sum_abs += std::fabs(w[t]);
    if (integer) (w[t] < 0 ? neg : pos) += (int64_t)w[t];
  }
  if (integer && sum_abs >= 2147483648.0) return QAOA_ERR_INVALID_ARG;
  if (!integer && !(sum_abs < 1e300)) return QAOA_ERR_INVALID_ARG;
  int fixed_shift = 0;
  if (!integer) {
    int e2 = 0;
    std::frexp(sum_abs > 0.0 ? sum_abs : 1.0, &e2);  // sum_abs < 2^e2: every partial sum stays below 2^62 + terms / 2
    fixed_shift = 62 - e2;
  }
  PuboArgs* a = new PuboArgs;
  int64_t t = 0;
  int rc = QAOA_OK;
  do {
    std::memset(a, 0, sizeof(PuboArgs));
    a->n = n;
    a->accumulate = t > 0;
    a->cost_dtype = cost_dtype;
    a->integer = integer;
    a->fixed_shift = fixed_shift;
    a->C = C_dev;
    a->nterms = (int)std::min<int64_t>(kPuboChunk, nterms - t);
    for (int k = 0; k < a->nterms; ++k) {
      a->mask[k] = masks[t + k];
      a->q[k] = integer ? (long long)w[t + k] : (long long)std::llrint(std::ldexp(w[t + k], fixed_shift));
    }
    rc = cuda_status(launch_pubo(*a, (cudaStream_t)stream));
    t += a->nterms;
  } while (rc == QAOA_OK && t < nterms);
  delete a;
  if (rc) return rc;
  if (desc) {
    desc->C_dev = C_dev;
    desc->dtype = cost_dtype;
    desc->cmin = integer ? neg : 1;
    desc->cmax = integer ? pos : 0;
  }
  return QAOA_OK;
}

int qaoa_apply_layers(int n, int dtype, void* psi_dev, const qaoa_cost_t* cost, const double* gamma,
                      const double* beta, int p, int init, double* expect_dev, void* ws_dev, size_t ws_bytes,
                      void* stream) {
  if (n < 1 || n > QAOA_MAX_N || !valid_dtype(dtype) || psi_dev == nullptr) return QAOA_ERR_INVALID_ARG;
  if (!angles_ok(gamma, beta, p) || (init != 0 && init != 1)) return QAOA_ERR_INVALID_ARG;
  if ((p > 0 || expect_dev) && !valid_cost(cost)) return QAOA_ERR_INVALID_ARG;
  const int64_t span = (cost && cost->dtype == QAOA_COST_I32 && cost->cmax >= cost->cmin)
                           ? cost->cmax - cost->cmin + 1 : 0;
  size_t need = 0;
  qaoa_workspace_size(n, dtype, QAOA_OP_LAYERS, p, 0, span, &need);
  if (need > 0 && (ws_dev == nullptr || ws_bytes < need)) return QAOA_ERR_WORKSPACE;
  const int B = sweep_tile_bits(dtype, false);
  const std::vector<Group> gs = plan_groups(n, B);
  std::vector<Sweep> sw;
  plan_forward((int)gs.size(), p, init != 0, sw);
  if (p == 0) {
    if (!init && !expect_dev) return QAOA_OK;
    Sweep s;
    s.group = 0;
    s.init = init != 0;
    s.load_user = !init;
    s.store_psi = init != 0;
    sw.push_back(s);
  }
  sw.back().store_user = true;
  int nout = 0;
  std::vector<int> ncontrib;
  if (expect_dev) {
    sw.back().ops.push_back(make_op(OP_RED_EXPECT, F_PSI, 0, (uint32_t)sw.back().red_slot.size()));
    sw.back().red_slot.push_back(0 * kMaxContrib + 0);
    sw.back().red_slot.push_back(1 * kMaxContrib + 0);
    nout = 2;
    ncontrib = {1, 1};
  }
  qaoa_cost_t dummy{nullptr, QAOA_COST_F64, 1, 0};
  Ctx c{n, dtype, cost ? cost : &dummy, (cudaStream_t)stream, (char*)ws_dev, ws_bytes};
  return run_sweeps(c, sw, gs, B, psi_dev, nullptr, gamma, beta, nullptr, p, nout, ncontrib, expect_dev);
}

int qaoa_expectation(int n, int dtype, const void* psi_dev, const qaoa_cost_t* cost, double* out_dev,
                     void* ws_dev, size_t ws_bytes, void* stream) {
  if (n < 1 || n > QAOA_MAX_N || !valid_dtype(dtype) || psi_dev == nullptr || out_dev == nullptr ||
      !valid_cost(cost))
    return QAOA_ERR_INVALID_ARG;
  // the last kHostResultBytes of the reported size are for qaoa_expectation_host's result
  if (ws_dev == nullptr || ws_bytes < kExpectPartialBytes) return QAOA_ERR_WORKSPACE;
  int grid = 0;
  {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t need = ((1ll << n) + 255) / 256;
    grid = (int)std::min<int64_t>(std::min<int64_t>(need, (int64_t)sms * 8), kGridCap);
  }
  double* partials = (double*)ws_dev;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = cuda_status(launch_expect(dtype, psi_dev, cost->C_dev, cost->dtype, n, partials, grid, s));
  if (rc) return rc;
  ReducePlan r;
  std::memset(&r, 0, sizeof(r));
  r.nout = 2;
  r.grid = grid;
  r.ncontrib[0] = r.ncontrib[1] = 1;
  r.scale[0] = r.scale[1] = 1.0;
  return cuda_status(launch_reduce(r, partials, out_dev, s));
}

int qaoa_expectation_host(int n, int dtype, const void* psi_dev, const qaoa_cost_t* cost, double* out_host,
                          void* ws_dev, size_t ws_bytes, void* stream) {
  if (out_host == nullptr) return QAOA_ERR_INVALID_ARG;
  size_t need = 0;
  if (qaoa_workspace_size(n, dtype, QAOA_OP_EXPECTATION, 0, 0, 0, &need)) return QAOA_ERR_INVALID_ARG;
  if (ws_dev == nullptr || ws_bytes < need) return QAOA_ERR_WORKSPACE;
  double* out_dev = (double*)((char*)ws_dev + kExpectPartialBytes);
  int rc = qaoa_expectation(n, dtype, psi_dev, cost, out_dev, ws_dev, kExpectPartialBytes, stream);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(out_host, out_dev, 2 * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return QAOA_ERR_CUDA;
  return cuda_status(cudaStreamSynchronize(s));
}

int qaoa_sample(int n, int dtype, const void* psi_dev, const qaoa_cost_t* cost, int64_t shots, uint64_t seed,
                uint64_t* z_dev, double* cost_dev, void* ws_dev, size_t ws_bytes, void* stream) {
  if (n < 1 || n > QAOA_MAX_N || !valid_dtype(dtype) || psi_dev == nullptr || !valid_cost(cost) || shots < 0)
    return QAOA_ERR_INVALID_ARG;
  if (shots > 0 && (z_dev == nullptr || cost_dev == nullptr)) return QAOA_ERR_INVALID_ARG;
  size_t need = 0;
  qaoa_workspace_size(n, dtype, QAOA_OP_SAMPLE, 0, shots, 0, &need);
  if (ws_dev == nullptr || ws_bytes < need) return QAOA_ERR_WORKSPACE;
  SampleArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n = n;
  a.dtype = dtype;
  a.psi = psi_dev;
  a.C = cost->C_dev;
  a.cost_dtype = cost->dtype;
  a.shots = shots;
  a.seed = seed;
  a.z = z_dev;
  a.cost = cost_dev;
  a.leaf = (double*)ws_dev;
  return cuda_status(launch_sample(a, (cudaStream_t)stream));
}

int qaoa_sample_host(int n, int dtype, const void* psi_dev, const qaoa_cost_t* cost, int64_t shots, uint64_t seed,
                     uint64_t* z_dev, double* cost_dev, uint64_t* z_host, double* cost_host, void* ws_dev,
                     size_t ws_bytes, void* stream) {
  if (shots > 0 && (z_host == nullptr || cost_host == nullptr)) return QAOA_ERR_INVALID_ARG;
  int rc = qaoa_sample(n, dtype, psi_dev, cost, shots, seed, z_dev, cost_dev, ws_dev, ws_bytes, stream);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (shots > 0) {
    if (cudaMemcpyAsync(z_host, z_dev, shots * sizeof(uint64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return QAOA_ERR_CUDA;
    if (cudaMemcpyAsync(cost_host, cost_dev, shots * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return QAOA_ERR_CUDA;
  }
  return cuda_status(cudaStreamSynchronize(s));
}

}  // extern "C"

// The adjoint gradient with angles either on the host (gamma, beta) or on the device
// (ang_dev = [gamma p | beta p]).
static int gradient_impl(int n, int dtype, void* psi_dev, void* lambda_dev, const qaoa_cost_t* cost,
                         const double* gamma, const double* beta, const double* ang_dev, int p, double* out_dev,
                         void* ws_dev, size_t ws_bytes, void* stream) {
  if (n < 1 || n > QAOA_MAX_N || !valid_dtype(dtype) || psi_dev == nullptr || lambda_dev == nullptr ||
      out_dev == nullptr || !valid_cost(cost) || p < 1 || p > QAOA_MAX_P)
    return QAOA_ERR_INVALID_ARG;
  if (ang_dev == nullptr && !angles_ok(gamma, beta, p)) return QAOA_ERR_INVALID_ARG;
  if (psi_dev == lambda_dev) return QAOA_ERR_INVALID_ARG;
  const int64_t span = (cost->dtype == QAOA_COST_I32 && cost->cmax >= cost->cmin) ? cost->cmax - cost->cmin + 1 : 0;
  size_t need = 0;
  qaoa_workspace_size(n, dtype, QAOA_OP_GRADIENT, p, 0, span, &need);
  if (ws_dev == nullptr || ws_bytes < need) return QAOA_ERR_WORKSPACE;
  const int B = sweep_tile_bits(dtype, true);
  const std::vector<Group> gs = plan_groups(n, B);
  const int k = (int)gs.size();
  std::vector<Sweep> sw;
  // outputs: 0 = E, 1 = norm, 2 + l = dE/dgamma_l, 2 + p + l = dE/dbeta_l
  const int nout = 2 * p + 2;
  std::vector<int> ncontrib(nout, 0);
  plan_gradient(k, p, sw, [&](Sweep& s, int out0, int outs) {
    const uint32_t acc = (uint32_t)s.red_slot.size();
    for (int i = 0; i < outs; ++i) {
      s.red_slot.push_back((out0 + i) * kMaxContrib + ncontrib[out0 + i]);
      ncontrib[out0 + i]++;
    }
    return acc;
  });
  sw.back().store_user = true;
  for (int o = 0; o < nout; ++o)
    if (ncontrib[o] > kMaxContrib) return QAOA_ERR_UNSUPPORTED;
  for (const Sweep& s : sw)
    if ((int)s.red_slot.size() > 255) return QAOA_ERR_UNSUPPORTED;
  Ctx c{n, dtype, cost, (cudaStream_t)stream, (char*)ws_dev, ws_bytes};
  return run_sweeps(c, sw, gs, B, psi_dev, lambda_dev, gamma, beta, ang_dev, p, nout, ncontrib, out_dev);
}

extern "C" {

int qaoa_gradient(int n, int dtype, void* psi_dev, void* lambda_dev, const qaoa_cost_t* cost, const double* gamma,
                  const double* beta, int p, double* out_dev, void* ws_dev, size_t ws_bytes, void* stream) {
  return gradient_impl(n, dtype, psi_dev, lambda_dev, cost, gamma, beta, nullptr, p, out_dev, ws_dev, ws_bytes,
                       stream);
}

int qaoa_gradient_dev(int n, int dtype, void* psi_dev, void* lambda_dev, const qaoa_cost_t* cost,
                      const double* angles_dev, int p, double* out_dev, void* ws_dev, size_t ws_bytes, void* stream) {
  if (angles_dev == nullptr) return QAOA_ERR_INVALID_ARG;
  return gradient_impl(n, dtype, psi_dev, lambda_dev, cost, nullptr, nullptr, angles_dev, p, out_dev, ws_dev,
                       ws_bytes, stream);
}


int qaoa_optimizer_state_size(int kind, int p, size_t* bytes) {
  if (bytes == nullptr || p < 1 || p > QAOA_MAX_P) return QAOA_ERR_INVALID_ARG;
  if (kind == QAOA_OPTIMIZER_ADAM) *bytes = (4 * (size_t)p + 1) * sizeof(double);
  else if (kind == QAOA_OPTIMIZER_LBFGS) *bytes = lbfgs_state_doubles(p, QAOA_LBFGS_MAX_M) * sizeof(double);
  else return QAOA_ERR_INVALID_ARG;
  return QAOA_OK;
}

int qaoa_optimize_adam(int n, int dtype, void* psi_dev, void* lambda_dev, const qaoa_cost_t* cost,
                       double* angles_dev, int p, int64_t steps, double lr, double beta1, double beta2, double eps,
                       double* history_dev, double* state_dev, int resume, void* ws_dev, size_t ws_bytes,
                       void* stream) {
  if (angles_dev == nullptr || steps < 0 || !(lr > 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) ||
      !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0) || p < 1 || p > QAOA_MAX_P || !valid_cost(cost) ||
      (resume != 0 && resume != 1) || (resume && state_dev == nullptr))
    return QAOA_ERR_INVALID_ARG;
  size_t need = 0;
  const int64_t span = (cost->dtype == QAOA_COST_I32 && cost->cmax >= cost->cmin) ? cost->cmax - cost->cmin + 1 : 0;
  int rc = qaoa_workspace_size(n, dtype, QAOA_OP_OPTIMIZE, p, 0, span, &need);
  if (rc) return rc;
  if (ws_dev == nullptr || ws_bytes < need) return QAOA_ERR_WORKSPACE;
  const size_t gbytes = need - adam_extra_bytes(p);
  char* extra = (char*)ws_dev + gbytes;
  double* state = state_dev ? state_dev : (double*)extra;
  long long* counter = (long long*)(state + 4 * p);
  double* gout = (double*)(extra + round256((4 * p + 1) * sizeof(double)));
  cudaStream_t s = (cudaStream_t)stream;
  long long row0 = 0;
  if (resume) {  // history rows count from this call's first step
    if (cudaMemcpyAsync(&row0, counter, sizeof(row0), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return QAOA_ERR_CUDA;
  } else if (cudaMemsetAsync(state, 0, (4 * p + 1) * sizeof(double), s) != cudaSuccess) {
    return QAOA_ERR_CUDA;
  }
  return replay_steps(s, steps, [&](cudaStream_t cur) {
    int r = gradient_impl(n, dtype, psi_dev, lambda_dev, cost, nullptr, nullptr, angles_dev, p, gout, ws_dev, gbytes,
                          (void*)cur);
    if (r) return r;
    return cuda_status(
        launch_adam(angles_dev, gout, state, counter, p, lr, beta1, beta2, eps, history_dev, row0, steps, cur));
  }, nullptr, 0);
}

int qaoa_optimize_lbfgs(int n, int dtype, void* psi_dev, void* lambda_dev, const qaoa_cost_t* cost,
                        double* angles_dev, int p, int64_t max_evals, int m, double gtol, double* history_dev,
                        double* info_dev, double* state_dev, int resume, void* ws_dev, size_t ws_bytes,
                        void* stream) {
  if (angles_dev == nullptr || max_evals < 0 || m < 1 || m > QAOA_LBFGS_MAX_M || !(gtol >= 0.0) || p < 1 ||
      p > QAOA_MAX_P || !valid_cost(cost) || (resume != 0 && resume != 1) || (resume && state_dev == nullptr))
    return QAOA_ERR_INVALID_ARG;
  size_t need = 0;
  const int64_t span = (cost->dtype == QAOA_COST_I32 && cost->cmax >= cost->cmin) ? cost->cmax - cost->cmin + 1 : 0;
  int rc = qaoa_workspace_size(n, dtype, QAOA_OP_LBFGS, p, 0, span, &need);
  if (rc) return rc;
  if (ws_dev == nullptr || ws_bytes < need) return QAOA_ERR_WORKSPACE;
  const size_t gbytes = need - lbfgs_extra_bytes(p);
  char* extra = (char*)ws_dev + gbytes;
  const size_t nstate = lbfgs_state_doubles(p, QAOA_LBFGS_MAX_M);
  double* state = state_dev ? state_dev : (double*)extra;
  double* gout = (double*)(extra + round256(nstate * sizeof(double)));
  cudaStream_t s = (cudaStream_t)stream;
  long long row0 = 0;
  if (resume) {
    double scal[16];
    if (cudaMemcpyAsync(scal, state, sizeof(scal), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return QAOA_ERR_CUDA;
    row0 = (long long)scal[3];                // evaluations so far
    if (scal[7] != 0.0) max_evals = 0;        // already finished: report only
    rc = cuda_status(launch_lbfgs_resume(angles_dev, state, p, s));
    if (rc) return rc;
  } else if (cudaMemsetAsync(state, 0, nstate * sizeof(double), s) != cudaSuccess) {
    return QAOA_ERR_CUDA;
  }
  rc = replay_steps(s, max_evals, [&](cudaStream_t cur) {
    int r = gradient_impl(n, dtype, psi_dev, lambda_dev, cost, nullptr, nullptr, angles_dev, p, gout, ws_dev, gbytes,
                          (void*)cur);
    if (r) return r;
    return cuda_status(launch_lbfgs(angles_dev, gout, state, p, m, gtol, 1e-4, history_dev, row0, max_evals, cur));
  }, state + 7, 16);
  if (rc) return rc;
  rc = cuda_status(launch_lbfgs_finish(angles_dev, state, p, info_dev, s));
  if (rc) return rc;
  return cuda_status(cudaStreamSynchronize(s));
}

int qaoa_gradient_host(int n, int dtype, void* psi_dev, void* lambda_dev, const qaoa_cost_t* cost,
                       const double* gamma, const double* beta, int p, double* out_dev, double* out_host,
                       void* ws_dev, size_t ws_bytes, void* stream) {
  if (out_host == nullptr) return QAOA_ERR_INVALID_ARG;
  int rc = qaoa_gradient(n, dtype, psi_dev, lambda_dev, cost, gamma, beta, p, out_dev, ws_dev, ws_bytes, stream);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(out_host, out_dev, (2 * p + 2) * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return QAOA_ERR_CUDA;
  return cuda_status(cudaStreamSynchronize(s));
}

// ------------------------------------------------------------ batched gradients

namespace {

struct BatchLayout {
  std::vector<BatchGraph> graphs;  // processing order: large-tile graphs, then small-tile, n descending
  std::vector<BatchPlan> plans;
  std::vector<int> edges;          // (u, v) pairs
  std::vector<double> ew;          // edge weights
  bool cost_f64 = false;           // some graph has float weights: float64 costs for all
  std::vector<int64_t> blk_off;
  std::vector<double> angles;      // processing order
  int n_large = 0;                 // graphs [0, n_large) use 2^12 tiles, the rest 2^10
  int n_grouped = 0;               // graphs [0, n_grouped) run as grouped one-graph sweeps
  size_t off_graphs = 0, off_plans = 0, off_blk = 0, off_edges = 0, off_ew = 0, off_angles = 0, head_bytes = 0;
  size_t off_queue = 0, off_trig = 0, off_psi = 0, off_lam = 0, off_C = 0, off_phase = 0, off_dtab = 0,
         off_turn = 0, off_gslot = 0, off_grow = 0, off_gpart = 0, total = 0;
};

int default_tile(int n) { return n <= 10 ? 0 : 1; }

// last layout holding group qubits [c, c + t) on tiles of 2^B with RB register bits
int last_layout(int B, int RB, int c, int t) {
  const int nr = (B + RB - 1) / RB;
  int last = 0;
  for (int k = 0; k < nr; ++k) {
    const int lo = std::max(0, B - RB * (k + 1)), hi = k == 0 ? B : std::max(0, B - RB * k);
    if (hi > c && lo < c + t) last = k;
  }
  return last;
}

// Whether a batched sweep can run the lean tile code (complex128, 2^12 tiles): full tiles with
// affine layout-0 addresses, groups of >= 3 qubits, whole 16-byte cost chunks per row, and
// in two-buffer sweeps every op on psi alone before lambda exists (the lean code applies
// mixers and phases to both buffers).
int batch_lean_last(const Sweep& s, const Group& g, int B, int RB, bool fx, bool cost_f64) {
  if (!fx || B != 12 || g.t + g.c != B || g.c > B - RB || g.t < 3) return -1;
  bool reads_c = false, lam_live = s.two && s.load_lam;
  for (uint32_t op : s.ops) {
    const uint32_t kind = op & 0xff;
    reads_c |= (kind == OP_PHASE || kind == OP_LAMBDA || kind == OP_RED_EXPECT || kind == OP_RED_CTERM);
    if (s.two && (kind == OP_MIX || kind == OP_PHASE) && !(op & F_LAM) && lam_live) return -1;
    if (kind == OP_LAMBDA) lam_live = true;
  }
  if (reads_c && !(g.j0 == 0 || (1 << g.c) >= (cost_f64 ? 2 : 4))) return -1;
  return last_layout(B, RB, g.c, g.t);
}

// the gradient plan of n qubits on 2^B tiles, accumulators = output indices
int batch_plan(int n, int B, int RB, bool fx, bool cost_f64, int p, BatchPlan& P) {
  std::memset(&P, 0, sizeof(P));
  const std::vector<Group> gs = plan_groups(n, B);
  std::vector<Sweep> sw;
  plan_gradient((int)gs.size(), p, sw, [](Sweep&, int out0, int) { return (uint32_t)out0; });
  if ((int)sw.size() > kBatchMaxSweeps) return QAOA_ERR_UNSUPPORTED;
  int tmax = 1;
  for (const Group& g : gs) tmax = std::max(tmax, g.t);
  P.n = n;
  P.fx_shift = fx_shift_for(tmax);
  const double amp0 = std::pow(2.0, -0.5 * n);
  P.init_fx = (long long)std::llrint(std::ldexp(amp0, P.fx_shift));
  P.init_f32 = (float)amp0;
  P.nsweeps = (int)sw.size();
  for (int i = 0; i < P.nsweeps; ++i) {
    const Sweep& s = sw[i];
    BatchSweep& b = P.sw[i];
    const Group& g = gs[s.group];
    if ((int)s.ops.size() > kBatchMaxOps) return QAOA_ERR_UNSUPPORTED;
    b.g = {n, g.j0, g.t, g.c, tiles_of(g, n)};
    b.load_fmt = s.init ? 2 : 0;
    // the final state is not needed: the last sweep stores nothing
    b.store_fmt = (i == P.nsweeps - 1 || !s.store_psi) ? -1 : 0;
    b.load_lam = s.two && s.load_lam;
    b.store_lam = s.two && s.store_lam;
    b.two = s.two;
    b.lean_last = batch_lean_last(s, g, B, RB, fx, cost_f64);
    b.nops = (int)s.ops.size();
    for (int k = 0; k < b.nops; ++k) {
      b.ops[k] = s.ops[k];
      const uint32_t kind = s.ops[k] & 0xff;
      if (kind == OP_PHASE || kind == OP_LAMBDA || kind == OP_RED_EXPECT || kind == OP_RED_CTERM) b.needs_cost = 1;
    }
  }
  return QAOA_OK;
}

// Grouped batched gradients: graphs of one size n run the one-graph gradient plan together,
// each sweep one launch of the lean kernel over all of them (GroupSlot: per-graph offsets,
// tables, angles; kGroupTiles tiles or more per block).  A plan qualifies when every sweep
// runs the lean code; smaller graphs stay in the persistent batch kernel.
constexpr int kGroupMinN = 15;   // below, the plan has groups of < 3 qubits (generic sweeps)
constexpr int kGroupTiles = 8;   // tiles per block and graph, at least (up to kGroupMaxBpg blocks)
constexpr int kGroupMaxBpg = 16;

struct GroupPlan {
  int B = 0;
  std::vector<Group> gs;
  std::vector<Sweep> sw;
  std::vector<int> ncontrib;
  int nout = 0;
  int bpg = 1;
};

static bool group_plan(int n, int dtype, int p, bool cost_f64, GroupPlan& G) {
  if (n < kGroupMinN) return false;
  G.B = sweep_tile_bits(dtype, true);
  G.gs = plan_groups(n, G.B);
  G.sw.clear();
  G.nout = 2 * p + 2;
  G.ncontrib.assign(G.nout, 0);
  plan_gradient((int)G.gs.size(), p, G.sw, [&](Sweep& s, int out0, int outs) {
    const uint32_t acc = (uint32_t)s.red_slot.size();
    for (int i = 0; i < outs; ++i) {
      s.red_slot.push_back((out0 + i) * kMaxContrib + G.ncontrib[out0 + i]);
      G.ncontrib[out0 + i]++;
    }
    return acc;
  });
  for (int o = 0; o < G.nout; ++o)
    if (G.ncontrib[o] > kMaxContrib) return false;
  int64_t tiles = 1;
  for (const Sweep& s : G.sw) {
    if ((int)s.ops.size() > kMaxOps || (int)s.red_slot.size() > kMaxAcc) return false;
    if (lean_kind(s, G.gs[s.group], G.B, dtype, cost_f64) == SWEEP_GENERIC) return false;
    tiles = std::max(tiles, tiles_of(G.gs[s.group], n));
  }
  G.bpg = (int)std::max<int64_t>(1, std::min<int64_t>(kGroupMaxBpg, tiles / kGroupTiles));
  return true;
}

int batch_layout(int dtype, int p, int ngraphs, const qaoa_graph_t* gs, const double* angles, const int32_t* tiles,
                 BatchLayout& L) {
  if (!valid_dtype(dtype) || p < 1 || p > QAOA_BATCH_MAX_P || ngraphs < 0 || ngraphs > QAOA_BATCH_MAX_GRAPHS)
    return QAOA_ERR_INVALID_ARG;
  if (ngraphs > 0 && gs == nullptr) return QAOA_ERR_INVALID_ARG;
  const bool fx = dtype == QAOA_C128;
  const size_t vs = fx ? 16 : 8;
  std::vector<int64_t> cmin(ngraphs), cmax(ngraphs);
  std::vector<int> tile(ngraphs);
  bool any_float = false;
  for (int i = 0; i < ngraphs; ++i) {
    const qaoa_graph_t& g = gs[i];
    if (qaoa_graph_check(&g, &cmin[i], &cmax[i]) != QAOA_OK) return QAOA_ERR_INVALID_ARG;
    if (g.weight_kind != QAOA_WEIGHT_INT) any_float = true;
    if (g.n > QAOA_BATCH_MAX_N || g.m > QAOA_BATCH_MAX_EDGES) return QAOA_ERR_UNSUPPORTED;
    tile[i] = tiles ? tiles[g.n] : default_tile(g.n);
    if (tile[i] != 0 && tile[i] != 1) return QAOA_ERR_INVALID_ARG;
  }
  if (angles != nullptr)
    for (int64_t i = 0; i < (int64_t)ngraphs * 2 * p; ++i)
      if (!std::isfinite(angles[i])) return QAOA_ERR_INVALID_ARG;
  std::vector<int> order(ngraphs);
  for (int i = 0; i < ngraphs; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    if (tile[a] != tile[b]) return tile[a] > tile[b];
    return gs[a].n > gs[b].n;
  });
  // plans per (n, tile)
  int plan_of[2][QAOA_MAX_N + 1];
  for (int t = 0; t < 2; ++t)
    for (int n = 0; n <= QAOA_MAX_N; ++n) plan_of[t][n] = -1;
  L = BatchLayout();
  L.cost_f64 = any_float;
  L.graphs.resize(ngraphs);
  L.blk_off.assign(ngraphs + 1, 0);
  L.angles.assign((size_t)ngraphs * 2 * p, 0.0);
  int64_t amps = 0, tab = 0, edge = 0;
  for (int k = 0; k < ngraphs; ++k) {
    const int i = order[k];
    const qaoa_graph_t& g = gs[i];
    BatchGraph& G = L.graphs[k];
    G.n = g.n;
    G.m = (int)g.m;
    G.out = i;
    if (plan_of[tile[i]][g.n] < 0) {
      BatchPlan P;
      const int rc = batch_plan(g.n, batch_tile_bits(tile[i]), batch_register_bits(dtype, tile[i]), fx, any_float, p, P);
      if (rc) return rc;
      plan_of[tile[i]][g.n] = (int)L.plans.size();
      L.plans.push_back(P);
    }
    G.plan = plan_of[tile[i]][g.n];
    double sum_abs = 0.0;
    for (int64_t e = 0; e < g.m; ++e) sum_abs += std::fabs(g.w ? g.w[e] : 1.0);
    int ls = 0;  // 2^lam_shift >= sum |w| >= max |C|
    while (ls < 62 && std::ldexp(1.0, ls) < sum_abs) ++ls;
    G.lam_shift = ls;
    const int64_t span = cmax[i] - cmin[i] + 1;
    G.cmin = L.cost_f64 ? 0 : (int)cmin[i];
    G.span = (!L.cost_f64 && span >= 1 && span <= QAOA_MAX_TABLE_SPAN) ? (int)span : 0;
    G.state = amps;
    G.cost = amps;
    amps += std::max<int64_t>((int64_t)1 << g.n, 64);  // 64-element (>= 256-byte) alignment
    G.table = tab;
    tab += (int64_t)p * G.span;
    G.edge = edge;
    for (int64_t e = 0; e < g.m; ++e) {
      L.edges.push_back(g.uv[2 * e]);
      L.edges.push_back(g.uv[2 * e + 1]);
      L.ew.push_back(g.w ? g.w[e] : 1.0);
    }
    edge += g.m;
    L.blk_off[k + 1] = L.blk_off[k] + (((int64_t)1 << g.n) + (1 << kBatchCostBits) - 1) / (1 << kBatchCostBits);
    if (angles != nullptr)
      for (int j = 0; j < 2 * p; ++j) L.angles[(size_t)k * 2 * p + j] = angles[(size_t)i * 2 * p + j];
    if (tile[i] == 1) L.n_large = k + 1;
  }
  // leading large-tile graphs whose size has an all-lean grouped plan
  size_t gpart = 0;
  {
    int k = 0;
    while (k < L.n_large) {
      int e = k;
      while (e < L.n_large && L.graphs[e].n == L.graphs[k].n) ++e;
      GroupPlan G;
      if (!group_plan(L.graphs[k].n, dtype, p, L.cost_f64, G)) break;
      gpart = std::max(gpart, (size_t)G.nout * kMaxContrib * (size_t)(e - k) * G.bpg * sizeof(double));
      k = e;
    }
    L.n_grouped = k;
  }
  if (L.edges.empty()) {
    L.edges.assign(2, 0);
    L.ew.assign(1, 0.0);
  }
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += round256(bytes);
    return at;
  };
  L.off_graphs = take(sizeof(BatchGraph) * std::max(ngraphs, 1));
  L.off_plans = take(sizeof(BatchPlan) * std::max<size_t>(L.plans.size(), 1));
  L.off_blk = take(sizeof(int64_t) * (ngraphs + 1));
  L.off_edges = take(sizeof(int) * L.edges.size());
  L.off_ew = take(sizeof(double) * L.ew.size());
  L.off_angles = take(sizeof(double) * std::max<size_t>(L.angles.size(), 1));
  L.head_bytes = o;
  L.off_queue = take(256);
  L.off_trig = take(sizeof(double) * 3 * p * std::max(ngraphs, 1));
  L.off_psi = take(vs * std::max<int64_t>(amps, 1));
  L.off_lam = take(vs * std::max<int64_t>(amps, 1));
  L.off_C = take((L.cost_f64 ? 8 : 4) * std::max<int64_t>(amps, 1));
  L.off_phase = take(vs * std::max<int64_t>(tab, 1));
  L.off_dtab = take(fx ? (size_t)16 * p * 196 * std::max(ngraphs, 1) : 0);
  L.off_turn = take(fx ? (size_t)16 * 3072 : 0);
  L.off_gslot = take(sizeof(GroupSlot) * std::max(L.n_grouped, 1));
  L.off_grow = take(sizeof(int) * std::max(L.n_grouped, 1));
  L.off_gpart = take(std::max<size_t>(gpart, 8));
  L.total = o;
  return QAOA_OK;
}

// the grouped sweeps of graphs [k0, k1) (one size; GroupSlots and output rows already on the
// device at slot and row)
static int run_group(int dtype, int p, const BatchLayout& L, const BatchArgs& b, int k0, int k1,
                     const GroupSlot* slot, const int* row, double* partials, cudaStream_t st) {
  const int n = L.graphs[k0].n, ng = k1 - k0;
  GroupPlan G;
  if (!group_plan(n, dtype, p, L.cost_f64, G)) return QAOA_ERR_UNSUPPORTED;
  const bool fx = dtype == QAOA_C128;
  int tmax = 1;
  for (const Group& g : G.gs) tmax = std::max(tmax, g.t);
  const int S = fx_shift_for(tmax);
  const double amp0 = std::pow(2.0, -0.5 * n);
  const int grid = ng * G.bpg;
  const size_t vs = fx ? 16 : 8;
  int max_span = 0;
  for (int k = k0; k < k1; ++k) max_span = std::max(max_span, L.graphs[k].span);
  for (const Sweep& s : G.sw) {
    SweepArgs a;
    std::memset(&a, 0, sizeof(a));
    a.psi = b.psi;
    a.lam = s.two ? b.lam : nullptr;
    a.C = b.C;
    a.cost_dtype = L.cost_f64 ? QAOA_COST_F64 : QAOA_COST_I32;
    const Group& g = G.gs[s.group];
    a.g = {n, g.j0, g.t, g.c, tiles_of(g, n)};
    a.tile_bits = G.B;
    a.load_fmt = s.init ? 2 : 0;
    a.store_fmt = s.store_psi ? 0 : -1;
    a.load_lam = s.load_lam;
    a.store_lam = s.store_lam;
    a.fx_shift = S;
    a.init_fx = (long long)std::llrint(std::ldexp(amp0, S));
    a.init_f32 = (float)amp0;
    a.nops = (int)s.ops.size();
    bool reads_c = false;
    for (size_t k = 0; k < s.ops.size(); ++k) {
      a.ops[k] = s.ops[k];
      const uint32_t kind = s.ops[k] & 0xff;
      reads_c |= (kind == OP_PHASE || kind == OP_LAMBDA || kind == OP_RED_EXPECT || kind == OP_RED_CTERM);
    }
    a.needs_cost = reads_c;
    a.np = p;
    a.dev_trig = b.trig;  // per graph: GroupSlot.trig
    a.phase_table = max_span > 0 ? b.phase : nullptr;
    a.span = max_span;  // shared-memory sizing; each graph's own span is in its slot
    a.smem_table_layer = -1;
    if (max_span > 0 && max_span <= kSmemTable) {
      for (uint32_t op : s.ops)
        if ((op & 0xff) == OP_PHASE) {
          a.smem_table_layer = (int)((op >> 16) & 0xff);
          break;
        }
    }
    a.d_table = b.dtab;
    a.turn_table = b.turn;
    a.nred = (int)s.red_slot.size();
    for (int r = 0; r < a.nred; ++r) a.red_slot[r] = s.red_slot[r];
    a.partials = partials;
    a.grid = grid;
    a.gslot = slot;
    a.gbpg = G.bpg;
    const double cb = L.cost_f64 ? 8.0 : 4.0;
    const double per = (double)vs * ((s.init ? 0 : 1) + (s.store_psi ? 1 : 0) + (s.two && s.load_lam ? 1 : 0) +
                                     (s.two && s.store_lam ? 1 : 0)) +
                       (reads_c ? cb : 0.0);
    a.algo_bytes = per * (double)(1ull << n) * ng;
    a.kind = lean_kind(s, g, G.B, dtype, L.cost_f64);
    if (a.kind == SWEEP_GENERIC) return QAOA_ERR_UNSUPPORTED;
    const int rc = cuda_status(launch_sweep(dtype, s.two, a, st));
    if (rc) return rc;
  }
  ReducePlan r;
  std::memset(&r, 0, sizeof(r));
  r.nout = G.nout;
  r.grid = grid;
  for (int o = 0; o < G.nout; ++o) {
    r.ncontrib[o] = G.ncontrib[o];
    r.scale[o] = 1.0;
  }
  return cuda_status(launch_group_reduce(r, ng, G.bpg, row, partials, b.out, st));
}

int batch_run(int dtype, int p, const BatchLayout& L, double* out_dev, void* ws_dev, size_t ws_bytes, void* stream) {
  if (ws_dev == nullptr || ws_bytes < L.total || ((uintptr_t)ws_dev & 255)) return QAOA_ERR_WORKSPACE;
  const int ng = (int)L.graphs.size();
  if (ng == 0) return QAOA_OK;
  if (out_dev == nullptr) return QAOA_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  char* ws = (char*)ws_dev;
  // one upload of the host-built header
  std::vector<char> head(L.head_bytes, 0);
  std::memcpy(head.data() + L.off_graphs, L.graphs.data(), sizeof(BatchGraph) * ng);
  std::memcpy(head.data() + L.off_plans, L.plans.data(), sizeof(BatchPlan) * L.plans.size());
  std::memcpy(head.data() + L.off_blk, L.blk_off.data(), sizeof(int64_t) * L.blk_off.size());
  std::memcpy(head.data() + L.off_edges, L.edges.data(), sizeof(int) * L.edges.size());
  std::memcpy(head.data() + L.off_ew, L.ew.data(), sizeof(double) * L.ew.size());
  std::memcpy(head.data() + L.off_angles, L.angles.data(), sizeof(double) * L.angles.size());
  if (cudaMemcpyAsync(ws, head.data(), L.head_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return QAOA_ERR_CUDA;
  if (cudaMemsetAsync(ws + L.off_queue, 0, 256, s) != cudaSuccess) return QAOA_ERR_CUDA;
  BatchArgs b;
  std::memset(&b, 0, sizeof(b));
  b.ngraphs = ng;
  b.p = p;
  b.dtype = dtype;
  b.graphs = (const BatchGraph*)(ws + L.off_graphs);
  b.plans = (const BatchPlan*)(ws + L.off_plans);
  b.edges = (const int*)(ws + L.off_edges);
  b.ew = (const double*)(ws + L.off_ew);
  b.cost_f64 = L.cost_f64;
  b.blk_off = (const int64_t*)(ws + L.off_blk);
  b.angles = (const double*)(ws + L.off_angles);
  b.psi = ws + L.off_psi;
  b.lam = ws + L.off_lam;
  b.C = ws + L.off_C;
  b.phase = ws + L.off_phase;
  b.dtab = dtype == QAOA_C128 ? ws + L.off_dtab : nullptr;
  b.turn = dtype == QAOA_C128 ? ws + L.off_turn : nullptr;
  b.trig = (double*)(ws + L.off_trig);
  b.out = out_dev;
  int rc = cuda_status(launch_batch_prep(b, L.blk_off[ng], s));
  if (rc) return rc;
  if (L.n_grouped > 0) {  // per-graph slots of the grouped sweeps (device addresses in this workspace)
    const bool fx = dtype == QAOA_C128;
    const size_t vs = fx ? 16 : 8;
    std::vector<GroupSlot> slots(L.n_grouped);
    std::vector<int> rows(L.n_grouped);
    for (int k = 0; k < L.n_grouped; ++k) {
      const BatchGraph& G = L.graphs[k];
      GroupSlot& g = slots[k];
      g.zoff = G.state;
      g.phase_table = G.span > 0 ? (const void*)((char*)b.phase + G.table * vs) : nullptr;
      g.cmin = G.cmin;
      g.span = G.span;
      g.d_table = fx ? (const void*)((char*)b.dtab + (size_t)k * p * 196 * sizeof(longlong2)) : nullptr;
      g.trig = b.trig + (size_t)k * 3 * p;
      g.lam_shift = G.lam_shift;
      rows[k] = G.out;
    }
    if (cudaMemcpyAsync(ws + L.off_gslot, slots.data(), sizeof(GroupSlot) * slots.size(), cudaMemcpyHostToDevice,
                        s) != cudaSuccess ||
        cudaMemcpyAsync(ws + L.off_grow, rows.data(), sizeof(int) * rows.size(), cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
      return QAOA_ERR_CUDA;
    int k = 0;
    while (k < L.n_grouped) {
      int e = k;
      while (e < L.n_grouped && L.graphs[e].n == L.graphs[k].n) ++e;
      rc = run_group(dtype, p, L, b, k, e, (const GroupSlot*)(ws + L.off_gslot) + k, (const int*)(ws + L.off_grow) + k,
                     (double*)(ws + L.off_gpart), s);
      if (rc) return rc;
      k = e;
    }
  }
  int* queue = (int*)(ws + L.off_queue);
  rc = cuda_status(launch_batch(b, 1, L.n_grouped, L.n_large - L.n_grouped, queue, s));
  if (rc) return rc;
  return cuda_status(launch_batch(b, 0, L.n_large, ng - L.n_large, queue + 1, s));
}

}  // namespace

int qaoa_batch_workspace_size(int dtype, int p, int ngraphs, const qaoa_graph_t* graphs, const int32_t* tiles,
                              size_t* bytes) {
  if (bytes == nullptr) return QAOA_ERR_INVALID_ARG;
  BatchLayout L;
  const int rc = batch_layout(dtype, p, ngraphs, graphs, nullptr, tiles, L);
  if (rc) return rc;
  *bytes = L.total;
  return QAOA_OK;
}

int qaoa_batch_gradient(int dtype, int ngraphs, const qaoa_graph_t* graphs, const double* angles, int p,
                        const int32_t* tiles, double* out_dev, void* ws_dev, size_t ws_bytes, void* stream) {
  if (ngraphs > 0 && angles == nullptr) return QAOA_ERR_INVALID_ARG;
  BatchLayout L;
  const int rc = batch_layout(dtype, p, ngraphs, graphs, angles, tiles, L);
  if (rc) return rc;
  return batch_run(dtype, p, L, out_dev, ws_dev, ws_bytes, stream);
}

// synthetic tuning instances: a ring plus chords (u, u + 3), integer weights 1..5
static void tune_graph(int n, int seed, std::vector<int>& uv, std::vector<double>& w) {
  std::set<std::pair<int, int>> seen;
  uv.clear();
  w.clear();
  for (int d : {1, 3})
    for (int u = 0; u < n; ++u) {
      const int v = (u + d) % n;
      if (u == v) continue;
      const std::pair<int, int> e{std::min(u, v), std::max(u, v)};
      if (!seen.insert(e).second) continue;
      uv.push_back(e.first);
      uv.push_back(e.second);
      w.push_back((double)(1 + (u * 7 + d + seed) % 5));
    }
}

int qaoa_batch_autotune_workspace_size(int dtype, int p, int n_hi, int graphs_per_n, size_t* bytes) {
  if (bytes == nullptr || n_hi < 2 || n_hi > QAOA_BATCH_MAX_N || graphs_per_n < 1 || graphs_per_n > 65536)
    return QAOA_ERR_INVALID_ARG;
  std::vector<int> uv;
  std::vector<double> w;
  tune_graph(n_hi, 0, uv, w);
  std::vector<qaoa_graph_t> gs(graphs_per_n, qaoa_graph_t{n_hi, (int64_t)w.size(), uv.data(), w.data(), QAOA_WEIGHT_INT});
  size_t b0 = 0, b1 = 0;
  const int32_t zero[QAOA_MAX_N + 1] = {0};
  int32_t one[QAOA_MAX_N + 1];
  for (int& x : one) x = 1;
  int rc = qaoa_batch_workspace_size(dtype, p, graphs_per_n, gs.data(), zero, &b0);
  if (rc) return rc;
  rc = qaoa_batch_workspace_size(dtype, p, graphs_per_n, gs.data(), one, &b1);
  if (rc) return rc;
  *bytes = std::max(b0, b1) + 256 + (size_t)graphs_per_n * (2 * p + 2) * sizeof(double);
  return QAOA_OK;
}

int qaoa_batch_autotune(int dtype, int p, int n_lo, int n_hi, int graphs_per_n, int32_t* tiles_out, double* ms_out,
                        void* ws_dev, size_t ws_bytes, void* stream) {
  if (tiles_out == nullptr || n_lo < 2 || n_lo > n_hi) return QAOA_ERR_INVALID_ARG;
  size_t need = 0;
  int rc = qaoa_batch_autotune_workspace_size(dtype, p, n_hi, graphs_per_n, &need);
  if (rc) return rc;
  if (ws_dev == nullptr || ws_bytes < need) return QAOA_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  double* out = (double*)((char*)ws_dev + (need - (size_t)graphs_per_n * (2 * p + 2) * sizeof(double)));
  for (int n = 0; n <= QAOA_MAX_N; ++n) tiles_out[n] = default_tile(n);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return QAOA_ERR_CUDA;
  std::vector<double> ang((size_t)graphs_per_n * 2 * p);
  for (size_t i = 0; i < ang.size(); ++i) ang[i] = 0.1 + 0.37 * (double)(i % 7);
  rc = QAOA_OK;
  for (int n = n_lo; n <= n_hi && rc == QAOA_OK; ++n) {
    std::vector<std::vector<int>> uvs(graphs_per_n);
    std::vector<std::vector<double>> ws(graphs_per_n);
    std::vector<qaoa_graph_t> gs(graphs_per_n);
    for (int i = 0; i < graphs_per_n; ++i) {
      tune_graph(n, i, uvs[i], ws[i]);
      gs[i] = qaoa_graph_t{n, (int64_t)ws[i].size(), uvs[i].data(), ws[i].data(), QAOA_WEIGHT_INT};
    }
    double best = 0.0;
    for (int t = 0; t < 2 && rc == QAOA_OK; ++t) {
      int32_t tiles[QAOA_MAX_N + 1];
      for (int& x : tiles) x = t;
      BatchLayout L;
      rc = batch_layout(dtype, p, graphs_per_n, gs.data(), ang.data(), tiles, L);
      float ms = 0.f;
      for (int rep = 0; rep < 2 && rc == QAOA_OK; ++rep) {  // warm-up, then timed
        cudaEventRecord(e0, s);
        rc = batch_run(dtype, p, L, out, ws_dev, ws_bytes, stream);
        cudaEventRecord(e1, s);
        if (rc == QAOA_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = QAOA_ERR_CUDA;
        if (rc == QAOA_OK) cudaEventElapsedTime(&ms, e0, e1);
      }
      if (ms_out) ms_out[2 * n + t] = ms;
      if (rc == QAOA_OK && (t == 0 || ms < best)) {
        best = ms;
        tiles_out[n] = t;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

// ------------------------------------------------------------ learned angle proposer

namespace {
struct ProposeLayout {
  std::vector<int> n, uv;
  std::vector<int64_t> edge_off;
  std::vector<double> w;
  size_t off_n = 0, off_eo = 0, off_uv = 0, off_w = 0, total = 0;
};

int propose_layout(int ngraphs, const qaoa_graph_t* graphs, ProposeLayout& L) {
  if (ngraphs < 0 || ngraphs > QAOA_BATCH_MAX_GRAPHS || (ngraphs > 0 && graphs == nullptr)) return QAOA_ERR_INVALID_ARG;
  L = ProposeLayout();
  L.edge_off.push_back(0);
  for (int i = 0; i < ngraphs; ++i) {
    const qaoa_graph_t& g = graphs[i];
    if (qaoa_graph_check(&g, nullptr, nullptr) != QAOA_OK) return QAOA_ERR_INVALID_ARG;
    L.n.push_back(g.n);
    for (int64_t e = 0; e < g.m; ++e) {
      L.uv.push_back(g.uv[2 * e]);
      L.uv.push_back(g.uv[2 * e + 1]);
      L.w.push_back(g.w ? g.w[e] : 1.0);
    }
    L.edge_off.push_back(L.edge_off.back() + g.m);
  }
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += round256(std::max<size_t>(bytes, 1));
    return at;
  };
  L.off_n = take(sizeof(int) * L.n.size());
  L.off_eo = take(sizeof(int64_t) * L.edge_off.size());
  L.off_uv = take(sizeof(int) * L.uv.size());
  L.off_w = take(sizeof(double) * L.w.size());
  L.total = o;
  return QAOA_OK;
}
}  // namespace

int64_t qaoa_proposer_param_count(int p) {
  if (p < 1 || p > QAOA_MAX_P) return -1;
  return proposer_param_count(p);
}

int qaoa_propose_workspace_size(int ngraphs, const qaoa_graph_t* graphs, size_t* bytes) {
  if (bytes == nullptr) return QAOA_ERR_INVALID_ARG;
  ProposeLayout L;
  const int rc = propose_layout(ngraphs, graphs, L);
  if (rc) return rc;
  *bytes = L.total;
  return QAOA_OK;
}

int qaoa_propose_angles(int ngraphs, const qaoa_graph_t* graphs, int p, const float* params_dev, double* angles_dev,
                        void* ws_dev, size_t ws_bytes, void* stream) {
  if (p < 1 || p > QAOA_MAX_P) return QAOA_ERR_INVALID_ARG;
  ProposeLayout L;
  int rc = propose_layout(ngraphs, graphs, L);
  if (rc) return rc;
  if (ngraphs == 0) return QAOA_OK;
  if (params_dev == nullptr || angles_dev == nullptr) return QAOA_ERR_INVALID_ARG;
  if (ws_dev == nullptr || ws_bytes < L.total) return QAOA_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<char> head(L.total, 0);
  std::memcpy(head.data() + L.off_n, L.n.data(), sizeof(int) * L.n.size());
  std::memcpy(head.data() + L.off_eo, L.edge_off.data(), sizeof(int64_t) * L.edge_off.size());
  if (!L.uv.empty()) std::memcpy(head.data() + L.off_uv, L.uv.data(), sizeof(int) * L.uv.size());
  if (!L.w.empty()) std::memcpy(head.data() + L.off_w, L.w.data(), sizeof(double) * L.w.size());
  char* ws = (char*)ws_dev;
  if (cudaMemcpyAsync(ws, head.data(), L.total, cudaMemcpyHostToDevice, s) != cudaSuccess) return QAOA_ERR_CUDA;
  ProposeArgs a;
  a.p = p;
  a.n = (const int*)(ws + L.off_n);
  a.edge_off = (const int64_t*)(ws + L.off_eo);
  a.uv = (const int*)(ws + L.off_uv);
  a.w = (const double*)(ws + L.off_w);
  a.params = params_dev;
  a.angles = angles_dev;
  return cuda_status(launch_propose(a, ngraphs, s));
}

int64_t qaoa_launch_count(void) { return g_launches.load(); }
void qaoa_launch_count_reset(void) { g_launches.store(0); }

int qaoa_timing_enable(int on) {
  std::lock_guard<std::mutex> lk(g_timing_mu);
  g_timing_on = on != 0;
  return QAOA_OK;
}

int qaoa_timing_read(double* ms, int64_t* launches, double* bytes, int64_t* dropped) {
  std::lock_guard<std::mutex> lk(g_timing_mu);
  for (int k = 0; k < 4; ++k) {
    if (ms) ms[k] = 0.0;
    if (launches) launches[k] = 0;
    if (bytes) bytes[k] = 0.0;
  }
  int rc = QAOA_OK;
  for (TimedLaunch& t : g_timed) {
    if (cudaEventSynchronize(t.e1) != cudaSuccess) rc = QAOA_ERR_CUDA;
    float f = 0.f;
    if (cudaEventElapsedTime(&f, t.e0, t.e1) != cudaSuccess) rc = QAOA_ERR_CUDA;
    if (t.kind >= 0 && t.kind < 4) {
      if (ms) ms[t.kind] += f;
      if (launches) launches[t.kind] += 1;
      if (bytes) bytes[t.kind] += t.bytes;
    }
    g_event_pool.push_back(t.e0);
    g_event_pool.push_back(t.e1);
  }
  g_timed.clear();
  if (dropped) *dropped = g_dropped;
  g_dropped = 0;
  return rc;
}

}  // extern "C"
