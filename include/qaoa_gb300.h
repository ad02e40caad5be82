/*
 * qaoa_gb300.h — C ABI of the GB300 MaxCut-QAOA statevector simulator.
 *
 * The method is the QAOA of arXiv 2407.13012 (CUAOA), Eq. 1:
 *   |psi> = U_M(beta_p) U_C(gamma_p) ... U_M(beta_1) U_C(gamma_1) |+>^n,
 *   U_C(gamma) = exp(-i gamma H_C), H_C = diag(C(z)) (Sec. II-A),
 *   U_M(beta)  = exp(-i beta sum_j X_j) = prod_j RX_j(2 beta).
 * The paper's mixer Hamiltonian H_M = -sum_j X_j (Sec. II-A) gives
 * R_x(-2 beta) (Sec. IV-B); this library uses RX(+2 beta), i.e. the paper's
 * angles with beta -> -beta.  Pass mixer angles negated to get the paper's
 * convention.
 *
 * Conventions shared by every call:
 *  - Amplitude index z in [0, 2^n); qubit j is bit j of z (the one-hot
 *    encoding of Eq. 3, variable i <-> 2^i).
 *  - C(z) = sum over edges (u,v) of w_uv * [bit u of z != bit v of z]
 *    (MaxCut, Sec. V).
 *  - State buffers are interleaved (re, im): QAOA_C128 = 2 x float64 per
 *    amplitude (16 B), QAOA_C64 = 2 x float32 (8 B).  Layout is index order.
 *  - Arithmetic.  QAOA_C64 computes in float32 (reductions in float64).
 *    QAOA_C128 stores float64 pairs between calls but, inside a call, holds
 *    the state as int64 fixed point with the fixed resolution 2^-54 (value =
 *    integer x 2^-54): an amplitude of magnitude 2^-k keeps 54 - k significant
 *    bits (39 at 2^-15, a typical amplitude at n = 30), not float64's 53.
 *    Each group mixer adds a rounding error of 2-norm about
 *    0.41 x 2^((n + t)/2 - 54) for a group of t <= 12 qubits; <C> and the
 *    gradient are reduced exactly in int128 and see far less (their error
 *    stays below 1e-10 x max(1, sum|w|) at every tested n <= 31).
 *  - Every pointer named *_dev is device memory owned by the caller; the
 *    library never allocates or frees device memory.  Host pointers are read
 *    during the call only.
 *  - All device work is enqueued on `stream` (a cudaStream_t passed as
 *    void*; NULL = legacy default stream) and is asynchronous unless the name
 *    ends in _host, in which case the call synchronises `stream` and writes
 *    host outputs before returning.
 *  - `ws_dev`/`ws_bytes`: caller-owned device scratch of at least
 *    qaoa_workspace_size() bytes, 256-byte aligned.  Its content on entry is
 *    ignored; calls that share one workspace must be ordered on a stream.
 *  - Return value: QAOA_OK or an error code.  Argument errors are detected
 *    on the host before anything is enqueued.  QAOA_ERR_CUDA reports a
 *    launch or runtime error (cudaGetLastError after each launch).
 *
 * Limits: 1 <= n <= 32; p <= QAOA_MAX_P.
 */
#ifndef QAOA_GB300_H
#define QAOA_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QAOA_MAX_N 32
#define QAOA_MAX_P 64

enum qaoa_status {
  QAOA_OK = 0,
  QAOA_ERR_INVALID_ARG = 1, /* bad pointer, size, graph or angle */
  QAOA_ERR_UNSUPPORTED = 2, /* valid but outside the library's limits */
  QAOA_ERR_CUDA = 3,        /* CUDA launch / runtime error */
  QAOA_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up */
  QAOA_ERR_WORKSPACE = 5    /* ws_bytes smaller than qaoa_workspace_size() */
};

enum qaoa_dtype { QAOA_C128 = 0, QAOA_C64 = 1 };
enum qaoa_cost_dtype { QAOA_COST_I32 = 0, QAOA_COST_F64 = 1 };
enum qaoa_weight_kind { QAOA_WEIGHT_INT = 0, QAOA_WEIGHT_F64 = 1 };
enum qaoa_op {
  QAOA_OP_COST = 0,
  QAOA_OP_LAYERS = 1,
  QAOA_OP_EXPECTATION = 2,
  QAOA_OP_SAMPLE = 3,
  QAOA_OP_GRADIENT = 4,
  QAOA_OP_OPTIMIZE = 5,
  QAOA_OP_LBFGS = 6
};

/*
 * Weighted graph on host memory (MaxCut instance, Sec. V).
 *  n            number of vertices = qubits, 1..32.
 *  m            number of edges, >= 0.
 *  uv           2*m int32: edge e joins uv[2e] and uv[2e+1].
 *  w            m float64 weights, or NULL for all weights 1.
 *  weight_kind  QAOA_WEIGHT_INT: every weight must be integral with
 *               sum |w| < 2^31; QAOA_WEIGHT_F64: any finite weights.
 * Rejected (QAOA_ERR_INVALID_ARG): u == v, a vertex outside [0, n), a
 * repeated edge (in either orientation), a non-finite weight, a non-integral
 * weight under QAOA_WEIGHT_INT.
 */
typedef struct qaoa_graph {
  int32_t n;
  int64_t m;
  const int32_t* uv;
  const double* w;
  int32_t weight_kind;
} qaoa_graph_t;

/*
 * Cost vector descriptor.  C_dev holds 2^n entries of `dtype` (device
 * memory, caller-owned).  For QAOA_COST_I32, [cmin, cmax] are bounds the
 * caller promises for every entry; the phase kernels then look
 * exp(-i gamma c) up in a table of cmax - cmin + 1 entries (when that span is
 * at most QAOA_MAX_TABLE_SPAN).  An entry outside the bounds is still handled
 * correctly (computed directly), so wrong bounds cost speed, never
 * correctness.  cmax < cmin means "unknown" (no table).  qaoa_cost_vector()
 * fills a descriptor with exact bounds.
 */
#define QAOA_MAX_TABLE_SPAN 16384
typedef struct qaoa_cost {
  const void* C_dev;
  int32_t dtype;
  int64_t cmin;
  int64_t cmax;
} qaoa_cost_t;

/* Library version as 10000*major + 100*minor + patch. */
int qaoa_version(void);

/* Static description of a status code (never NULL). */
const char* qaoa_strerror(int status);

/*
 * Validate a graph on the host without touching the GPU.  Returns QAOA_OK or
 * QAOA_ERR_INVALID_ARG; on success, if non-NULL, *cmin/*cmax receive integer
 * bounds on C(z) (sum of negative / positive weights) for integer graphs.
 */
int qaoa_graph_check(const qaoa_graph_t* g, int64_t* cmin, int64_t* cmax);

/*
 * Cost vector of a general polynomial objective in 0-1 variables (Eq. 3):
 *   C(z) = sum_t w_t prod_{i in T_t} z_i,
 * term t given by the bit mask masks[t] of its variables T_t (bit i = variable
 * i = qubit i; mask 0 is a constant term).  MaxCut is the special case with
 * terms {u}: w, {v}: w, {u, v}: -2w per edge.  Host arrays masks[nterms],
 * w[nterms]; nterms <= QAOA_MAX_PUBO_TERMS.  weight_kind QAOA_WEIGHT_INT
 * (integral weights, sum |w| < 2^31): exact, int32 or float64 costs;
 * QAOA_WEIGHT_F64: float64 costs from weights quantised to one common fixed
 * point and summed exactly (one rounding per 2048 terms).  Fills *desc as
 * qaoa_cost_vector does (integer bounds = sums of the negative / positive
 * weights).  Errors: QAOA_ERR_INVALID_ARG for a variable outside [0, n), a
 * non-finite or (INT) non-integral weight, or I32 costs with float weights.
 * Every downstream call (layers, expectation, sampling, gradients) takes the
 * result like a MaxCut cost vector.
 */
#define QAOA_MAX_PUBO_TERMS (1 << 24)
int qaoa_cost_vector_pubo(int n, int64_t nterms, const uint32_t* masks, const double* w,
                          int weight_kind, void* C_dev, int cost_dtype, qaoa_cost_t* desc,
                          void* stream);

/*
 * Bytes of device scratch the call `op` (enum qaoa_op) needs for n qubits,
 * state dtype `dtype`, depth p (QAOA_OP_LAYERS / QAOA_OP_GRADIENT; ignored
 * otherwise), `shots` (QAOA_OP_SAMPLE; ignored otherwise) and cost range
 * `cost_span` = cmax - cmin + 1 of the integer cost vector's descriptor (0
 * when there is no table: float costs or unknown bounds).  Host-only;
 * writes *bytes.
 */
int qaoa_workspace_size(int n, int dtype, int op, int p, int64_t shots, int64_t cost_span,
                        size_t* bytes);

/*
 * S1 — cost vector (Sec. IV-A, Eq. 3; "the precomputation of the cost
 * Hamiltonian", Sec. I): fill C_dev[z] = C(z) for all z in [0, 2^n).
 *  cost_dtype QAOA_COST_I32: int32 values, exact; needs an integer graph.
 *  cost_dtype QAOA_COST_F64: float64 values.  Integer graphs: exact.  Float
 *    weights: the sum of the edge weights quantised to a common binary
 *    fixed point with 2^-(62 - ceil(log2(sum|w| + 1))) resolution, summed
 *    exactly, rounded once to float64 (|error| <= (m+1) 2^-52 max(1, sum|w|)).
 * C_dev holds 2^n elements of the chosen type.  No workspace.  If desc is
 * non-NULL it is filled with {C_dev, cost_dtype, cmin, cmax}: the sums of the
 * negative and of the positive weights for integer graphs, cmax < cmin for
 * float weights.
 */
int qaoa_cost_vector(const qaoa_graph_t* g, void* C_dev, int cost_dtype, qaoa_cost_t* desc,
                     void* stream);

/*
 * S2+S3 — apply p QAOA layers in place (Eq. 1; Sec. IV-B):
 * for l = 0..p-1: psi_z *= exp(-i gamma[l] C(z)), then RX(2 beta[l]) on every
 * qubit.  init = 1 starts from |+>^n (psi_dev is write-only then); init = 0
 * continues from the state in psi_dev.  gamma/beta are host arrays of p
 * doubles.  p = 0 with init = 1 just writes |+>^n.
 *  expect_dev: optional (may be NULL) device double[2] receiving
 *    [<C>, <psi|psi>] of the final state, fused into the last sweep.
 */
int qaoa_apply_layers(int n, int dtype, void* psi_dev, const qaoa_cost_t* cost,
                      const double* gamma, const double* beta, int p, int init,
                      double* expect_dev, void* ws_dev, size_t ws_bytes, void* stream);

/*
 * S4 — expectation value (Sec. IV-D): out_dev[0] = sum_z C(z) |psi_z|^2,
 * out_dev[1] = sum_z |psi_z|^2 (device doubles; deterministic reduction
 * order, float64 accumulation).
 */
int qaoa_expectation(int n, int dtype, const void* psi_dev, const qaoa_cost_t* cost,
                     double* out_dev, void* ws_dev, size_t ws_bytes, void* stream);

/* As qaoa_expectation, then synchronise and copy the two doubles to out_host. */
int qaoa_expectation_host(int n, int dtype, const void* psi_dev, const qaoa_cost_t* cost,
                          double* out_host, void* ws_dev, size_t ws_bytes, void* stream);

/*
 * qaoa_expectation without a workspace argument, for callers that cannot
 * allocate device memory (they run inside an allocator or pool callback, on
 * a teardown path, or inside a host that owns all device memory).  The paper
 * has no counterpart; this is a deployment convenience.
 *  Scratch: a fixed 256 KiB array in device global memory defined by the
 *    library (reduction partials for up to 2048 blocks; enough for every n in
 *    1..32).  Each GPU that loads the library holds it until the process exits.
 *    The call allocates nothing: no cudaMalloc/cudaFree, no library allocator.
 *  Set-up: the first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.
 *  Sharing: every call uses the same array; each call writes every scratch
 *    entry it later reads, so no clearing is needed, but calls that overlap on
 *    the GPU (different streams, or different host threads) race and must be
 *    serialised by the caller.
 *  Errors: as qaoa_expectation; QAOA_ERR_UNSUPPORTED if a size would need more
 *    scratch than the array holds.
 */
int qaoa_expectation_noalloc(int n, int dtype, const void* psi_dev, const qaoa_cost_t* cost,
                             double* out_dev, void* stream);

/*
 * S5+S6 — draw `shots` bitstrings from |psi_z|^2 on the device (Sec. IV-D)
 * and return each with its objective value.  Uniforms: u_i (i = 0..shots-1)
 * is the i-th 53-bit uniform of the SplitMix64 counter stream keyed by
 * (seed, "sample"): base = mix64(mix64(seed) ^ 0x5f5f656c706d6173),
 * x_i = mix64(base + (i+1) * 0x9E3779B97F4A7C15), u_i = (x_i >> 11) * 2^-53.
 * Rule: z_i = min{z : P(z) > u_i * P_total} with P the inclusive prefix sum
 * of |psi|^2 in index order; a target at or past the end yields the last z
 * of nonzero probability.  Outputs: z_dev[i] (uint64), cost_dev[i] =
 * C(z_i) as float64 (exact copy of the cost vector entry).  Shot order is
 * draw order.  shots may be 0.
 */
int qaoa_sample(int n, int dtype, const void* psi_dev, const qaoa_cost_t* cost, int64_t shots,
                uint64_t seed, uint64_t* z_dev, double* cost_dev, void* ws_dev, size_t ws_bytes,
                void* stream);

/* As qaoa_sample, then synchronise and copy z and cost to the host arrays. */
int qaoa_sample_host(int n, int dtype, const void* psi_dev, const qaoa_cost_t* cost,
                     int64_t shots, uint64_t seed, uint64_t* z_dev, double* cost_dev,
                     uint64_t* z_host, double* cost_host, void* ws_dev, size_t ws_bytes,
                     void* stream);

/*
 * S7 — adjoint gradient of E = <C> (Sec. II-B; QAOA form Sec. IV-C).
 * Runs the forward pass from |+>^n into psi_dev, sets lambda = C psi, then
 * walks the layers backwards uncomputing both states, with
 *   dE/dbeta_l  = 2 Im <lambda| sum_j X_j |psi>  (before U_M(beta_l)^dagger)
 *   dE/dgamma_l = 2 Im <lambda| C |psi>          (before U_C(gamma_l)^dagger).
 * out_dev (device, 2p+2 doubles): [E, <psi|psi>, dE/dgamma_1..p,
 * dE/dbeta_1..p].  psi_dev and lambda_dev are 2^n-amplitude buffers of
 * `dtype`; on return psi_dev holds the uncomputed state (|+>^n up to
 * rounding) and lambda_dev is unspecified.
 */
int qaoa_gradient(int n, int dtype, void* psi_dev, void* lambda_dev, const qaoa_cost_t* cost,
                  const double* gamma, const double* beta, int p, double* out_dev, void* ws_dev,
                  size_t ws_bytes, void* stream);

/*
 * As qaoa_gradient with the angles in device memory: angles_dev holds
 * [gamma_1..p, beta_1..p] (2p doubles, read on the stream).  Nothing is read
 * from the host, so the call can be captured in a CUDA graph after a first
 * uncaptured call with the same sizes.
 */
int qaoa_gradient_dev(int n, int dtype, void* psi_dev, void* lambda_dev, const qaoa_cost_t* cost,
                      const double* angles_dev, int p, double* out_dev, void* ws_dev, size_t ws_bytes,
                      void* stream);

/*
 * Gradient-based training of the angles (the paper offers L-BFGS and BFGS
 * optimisers driven by the adjoint gradient, Sec. V-B): `steps` steps of Adam
 * ascent on E = <C>, entirely on the device.  Each step runs qaoa_gradient_dev at
 * angles_dev, then updates angles_dev in place:
 *   m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
 *   angles += lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps),  t = 1, 2, ...
 * with g = dE/d[gamma, beta] and m = v = 0 at the start.  The first step runs
 * directly; the remaining steps replay a CUDA graph of one step on `stream`
 * (given the legacy default stream, NULL, the graph runs on a private blocking
 * stream ordered after it), with no host round trip inside.
 * history_dev (optional): steps x (4p + 2) doubles; row t = [E, <psi|psi>,
 * dE/dgamma, dE/dbeta, gamma, beta] at the angles step t started from.
 * Workspace: qaoa_workspace_size(..., QAOA_OP_OPTIMIZE, p, ...).  The call
 * synchronises `stream` before returning.  On return angles_dev holds the final
 * angles; psi_dev and lambda_dev are scratch.
 */
int qaoa_optimize_adam(int n, int dtype, void* psi_dev, void* lambda_dev, const qaoa_cost_t* cost,
                       double* angles_dev, int p, int64_t steps, double lr, double beta1,
                       double beta2, double eps, double* history_dev, double* state_dev, int resume,
                       void* ws_dev, size_t ws_bytes, void* stream);

/*
 * L-BFGS ascent on E = <C> over the angles, entirely on the device (the paper
 * optimises the angles with L-BFGS on the adjoint gradient, Sec. V-B).  Each
 * evaluation runs qaoa_gradient_dev at angles_dev and then one step of an
 * L-BFGS state machine on the device: Armijo backtracking (c1 = 1e-4) with
 * safeguarded quadratic interpolation; accepted steps store (s, y) when
 * s.y > 0 (at most m <= QAOA_LBFGS_MAX_M pairs) and take the two-loop
 * direction with H0 = s.y / y.y (the first step: -g / max(1, |g|)).  The run
 * ends after max_evals evaluations, when |dE/dangles|_inf < gtol (converged)
 * or when the step falls below 1e-12 (no progress).  As for Adam, the first
 * evaluation runs directly and the rest replay a CUDA graph; the host reads a
 * device flag every 16 evaluations to stop early.
 * history_dev (optional): max_evals x (4p + 2) doubles, one row per evaluation
 * (accepted or not) = [E, <psi|psi>, dE/dgamma, dE/dbeta, gamma, beta].
 * info_dev (optional): 4 doubles [E at the final angles, accepted steps,
 * evaluations, status 0 = evaluations used up, 1 = converged, 2 = no progress].
 * On return angles_dev holds the best accepted angles.  Workspace:
 * qaoa_workspace_size(..., QAOA_OP_LBFGS, p, ...).  Synchronises `stream`.
 */
#define QAOA_LBFGS_MAX_M 16
int qaoa_optimize_lbfgs(int n, int dtype, void* psi_dev, void* lambda_dev, const qaoa_cost_t* cost,
                        double* angles_dev, int p, int64_t max_evals, int m, double gtol,
                        double* history_dev, double* info_dev, double* state_dev, int resume,
                        void* ws_dev, size_t ws_bytes, void* stream);

/*
 * Checkpoint / resume of the optimisers.  state_dev (optional, device,
 * qaoa_optimizer_state_size() bytes, caller-owned) holds the optimiser's whole
 * state: Adam's moments and step count, or the L-BFGS machine (point, gradient,
 * direction, step, pair history, counters).  With state_dev == NULL the state
 * lives in the workspace and every call starts afresh (resume must be 0).  With
 * resume = 1 the call continues from state_dev: saved angles plus saved state
 * give exactly the trajectory of one uninterrupted run (history rows of the
 * call are numbered from its own first step).  The state is a few KB; copying
 * it and the angles to host memory is the checkpoint.
 */
enum qaoa_optimizer { QAOA_OPTIMIZER_ADAM = 0, QAOA_OPTIMIZER_LBFGS = 1 };
int qaoa_optimizer_state_size(int kind, int p, size_t* bytes);

/* As qaoa_gradient, then synchronise and copy the 2p+2 doubles to out_host. */
int qaoa_gradient_host(int n, int dtype, void* psi_dev, void* lambda_dev,
                       const qaoa_cost_t* cost, const double* gamma, const double* beta, int p,
                       double* out_dev, double* out_host, void* ws_dev, size_t ws_bytes,
                       void* stream);

/*
 * Learned angle proposer: fused inference of a message-passing network that
 * maps each graph to 2p starting angles [gamma_1..p | beta_1..p] for the
 * optimisers above (the paper starts them from fixed schedules, Sec. II-A; the
 * network and its training are this library's addition).  With A the weighted
 * adjacency, d_v the degree and s_v = sum_u A_vu (float32 throughout):
 *   h_v = relu([d_v / 4, s_v / 2] W_in + b_in);
 *   QAOA_PROPOSER_LAYERS times: h_v = relu(h_v W_s + ((sum_u A_vu h_u) / max(1, d_v)) W_m + b);
 *   angles = relu([mean_v h_v, max_v h_v] W_1 + b_1) W_2 + b_2.
 * params_dev: qaoa_proposer_param_count(p) floats (device), row-major
 * (in x out) matrices in the order W_in (2 x H), b_in, (W_s, W_m (H x H), b) per
 * layer, W_1 (2H x H), b_1, W_2 (H x 2p), b_2, with H = QAOA_PROPOSER_HIDDEN.
 * graphs: host, n <= 32, any weights (checked as by qaoa_graph_check).
 * angles_dev: ngraphs x 2p doubles.  One CTA per graph, one launch; the graph
 * arrays are copied to ws_dev (qaoa_propose_workspace_size bytes) on `stream`.
 */
#define QAOA_PROPOSER_HIDDEN 64
#define QAOA_PROPOSER_LAYERS 3
int64_t qaoa_proposer_param_count(int p);
int qaoa_propose_workspace_size(int ngraphs, const qaoa_graph_t* graphs, size_t* bytes);
int qaoa_propose_angles(int ngraphs, const qaoa_graph_t* graphs, int p, const float* params_dev,
                        double* angles_dev, void* ws_dev, size_t ws_bytes, void* stream);

/*
 * Launch accounting (for benchmarks): number of kernels this library has
 * launched in this process since the last reset.  Host-only.
 */
int64_t qaoa_launch_count(void);
void qaoa_launch_count_reset(void);

/*
 * Per-kernel timing (for benchmarks).  While enabled, the library records a
 * CUDA event pair around every launch on the launching stream, by kernel
 * class: 0 = layer sweep, 1 = cost vector, 2 = sampling sweeps, 3 = small
 * reductions / tables / scans.  qaoa_timing_read() synchronises the recorded
 * events and writes, per class (arrays of 4, any may be NULL), the summed
 * milliseconds, the launch count and the algorithmic HBM bytes of those
 * launches (each state, lambda and cost-vector element read or written once
 * per launch), then clears them.  At most 65536 launches are recorded between
 * reads; later ones are counted in *dropped but not timed.
 */
int qaoa_timing_enable(int on);
int qaoa_timing_read(double* ms, int64_t* launches, double* bytes, int64_t* dropped);

/*
 * Batched adjoint gradients of many small graphs (the batched workload: thousands
 * of graphs of uneven n, each with its own angles).  Each graph gets exactly
 * what qaoa_gradient computes from |+>: [E, <psi|psi>, dE/dgamma_1..p,
 * dE/dbeta_1..p] (Eq. 1, Sec. IV-D).  Integer weights give int32 costs and
 * phase tables; if any graph has float weights, every graph gets float64 costs
 * (the weights in one common fixed point, summed exactly and rounded once, as
 * qaoa_cost_vector does) and directly computed phases.
 * Graphs on 2^12 tiles whose size has an all-lean one-graph plan (n >= 16
 * complex128, n >= 18 complex64) run grouped: each sweep of that plan is one
 * launch for all graphs of the size.  The rest run in one persistent launch per
 * tile size: each CTA takes the next graph (largest n first) and runs its whole
 * plan.  The paper evaluates graphs one at a time; batching is this library's
 * addition.
 *  graphs      ngraphs host descriptors (n <= QAOA_BATCH_MAX_N,
 *              m <= QAOA_BATCH_MAX_EDGES); checked as by qaoa_graph_check.
 *  angles      host, ngraphs x 2p doubles: row i = [gamma_1..p | beta_1..p]
 *              of graph i.  1 <= p <= QAOA_BATCH_MAX_P.
 *  tiles       optional host array of QAOA_MAX_N + 1 int32 indexed by n: 0 =
 *              2^10-amplitude tiles, 1 = 2^12 (NULL: 0 for n <= 10, else 1),
 *              e.g. from qaoa_batch_autotune.
 *  out_dev     device, ngraphs x (2p + 2) doubles, row i for graph i.
 *  ws_dev      at least qaoa_batch_workspace_size() bytes (256-byte aligned);
 *              it holds every graph's cost vector, state and lambda buffers.
 * Errors: QAOA_ERR_INVALID_ARG (a bad graph, angle or pointer),
 * QAOA_ERR_UNSUPPORTED (a graph past the limits),
 * QAOA_ERR_WORKSPACE.  The graph and angle arrays are read before the call
 * returns; the copy of them to the workspace is enqueued on `stream`.
 */
#define QAOA_BATCH_MAX_N 26
#define QAOA_BATCH_MAX_P 12
#define QAOA_BATCH_MAX_EDGES 512
#define QAOA_BATCH_MAX_GRAPHS (1 << 20)
int qaoa_batch_workspace_size(int dtype, int p, int ngraphs, const qaoa_graph_t* graphs,
                              const int32_t* tiles, size_t* bytes);
int qaoa_batch_gradient(int dtype, int ngraphs, const qaoa_graph_t* graphs, const double* angles,
                        int p, const int32_t* tiles, double* out_dev, void* ws_dev, size_t ws_bytes,
                        void* stream);

/*
 * Tile-size autotuner for qaoa_batch_gradient: for each n in [n_lo, n_hi]
 * times a batch of graphs_per_n synthetic graphs of n vertices (a ring plus
 * (u, u + 3) chords, integer weights 1..5) with 2^10 and with 2^12 tiles (one
 * warm-up run each, then one run timed with CUDA events on `stream`) and sets
 * tiles_out[n] (QAOA_MAX_N + 1 entries; entries outside [n_lo, n_hi] get the
 * default) to the faster.  ms_out (optional, 2 * (QAOA_MAX_N + 1) doubles)
 * receives the times at [2n + tile].  Synchronises `stream`.  Workspace:
 * qaoa_batch_autotune_workspace_size().
 */
int qaoa_batch_autotune_workspace_size(int dtype, int p, int n_hi, int graphs_per_n, size_t* bytes);
int qaoa_batch_autotune(int dtype, int p, int n_lo, int n_hi, int graphs_per_n, int32_t* tiles_out,
                        double* ms_out, void* ws_dev, size_t ws_bytes, void* stream);

/*
 * Constraint-preserving QAOA on a Hamming-weight subspace.  The paper names
 * constraint-preserving mixers that shrink the simulated search space as future
 * work (Sec. VI) without fixing one; this library takes the ring XY mixer of the
 * quantum alternating operator ansatz (Hadfield et al., Algorithms 12(2):34, 2019)
 * for the constraint popcount(z) = k (for MaxCut with k = n/2: graph bisection).
 *  - Feasible set F_k = {z in [0, 2^n) : popcount(z) = k}, binom(n, k) states.
 *    A subspace state holds binom(n, k) amplitudes (QAOA_C128 / QAOA_C64,
 *    interleaved as above) in RANK ORDER: the states of F_k by increasing z
 *    (rank(z) = sum_i binom(c_i, i) over the set bits c_1 < ... < c_k).
 *  - Layer l (Eq. 1 with the mixer replaced): psi_z *= exp(-i gamma_l C(z)), then
 *    the pair gates exp(-i beta_l (X_a X_b + Y_a Y_b) / 2) on the ring pairs
 *    (j, j+1 mod n) in parity order: even j < n-1, then odd j < n-1, then the
 *    closing pair (n-1, 0) (n = 2: the single pair (0, 1); n = 1: none).
 *  - init = 1 starts from the uniform superposition over F_k (Dicke state).
 *  - Arithmetic: complex64 states in float32 (phases from float64 angles reduced
 *    mod 2 pi).  complex128 states are float64 in memory; the forward layers
 *    gather tiles of up to 9 consecutive qubits into int64 fixed point with a
 *    scale of their own (value = integer x 2^-(56 - E), every component of the
 *    tile below 2^E, any state norm) and round each rotated part once, the
 *    adjoint pass likewise for psi and lambda (gradient terms as exact 128-bit
 *    products); the closing pair and the final reductions run in float64.
 * Limits: 1 <= n <= QAOA_XY_MAX_N, 0 <= k <= n, m <= QAOA_XY_MAX_EDGES; the
 * caller sizes every buffer with qaoa_xy_dim().  Graphs are validated as in
 * qaoa_graph_check() except for these limits.
 */
#define QAOA_XY_MAX_N 40
#define QAOA_XY_MAX_EDGES 1024

/* *dim = binom(n, k), the number of amplitudes and cost entries.  Host-only. */
int qaoa_xy_dim(int n, int k, int64_t* dim);

/*
 * Bytes of device scratch for qaoa_xy_apply_layers (depth p, integer cost span
 * cmax - cmin + 1 of the descriptor, 0 when there is no phase table) and, with
 * p = 0 and span 0, for qaoa_xy_expectation.  Host-only.
 */
int qaoa_xy_workspace_size(int n, int k, int dtype, int p, int64_t cost_span, size_t* bytes);

/*
 * Cost of every feasible state (Sec. IV-A restricted to F_k): C_dev[r] = C(z_r)
 * for the state z_r of rank r, binom(n, k) entries of cost_dtype.  Integer
 * weights: exact (int32 or float64).  Float weights: float64, quantised to one
 * common fixed point and summed exactly as qaoa_cost_vector does.  desc as in
 * qaoa_cost_vector (bounds are those of the whole cut, valid on F_k).  No
 * workspace.  Errors: QAOA_ERR_INVALID_ARG (bad graph, k, pointer or dtype).
 */
int qaoa_xy_cost_vector(const qaoa_graph_t* g, int k, void* C_dev, int cost_dtype, qaoa_cost_t* desc,
                        void* stream);

/*
 * p layers in place on a subspace state (see above); gamma/beta are host arrays
 * of p doubles.  expect_dev: optional device double[2] receiving [<C>, <psi|psi>]
 * of the final state (float64, fixed reduction order).  cost: a descriptor from
 * qaoa_xy_cost_vector for the same (n, k).  Errors: QAOA_ERR_INVALID_ARG (sizes,
 * pointers, non-finite angles, a workspace not 256-byte aligned),
 * QAOA_ERR_WORKSPACE (ws_bytes below qaoa_xy_workspace_size), QAOA_ERR_CUDA.
 */
int qaoa_xy_apply_layers(int n, int k, int dtype, void* psi_dev, const qaoa_cost_t* cost, const double* gamma,
                         const double* beta, int p, int init, double* expect_dev, void* ws_dev, size_t ws_bytes,
                         void* stream);

/* [<C>, <psi|psi>] of a subspace state into out_dev (device double[2]). */
int qaoa_xy_expectation(int n, int k, int dtype, const void* psi_dev, const qaoa_cost_t* cost, double* out_dev,
                        void* ws_dev, size_t ws_bytes, void* stream);

/* Bytes of device scratch for qaoa_xy_sample.  Host-only. */
int qaoa_xy_sample_workspace_size(int n, int k, size_t* bytes);

/*
 * Bitstring samples of a subspace state (the sampling of Sec. IV-D over F_k): with
 * P the running sum of |psi_r|^2 in rank order, shot i draws u_i from the same
 * SplitMix64 stream as qaoa_sample (seed, i) and takes the rank
 * r_i = min{r : P(r) > u_i P_total} (the last rank with nonzero probability when
 * rounding puts the target past the end); z_dev[i] receives the state of F_k with
 * that rank (a bitstring with k ones) and cost_dev[i] = C(z_i) from the subspace
 * cost vector.  Rank order is increasing z, so this equals qaoa_sample on the state
 * embedded in 2^n amplitudes.  Errors as for qaoa_sample; QAOA_ERR_WORKSPACE below
 * qaoa_xy_sample_workspace_size.
 */
int qaoa_xy_sample(int n, int k, int dtype, const void* psi_dev, const qaoa_cost_t* cost, int64_t shots,
                   uint64_t seed, uint64_t* z_dev, double* cost_dev, void* ws_dev, size_t ws_bytes, void* stream);

/* Bytes of device scratch for qaoa_xy_gradient (depth p, integer cost span as
 * for qaoa_xy_workspace_size).  Host-only. */
int qaoa_xy_gradient_workspace_size(int n, int k, int dtype, int p, int64_t cost_span, size_t* bytes);

/*
 * Adjoint gradient on F_k (the adjoint method of Sec. II-B and IV-C applied to the
 * subspace circuit): every gate is exp(-i theta H_g) -- the cost unitary of layer l
 * (H = diag(C), theta = gamma_l) and each ring pair gate (H = (X_a X_b + Y_a Y_b)/2,
 * theta = beta_l) -- and dE/dtheta_g = 2 Im <lambda_g|H_g|psi_g> with psi_g the
 * state right after gate g and lambda_g the later gates undone on C psi_final.
 * The call runs the p forward layers from the Dicke state into psi_dev, sets
 * lambda = C psi in lam_dev (two distinct buffers of binom(n, k) amplitudes,
 * caller-owned), then walks the gates backwards, undoing each on both buffers
 * after taking its term.  out_dev (device, 2p + 2 doubles): [E, <psi|psi>,
 * dE/dgamma_1..p, dE/dbeta_1..p]; psi_dev ends back at the Dicke state (up to
 * rounding).  Every sum is float64 with a fixed order.  Errors as for
 * qaoa_xy_apply_layers, QAOA_ERR_WORKSPACE below
 * qaoa_xy_gradient_workspace_size.
 */
int qaoa_xy_gradient(int n, int k, int dtype, void* psi_dev, void* lam_dev, const qaoa_cost_t* cost,
                     const double* gamma, const double* beta, int p, double* out_dev, void* ws_dev, size_t ws_bytes,
                     void* stream);

#ifdef __cplusplus
}
#endif

#endif /* QAOA_GB300_H */
