// Batched adjoint gradients: thousands of small graphs (n ~ 8..20).
//
// The per-graph computation is the plain method (cost vector, Eq. 1's p layers, <C>, and
// the adjoint gradient of Sec. IV-D); only the scheduling differs from the one-graph path.
// One prep launch builds every graph's cost vector and tables.  Then the graphs run in one
// of two ways, by size (the host decides, capi.cu):
//  * grouped sweeps (the larger graphs, whose one-graph plan is all lean sweeps): the graphs
//    of one size run the one-graph gradient plan together, each sweep one launch of the
//    one-graph lean kernel over all of them, each block on its own graph's tiles, tables and
//    angles (GroupSlot), then one reduction per size;
//  * the persistent kernel below (the rest): one CTA owns one graph at a time and runs the
//    graph's whole sweep plan over the graph's own buffers, tile after tile, with CTA
//    barriers between sweeps, writing the graph's outputs from its block accumulators.
//    complex128 sweeps on full 2^12 tiles use the lean tile code, the rest the generic
//    program (for complex64 the lean form spilled and measured slower).  Graphs come off a
//    work counter largest first (longest-processing-time order).  Small graphs (n <= 10)
//    run on 2^10-amplitude tiles, larger ones on 2^12; the host may pick per qubit count
//    from measured times.
#include "batch_kernel.cuh"

namespace qaoa {
namespace {

constexpr int kPrepThreads = 256;
constexpr int kMaxBatchEdges = 512;
static_assert(QAOA_BATCH_MAX_EDGES <= kMaxBatchEdges, "edge staging holds every edge of a graph");
static_assert(QAOA_BATCH_MAX_N < 32, "cost-vector indices in 32 bits");

// One launch prepares every graph: blocks [0, cost_blocks) build the cost vectors (2^12
// entries per block, C(z) = sum over edges of w [z_u != z_v], Sec. III-B's MaxCut cost, int32
// for integer weights; float weights are quantised once to a common fixed point,
// 2^-(62 - e) with sum |w| < 2^e, summed exactly in int64 and rounded once to float64, as the
// one-graph cost kernel does); the next ngraphs blocks build each graph's per-layer terms and
// tables; the last block (fixed point) builds the shared turn tables.
__global__ void __launch_bounds__(kPrepThreads) batch_prep_kernel(const __grid_constant__ BatchArgs b,
                                                                   int64_t cost_blocks) {
  __shared__ int2 e_s[kMaxBatchEdges];
  __shared__ int wi_s[kMaxBatchEdges];        // integer weights
  __shared__ long long wq_s[kMaxBatchEdges];  // float weights in fixed point
  __shared__ int shift_s;
  const int64_t blk = blockIdx.x;
  const int tid = threadIdx.x;
  const int p = b.p;
  const bool fx = b.dtype == QAOA_C128;
  if (blk < cost_blocks) {
    int lo = 0, hi = b.ngraphs - 1;  // last graph with blk_off <= blk
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (b.blk_off[mid] <= blk) lo = mid;
      else hi = mid - 1;
    }
    const BatchGraph G = b.graphs[lo];
    if (tid == 0) {
      int sh = 0;
      if (b.cost_f64) {  // sum |w| in edge order, as the host does for the one-graph kernel
        double sa = 0.0;
        for (int k = 0; k < G.m; ++k) sa += fabs(b.ew[G.edge + k]);
        int e2 = 0;
        frexp(sa > 0.0 ? sa : 1.0, &e2);
        sh = 62 - e2;
      }
      shift_s = sh;
    }
    __syncthreads();
    for (int k = tid; k < G.m; k += kPrepThreads) {
      e_s[k] = make_int2(b.edges[2 * (G.edge + k)], b.edges[2 * (G.edge + k) + 1]);
      const double w = b.ew[G.edge + k];
      if (b.cost_f64) wq_s[k] = llrint(ldexp(w, shift_s));
      else wi_s[k] = (int)w;
    }
    __syncthreads();
    // n <= QAOA_BATCH_MAX_N < 32: 32-bit indices
    const uint32_t z0 = (uint32_t)(blk - b.blk_off[lo]) << kBatchCostBits;
    const uint32_t zend = min(z0 + (1u << kBatchCostBits), 1u << G.n);
    if (b.cost_f64) {
      for (uint32_t z = z0 + tid; z < zend; z += kPrepThreads) {
        long long c = 0;
        for (int k = 0; k < G.m; ++k)
          if (((z >> e_s[k].x) ^ (z >> e_s[k].y)) & 1u) c += wq_s[k];
        ((double*)b.C)[G.cost + (int64_t)z] = ldexp((double)c, -shift_s);
      }
    } else {
      for (uint32_t z = z0 + tid; z < zend; z += kPrepThreads) {
        int c = 0;
        for (int k = 0; k < G.m; ++k) c += (int)(((z >> e_s[k].x) ^ (z >> e_s[k].y)) & 1u) * wi_s[k];
        ((int*)b.C)[G.cost + (int64_t)z] = c;
      }
    }
    return;
  }
  const int64_t gi = blk - cost_blocks;
  if (gi < b.ngraphs) {
    const BatchGraph G = b.graphs[gi];
    const double* ang = b.angles + gi * 2 * p;
    double* trig = b.trig + gi * 3 * p;
    for (int l = tid; l < p; l += kPrepThreads) {
      trig[l] = ang[l] / (2.0 * 3.141592653589793238);
      double sn, cs;
      sincos(ang[p + l], &sn, &cs);
      trig[p + l] = cs;
      trig[2 * p + l] = sn;
    }
    const int64_t nph = (int64_t)p * G.span;
    for (int64_t i = tid; i < nph; i += kPrepThreads) {
      const int l = (int)(i / G.span);
      const double th = ang[l] * (double)(G.cmin + (i - (int64_t)l * G.span));
      if (fx) ((longlong2*)b.phase)[G.table + i] = unit_q62(th);
      else ((float2*)b.phase)[G.table + i] = unit_f32(th);
    }
    if (fx)
      for (int i = tid; i < p * 196; i += kPrepThreads)
        ((longlong2*)b.dtab)[gi * p * 196 + i] = d_entry(ang[p + i / 196], i % 196);
    return;
  }
  if (fx)
    for (int j = tid; j < 3 * 1024; j += kPrepThreads) ((longlong2*)b.turn)[j] = turn_entry(j);
}

// The persistent kernel: graphs [first, first + count) of the processing order, taken from
// *queue one at a time by each CTA.
}  // namespace

int batch_tile_bits(int tile) { return tile == 0 ? CfgXS::B : CfgXB::B; }
int batch_register_bits(int dtype, int tile) {
  if (tile == 0) return dtype == QAOA_C128 ? CfgXS::RB : CfgFS::RB;
  return dtype == QAOA_C128 ? CfgXB::RB : CfgFB::RB;
}

cudaError_t launch_batch_prep(const BatchArgs& b, int64_t cost_blocks, cudaStream_t s) {
  const int64_t blocks = cost_blocks + b.ngraphs + 1;
  note_launch(1, s, true);
  batch_prep_kernel<<<(unsigned)blocks, kPrepThreads, 0, s>>>(b, cost_blocks);
  note_launch(1, s, false);
  return cudaGetLastError();
}

cudaError_t launch_batch(const BatchArgs& b, int tile, int first, int count, int* queue, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  note_launch(0, s, true);
  cudaError_t e;
  if (b.dtype == QAOA_C128)
    e = tile == 0 ? launch_batch_cfg<CfgXS, true, false>(b, first, count, queue, s)
                  : launch_batch_c128_large(b, first, count, queue, s);
  else
    e = tile == 0 ? launch_batch_cfg<CfgFS, false, false>(b, first, count, queue, s)
                  : launch_batch_cfg<CfgFB, false, false>(b, first, count, queue, s);
  note_launch(0, s, false);
  return e;
}

}  // namespace qaoa
