// Batched adjoint gradients: thousands of small graphs (n ~ 8..20) in one persistent launch.
//
// The per-graph computation is the plain method (cost vector, Eq. 1's p layers, <C>, and
// the adjoint gradient of Sec. IV-D); only the scheduling differs from the one-graph path.
// One CTA owns one graph at a time: it runs the graph's whole sweep plan over the graph's
// own state buffers, tile after tile, with CTA barriers between sweeps, and writes the
// graph's outputs from its block accumulators, so no launch boundary or cross-CTA reduction
// separates the sweeps.  complex128 sweeps on full 2^12 tiles use the lean tile code
// (compile-time layout sequences; forward sweeps on psi alone), the rest the generic
// program (for complex64 the lean form spilled and measured slower).  Graphs come off a work counter largest first, which balances the
// CTAs (longest-processing-time order).  Small graphs (n <= 10) run on 2^10-amplitude tiles,
// larger ones on 2^12; the host may pick per qubit count from measured times.
#include "batch_kernel.cuh"

namespace qaoa {
namespace {

constexpr int kPrepThreads = 256;
constexpr int kMaxBatchEdges = 512;

// One launch prepares every graph: blocks [0, cost_blocks) build the cost vectors (2^12
// entries per block, C(z) = sum over edges of w [z_u != z_v], Sec. III-B's MaxCut cost,
// int32 for integer weights, else float64 summed in edge order);
// the next ngraphs blocks build each graph's per-layer terms and tables; the last block
// (fixed point) builds the shared turn tables.
__global__ void __launch_bounds__(kPrepThreads) batch_prep_kernel(const __grid_constant__ BatchArgs b,
                                                                   int64_t cost_blocks) {
  __shared__ int2 e_s[kMaxBatchEdges];
  __shared__ double w_s[kMaxBatchEdges];
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
    for (int k = tid; k < G.m; k += kPrepThreads) {
      e_s[k] = make_int2(b.edges[2 * (G.edge + k)], b.edges[2 * (G.edge + k) + 1]);
      w_s[k] = b.ew[G.edge + k];
    }
    __syncthreads();
    const uint64_t z0 = (uint64_t)(blk - b.blk_off[lo]) << kBatchCostBits;
    const uint64_t zend = 1ull << G.n;
    for (uint64_t z = z0 + tid; z < z0 + (1ull << kBatchCostBits) && z < zend; z += kPrepThreads) {
      if (b.cost_f64) {  // float64 sum in edge order
        double c = 0.0;
        for (int k = 0; k < G.m; ++k)
          if (((z >> e_s[k].x) ^ (z >> e_s[k].y)) & 1ull) c += w_s[k];
        ((double*)b.C)[G.cost + (int64_t)z] = c;
      } else {
        int c = 0;
        for (int k = 0; k < G.m; ++k)
          if (((z >> e_s[k].x) ^ (z >> e_s[k].y)) & 1ull) c += (int)w_s[k];
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
