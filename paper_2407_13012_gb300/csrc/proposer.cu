// Learned angle proposer: fused inference of a small message-passing network that maps a
// weighted graph to 2p QAOA angles [gamma_1..p, beta_1..p] (a warm start for the optimiser;
// the paper starts from fixed schedules such as the linear ramp of Sec. II-A).
//
// Network (hidden width H = 64, float32), for a graph with n <= 32 vertices, adjacency
// weights A (A_uv = w_uv), degree d_v and weighted degree s_v = sum_u A_uv:
//   x_v   = [d_v / 4, s_v / 2]
//   h_v   = relu(x_v W_in + b_in)
//   3 x:  m_v = (sum_u A_vu h_u) / max(1, d_v);  h_v = relu(h_v W_s + m_v W_m + b)
//   g     = [mean_v h_v, max_v h_v]
//   out   = relu(g W_1 + b_1) W_2 + b_2                       (2p values)
// Parameters are one float32 vector, row-major matrices (in x out) in the order
// W_in, b_in, (W_s, W_m, b) x 3, W_1, b_1, W_2, b_2.
// One CTA runs one graph: the adjacency and the activations live in shared memory and the
// whole network is one launch for all graphs.
#include "internal.h"

#include <cuda_runtime.h>

namespace qaoa {
namespace {

constexpr int kH = QAOA_PROPOSER_HIDDEN;
constexpr int kNMax = 32;
constexpr int kPT = 128;  // threads per CTA

struct Offs {
  int win, bin, ws[QAOA_PROPOSER_LAYERS], wm[QAOA_PROPOSER_LAYERS], b[QAOA_PROPOSER_LAYERS], w1, b1, w2, b2, total;
};
__host__ __device__ inline Offs offsets(int p) {
  Offs o;
  int k = 0;
  o.win = k;
  k += 2 * kH;
  o.bin = k;
  k += kH;
  for (int l = 0; l < QAOA_PROPOSER_LAYERS; ++l) {
    o.ws[l] = k;
    k += kH * kH;
    o.wm[l] = k;
    k += kH * kH;
    o.b[l] = k;
    k += kH;
  }
  o.w1 = k;
  k += 2 * kH * kH;
  o.b1 = k;
  k += kH;
  o.w2 = k;
  k += kH * 2 * p;
  o.b2 = k;
  k += 2 * p;
  o.total = k;
  return o;
}

__global__ void __launch_bounds__(kPT) propose_kernel(const __grid_constant__ ProposeArgs a) {
  __shared__ float A[kNMax][kNMax + 1];
  __shared__ float deg[kNMax], wdeg[kNMax];
  __shared__ float h[kNMax][kH], m[kNMax][kH], t[kNMax][kH];
  __shared__ float gvec[2 * kH], zvec[kH];
  const int gi = blockIdx.x, tid = threadIdx.x;
  const int n = a.n[gi];
  const int64_t e0 = a.edge_off[gi], e1 = a.edge_off[gi + 1];
  const Offs o = offsets(a.p);
  const float* P = a.params;
  for (int i = tid; i < kNMax * (kNMax + 1); i += kPT) (&A[0][0])[i] = 0.f;
  if (tid < kNMax) deg[tid] = 0.f;
  __syncthreads();
  for (int64_t e = e0 + tid; e < e1; e += kPT) {
    const int u = a.uv[2 * e], v = a.uv[2 * e + 1];
    const float w = (float)a.w[e];
    A[u][v] = w;
    A[v][u] = w;
    atomicAdd(&deg[u], 1.f);  // integer counts: exact in any order
    atomicAdd(&deg[v], 1.f);
  }
  __syncthreads();
  if (tid < n) {
    float s = 0.f;
    for (int u = 0; u < n; ++u) s += A[tid][u];
    wdeg[tid] = s;
  }
  __syncthreads();
  // input layer
  for (int idx = tid; idx < n * kH; idx += kPT) {
    const int v = idx / kH, j = idx % kH;
    const float x0 = deg[v] * 0.25f, x1 = wdeg[v] * 0.5f;
    h[v][j] = fmaxf(0.f, fmaf(x0, __ldg(P + o.win + j), fmaf(x1, __ldg(P + o.win + kH + j), __ldg(P + o.bin + j))));
  }
  __syncthreads();
  for (int l = 0; l < QAOA_PROPOSER_LAYERS; ++l) {
    for (int idx = tid; idx < n * kH; idx += kPT) {  // neighbour mean
      const int v = idx / kH, k = idx % kH;
      float s = 0.f;
      for (int u = 0; u < n; ++u) s = fmaf(A[v][u], h[u][k], s);
      m[v][k] = s / fmaxf(1.f, deg[v]);
    }
    __syncthreads();
    for (int idx = tid; idx < n * kH; idx += kPT) {
      const int v = idx / kH, j = idx % kH;
      float s = __ldg(P + o.b[l] + j);
      for (int k = 0; k < kH; ++k) {
        s = fmaf(h[v][k], __ldg(P + o.ws[l] + k * kH + j), s);
        s = fmaf(m[v][k], __ldg(P + o.wm[l] + k * kH + j), s);
      }
      t[v][j] = fmaxf(0.f, s);
    }
    __syncthreads();
    for (int idx = tid; idx < n * kH; idx += kPT) h[idx / kH][idx % kH] = t[idx / kH][idx % kH];
    __syncthreads();
  }
  // readout
  if (tid < kH) {
    float s = 0.f, mx = 0.f;  // activations are >= 0
    for (int v = 0; v < n; ++v) {
      s += h[v][tid];
      mx = fmaxf(mx, h[v][tid]);
    }
    gvec[tid] = s / (float)n;
    gvec[kH + tid] = mx;
  }
  __syncthreads();
  if (tid < kH) {
    float s = __ldg(P + o.b1 + tid);
    for (int k = 0; k < 2 * kH; ++k) s = fmaf(gvec[k], __ldg(P + o.w1 + k * kH + tid), s);
    zvec[tid] = fmaxf(0.f, s);
  }
  __syncthreads();
  const int np2 = 2 * a.p;
  if (tid < np2) {
    float s = __ldg(P + o.b2 + tid);
    for (int k = 0; k < kH; ++k) s = fmaf(zvec[k], __ldg(P + o.w2 + k * np2 + tid), s);
    a.angles[(int64_t)gi * np2 + tid] = (double)s;
  }
}

}  // namespace

int64_t proposer_param_count(int p) { return offsets(p).total; }

cudaError_t launch_propose(const ProposeArgs& a, int ngraphs, cudaStream_t s) {
  if (ngraphs <= 0) return cudaSuccess;
  note_launch(3, s, true);
  propose_kernel<<<ngraphs, kPT, 0, s>>>(a);
  note_launch(3, s, false);
  return cudaGetLastError();
}

}  // namespace qaoa
