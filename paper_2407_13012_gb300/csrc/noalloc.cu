// qaoa_expectation_noalloc: the expectation value without a caller-supplied workspace.
//
// Some callers cannot call cudaMalloc: code that runs where the allocator is off
// limits (inside a custom allocator, a memory-pool callback or a signal/teardown
// path), hosts that hand out only fixed buffers, or embedders whose device memory
// is entirely owned by another framework.  For them this entry point takes its
// reduction scratch from a fixed array in device global memory that the library
// defines at file scope.  The array is created when the library is loaded on a
// GPU and every GPU that loads the library holds it until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"

namespace {

// Reduction partials for qaoa_expectation (2 outputs x 8 slots x 2048 blocks doubles,
// 256 KiB): the workspace qaoa_expectation itself needs, without the host-result slot.
constexpr size_t kScratchBytes = qaoa::kExpectPartialBytes;
static __device__ __align__(256) unsigned char g_expect_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[64] = {};  // per device: device address of g_expect_scratch

// Host code cannot use &g_expect_scratch as a device pointer (it names a host-side
// stand-in); ask the runtime for the device address once per device.
int scratch_for_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return QAOA_ERR_CUDA;
  if (dev < 0 || dev >= 64) return QAOA_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_expect_scratch) != cudaSuccess || p == nullptr) return QAOA_ERR_CUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return QAOA_OK;
}

}  // namespace

extern "C" int qaoa_expectation_noalloc(int n, int dtype, const void* psi_dev, const qaoa_cost_t* cost,
                                        double* out_dev, void* stream) {
  size_t need = 0;
  int rc = qaoa_workspace_size(n, dtype, QAOA_OP_EXPECTATION, 0, 0, 0, &need);
  if (rc) return rc;
  // the reported size is qaoa_expectation's partials plus qaoa_expectation_host's result slot
  if (need - qaoa::kHostResultBytes > kScratchBytes) return QAOA_ERR_UNSUPPORTED;
  void* scratch = nullptr;
  rc = scratch_for_current_device(&scratch);
  if (rc) return rc;
  // Every slot of the scratch that qaoa_expectation reads is written earlier in the
  // same call, so nothing has to be cleared between calls.
  return qaoa_expectation(n, dtype, psi_dev, cost, out_dev, scratch, kScratchBytes, stream);
}
