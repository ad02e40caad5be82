// The complex128 batched kernel on 2^12-amplitude tiles with the lean tile code, in a
// translation unit of its own so that it compiles in parallel with the rest.
#include "batch_kernel.cuh"

namespace qaoa {

cudaError_t launch_batch_c128_large(const BatchArgs& b, int first, int count, int* queue, cudaStream_t s) {
  return launch_batch_cfg<CfgXB, true, true>(b, first, count, queue, s);
}

}  // namespace qaoa
