// Batched product kernel, fp32 working precision.
#include "batch_kern.cuh"

namespace hodlr {

cudaError_t launch_batch_f32(int grid, int threads, const BItem* items, const int32_t* first, const int32_t* list,
                             cudaStream_t s) {
  return launch_batch_w<float>(grid, threads, items, first, list, s);
}

}  // namespace hodlr
