// Batched product kernel, fp64 working precision.
#include "batch_kern.cuh"

namespace hodlr {

cudaError_t launch_batch_f64(int grid, int threads, const BItem* items, const int32_t* first, const int32_t* list,
                             cudaStream_t s) {
  return launch_batch_w<double>(grid, threads, items, first, list, s);
}

}  // namespace hodlr
