// Partitioned product kernels, fp32 working precision.
#include "batch_kern.cuh"

namespace hodlr {

cudaError_t launch_part_f32(int step, const BItem& b, int lf0, int lf1, int grid, int threads, cudaStream_t s) {
  return launch_part_w<float>(step, b, lf0, lf1, grid, threads, s);
}

}  // namespace hodlr
