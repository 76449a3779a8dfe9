// On-the-fly FP64 dense kernel-matrix product b = A x (a checker for HODLR
// products at sizes where A cannot be stored).  Entries A_ij = f(r_ij) +
// diag*delta_ij of the eq. (4.1) kernels and the synthetic workloads are
// generated in registers and never stored.  One warp per output row; lanes
// stride over the columns j, then a fixed shuffle tree: deterministic.
#include "hodlr_internal.cuh"

namespace hodlr {

namespace {

constexpr int kDenseThreads = 256;
constexpr int kDenseCols = 8;  // right-hand sides per pass

__global__ void __launch_bounds__(kDenseThreads)
dense_kernel_matvec_kernel(int n, int dim, const double* __restrict__ pts, int kind, double c,
                           double len2, double diag, int nrows, const int32_t* __restrict__ rows,
                           int nrhs, const double* __restrict__ X, int64_t ldx,
                           double* __restrict__ B, int64_t ldb) {
  const int warp = (blockIdx.x * kDenseThreads + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= nrows) return;
  const int i = rows ? rows[warp] : warp;
  if (i < 0 || i >= n) {  // an invalid row index yields NaN, never an out-of-range read
    for (int q = lane; q < nrhs; q += 32) B[(int64_t)warp * ldb + q] = __longlong_as_double(0x7ff8000000000000ll);
    return;
  }
  for (int c0 = 0; c0 < nrhs; c0 += kDenseCols) {
    const int nc = min(kDenseCols, nrhs - c0);
    double acc[kDenseCols];
#pragma unroll
    for (int q = 0; q < kDenseCols; ++q) acc[q] = 0.0;
    for (int j = lane; j < n; j += 32) {
      const double a = kernel_entry(pts, dim, i, j, kind, c, len2, diag);
      const double* xr = X + (int64_t)j * ldx + c0;
#pragma unroll
      for (int q = 0; q < kDenseCols; ++q)
        if (q < nc) acc[q] = fma(a, xr[q], acc[q]);
    }
#pragma unroll
    for (int q = 0; q < kDenseCols; ++q) {
      double v = acc[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0 && q < nc) B[(int64_t)warp * ldb + c0 + q] = v;
    }
  }
}

}  // namespace

cudaError_t launch_dense_kernel_matvec(int n, int dim, const double* pts, int kind, double c,
                                       double len2, double diag, int nrows, const int32_t* rows,
                                       int nrhs, const double* X, int64_t ldx, double* B,
                                       int64_t ldb, cudaStream_t s) {
  const int warps_per_block = kDenseThreads / 32;
  const int grid = (nrows + warps_per_block - 1) / warps_per_block;
  dense_kernel_matvec_kernel<<<grid, kDenseThreads, 0, s>>>(n, dim, pts, kind, c, len2, diag,
                                                            nrows, rows, nrhs, X, ldx, B, ldb);
  return cudaGetLastError();
}

}  // namespace hodlr
