// Import-time kernels: block norms for the precision rule (Algorithm 3.2,
// the nrm / nrmAll quantities) and conversion of the fp64 generators into
// their storage formats (Algorithm 3.2, "store U, V in u_k"; leaves in u).
#include "hodlr_internal.cuh"

namespace hodlr {

namespace {

constexpr int kNormThreads = 256;

// One CTA per task: sum of squares and max |x| of `count` consecutive fp64
// values.  Fixed per-thread order plus a fixed tree: deterministic.
__global__ void __launch_bounds__(kNormThreads)
norms_kernel(const double* __restrict__ staging, const NormTask* __restrict__ tasks,
             double* __restrict__ sumsq, double* __restrict__ amax) {
  __shared__ double s_sum[kNormThreads];
  __shared__ double s_max[kNormThreads];
  const NormTask t = tasks[blockIdx.x];
  const double* p = staging + t.src;
  double acc = 0.0, mx = 0.0;
  for (int64_t i = threadIdx.x; i < t.count; i += kNormThreads) {
    double v = p[i];
    acc = fma(v, v, acc);
    mx = fmax(mx, fabs(v));
  }
  s_sum[threadIdx.x] = acc;
  s_max[threadIdx.x] = mx;
  __syncthreads();
  for (int w = kNormThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      s_sum[threadIdx.x] += s_sum[threadIdx.x + w];
      s_max[threadIdx.x] = fmax(s_max[threadIdx.x], s_max[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    sumsq[blockIdx.x] = s_sum[0];
    amax[blockIdx.x] = s_max[0];
  }
}

// One CTA per column: rows of the fp64 staging (row-major, stride
// src_stride) -> one contiguous padded column of the pool, rounded to the
// column's format after multiplying by the block's power-of-two scale.
__global__ void pack_kernel(const double* __restrict__ staging, const PackTask* __restrict__ tasks,
                            uint8_t* __restrict__ pool) {
  const PackTask t = tasks[blockIdx.x];
  const int eb = prec_bytes(t.prec);
  for (int p = threadIdx.x; p < t.pm; p += blockDim.x) {
    double v = p < t.m ? staging[t.src + (int64_t)p * t.src_stride] * t.scale : 0.0;
    store1(pool + t.dst + (int64_t)p * eb, t.prec, v);
  }
}

// Inverse of pack_kernel: decoded value / scale back into the staging.
__global__ void unpack_kernel(const uint8_t* __restrict__ pool, const PackTask* __restrict__ tasks,
                              double* __restrict__ staging) {
  const PackTask t = tasks[blockIdx.x];
  const int eb = prec_bytes(t.prec);
  for (int p = threadIdx.x; p < t.m; p += blockDim.x) {
    double v = load1_f64(pool + t.dst + (int64_t)p * eb, t.prec);
    staging[t.src + (int64_t)p * t.src_stride] = v / t.scale;
  }
}

}  // namespace

cudaError_t launch_norms(const double* staging, const NormTask* tasks, int ntasks,
                         double* sumsq, double* amax, cudaStream_t s) {
  if (ntasks == 0) return cudaSuccess;
  norms_kernel<<<ntasks, kNormThreads, 0, s>>>(staging, tasks, sumsq, amax);
  return cudaGetLastError();
}

cudaError_t launch_pack(const double* staging, const PackTask* tasks, int ntasks, uint8_t* pool,
                        cudaStream_t s) {
  if (ntasks == 0) return cudaSuccess;
  pack_kernel<<<ntasks, 128, 0, s>>>(staging, tasks, pool);
  return cudaGetLastError();
}

cudaError_t launch_unpack(const uint8_t* pool, const PackTask* tasks, int ntasks, double* staging,
                          cudaStream_t s) {
  if (ntasks == 0) return cudaSuccess;
  unpack_kernel<<<ntasks, 128, 0, s>>>(pool, tasks, staging);
  return cudaGetLastError();
}

}  // namespace hodlr
