// Import-time kernels: block norms for the precision rule (Algorithm 3.2,
// the nrm / nrmAll quantities) and conversion of the fp64 generators into
// their storage formats (Algorithm 3.2, "store U, V in u_k"; leaves in u).
#include <algorithm>

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

// One warp per column segment: rows of the fp64 staging (row-major, stride
// src_stride) -> one contiguous padded column segment of the pool, rounded
// to the column's format after multiplying by the block's power-of-two scale.
constexpr int kPackWarps = 8;

__global__ void pack_kernel(const double* __restrict__ staging, const PackTask* __restrict__ tasks,
                            int ntasks, uint8_t* __restrict__ pool) {
  const int task = blockIdx.x * kPackWarps + (threadIdx.x >> 5);
  if (task >= ntasks) return;
  const PackTask t = tasks[task];
  const int eb = prec_bytes(t.prec);
  const int64_t ds = t.dst_stride ? t.dst_stride : eb;
  for (int p = threadIdx.x & 31; p < t.pm; p += 32) {
    double v = p < t.m ? staging[t.src + (int64_t)p * t.src_stride] * t.scale : 0.0;
    store1(pool + t.dst + (int64_t)p * ds, t.prec, v);
  }
}

// Inverse of pack_kernel: decoded value / scale back into the staging.
__global__ void unpack_kernel(const uint8_t* __restrict__ pool, const PackTask* __restrict__ tasks,
                              int ntasks, double* __restrict__ staging) {
  const int task = blockIdx.x * kPackWarps + (threadIdx.x >> 5);
  if (task >= ntasks) return;
  const PackTask t = tasks[task];
  const int eb = prec_bytes(t.prec);
  const int64_t ds = t.dst_stride ? t.dst_stride : eb;
  for (int p = threadIdx.x & 31; p < t.m; p += 32) {
    double v = load1_f64(pool + t.dst + (int64_t)p * ds, t.prec);
    staging[t.src + (int64_t)p * t.src_stride] = v / t.scale;
  }
}

// 32-bit words at given byte offsets (tile headers).
__global__ void put_words_kernel(uint8_t* __restrict__ pool, const int64_t* __restrict__ off,
                                 const uint32_t* __restrict__ val, int64_t count) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x)
    *reinterpret_cast<uint32_t*>(pool + off[e]) = val[e];
}

}  // namespace

cudaError_t launch_put_words(uint8_t* pool, const int64_t* off, const uint32_t* val, int64_t count,
                             cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  put_words_kernel<<<(int)std::min<int64_t>((count + 255) / 256, 4096), 256, 0, s>>>(pool, off, val, count);
  return cudaGetLastError();
}

cudaError_t launch_norms(const double* staging, const NormTask* tasks, int ntasks,
                         double* sumsq, double* amax, cudaStream_t s) {
  if (ntasks == 0) return cudaSuccess;
  norms_kernel<<<ntasks, kNormThreads, 0, s>>>(staging, tasks, sumsq, amax);
  return cudaGetLastError();
}

cudaError_t launch_pack(const double* staging, const PackTask* tasks, int ntasks, uint8_t* pool,
                        cudaStream_t s) {
  if (ntasks == 0) return cudaSuccess;
  pack_kernel<<<(ntasks + kPackWarps - 1) / kPackWarps, 32 * kPackWarps, 0, s>>>(staging, tasks, ntasks, pool);
  return cudaGetLastError();
}

cudaError_t launch_unpack(const uint8_t* pool, const PackTask* tasks, int ntasks, double* staging,
                          cudaStream_t s) {
  if (ntasks == 0) return cudaSuccess;
  unpack_kernel<<<(ntasks + kPackWarps - 1) / kPackWarps, 32 * kPackWarps, 0, s>>>(pool, tasks, ntasks, staging);
  return cudaGetLastError();
}

}  // namespace hodlr
