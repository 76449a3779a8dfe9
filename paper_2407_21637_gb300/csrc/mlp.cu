// Block-rank predictor: a 11-64-64-64-1 multilayer perceptron (relu hidden
// layers, fp16 weights, fp32 arithmetic) that predicts log2(rank + 1) of an
// off-diagonal block from features computed from a few of its generated
// entries, to size the first sketch of hodlr_build (the adaptive rule still
// decides every rank; a block whose sketch falls short is redone).
//
// Parameter vector (P = 9153): W1 (64 x 11, row-major), b1 (64), W2 (64 x 64),
// b2, W3 (64 x 64), b3, W4 (1 x 64), b4 (1).
//
//  features  per block (k, i): k / 12, log2(m) / 20, log10(eps) / 10 and the
//            log10 of eight row norms of the block (rows (2j + 1) m / 16,
//            all of its columns) over the largest of them, / 10;
//  forward   one warp per sample (two hidden units per lane, inputs broadcast
//            by shuffles), the weights in shared memory;
//  backward  per-sample deltas, then one thread per parameter summing over
//            the samples in order (no atomics: reproducible);
//  adam      one thread per parameter on fp32 master weights, fp16 copy.
#include <algorithm>
#include <cmath>
#include <vector>

#include "handle.cuh"

namespace hodlr {
namespace {

constexpr int kIn = 11, kHid = 64;
constexpr int kP = kHid * kIn + kHid + 2 * (kHid * kHid + kHid) + kHid + 1;   // 9153
constexpr int oW1 = 0, oB1 = oW1 + kHid * kIn, oW2 = oB1 + kHid, oB2 = oW2 + kHid * kHid, oW3 = oB2 + kHid,
              oB3 = oW3 + kHid * kHid, oW4 = oB3 + kHid, oB4 = oW4 + kHid;
static_assert(oB4 + 1 == kP, "parameter layout");
constexpr int kAct = 3 * kHid;   // saved pre-activations z1, z2, z3 per sample

struct FBlock {
  int32_t r0, m, c0, mc, k;
};

// features of one block per CTA
__global__ void __launch_bounds__(256) features_kernel(const double* __restrict__ pts, int dim, int kind, double c,
                                                       double len2, double diag, const FBlock* __restrict__ blocks,
                                                       double eps, float* __restrict__ feat) {
  __shared__ double red[8][8];
  const FBlock b = blocks[blockIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // warp j: the norm of row (2j + 1) m / 16 of the block
  const int row = b.r0 + (int)(((int64_t)(2 * warp + 1) * b.m) / 16);
  double s = 0.0;
  for (int j = lane; j < b.mc; j += 32) {
    const double a = kernel_entry(pts, dim, row, b.c0 + j, kind, c, len2, diag);
    s = fma(a, a, s);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) red[warp][0] = sqrt(s);
  __syncthreads();
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int j = 0; j < 8; ++j) mx = fmax(mx, red[j][0]);
    float* f = feat + (int64_t)blockIdx.x * kIn;
    f[0] = (float)(b.k / 12.0);
    f[1] = (float)(log2((double)b.m) / 20.0);
    f[2] = (float)(log10(eps) / 10.0);
    for (int j = 0; j < 8; ++j) f[3 + j] = (float)(log10(red[j][0] / (mx > 0.0 ? mx : 1.0) + 1e-30) / 10.0);
  }
}

// One warp per sample: lane l holds hidden units l and l + 32; the inputs of
// a layer are broadcast from their lanes by shuffles, and every sum runs
// over its inputs in ascending order from the bias (the order of the
// layer definitions).  Weight matrices sit transposed in shared memory
// (input-major), so the lanes of one input read consecutive words.
constexpr int kMlpThreads = 256;

__device__ __forceinline__ int mlp_wt(int p) {   // parameter index -> shared-memory index
  if (p < oB1) return oW1 + (p % kIn) * kHid + p / kIn;
  if (p >= oW2 && p < oB2) return oW2 + ((p - oW2) % kHid) * kHid + (p - oW2) / kHid;
  if (p >= oW3 && p < oB3) return oW3 + ((p - oW3) % kHid) * kHid + (p - oW3) / kHid;
  return p;
}

// y and the pre-activations z1, z2, z3
__global__ void __launch_bounds__(kMlpThreads) forward_kernel(const __half* __restrict__ w16, int S,
                                                              const float* __restrict__ X, float* __restrict__ y,
                                                              float* __restrict__ act) {
  __shared__ float w[kP];
  for (int e = threadIdx.x; e < kP; e += blockDim.x) w[mlp_wt(e)] = __half2float(w16[e]);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int nwarp = (int)(gridDim.x * blockDim.x) >> 5;
  for (int s = (int)(blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < S; s += nwarp) {
    const float x = lane < kIn ? X[(int64_t)s * kIn + lane] : 0.0f;
    float* za = act ? act + (int64_t)s * kAct : nullptr;
    float z0 = w[oB1 + lane], z1 = w[oB1 + 32 + lane];
#pragma unroll
    for (int j = 0; j < kIn; ++j) {
      const float xj = __shfl_sync(0xffffffffu, x, j);
      z0 = fmaf(w[oW1 + j * kHid + lane], xj, z0);
      z1 = fmaf(w[oW1 + j * kHid + 32 + lane], xj, z1);
    }
    if (za) { za[lane] = z0; za[32 + lane] = z1; }
    float h0 = fmaxf(z0, 0.0f), h1 = fmaxf(z1, 0.0f);
#pragma unroll
    for (int layer = 0; layer < 2; ++layer) {
      const int oW = layer ? oW3 : oW2, oB = layer ? oB3 : oB2;
      z0 = w[oB + lane];
      z1 = w[oB + 32 + lane];
#pragma unroll
      for (int j = 0; j < kHid; ++j) {
        const float hj = __shfl_sync(0xffffffffu, j < 32 ? h0 : h1, j & 31);
        z0 = fmaf(w[oW + j * kHid + lane], hj, z0);
        z1 = fmaf(w[oW + j * kHid + 32 + lane], hj, z1);
      }
      if (za) { za[(layer + 1) * kHid + lane] = z0; za[(layer + 1) * kHid + 32 + lane] = z1; }
      h0 = fmaxf(z0, 0.0f);
      h1 = fmaxf(z1, 0.0f);
    }
    float o = w[oB4];   // every lane forms the same sum, in order
#pragma unroll
    for (int j = 0; j < kHid; ++j) o = fmaf(w[oW4 + j], __shfl_sync(0xffffffffu, j < 32 ? h0 : h1, j & 31), o);
    if (lane == 0) y[s] = o;
  }
}

// per-sample deltas d1, d2, d3 (dL/dz of each hidden layer) from dy; the
// weights in their own (output-major) layout: the lanes of one output row
// read consecutive words
__global__ void __launch_bounds__(kMlpThreads) delta_kernel(const __half* __restrict__ w16, int S,
                                                            const float* __restrict__ act, const float* __restrict__ dy,
                                                            float* __restrict__ del) {
  __shared__ float w[kP];
  for (int e = threadIdx.x; e < kP; e += blockDim.x) w[e] = __half2float(w16[e]);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int nwarp = (int)(gridDim.x * blockDim.x) >> 5;
  for (int s = (int)(blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < S; s += nwarp) {
    const float* z = act + (int64_t)s * kAct;
    float* d = del + (int64_t)s * kAct;
    const float g = dy[s];
    float d0 = z[2 * kHid + lane] > 0.0f ? g * w[oW4 + lane] : 0.0f;   // d3
    float d1 = z[2 * kHid + 32 + lane] > 0.0f ? g * w[oW4 + 32 + lane] : 0.0f;
    d[2 * kHid + lane] = d0;
    d[2 * kHid + 32 + lane] = d1;
#pragma unroll
    for (int layer = 1; layer >= 0; --layer) {   // d2 = (W3^T d3) * relu'(z2), d1 = (W2^T d2) * relu'(z1)
      const int oW = layer ? oW3 : oW2;
      float t0 = 0.0f, t1 = 0.0f;
#pragma unroll
      for (int i = 0; i < kHid; ++i) {
        const float di = __shfl_sync(0xffffffffu, i < 32 ? d0 : d1, i & 31);
        t0 = fmaf(w[oW + i * kHid + lane], di, t0);
        t1 = fmaf(w[oW + i * kHid + 32 + lane], di, t1);
      }
      d0 = z[layer * kHid + lane] > 0.0f ? t0 : 0.0f;
      d1 = z[layer * kHid + 32 + lane] > 0.0f ? t1 : 0.0f;
      d[layer * kHid + lane] = d0;
      d[layer * kHid + 32 + lane] = d1;
    }
  }
}

// CTAs for S samples at one warp each (at most two per SM's worth: each CTA
// loads all the weights once)
static unsigned mlp_grid(int S) {
  const int per = kMlpThreads / 32;
  return (unsigned)std::max(1, std::min((S + per - 1) / per, 2 * 152));
}

// one thread per parameter: the sum over samples (in order) of delta x input
__global__ void __launch_bounds__(256) grad_kernel(int S, const float* __restrict__ X, const float* __restrict__ act,
                                                   const float* __restrict__ del, const float* __restrict__ dy,
                                                   float* __restrict__ grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kP) return;
  // which layer, output unit i and input j (j = -1: bias)
  int layer, i, j;
  if (p < oB1) { layer = 0; i = p / kIn; j = p % kIn; }
  else if (p < oW2) { layer = 0; i = p - oB1; j = -1; }
  else if (p < oB2) { layer = 1; i = (p - oW2) / kHid; j = (p - oW2) % kHid; }
  else if (p < oW3) { layer = 1; i = p - oB2; j = -1; }
  else if (p < oB3) { layer = 2; i = (p - oW3) / kHid; j = (p - oW3) % kHid; }
  else if (p < oW4) { layer = 2; i = p - oB3; j = -1; }
  else if (p < oB4) { layer = 3; i = 0; j = p - oW4; }
  else { layer = 3; i = 0; j = -1; }
  float g = 0.0f;
  for (int s = 0; s < S; ++s) {
    const float dl = layer == 3 ? dy[s] : del[(int64_t)s * kAct + layer * kHid + i];
    float in;
    if (j < 0) in = 1.0f;
    else if (layer == 0) in = X[(int64_t)s * kIn + j];
    else in = fmaxf(act[(int64_t)s * kAct + (layer - 1) * kHid + j], 0.0f);
    g = fmaf(dl, in, g);
  }
  grad[p] = g;
}

// dy = 2 (y - t) / S and the mean squared error (one CTA, fixed order)
__global__ void __launch_bounds__(1024) loss_kernel(int S, const float* __restrict__ y, const float* __restrict__ t,
                                                    float* __restrict__ dy, float* __restrict__ loss) {
  __shared__ float red[32];
  float acc = 0.0f;
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    const float e = y[s] - t[s];
    dy[s] = 2.0f * e / (float)S;
    acc = fmaf(e, e, acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float tot = 0.0f;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) tot += red[q];
    *loss = tot / (float)S;
  }
}

__global__ void adam_kernel(int P, float* __restrict__ w32, __half* __restrict__ w16, float* __restrict__ m,
                            float* __restrict__ v, const float* __restrict__ g, int step, float lr) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float mm = b1 * m[p] + (1.0f - b1) * g[p];
  const float vv = b2 * v[p] + (1.0f - b2) * g[p] * g[p];
  m[p] = mm;
  v[p] = vv;
  const float mh = mm / (1.0f - powf(b1, (float)step));
  const float vh = vv / (1.0f - powf(b2, (float)step));
  const float wn = w32[p] - lr * mh / (sqrtf(vh) + eps);
  w32[p] = wn;
  w16[p] = __float2half_rn(wn);
}

}  // namespace
}  // namespace hodlr

using namespace hodlr;

extern "C" hodlr_status hodlr_mlp_features(const hodlr_kernel* kernel, const double* points, int32_t n, int32_t depth,
                                           double eps, float* feat, void* stream) {
  if (!kernel || !points || !feat) return set_error(HODLR_EINVAL, "null argument");
  if (kernel->dim < 1 || kernel->dim > 3 || kernel->kind < 0 || kernel->kind > 3)
    return set_error(HODLR_EINVAL, "bad kernel");
  if (n < 1 || depth < 1 || depth > HODLR_MAX_DEPTH || (int64_t(1) << depth) > n)
    return set_error(HODLR_EINVAL, "bad n/depth");
  if (!(eps > 0.0)) return set_error(HODLR_EINVAL, "eps must be positive");
  // the cluster tree (ceil-half split) and the blocks in node order
  std::vector<std::vector<std::pair<int, int>>> lv(depth + 1);
  lv[0].push_back({0, n});
  for (int k = 0; k < depth; ++k)
    for (auto& nd : lv[k]) {
      const int left = (nd.second + 1) / 2;
      lv[k + 1].push_back({nd.first, left});
      lv[k + 1].push_back({nd.first + left, nd.second - left});
    }
  std::vector<FBlock> bl;
  for (int k = 1; k <= depth; ++k)
    for (int i = 0; i < (1 << k); ++i)
      bl.push_back({lv[k][i].first, lv[k][i].second, lv[k][i ^ 1].first, lv[k][i ^ 1].second, k});
  cudaStream_t s = (cudaStream_t)stream;
  FBlock* d_bl = nullptr;
  cudaError_t e = cudaMalloc(&d_bl, bl.size() * sizeof(FBlock));
  if (e != cudaSuccess) return set_error(HODLR_ENOMEM, "hodlr_mlp_features");
  e = cudaMemcpyAsync(d_bl, bl.data(), bl.size() * sizeof(FBlock), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    features_kernel<<<(unsigned)bl.size(), 256, 0, s>>>(points, kernel->dim, kernel->kind, kernel->c, kernel->len2,
                                                        kernel->diag, d_bl, eps, feat);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_bl);
  return e == cudaSuccess ? HODLR_OK : set_cuda_error(e, "hodlr_mlp_features");
}

extern "C" hodlr_status hodlr_mlp_forward(const uint16_t* w16, int32_t S, const float* X, float* y, float* act,
                                          void* stream) {
  if (!w16 || !X || !y || S < 0) return set_error(HODLR_EINVAL, "bad hodlr_mlp_forward arguments");
  if (S == 0) return HODLR_OK;
  forward_kernel<<<mlp_grid(S), kMlpThreads, 0, (cudaStream_t)stream>>>(
      reinterpret_cast<const __half*>(w16), S, X, y, act);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HODLR_OK : set_cuda_error(e, "hodlr_mlp_forward");
}

extern "C" hodlr_status hodlr_mlp_loss(int32_t S, const float* y, const float* t, float* dy, float* loss,
                                       void* stream) {
  if (!y || !t || !dy || !loss || S < 1) return set_error(HODLR_EINVAL, "bad hodlr_mlp_loss arguments");
  loss_kernel<<<1, 1024, 0, (cudaStream_t)stream>>>(S, y, t, dy, loss);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HODLR_OK : set_cuda_error(e, "hodlr_mlp_loss");
}

extern "C" hodlr_status hodlr_mlp_backward(const uint16_t* w16, int32_t S, const float* X, const float* act,
                                           const float* dy, float* grad, float* work, void* stream) {
  if (!w16 || !X || !act || !dy || !grad || !work || S < 1)
    return set_error(HODLR_EINVAL, "bad hodlr_mlp_backward arguments");
  cudaStream_t s = (cudaStream_t)stream;
  delta_kernel<<<mlp_grid(S), kMlpThreads, 0, s>>>(reinterpret_cast<const __half*>(w16), S, act, dy, work);
  grad_kernel<<<(unsigned)((kP + 255) / 256), 256, 0, s>>>(S, X, act, work, dy, grad);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HODLR_OK : set_cuda_error(e, "hodlr_mlp_backward");
}

extern "C" hodlr_status hodlr_mlp_adam(float* w32, uint16_t* w16, float* m, float* v, const float* grad, int32_t step,
                                       float lr, void* stream) {
  if (!w32 || !w16 || !m || !v || !grad || step < 1) return set_error(HODLR_EINVAL, "bad hodlr_mlp_adam arguments");
  adam_kernel<<<(kP + 255) / 256, 256, 0, (cudaStream_t)stream>>>(kP, w32, reinterpret_cast<__half*>(w16), m, v, grad,
                                                                  step, lr);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HODLR_OK : set_cuda_error(e, "hodlr_mlp_adam");
}

extern "C" int32_t hodlr_mlp_num_params(void) { return kP; }
