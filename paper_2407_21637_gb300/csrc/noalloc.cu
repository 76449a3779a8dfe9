// hodlr_matvec_noalloc: the HODLR product without any device allocation.
//
// hodlr_matvec keeps its scratch (the partial sums of V^T X and a grid
// barrier counter) in buffers the handle allocated when it was created.
// This variant keeps that scratch in one file-scope device array instead, so
// a call never reaches cudaMalloc, and it does not touch the handle's own
// scratch.  It is meant for callers that cannot allocate device memory at
// the point of the call: for instance a process whose device memory is
// already fully reserved by another allocator (a framework's caching
// allocator or a pre-partitioned pool), or code on a latency-critical path
// that must not enter the driver's allocator.
//
// The array is a fixed, modest size (kNoAllocScratchBytes); every GPU that
// loads this library holds it until the process exits.  It runs the
// CUDA-core streamed product (stream.cu) in batches of columns that fit the
// array.
#include <algorithm>

#include "handle.cuh"

namespace hodlr {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(256) << 10;   // 256 KiB per device

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

}  // namespace
}  // namespace hodlr

using namespace hodlr;

extern "C" hodlr_status hodlr_matvec_noalloc(hodlr_t h, int32_t nrhs, const void* X, int64_t ldx,
                                             void* B, int64_t ldb, int32_t xb_prec, void* stream) {
  if (!h) return set_error(HODLR_EINVAL, "null handle");
  if (nrhs < 0) return set_error(HODLR_EINVAL, "nrhs < 0");
  if (nrhs == 0) return HODLR_OK;
  if (!X || !B) return set_error(HODLR_EINVAL, "null X/B");
  if (ldx < nrhs || ldb < nrhs) return set_error(HODLR_EINVAL, "leading dimension < nrhs");
  if (xb_prec != h->work) return set_error(HODLR_EINVAL, "X/B type must equal the working precision");
  const size_t es = prec_bytes(h->work);
  const char* xb = (const char*)X;
  char* bb = (char*)B;
  const size_t span_x = ((size_t)(h->n - 1) * ldx + nrhs) * es;
  const size_t span_b = ((size_t)(h->n - 1) * ldb + nrhs) * es;
  if (!(xb + span_x <= bb || bb + span_b <= xb)) return set_error(HODLR_EINVAL, "X and B overlap");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_cuda_error(e, "cudaGetDevice");
  if (dev != h->device) return set_error(HODLR_EINVAL, "the current device differs from the handle's device");

  // scratch layout: the grid counter (kSyncHeadBytes), then the partial
  // slots of one batch of nb columns (st_p_rows * nb values)
  const size_t counter_bytes = kSyncHeadBytes;
  const size_t per_col = (size_t)std::max(h->hd.st_p_rows, 1) * es;
  if (counter_bytes + per_col > kNoAllocScratchBytes)
    return set_error(HODLR_EINVAL, "matrix too large for the 256 KiB static scratch of hodlr_matvec_noalloc "
                                   "(use hodlr_matvec)");
  if (!h->use_stream)
    return set_error(HODLR_EINVAL, "ranks too large for the streamed product that hodlr_matvec_noalloc runs "
                                   "(use hodlr_matvec)");
  const int nb_max = (int)std::min<size_t>(std::min<size_t>((size_t)nrhs, (size_t)h->batch),
                                           (kNoAllocScratchBytes - counter_bytes) / per_col);
  // In host code the array's name stands in for the symbol; the address a
  // kernel may use is looked up here, on the current device, on every call
  // (a lookup allocates nothing and enqueues nothing).
  void* base = nullptr;
  e = cudaGetSymbolAddress(&base, g_noalloc_scratch);
  if (e != cudaSuccess) return set_cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
  unsigned long long* sync = (unsigned long long*)base;
  void* partials = (char*)base + counter_bytes;
  cudaStream_t s = (cudaStream_t)stream;
  // The array keeps the previous call's contents: the counter must start at
  // zero (every partial slot is written before it is read).
  e = cudaMemsetAsync(sync, 0, counter_bytes, s);
  if (e != cudaSuccess) return set_cuda_error(e, "cudaMemsetAsync(grid counter)");
  unsigned long long base_count = 0;
  for (int c0 = 0; c0 < nrhs; c0 += nb_max) {
    const int nb = std::min(nb_max, nrhs - c0);
    e = launch_stream(h->hd, h->work, nb, xb + c0 * es, ldx, bb + c0 * es, ldb, partials, sync, base_count, s,
                      nullptr);
    if (e != cudaSuccess) return set_cuda_error(e, "hodlr_matvec_noalloc launch");
    base_count += stream_sync_step(h->hd);
  }
  return HODLR_OK;
}
