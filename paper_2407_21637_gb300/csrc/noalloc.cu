// hodlr_matvec_noalloc: the HODLR product without any device allocation.
//
// hodlr_matvec keeps its scratch (the partial sums of V^T X, the gathered
// V^T X results and a grid barrier counter) in buffers the handle
// allocated when it was created.  This variant keeps that scratch in one
// file-scope device array instead, so a call never reaches cudaMalloc, and
// it does not touch the handle's own scratch.  It is meant for callers that
// cannot allocate device memory at the point of the call: for instance a
// process whose device memory is already fully reserved by another
// allocator (a framework's caching allocator or a pre-partitioned pool), or
// code on a latency-critical path that must not enter the driver's
// allocator.
//
// The array is a fixed, modest size (kNoAllocScratchBytes); every GPU that
// loads this library holds it until the process exits.
#include <mutex>

#include "handle.cuh"

namespace hodlr {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(4) << 20;   // 4 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// The device address of the array on the current device.  In host code the
// array's name only stands in for the symbol; the address a kernel may use
// comes from cudaGetSymbolAddress, taken once per device with that device
// current (the first call on each device does it).
hodlr_status scratch_for_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_cuda_error(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return set_error(HODLR_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return set_cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return HODLR_OK;
}

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

  // scratch layout: the grid counter (kSyncHeadBytes), then, per batch of
  // nb columns, the gathered Y (y_rows * nb values + 4 of slack, rounded to
  // 256 bytes) and the partial sums (p_rows * nb values)
  const size_t counter_bytes = kSyncHeadBytes;
  const size_t per_col = ((size_t)h->hd.y_rows + (size_t)h->hd.p_rows) * es;
  const size_t fixed = counter_bytes + 4 * es + 512;
  if (fixed + per_col > kNoAllocScratchBytes)
    return set_error(HODLR_EINVAL, "matrix too large for the 4 MiB static scratch of hodlr_matvec_noalloc "
                                   "(use hodlr_matvec)");
  const int nb_max = (int)std::min<size_t>(std::min<size_t>((size_t)nrhs, (size_t)h->batch),
                                           (kNoAllocScratchBytes - fixed) / per_col);
  void* base = nullptr;
  hodlr_status st = scratch_for_current_device(&base);
  if (st != HODLR_OK) return st;
  unsigned long long* sync = (unsigned long long*)base;
  char* ybuf = (char*)base + counter_bytes;
  cudaStream_t s = (cudaStream_t)stream;
  // The array keeps the previous call's contents: the counter must start at
  // zero.
  cudaError_t e = cudaMemsetAsync(sync, 0, counter_bytes, s);
  if (e != cudaSuccess) return set_cuda_error(e, "cudaMemsetAsync(grid counter)");
  unsigned long long base_count = 0;
  for (int c0 = 0; c0 < nrhs; c0 += nb_max) {
    const int nb = std::min(nb_max, nrhs - c0);
    void* Y = ybuf;
    void* partials = ybuf + (((size_t)h->hd.y_rows * nb + 4) * es + 255) / 256 * 256;
    e = launch_matvec(h->hd, h->work, nb, xb + c0 * es, ldx, bb + c0 * es, ldb, Y, partials, sync, base_count,
                      s, nullptr);
    if (e != cudaSuccess) return set_cuda_error(e, "hodlr_matvec_noalloc launch");
    base_count += matvec_sync_step(h->hd);
  }
  return HODLR_OK;
}
