// Leaf products D_i X[I_i] and the products V_j^T X[I_j] of Algorithm 3.3
// on the fifth-generation tensor cores (tcgen05), for fp32 work with many
// right-hand sides.
//
// The product kernel (matvec.cu) does both on CUDA cores; with 16 or more
// right-hand sides they are dense contractions worth the tensor cores.  Per
// group of up to 128 rows,
//     C (128 x N) = A (128 x m) * X[I] (m x N),   N = R rounded up to 16,
// accumulated in tensor memory (TMEM, fp32).  A leaf group's A is up to 128
// rows of the leaf block D_i (I = I_i), written to B; a V group's A is up to
// 128 columns of fp32 generators V_j restricted to the rows I of one V
// chunk (the chunks of one leaf at several levels), written to the chunks'
// partial rows, which the product kernel then sums per node.  fp32 is kept
// by splitting every fp32 value x into hi + lo with hi = tf32(x) (round to
// nearest) and lo = tf32(x - hi); per K step two MMAs of width 2N,
//     A_hi [X_hi | X_lo] + A_lo [X_hi | X_lo],
// give all four partial products in two accumulator halves that the
// epilogue adds.  The error per product is at most about 2 * 2^-22 |a| |x|
// (the rounding of the two lo parts), far inside the elementwise bound the
// product is tested against.
//
// Per CTA (persistent, one per SM): sixteen converter warps keep a ring of
// three stages with cp.async: a K-chunk of 64 columns of A for 128 rows
// (placed in the 128-byte-swizzled K-major layout, two atoms along K) and
// the matching 64 rows of X.  Once a chunk has landed they split it: A's hi and lo parts go to
// tensor memory (tcgen05.st, lane = row), X is transposed into N x 32 hi
// and lo tiles in shared memory (two operand buffers each).  One thread
// issues the MMAs (tcgen05.mma.kind::tf32, A from tensor memory, B from a
// shared-memory descriptor) and commits them to the buffer's mbarrier,
// which frees it for the next chunk.  Groups alternate between two
// accumulators in TMEM, so that four epilogue warps (one per TMEM lane
// quadrant) read one group's result (tcgen05.ld) and write it out while the
// next group accumulates.  Every wait is bounded (two seconds) and records
// an error code; the CTA always frees its tensor memory before it exits.
#include <algorithm>

#include "hodlr_internal.cuh"

namespace hodlr {

namespace {

constexpr int kConvWarps = 16;
constexpr int kConvThreads = 32 * kConvWarps;
constexpr int kEpiWarps = 4;                    // one per TMEM lane quadrant
constexpr int kTcThreads = kConvThreads + 32 + 32 * kEpiWarps;   // converters, the MMA warp, epilogue
constexpr int kTcM = 128;                       // rows per group (MMA M)
constexpr int kKc = 64;                         // K-chunk: 64 fp32 = two 128-byte swizzle atoms along K
constexpr int kKa = kKc / 32;                   // swizzle atoms along K per chunk
constexpr unsigned long long kTcWaitNs = 2000000000ull;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long gns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void bar_init(uint64_t* b, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ bool bar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity), "r"(1000000u)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool bar_wait(uint64_t* b, uint32_t parity, int* err, int code) {
  if (bar_try(b, parity)) return true;
  const unsigned long long t0 = gns();
  while (!bar_try(b, parity))
    if (gns() - t0 > kTcWaitNs) {
      atomicExch(err, code);
      return false;
    }
  return true;
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows
// of 128 bytes, groups of 8 rows 1024 bytes apart, 1024-byte aligned base.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);   // start address
  d |= (uint64_t)1 << 16;                      // leading byte offset (unused with this swizzle)
  d |= (uint64_t)(1024 >> 4) << 32;            // stride byte offset: 8 rows x 128 bytes
  d |= (uint64_t)1 << 46;                      // descriptor version
  d |= (uint64_t)2 << 61;                      // 128-byte swizzle
  return d;
}
// Instruction descriptor: D fp32, A and B tf32, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// Byte offset of the 16-byte group g (4 fp32) of row r in a 128-byte-swizzled
// K-major tile.
__device__ __forceinline__ uint32_t sw128(int r, int g) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((g ^ (r & 7)) << 4));
}
// The same for a chunk of kKc values per row: atom column g / 8 (32 values
// of K for all `rows` rows), then sw128 within it.
__device__ __forceinline__ uint32_t swk(int r, int g, int rows) {
  return (uint32_t)((g >> 3) * rows * 128) + sw128(r, g & 7);
}
// x rounded to tf32 (10 fraction bits) to nearest, ties away from zero, on
// the bit pattern: half a unit of the 13 dropped bits is added to the
// magnitude and the dropped bits are cleared (a carry into the exponent is
// the rounding up to the next binade).  Two integer operations on the full-
// rate pipes; finite x only.
__device__ __forceinline__ uint32_t tf32_rna(float x) { return (__float_as_uint(x) + 0x1000u) & 0xffffe000u; }
__device__ __forceinline__ void split(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_rna(x);
  lo = tf32_rna(x - __uint_as_float(hi));
}
__device__ __forceinline__ void sts4(uint32_t a, uint32_t x, uint32_t y, uint32_t z, uint32_t w) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(x), "r"(y), "r"(z), "r"(w) : "memory");
}

// D (+)= A B, A in tensor memory (128 lanes = rows, one tf32 per column), B from
// a shared-memory descriptor.
__device__ __forceinline__ void mma_tf32_tmem_a(uint32_t tmem_d, uint32_t tmem_a, uint64_t bdesc, uint32_t idesc,
                                                uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(tmem_d),
      "r"(tmem_a), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// 16 consecutive 32-bit columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
      "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void mma_commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(b))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive fp32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void bar_conv() {
  asm volatile("bar.sync 1, %0;" ::"r"(kConvThreads) : "memory");
}
__device__ __forceinline__ uint4 lds16(uint32_t a) {
  uint4 v;
  asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
  return v;
}
__device__ __forceinline__ float lds1f(uint32_t a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
  return v;
}

// Shared memory (every part 1024-byte aligned):
//  raw ring, kTcRaw stages: A (128 x 64 fp32, placed by cp.async in the
//    128-byte-swizzled K-major layout, two atom columns of 32 values) and X
//    (64 x N fp32, row-major as loaded);
//  two operand buffers [X_hi | X_lo]^T (2N rows x 64 tf32, K-major, 128-byte
//    swizzle).
// Tensor memory (512 columns): two accumulators of 2N columns (columns
// 128 a: the products with X_hi in the first N, with X_lo in the next N)
// and two A operand buffers (columns kTmemA + 128 b: A_hi in 64 columns,
// A_lo in the next 64; lane = row of A).
constexpr int kTcRaw = 3;
constexpr uint32_t kTmemAcc = 128;
constexpr uint32_t kTmemA = 2 * kTmemAcc;        // A buffer b: hi at kTmemA + 2 kKc b, lo kKc columns further
constexpr uint32_t kTmemCols = 512;
__host__ __device__ inline uint32_t tc_raw_bytes(int N) { return (uint32_t)kTcM * kKc * 4 + (uint32_t)N * kKc * 4; }
__host__ __device__ inline uint32_t tc_op_bytes(int N) { return 2u * (uint32_t)N * kKc * 4; }
__host__ __device__ inline uint32_t tc_smem_bytes(int N) {
  return 1024 + kTcRaw * tc_raw_bytes(N) + 2 * tc_op_bytes(N) + 256;
}

template <int N>
__global__ void __launch_bounds__(kTcThreads, 1)
leaf_tc_kernel(const TcGroup* __restrict__ groups, const int32_t* __restrict__ cta_first,
               const TcVRow* __restrict__ vrows,
               const uint8_t* __restrict__ pool, const float* __restrict__ X, int64_t ldx, int R,
               float* __restrict__ B, int64_t ldb, float* __restrict__ partials, uint32_t tmem_cols, int* err) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr uint32_t ab = kTcM * kKc * 4, xb = (uint32_t)N * kKc * 4;
  constexpr uint32_t rb = ab + xb, ob = 2 * xb;
  static_assert(2 * N <= (int)kTmemAcc, "accumulator wider than its TMEM slot");
  const uint32_t raw0 = su32(base), op0 = raw0 + kTcRaw * rb;
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + kTcRaw * rb + 2 * ob);
  uint64_t* conv_done = bars;          // [2], kConvThreads arrivals
  uint64_t* mma_done = bars + 2;       // [2], one commit
  uint64_t* acc_full = bars + 4;       // [2] accumulator buffers, one commit
  uint64_t* acc_empty = bars + 6;      // [2], kEpiWarps arrivals
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 8);
  int* abort_flag = reinterpret_cast<int*>(bars + 9);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int b = 0; b < 2; ++b) {
      bar_init(&conv_done[b], kConvThreads);
      bar_init(&mma_done[b], 1);
      bar_init(&acc_full[b], 1);
      bar_init(&acc_empty[b], kEpiWarps);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kConvWarps) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  constexpr uint32_t idesc = idesc_tf32(kTcM, 2 * N);   // B = [X_hi | X_lo]
  const bool x16 = (ldx % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);

  // this CTA's chunks, in order: (group, K-chunk) (unrolled: the loads of
  // several groups in flight together)
  const int g0 = __ldg(cta_first + blockIdx.x), g1 = __ldg(cta_first + blockIdx.x + 1);   // this CTA's groups
  int total = 0;
#pragma unroll 8
  for (int g = g0; g < g1; ++g) total += (__ldg(&groups[g].m) + kKc - 1) / kKc;

  if (warp < kConvWarps) {
    const int t = threadIdx.x;
    // fixed per thread: A pieces (row rr + kAR i, 16-byte group cg),
    // X pieces (piece p = t + kConvThreads j: row p / (N / 4), columns
    // 4 (p % (N / 4)) .. + 3) and B pieces (row p % N, 16-byte group p / N)
    constexpr int n4 = N / 4;
    constexpr int XP = (kKc * n4 + kConvThreads - 1) / kConvThreads;   // X pieces per thread
    constexpr int BP = (N * (kKc / 4) + kConvThreads - 1) / kConvThreads;
    constexpr int kAR = kConvThreads / 8;   // A rows per pass of all converter threads
    constexpr int kAP = kTcM / kAR;         // A pieces per thread
    static_assert(kAP * kAR == kTcM && kAR % 32 == 0, "converter threads must tile the 128 A rows");
    const int rr = t >> 3, cg = t & 7;
    // A split: warp w takes TMEM lanes 32 (w % 4) .. + 31 (row = lane) and
    // columns 16 (w / 4) .. + 15 of the chunk
    static_assert(kConvWarps == 16, "four warps per TMEM lane quadrant");
    const int aq = warp & 3, akq = warp >> 2;
    const int arow = 32 * aq + lane;
    const uint32_t alane = (uint32_t)(32 * aq) << 16;
    // load cursor state (per group).  load_group only issues the loads of
    // a group's fields and row offsets; they are first used by the next
    // chunk's copies, so their latency overlaps the conversion in between.
    int lg = g0, lkc = 0;
    int64_t aoff[kAP];   // byte offset of each A row's first element, -1: no row
    int lm = 0, lxrow = 0;
    auto load_group = [&](int g) {
      const TcGroup* G = groups + g;
      lm = __ldg(&G->m);
      lxrow = __ldg(&G->xrow0);
#pragma unroll
      for (int i = 0; i < kAP; ++i) aoff[i] = __ldg(&vrows[(size_t)g * kTcM + rr + kAR * i].off);
    };
    if (lg < g1) load_group(lg);
    auto issue = [&](int u) {
      if (u < total) {
        const int k0 = lkc * kKc;
        const uint32_t ra = raw0 + (uint32_t)(u % kTcRaw) * rb, rx = ra + ab;
        const int lmp = (lm + 3) & ~3;
#pragma unroll
        for (int a = 0; a < kKa; ++a) {
          const int gk = cg + 8 * a;   // 16-byte group of the chunk
          const bool kin = 4 * gk + k0 < lmp;
#pragma unroll
          for (int i = 0; i < kAP; ++i) {
            const bool ok = aoff[i] >= 0 && kin;
            cp_async16(ra + swk(rr + kAR * i, gk, kTcM),
                       ok ? (const void*)(pool + aoff[i] + (size_t)(k0 + 4 * gk) * 4) : (const void*)pool, ok ? 16u : 0u);
          }
        }
        const float* xbase = X + (int64_t)lxrow * ldx;
#pragma unroll
        for (int j = 0; j < XP; ++j) {
          const int p = t + kConvThreads * j;
          if (XP * kConvThreads == kKc * n4 || p < kKc * n4) {
            const int k = p / n4, n = 4 * (p % n4);
            const bool rok = k0 + k < lm;
            const float* xr = xbase + (int64_t)(k0 + k) * ldx + n;
            const uint32_t dst = rx + (uint32_t)((k * N + n) * 4);
            if (x16) {
              const int cnt = rok ? max(0, min(4, R - n)) : 0;
              cp_async16(dst, cnt ? (const void*)xr : (const void*)X, (uint32_t)(cnt * 4));
            } else {
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const bool ok = rok && n + e < R;
                cp_async4(dst + 4u * e, ok ? (const void*)(xr + e) : (const void*)X, ok ? 4u : 0u);
              }
            }
          }
        }
        if (++lkc * kKc >= lm) {
          lkc = 0;
          ++lg;
          if (lg < g1) load_group(lg);
        }
      }
      cp_async_commit();
    };
    // prologue: chunks 0 .. kTcRaw - 2 in flight
#pragma unroll 1
    for (int u = 0; u < kTcRaw - 1; ++u) issue(u);
    int cg_idx = g0, ckc = 0;   // compute cursor
    int cm = cg_idx < g1 ? __ldg(&groups[cg_idx].m) : 0;
    int crows = cg_idx < g1 ? __ldg(&groups[cg_idx].rows) : 0;
#pragma unroll 1
    for (int u = 0; u < total; ++u) {
      const int r = u % kTcRaw, b = u & 1;
      const uint32_t ra = raw0 + (uint32_t)r * rb, rx = ra + ab;
      const uint32_t oa = op0 + (uint32_t)b * ob;
      // chunk u's copies have landed (the kTcRaw - 2 after it may be pending)
      cp_async_wait<kTcRaw - 2>();
      bar_conv();   // everybody's copies; everybody is done with raw stage (u - 1) % kTcRaw
      // the operand buffer of chunk u - 2 is free once its MMAs are done
      bool ok = !*(volatile int*)abort_flag;
      if (ok && u >= 2) ok = bar_wait(&mma_done[b], (uint32_t)(((u >> 1) - 1) & 1), err, 21);
      if (!ok) *(volatile int*)abort_flag = 1;
      tc_fence_after();
      // refill the raw stage of chunk u - 1 with chunk u + kTcRaw - 1
      issue(u + kTcRaw - 1);
      // A: split into hi and lo, into tensor memory (a quadrant past the
      // group's valid rows is skipped; rows past them in a quadrant reach
      // only accumulator rows that the epilogue does not write)
      if (32 * aq < crows) {
        uint32_t h[16], l[16];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const uint4 v = lds16(ra + swk(arow, 4 * akq + j, kTcM));
          split(__uint_as_float(v.x), h[4 * j + 0], l[4 * j + 0]);
          split(__uint_as_float(v.y), h[4 * j + 1], l[4 * j + 1]);
          split(__uint_as_float(v.z), h[4 * j + 2], l[4 * j + 2]);
          split(__uint_as_float(v.w), h[4 * j + 3], l[4 * j + 3]);
        }
        const uint32_t ta = tmem + alane + kTmemA + 2u * kKc * (uint32_t)b + 16u * (uint32_t)akq;
        tmem_st16(ta, h);
        tmem_st16(ta + kKc, l);
      }
      // B = X^T: thread (n, k-group of 4), consecutive threads take consecutive n
#pragma unroll
      for (int j = 0; j < BP; ++j) {
        const int p = t + kConvThreads * j;
        if (BP * kConvThreads == N * (kKc / 4) || p < N * (kKc / 4)) {
          const int n = p % N, kg = p / N;
          uint32_t h[4], l[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) split(lds1f(rx + (uint32_t)(((4 * kg + e) * N + n) * 4)), h[e], l[e]);
          sts4(oa + swk(n, kg, 2 * N), h[0], h[1], h[2], h[3]);
          sts4(oa + swk(N + n, kg, 2 * N), l[0], l[1], l[2], l[3]);
        }
      }
      // TMEM stores complete, generic-proxy stores -> visible to the tensor
      // cores (async proxy)
      tmem_wait_st();
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc_fence_before();
      bar_arrive(&conv_done[b]);
      if (++ckc * kKc >= cm) {
        ckc = 0;
        ++cg_idx;
        cm = cg_idx < g1 ? __ldg(&groups[cg_idx].m) : 0;
        crows = cg_idx < g1 ? __ldg(&groups[cg_idx].rows) : 0;
      }
    }
    cp_async_wait<0>();
  } else if (warp == kConvWarps) {
    // ================= MMA issuer =================
    // group number gc accumulates into TMEM columns kTmemAcc (gc & 1); per
    // 8-wide K step, A_hi [X_hi | X_lo] + A_lo [X_hi | X_lo]
    int ckc = 0, cg_idx = g0, gc = 0;
    int cm = cg_idx < g1 ? __ldg(&groups[cg_idx].m) : 0;
#pragma unroll 1
    for (int u = 0; u < total; ++u) {
      const int b = u & 1;
      const uint32_t acc = tmem + (uint32_t)(gc & 1) * kTmemAcc;
      const bool last = (ckc + 1) * kKc >= cm;
      if (lane == 0) {
        bool ok = !*(volatile int*)abort_flag;
        // a group's first chunk: its accumulator buffer must have been read
        if (ok && ckc == 0 && gc >= 2) ok = bar_wait(&acc_empty[gc & 1], (uint32_t)(((gc >> 1) - 1) & 1), err, 24);
        if (ok) ok = bar_wait(&conv_done[b], (uint32_t)((u >> 1) & 1), err, 22);
        if (ok && !*(volatile int*)abort_flag) {
          tc_fence_after();
          const uint32_t oa = op0 + (uint32_t)b * ob;
          const uint32_t ah = tmem + kTmemA + 2u * kKc * (uint32_t)b, al = ah + kKc;
#pragma unroll
          for (int ks = 0; ks < kKc / 8; ++ks) {
            // 2N rows: X_hi^T, then X_lo^T; atom column ks / 4, 8 tf32 = 32 bytes along K within it
            const uint64_t bd = desc_sw128(oa + (uint32_t)((ks >> 2) * 2 * N * 128));
            const uint64_t adv = (uint64_t)((ks & 3) * 32) >> 4;
            const uint32_t ac = (uint32_t)(ks * 8);          // 8 tf32 = 8 TMEM columns
            mma_tf32_tmem_a(acc, ah + ac, bd + adv, idesc, (ckc > 0 || ks > 0) ? 1u : 0u);
            mma_tf32_tmem_a(acc, al + ac, bd + adv, idesc, 1u);
          }
        } else {
          *(volatile int*)abort_flag = 1;
        }
        mma_commit(&mma_done[b]);
        if (last) mma_commit(&acc_full[gc & 1]);
      }
      __syncwarp();
      if (last) {
        ckc = 0;
        ++cg_idx;
        cm = cg_idx < g1 ? __ldg(&groups[cg_idx].m) : 0;
        ++gc;
      } else {
        ++ckc;
      }
    }
  } else {
    // ================= epilogue: accumulator -> B or partial rows =================
    // warp kConvWarps + 1 + e reads TMEM lanes 32 q .. 32 q + 31, q = warp % 4
    const int q = warp & 3;
    const int row = 32 * q + lane;
    int gc = 0;
#pragma unroll 1
    for (int g = g0; g < g1; ++g, ++gc) {
      const TcGroup* G = groups + g;
      const bool okw = bar_wait(&acc_full[gc & 1], (uint32_t)((gc >> 1) & 1), err, 23) && !*(volatile int*)abort_flag;
      tc_fence_after();
      const int vt = __ldg(&G->vtab);
      bool rok;
      float* brow;
      bool vec;
      if (vt < 0) {
        rok = row < __ldg(&G->rows);
        brow = B + (int64_t)(__ldg(&G->row0) + row) * ldb;
        vec = (R == N) && (ldb % 4 == 0) && ((reinterpret_cast<uintptr_t>(B) & 15) == 0);
      } else {
        const int pr = __ldg(&vrows[vt + row].prow);
        rok = pr >= 0;
        brow = partials + (int64_t)max(pr, 0) * R;
        vec = (R == N) && ((reinterpret_cast<uintptr_t>(partials) & 15) == 0);
      }
      const uint32_t acc = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(gc & 1) * kTmemAcc;
#pragma unroll
      for (int c0 = 0; c0 < N; c0 += 16) {
        float v[16], w[16];
        tmem_ld16(acc + (uint32_t)c0, v);
        tmem_ld16(acc + (uint32_t)(N + c0), w);
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] += w[j];
        if (okw && rok) {
          if (vec) {
#pragma unroll
            for (int j = 0; j < 16; j += 4)
              *reinterpret_cast<float4*>(brow + c0 + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (c0 + j < R) brow[c0 + j] = v[j];
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) bar_arrive(&acc_empty[gc & 1]);
    }
  }
  __syncthreads();
  if (warp == kConvWarps) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
  }
}

}  // namespace

size_t leaf_tc_smem(int N) { return tc_smem_bytes(N); }

namespace {
template <int N>
cudaError_t launch_n(const TcGroup* groups, const int32_t* cta_first, int ncta, const TcVRow* vrows,
                     const uint8_t* pool,
                     const float* X, int64_t ldx, int nrhs, float* B, int64_t ldb, float* partials, int* err,
                     cudaStream_t s) {
  const uint32_t cols = kTmemCols;   // two accumulators, two A operand buffers
  const size_t smem = leaf_tc_smem(N);
  static size_t smem_set = 0;   // per instantiation
  if (smem > smem_set) {
    cudaError_t e = cudaFuncSetAttribute(leaf_tc_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    smem_set = smem;
  }
  leaf_tc_kernel<N><<<ncta, kTcThreads, smem, s>>>(groups, cta_first, vrows, pool, X, ldx, nrhs, B, ldb, partials,
                                                    cols, err);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_leaf_tc(const TcGroup* groups, const int32_t* cta_first, int ncta, const TcVRow* vrows,
                           const uint8_t* pool,
                           const float* X, int64_t ldx, int nrhs, float* B, int64_t ldb, float* partials,
                           int* err, cudaStream_t s) {
  if (ncta == 0 || nrhs == 0) return cudaSuccess;
  const int N = (nrhs + 15) / 16 * 16;
  if (N < 16 || N > kTcMaxCols) return cudaErrorInvalidValue;
  switch (N) {
    case 16: return launch_n<16>(groups, cta_first, ncta, vrows, pool, X, ldx, nrhs, B, ldb, partials, err, s);
    case 32: return launch_n<32>(groups, cta_first, ncta, vrows, pool, X, ldx, nrhs, B, ldb, partials, err, s);
    case 48: return launch_n<48>(groups, cta_first, ncta, vrows, pool, X, ldx, nrhs, B, ldb, partials, err, s);
    default: return launch_n<64>(groups, cta_first, ncta, vrows, pool, X, ldx, nrhs, B, ldb, partials, err, s);
  }
}

}  // namespace hodlr
