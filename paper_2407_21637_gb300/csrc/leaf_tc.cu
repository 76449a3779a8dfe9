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
// partial rows, which the product kernel then sums per node.  fp32 is kept by the usual
// three-pass split: every fp32 value x becomes hi + lo with hi = tf32(x)
// (round to nearest) and lo = tf32(x - hi), and
//     D X ~ D_hi X_hi + D_hi X_lo + D_lo X_hi,
// whose error per product is at most about 3 * 2^-22 |d| |x| (the dropped
// D_lo X_lo term and the rounding of the lo parts), far inside the
// elementwise bound the product is tested against.
//
// Per CTA (persistent, one per SM): eight converter warps keep a ring of
// two to four stages in flight with cp.async: a K-chunk of 32 columns of D
// for 128 rows (placed directly in the tensor cores' K-major layout with the
// 128-byte swizzle) and the matching 32 rows of X.  Once a chunk has landed
// they split it in shared memory (D's hi part over the raw values, lo beside
// it; X transposed into N x 32 hi and lo tiles); one thread issues the MMAs
// (tcgen05.mma.kind::tf32, A and B from shared-memory descriptors) and
// commits them to the stage's mbarrier, which frees the stage for the next
// copies.  After a group's last chunk the four epilogue warps read the
// accumulator (tcgen05.ld) and write B.  Every wait is bounded (two seconds)
// and records an error code; the CTA always frees its tensor memory before
// it exits.
#include <algorithm>

#include "hodlr_internal.cuh"

namespace hodlr {

namespace {

constexpr int kConvWarps = 8;
constexpr int kConvThreads = 32 * kConvWarps;
constexpr int kTcThreads = kConvThreads + 32;   // + the MMA warp
constexpr int kTcM = 128;                       // rows per group (MMA M)
constexpr int kKc = 32;                         // K-chunk: 32 fp32 = one 128-byte swizzle row
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
__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void split(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_rna(x);
  lo = tf32_rna(x - __uint_as_float(hi));
}
__device__ __forceinline__ void sts4(uint32_t a, uint32_t x, uint32_t y, uint32_t z, uint32_t w) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(x), "r"(y), "r"(z), "r"(w) : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
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
//  raw ring, kTcRaw stages: A (128 x 32 fp32 of D, placed by cp.async in the
//    swizzled K-major layout) and X (32 x N fp32, row-major as loaded);
//  two operand buffers: A_hi, A_lo (128 x 32 tf32) and B_hi, B_lo (X^T,
//    N x 32 tf32), all K-major with the 128-byte swizzle.
constexpr int kTcRaw = 4;
__host__ __device__ inline uint32_t tc_raw_bytes(int N) { return (uint32_t)kTcM * kKc * 4 + (uint32_t)N * kKc * 4; }
__host__ __device__ inline uint32_t tc_op_bytes(int N) { return 2u * kTcM * kKc * 4 + 2u * (uint32_t)N * kKc * 4; }
__host__ __device__ inline uint32_t tc_smem_bytes(int N) {
  return 1024 + kTcRaw * tc_raw_bytes(N) + 2 * tc_op_bytes(N) + 256;
}

template <int N>
__global__ void __launch_bounds__(kTcThreads, 1)
leaf_tc_kernel(const TcGroup* __restrict__ groups, int ngroups, const TcVRow* __restrict__ vrows,
               const uint8_t* __restrict__ pool, const float* __restrict__ X, int64_t ldx, int R,
               float* __restrict__ B, int64_t ldb, float* __restrict__ partials, uint32_t tmem_cols, int* err) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr uint32_t ab = kTcM * kKc * 4, xb = (uint32_t)N * kKc * 4;
  constexpr uint32_t rb = ab + xb, ob = 2 * ab + 2 * xb;
  const uint32_t raw0 = su32(base), op0 = raw0 + kTcRaw * rb;
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + kTcRaw * rb + 2 * ob);
  uint64_t* conv_done = bars;          // [2], kConvThreads arrivals
  uint64_t* mma_done = bars + 2;       // [2], one commit
  uint64_t* acc_ready = bars + 4;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 5);
  int* abort_flag = reinterpret_cast<int*>(bars + 6);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int b = 0; b < 2; ++b) {
      bar_init(&conv_done[b], kConvThreads);
      bar_init(&mma_done[b], 1);
    }
    bar_init(acc_ready, 1);
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
  constexpr uint32_t idesc = idesc_tf32(kTcM, N);
  const bool x16 = (ldx % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);

  // this CTA's chunks, in order: (group, K-chunk)
  int total = 0;
  for (int g = blockIdx.x; g < ngroups; g += gridDim.x) total += (__ldg(&groups[g].m) + kKc - 1) / kKc;

  if (warp < kConvWarps) {
    const int t = threadIdx.x;
    // fixed per thread: A pieces (row rr + 32 i = tile i, 16-byte group cg),
    // X pieces (row kx + 256 / (N / 4) * j, columns nx .. nx + 3) and B
    // pieces (row nb, 16-byte group kb + 256 / N * j)
    constexpr int n4 = N / 4;
    constexpr int XP = (kKc * n4 + kConvThreads - 1) / kConvThreads;   // X pieces per thread
    constexpr int BP = (N * (kKc / 4) + kConvThreads - 1) / kConvThreads;
    const int rr = t >> 3, cg = t & 7;
    const uint32_t so0 = sw128(rr, cg);   // + 4096 * i for tile i
    // load cursor state (per group)
    int lg = blockIdx.x, lkc = 0;
    const uint8_t* asrc[4];
    bool aok[4];
    int lm = 0, lmp = 0;
    const float* xbase = X;
    auto load_group = [&](int g) {
      const TcGroup* G = groups + g;
      lm = __ldg(&G->m);
      lmp = (lm + 3) & ~3;
      const int vt = __ldg(&G->vtab);
      if (vt < 0) {
        // leaf group: tile i holds rows 32 i .. 32 i + 31, row-major (stride lmp)
        const int ntl = __ldg(&G->ntl);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          aok[i] = i < ntl;
          asrc[i] = aok[i] ? pool + __ldg(&G->doff[i]) + ((size_t)rr * lmp + 4 * cg) * 4 : pool;
        }
      } else {
        // V group: row 32 i + rr is one V column, K contiguous
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const TcVRow* e = vrows + vt + 32 * i + rr;
          aok[i] = __ldg(&e->prow) >= 0;
          asrc[i] = aok[i] ? pool + __ldg(&e->off) + (size_t)cg * 16 : pool;
        }
      }
      xbase = X + (int64_t)__ldg(&G->xrow0) * ldx;
    };
    if (lg < ngroups) load_group(lg);
    auto issue = [&](int u) {
      if (u < total) {
        const int k0 = lkc * kKc;
        const uint32_t ra = raw0 + (uint32_t)(u % kTcRaw) * rb, rx = ra + ab;
        const bool kin = 4 * cg + k0 < lmp;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const bool ok = aok[i] && kin;
          cp_async16(ra + so0 + 4096u * i, ok ? (const void*)(asrc[i] + (size_t)k0 * 4) : (const void*)pool,
                     ok ? 16u : 0u);
        }
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
          lg += gridDim.x;
          if (lg < ngroups) load_group(lg);
        }
      }
      cp_async_commit();
    };
    // prologue: chunks 0 .. kTcRaw - 2 in flight
#pragma unroll 1
    for (int u = 0; u < kTcRaw - 1; ++u) issue(u);
    int cg_idx = blockIdx.x, ckc = 0, gcount = 0;   // compute cursor
    int cm = cg_idx < ngroups ? __ldg(&groups[cg_idx].m) : 0;
    int crows = cg_idx < ngroups ? __ldg(&groups[cg_idx].rows) : 0;
#pragma unroll 1
    for (int u = 0; u < total; ++u) {
      const int r = u % kTcRaw, b = u & 1;
      const uint32_t ra = raw0 + (uint32_t)r * rb, rx = ra + ab;
      const uint32_t oa = op0 + (uint32_t)b * ob;
      // chunk u's copies have landed (chunks u + 1 and u + 2 may be pending)
      cp_async_wait<kTcRaw - 2>();
      bar_conv();   // everybody's copies; everybody is done with raw stage (u - 1) % kTcRaw
      // the operand buffer of chunk u - 2 is free once its MMAs are done
      bool ok = !*(volatile int*)abort_flag;
      if (ok && u >= 2) ok = bar_wait(&mma_done[b], (uint32_t)(((u >> 1) - 1) & 1), err, 21);
      if (!ok) *(volatile int*)abort_flag = 1;
      // refill the raw stage of chunk u - 1 with chunk u + kTcRaw - 1
      issue(u + kTcRaw - 1);
      // A: split into hi and lo (rows past the group's valid rows keep
      // whatever the buffer held: they only reach accumulator rows that the
      // epilogue does not write)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (32 * i + rr >= crows) continue;
        const uint32_t o = so0 + 4096u * i;
        const uint4 v = lds16(ra + o);
        uint32_t h0, l0, h1, l1, h2, l2, h3, l3;
        split(__uint_as_float(v.x), h0, l0);
        split(__uint_as_float(v.y), h1, l1);
        split(__uint_as_float(v.z), h2, l2);
        split(__uint_as_float(v.w), h3, l3);
        sts4(oa + o, h0, h1, h2, h3);
        sts4(oa + ab + o, l0, l1, l2, l3);
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
          const uint32_t o = sw128(n, kg);
          sts4(oa + 2 * ab + o, h[0], h[1], h[2], h[3]);
          sts4(oa + 2 * ab + xb + o, l[0], l[1], l[2], l[3]);
        }
      }
      // generic-proxy stores -> visible to the tensor cores (async proxy)
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      bar_arrive(&conv_done[b]);
      // end of a group: epilogue by warps 0..3 (one TMEM lane quadrant each)
      if (++ckc * kKc >= cm) {
        if (warp < 4) {
          const TcGroup* G = groups + cg_idx;
          const bool okw = bar_wait(acc_ready, (uint32_t)(gcount & 1), err, 23) && !*(volatile int*)abort_flag;
          tc_fence_after();
          const int row = 32 * warp + lane;
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
#pragma unroll
          for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
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
        }
        ckc = 0;
        cg_idx += gridDim.x;
        cm = cg_idx < ngroups ? __ldg(&groups[cg_idx].m) : 0;
        crows = cg_idx < ngroups ? __ldg(&groups[cg_idx].rows) : 0;
        ++gcount;
        // the accumulator may be overwritten once the epilogue has read it
        asm volatile("bar.sync 2, %0;" ::"r"(kConvThreads + 32) : "memory");
      }
    }
    cp_async_wait<0>();
  } else {
    // ================= MMA issuer (warp kConvWarps) =================
    int ckc = 0, cg_idx = blockIdx.x;
    int cm = cg_idx < ngroups ? __ldg(&groups[cg_idx].m) : 0;
#pragma unroll 1
    for (int u = 0; u < total; ++u) {
      const int b = u & 1;
      if (lane == 0) {
        if (bar_wait(&conv_done[b], (uint32_t)((u >> 1) & 1), err, 22) && !*(volatile int*)abort_flag) {
          tc_fence_after();
          const uint32_t oa = op0 + (uint32_t)b * ob;
          const uint64_t ah = desc_sw128(oa), al = desc_sw128(oa + ab);
          const uint64_t bh = desc_sw128(oa + 2 * ab), bl = desc_sw128(oa + 2 * ab + xb);
#pragma unroll
          for (int ks = 0; ks < kKc / 8; ++ks) {
            const uint64_t adv = (uint64_t)(ks * 32) >> 4;   // 8 tf32 = 32 bytes along K
            mma_tf32(tmem, ah + adv, bh + adv, idesc, (ckc > 0 || ks > 0) ? 1u : 0u);
            mma_tf32(tmem, ah + adv, bl + adv, idesc, 1u);
            mma_tf32(tmem, al + adv, bh + adv, idesc, 1u);
          }
        } else {
          *(volatile int*)abort_flag = 1;
        }
        mma_commit(&mma_done[b]);
      }
      __syncwarp();
      if (++ckc * kKc >= cm) {
        if (lane == 0) mma_commit(acc_ready);
        ckc = 0;
        cg_idx += gridDim.x;
        cm = cg_idx < ngroups ? __ldg(&groups[cg_idx].m) : 0;
        // wait for the epilogue before the next group overwrites the accumulator
        asm volatile("bar.sync 2, %0;" ::"r"(kConvThreads + 32) : "memory");
        tc_fence_after();
      }
    }
  }
  __syncthreads();
  if (warp == kConvWarps) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
  }
}

int tc_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  }
  return n;
}

}  // namespace

size_t leaf_tc_smem(int N) { return tc_smem_bytes(N); }

namespace {
template <int N>
cudaError_t launch_n(const TcGroup* groups, int ngroups, const TcVRow* vrows, const uint8_t* pool,
                     const float* X, int64_t ldx, int nrhs, float* B, int64_t ldb, float* partials, int* err,
                     cudaStream_t s) {
  uint32_t cols = 32;
  while (cols < (uint32_t)N) cols <<= 1;
  const size_t smem = leaf_tc_smem(N);
  static size_t smem_set = 0;   // per instantiation
  if (smem > smem_set) {
    cudaError_t e = cudaFuncSetAttribute(leaf_tc_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    smem_set = smem;
  }
  const int grid = std::min(ngroups, tc_sms());
  leaf_tc_kernel<N><<<grid, kTcThreads, smem, s>>>(groups, ngroups, vrows, pool, X, ldx, nrhs, B, ldb, partials,
                                                    cols, err);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_leaf_tc(const TcGroup* groups, int ngroups, const TcVRow* vrows, const uint8_t* pool,
                           const float* X, int64_t ldx, int nrhs, float* B, int64_t ldb, float* partials,
                           int* err, cudaStream_t s) {
  if (ngroups == 0 || nrhs == 0) return cudaSuccess;
  const int N = (nrhs + 15) / 16 * 16;
  if (N < 16 || N > kTcMaxCols) return cudaErrorInvalidValue;
  switch (N) {
    case 16: return launch_n<16>(groups, ngroups, vrows, pool, X, ldx, nrhs, B, ldb, partials, err, s);
    case 32: return launch_n<32>(groups, ngroups, vrows, pool, X, ldx, nrhs, B, ldb, partials, err, s);
    case 48: return launch_n<48>(groups, ngroups, vrows, pool, X, ldx, nrhs, B, ldb, partials, err, s);
    default: return launch_n<64>(groups, ngroups, vrows, pool, X, ldx, nrhs, B, ldb, partials, err, s);
  }
}

}  // namespace hodlr
