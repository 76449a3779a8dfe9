// Device helpers shared by the product kernels: bounded mbarrier waits,
// bulk asynchronous copies, explicit shared-memory accesses, decoding of the
// storage formats, and the bounded grid-counter wait.
#pragma once

#include <type_traits>

#include "hodlr_internal.cuh"

namespace hodlr {

constexpr unsigned long long kWaitLimitNs = 2000000000ull;   // every wait gives up after 2 s

template <typename W> struct WorkPrec;
template <> struct WorkPrec<float> { static constexpr int value = HODLR_FP32; };
template <> struct WorkPrec<double> { static constexpr int value = HODLR_FP64; };

// ---- PTX helpers ----------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// One test of the phase; a thread whose phase is not complete is suspended
// in hardware until it completes or about kSuspendNs pass (no busy polling
// of shared memory by waiting warps).
constexpr uint32_t kSuspendNs = 1000000;
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendNs)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: polls for a short while (the common case: the phase
// completes within microseconds), then sleeps in try_wait; false (and the
// error word set) if the phase has not completed within kWaitLimitNs.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err, int code) {
  for (int k = 0; k < 4; ++k)
    if (mbar_test_wait(bar, parity)) return true;
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > kWaitLimitNs) break;
  }
  atomicExch(err, code);
  return false;
}
// Bulk asynchronous copy global -> shared (16-byte aligned, size multiple of 16).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

template <typename W>
__device__ __forceinline__ W warp_sum(W v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// CPL consecutive values of a row (8- or 16-byte aligned when CPL = 2, 16
// when CPL = 4, fp32 only).
template <typename W, int CPL>
__device__ __forceinline__ void load_cols(const W* p, bool global, W (&v)[CPL]) {
  static_assert(CPL <= 2 || (CPL == 4 && sizeof(W) == 4), "four columns per lane in fp32 only");
  if constexpr (CPL == 1) {
    v[0] = global ? __ldg(p) : *p;
  } else if constexpr (CPL == 4) {
    const float4 t = global ? __ldg(reinterpret_cast<const float4*>(p)) : *reinterpret_cast<const float4*>(p);
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
  } else if constexpr (sizeof(W) == 4) {
    const float2 t = global ? __ldg(reinterpret_cast<const float2*>(p)) : *reinterpret_cast<const float2*>(p);
    v[0] = t.x;
    v[1] = t.y;
  } else {
    const double2 t = global ? __ldg(reinterpret_cast<const double2*>(p)) : *reinterpret_cast<const double2*>(p);
    v[0] = t.x;
    v[1] = t.y;
  }
}
template <typename W, int CPL>
__device__ __forceinline__ void store_cols(W* p, const W (&v)[CPL]) {
  if constexpr (CPL == 1) {
    *p = v[0];
  } else if constexpr (CPL == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else if constexpr (sizeof(W) == 4) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  } else {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  }
}

// ---- explicit shared-memory accesses (addresses in the shared window) ----
// The hot loops address shared memory through these so that every access is
// a shared-memory instruction, whatever the compiler can prove about a
// pointer (a generic access that may go to global memory is much slower).
__device__ __forceinline__ float sld_f32(uint32_t a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ double sld_f64(uint32_t a) {
  double v;
  asm volatile("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ uint32_t sld_u32(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ uint16_t sld_u16(uint32_t a) {
  uint16_t v;
  asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ uint16_t sld_u8(uint32_t a) {
  uint16_t v;
  asm volatile("ld.shared.u8 %0, [%1];" : "=h"(v) : "r"(a));
  return v;
}
template <typename W>
__device__ __forceinline__ W sld(uint32_t a) {
  if constexpr (sizeof(W) == 4) return sld_f32(a);
  else return sld_f64(a);
}
template <typename W>
__device__ __forceinline__ void sst(uint32_t a, W v) {
  if constexpr (sizeof(W) == 4) asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
  else asm volatile("st.shared.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory");
}
// CPL consecutive values of W (8- or 16-byte aligned when CPL = 2)
template <typename W, int CPL>
__device__ __forceinline__ void sld_cols(uint32_t a, W (&v)[CPL]) {
  if constexpr (CPL == 1) {
    v[0] = sld<W>(a);
  } else if constexpr (CPL == 4) {
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]) : "r"(a));
  } else if constexpr (sizeof(W) == 4) {
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v[0]), "=f"(v[1]) : "r"(a));
  } else {
    asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(v[0]), "=d"(v[1]) : "r"(a));
  }
}
template <typename W, int CPL>
__device__ __forceinline__ void sst_cols(uint32_t a, const W (&v)[CPL]) {
#pragma unroll
  for (int j = 0; j < CPL; ++j) sst<W>(a + j * (uint32_t)sizeof(W), v[j]);
}
// four consecutive fp32 values (16-byte aligned)
__device__ __forceinline__ float4 sld_v4f32(uint32_t a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
  return v;
}
__device__ __forceinline__ void sst_v4f32(uint32_t a, float4 v) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
               : "memory");
}
// N consecutive values of W (16-byte aligned, N a multiple of 4)
template <typename W, int N>
__device__ __forceinline__ void sld_vec(uint32_t a, W (&v)[N]) {
  if constexpr (sizeof(W) == 4) {
#pragma unroll
    for (int j4 = 0; j4 < N / 4; ++j4) {
      const float4 t = sld_v4f32(a + 16u * j4);
      v[4 * j4 + 0] = t.x;
      v[4 * j4 + 1] = t.y;
      v[4 * j4 + 2] = t.z;
      v[4 * j4 + 3] = t.w;
    }
  } else {
#pragma unroll
    for (int j2 = 0; j2 < N / 2; ++j2)
      asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(v[2 * j2]), "=d"(v[2 * j2 + 1]) : "r"(a + 16u * j2));
  }
}
// one element of storage format P (compile time), decoded into W
template <typename W, int P>
__device__ __forceinline__ W sld_fmt(uint32_t a) {
  if constexpr (P == HODLR_FP64) {
    return (W)sld_f64(a);
  } else if constexpr (P == HODLR_FP32) {
    return (W)sld_f32(a);
  } else if constexpr (P == HODLR_FP16) {
    return (W)__half2float(__ushort_as_half(sld_u16(a)));
  } else if constexpr (P == HODLR_BF16) {
    return (W)__uint_as_float(((uint32_t)sld_u16(a)) << 16);
  } else {
    __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)sld_u8(a), P == HODLR_E4M3 ? __NV_E4M3 : __NV_E5M2);
    return (W)__half2float(*reinterpret_cast<__half*>(&h));
  }
}

// Calls f with the storage format as a compile-time constant (an if-chain,
// fp32 first).
template <typename F>
__device__ __forceinline__ void with_format(int tier, F&& f) {
  if (tier == HODLR_FP32) f(std::integral_constant<int, HODLR_FP32>{});
  else if (tier == HODLR_BF16) f(std::integral_constant<int, HODLR_BF16>{});
  else if (tier == HODLR_FP16) f(std::integral_constant<int, HODLR_FP16>{});
  else if (tier == HODLR_FP64) f(std::integral_constant<int, HODLR_FP64>{});
  else if (tier == HODLR_E4M3) f(std::integral_constant<int, HODLR_E4M3>{});
  else f(std::integral_constant<int, HODLR_E5M2>{});
}

// Bounded wait until the grid counter reaches target (acquire).
__device__ __forceinline__ bool grid_wait(unsigned long long* counter, unsigned long long target, int* err) {
  const unsigned long long t0 = global_ns();
  while (true) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(counter) : "memory");
    if (v >= target) return true;
    if (global_ns() - t0 > kWaitLimitNs) {
      atomicExch(err, 5);
      return false;
    }
    __nanosleep(64);
  }
}

// One element of storage format P (compile time) from global memory, in W.
template <typename W, int P>
__device__ __forceinline__ W gld_fmt(const uint8_t* p) {
  if constexpr (P == HODLR_FP64) {
    return (W)__ldg(reinterpret_cast<const double*>(p));
  } else if constexpr (P == HODLR_FP32) {
    return (W)__ldg(reinterpret_cast<const float*>(p));
  } else if constexpr (P == HODLR_FP16) {
    return (W)__half2float(__ushort_as_half(__ldg(reinterpret_cast<const unsigned short*>(p))));
  } else if constexpr (P == HODLR_BF16) {
    return (W)__uint_as_float(((uint32_t)__ldg(reinterpret_cast<const unsigned short*>(p))) << 16);
  } else {
    __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)__ldg(reinterpret_cast<const unsigned char*>(p)),
                                           P == HODLR_E4M3 ? __NV_E4M3 : __NV_E5M2);
    return (W)__half2float(*reinterpret_cast<__half*>(&h));
  }
}

}  // namespace hodlr
