// Internal data structures and device helpers of libhodlr.
//
// Storage layout in HBM (one pool per handle):
//  * padded row space: leaf l occupies padded rows [prow0_l, prow0_l + pm_l)
//    with pm_l = m_l rounded up to a multiple of 16; a node at any level covers
//    the padded rows of its leaves, so every tile of 4 rows that starts on a
//    multiple of 4 inside a leaf is 16-byte aligned in every format;
//  * generators are stored column by column ("rank-major"): column c of U_i is
//    pm_i contiguous elements of the block's storage format, padding zeroed.
//    Threads run along rows, so loads of every format are coalesced and no
//    rank padding is needed;
//  * leaves D_i are stored column-major with the same padded row length;
//  * fp16/e4m3/e5m2 generators hold s*U, s*V with a per-block power-of-two s;
//    the kernels multiply by 1/s (exact).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include "../../include/hodlr.h"

namespace hodlr {

constexpr int kRowPad = 16;          // padded leaf length multiple (elements)
constexpr int kP2Rows = 32;          // rows per product tile (phase 2)
constexpr int kP1Rows = 4096;        // padded rows per phase-1 work item (whole leaves)
constexpr int kP1MaxLeaves = 256;    // leaves per phase-1 work item at most
constexpr int kMaxLeaf = 1024;       // largest leaf supported by the product kernels
constexpr int kPrecCount = 6;

struct NodeDev {
  int32_t level, idx;
  int32_t row0, m;        // real rows
  int32_t prow0, pm;      // padded rows
  int32_t rU, rV;         // rank of U_i (block (i,i^1)) and of V_i (block (i^1,i))
  int32_t tierU, tierV;   // hodlr_prec of U_i and of V_i
  double invsU, invsV;    // 1/s of U_i and V_i (1 for unscaled formats)
  int64_t offU, offV;     // byte offsets of column 0 in the pool
  int32_t yoff;           // Y_i = V_i^T X lives at rows [yoff, yoff+rV) of the Y buffer
  int32_t pad_;
};

struct LeafDev {
  int32_t row0, m, prow0, pm;
  int64_t offD;           // byte offset of column 0 (working precision)
  int32_t node;           // node index of the leaf (level depth), -1 when depth == 0
  int32_t pad_;
};

// Phase-1 work item: V_node^T X over the leaves [leaf0, leaf0 + nleaf) of node.
struct P1Item {
  int32_t node, leaf0, nleaf;
  int32_t item_in_node, nitems;   // position among the node's items
  int32_t poff;                   // partial sums at rows [poff, poff + rV) of the partial buffer
};

// Phase-2 work item: rows [t0, t0 + kP2Rows) of a leaf.
struct P2Item {
  int32_t leaf, t0;
};

// Device-resident description of a handle (passed by value to kernels).
struct HandleDev {
  const NodeDev* nodes;
  const LeafDev* leaves;
  const P1Item* p1;
  const P2Item* p2;
  const uint8_t* pool;
  int32_t n, depth, n_nodes, n_leaves;
  int32_t n_p1, n_p2;
  int32_t y_rows, p_rows;         // rows (rank units) of the Y and partial buffers
  int32_t sum_r_max;              // max over leaves of sum_k rU(ancestor_k)
  int32_t leaf_pm_max;
};

__host__ __device__ inline int node_index(int k, int i) { return (1 << k) - 2 + i; }

__host__ __device__ inline int prec_bytes(int p) {
  switch (p) {
    case HODLR_FP64: return 8;
    case HODLR_FP32: return 4;
    case HODLR_FP16: return 2;
    case HODLR_BF16: return 2;
    default: return 1;
  }
}

// ---- decoding of the storage formats into the working precision ----------
// Loads 4 consecutive elements (16-byte aligned group of 4) of format P and
// converts them exactly (or, for fp64 -> fp32 work, with one rounding).
template <typename W>
struct Vec4 { W x, y, z, w; };

template <typename W>
__device__ __forceinline__ Vec4<W> load4(const uint8_t* base, int prec) {
  Vec4<W> r;
  switch (prec) {
    case HODLR_FP64: {
      const double2* p = reinterpret_cast<const double2*>(base);
      double2 a = __ldg(p), b = __ldg(p + 1);
      r.x = (W)a.x; r.y = (W)a.y; r.z = (W)b.x; r.w = (W)b.y;
      break;
    }
    case HODLR_FP32: {
      float4 a = __ldg(reinterpret_cast<const float4*>(base));
      r.x = (W)a.x; r.y = (W)a.y; r.z = (W)a.z; r.w = (W)a.w;
      break;
    }
    case HODLR_FP16: {
      uint2 a = __ldg(reinterpret_cast<const uint2*>(base));
      __half2 h0 = *reinterpret_cast<__half2*>(&a.x), h1 = *reinterpret_cast<__half2*>(&a.y);
      float2 f0 = __half22float2(h0), f1 = __half22float2(h1);
      r.x = (W)f0.x; r.y = (W)f0.y; r.z = (W)f1.x; r.w = (W)f1.y;
      break;
    }
    case HODLR_BF16: {
      uint2 a = __ldg(reinterpret_cast<const uint2*>(base));
      r.x = (W)__uint_as_float(a.x << 16); r.y = (W)__uint_as_float(a.x & 0xffff0000u);
      r.z = (W)__uint_as_float(a.y << 16); r.w = (W)__uint_as_float(a.y & 0xffff0000u);
      break;
    }
    case HODLR_E4M3:
    case HODLR_E5M2: {
      uint32_t a = __ldg(reinterpret_cast<const unsigned int*>(base));
      __nv_fp8_interpretation_t it = prec == HODLR_E4M3 ? __NV_E4M3 : __NV_E5M2;
      __half2_raw h0 = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(a & 0xffffu), it);
      __half2_raw h1 = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(a >> 16), it);
      float2 f0 = __half22float2(*reinterpret_cast<__half2*>(&h0));
      float2 f1 = __half22float2(*reinterpret_cast<__half2*>(&h1));
      r.x = (W)f0.x; r.y = (W)f0.y; r.z = (W)f1.x; r.w = (W)f1.y;
      break;
    }
    default:
      r.x = r.y = r.z = r.w = (W)0;
  }
  return r;
}

// One element of format P decoded to double (exact).
__device__ __forceinline__ double load1_f64(const uint8_t* base, int prec) {
  switch (prec) {
    case HODLR_FP64: return *reinterpret_cast<const double*>(base);
    case HODLR_FP32: return (double)*reinterpret_cast<const float*>(base);
    case HODLR_FP16: return (double)__half2float(*reinterpret_cast<const __half*>(base));
    case HODLR_BF16: {
      uint16_t b = *reinterpret_cast<const uint16_t*>(base);
      return (double)__uint_as_float(((uint32_t)b) << 16);
    }
    case HODLR_E4M3:
    case HODLR_E5M2: {
      __half_raw h = __nv_cvt_fp8_to_halfraw(*reinterpret_cast<const __nv_fp8_storage_t*>(base),
                                             prec == HODLR_E4M3 ? __NV_E4M3 : __NV_E5M2);
      return (double)__half2float(*reinterpret_cast<__half*>(&h));
    }
  }
  return 0.0;
}

// ---- encoding: fp64 -> format, round to nearest, ties to even ------------
// Narrow formats go through fp32 with round-to-odd, which makes the second
// rounding (to nearest even) equal to a single rounding from fp64 because
// fp32 keeps at least two more significand bits than every narrow target.
__device__ __forceinline__ float f64_to_f32_round_odd(double x) {
  float f = __double2float_rz(x);
  if ((double)f != x) f = __uint_as_float(__float_as_uint(f) | 1u);
  return f;
}

__device__ __forceinline__ void store1(uint8_t* base, int prec, double x) {
  switch (prec) {
    case HODLR_FP64: *reinterpret_cast<double*>(base) = x; break;
    case HODLR_FP32: *reinterpret_cast<float*>(base) = __double2float_rn(x); break;
    case HODLR_FP16:
      *reinterpret_cast<__half*>(base) = __float2half_rn(f64_to_f32_round_odd(x));
      break;
    case HODLR_BF16:
      *reinterpret_cast<__nv_bfloat16*>(base) = __float2bfloat16_rn(f64_to_f32_round_odd(x));
      break;
    case HODLR_E4M3:
      *reinterpret_cast<__nv_fp8_storage_t*>(base) =
          __nv_cvt_float_to_fp8(f64_to_f32_round_odd(x), __NV_SATFINITE, __NV_E4M3);
      break;
    case HODLR_E5M2:
      *reinterpret_cast<__nv_fp8_storage_t*>(base) =
          __nv_cvt_float_to_fp8(f64_to_f32_round_odd(x), __NV_SATFINITE, __NV_E5M2);
      break;
  }
}

// ---- kernel-matrix entries (eq. (4.1) and the synthetic workloads) ---------
// A_ij = f(r_ij) + diag*delta_ij; at i == j, f is f(0) where finite, else 0.
__device__ __forceinline__ double kernel_entry(const double* __restrict__ pts, int dim, int i, int j,
                                               int kind, double c, double len2, double diag) {
  if (kind == 3) {  // 1/(x_i - x_j), 1D; 0 at i == j plus diag
    if (i == j) return diag;
    return 1.0 / (pts[i] - pts[j]);
  }
  double r2 = 0.0;
  for (int d = 0; d < dim; ++d) {
    const double t = pts[(int64_t)i * dim + d] - pts[(int64_t)j * dim + d];
    r2 = fma(t, t, r2);
  }
  double f;
  if (kind == 1) {
    f = exp(-r2 / len2);
  } else if (i == j) {
    // f(0) where it is finite, 0 for the singular kernels
    f = c > 0.0 ? (kind == 0 ? 1.0 / c : log(c)) : 0.0;
  } else {
    const double r = sqrt(r2);
    f = kind == 0 ? 1.0 / (r + c) : log(r + c);
  }
  return i == j ? f + diag : f;
}

// ---- kernel launchers implemented in the .cu files -------------------------
struct PackTask {          // one column of one generator or leaf
  int64_t src;             // element offset of (row 0, column c) in the fp64 staging
  int32_t src_stride;      // elements between consecutive rows in the staging
  int32_t m, pm;           // rows, padded rows
  int64_t dst;             // byte offset of the column in the pool
  int32_t prec;
  int32_t pad_;
  double scale;            // multiply before rounding (power of two)
};

struct NormTask {          // sum of squares and max |.| of one fp64 matrix
  int64_t src;
  int64_t count;
};

cudaError_t launch_norms(const double* staging, const NormTask* tasks, int ntasks,
                         double* sumsq, double* amax, cudaStream_t s);
cudaError_t launch_pack(const double* staging, const PackTask* tasks, int ntasks,
                        uint8_t* pool, cudaStream_t s);
cudaError_t launch_unpack(const uint8_t* pool, const PackTask* tasks, int ntasks,
                          double* staging, cudaStream_t s);

// ev (may be null): three events recorded before phase 1, between the phases
// and after phase 2.
cudaError_t launch_matvec(const HandleDev& hd, int work, int nrhs, const void* X, int64_t ldx,
                          void* B, int64_t ldb, void* Y, void* partials, unsigned* counters,
                          cudaStream_t s, cudaEvent_t* ev);

cudaError_t launch_dense_kernel_matvec(int n, int dim, const double* pts, int kind, double c,
                                       double len2, double diag, int nrows, const int32_t* rows,
                                       int nrhs, const double* X, int64_t ldx, double* B,
                                       int64_t ldb, cudaStream_t s);

}  // namespace hodlr
