// Batched HODLR products: many stored matrices (any sizes, ranks, formats;
// one working precision), each with its own X and B, in one persistent
// launch.  Each matrix's product (Algorithm 3.3) runs inside one CTA, so the
// launch needs no grid-wide dependency; the matrices are dealt to the CTAs
// longest first (by bytes) when the batch is planned.
//
// Per matrix, inside its CTA (warps over independent units, CTA barriers
// between the steps, every sum in a fixed order):
//   1. V^T X in units (node q, up to kLeavesPerUnit leaves of q's rows):
//      lanes over rows, a warp-reduced partial per unit and column of V_q;
//   2. Y_q = (sum of q's unit partials, in unit order) x the power-of-two
//      scales of V_q and U_{q^1};
//   3. per leaf (its X rows staged once in the warp's shared-memory slice)
//      and per 32-row tile of it (lane = row): D X from the tile's
//      interleaved leaf-block part, plus sum_k U_{a_k}[rows, :] Y_{a_k ^ 1}
//      from the tile's header and U region (a_k the level-k ancestor), the
//      U columns through shared memory in double-buffered pieces.
//
// hodlr_batch_create uploads the work list and allocates the scratch once;
// hodlr_batch_run is one kernel launch that allocates and copies nothing.
#include <algorithm>
#include <numeric>
#include <queue>
#include <vector>

#include "dev_common.cuh"
#include "handle.cuh"

namespace hodlr {
namespace {

constexpr int kLeavesPerUnit = 8;   // leaves of rows per V^T X unit
constexpr int kBatchMaxCols = 16;   // right-hand sides per matrix at most

struct BItem {
  const uint8_t* pool;
  const NodeDev* nodes;
  const LeafDev* leaves;
  const P2Tile* tiles;
  const int4* units;      // (node, first leaf, end leaf, first partial row)
  const int32_t* node_u;  // [nnodes + 1]: the node's units
  const int32_t* yoff;    // [nnodes]: first row of Y_q
  const int32_t* leaf_t0; // [nleaves + 1]: the leaf's first tile
  void* Y;                // rows x R
  void* P;                // partial rows x R
  const void* X;
  void* B;
  int64_t ldx, ldb;
  int32_t depth, R, nnodes, nunits, ntiles, nleaves;
  int32_t xvec;           // X rows load as 16-byte vectors (R and ldx multiples of 16 / sizeof, X aligned)
  int32_t rb;             // R rounded up to 1, 2, 4, 8 or 16: the item's column block and Y's row stride
};

constexpr int kXSlice = 8192;       // bytes of shared memory per warp for a leaf's X rows
constexpr int kUPiece = 3072;       // and for each of two pieces of a tile's U columns
constexpr int kSlice = kXSlice + 2 * kUPiece;

__device__ __forceinline__ int fmt_bytes(int tier) {
  return tier == HODLR_FP64 ? 8 : tier == HODLR_FP32 ? 4 : (tier == HODLR_E4M3 || tier == HODLR_E5M2) ? 1 : 2;
}

// 16-byte asynchronous global -> shared copies (completion per commit group)
__device__ __forceinline__ void bcp16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void bcp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void bcp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// One stored value of format P from shared memory, in the working precision
template <typename W, int P>
__device__ __forceinline__ W lds_fmt(const uint8_t* p) {
  if constexpr (P == HODLR_FP64) {
    return (W)*reinterpret_cast<const double*>(p);
  } else if constexpr (P == HODLR_FP32) {
    return (W)*reinterpret_cast<const float*>(p);
  } else if constexpr (P == HODLR_FP16) {
    return (W)__half2float(__ushort_as_half(*reinterpret_cast<const unsigned short*>(p)));
  } else if constexpr (P == HODLR_BF16) {
    return (W)__uint_as_float(((uint32_t)*reinterpret_cast<const unsigned short*>(p)) << 16);
  } else {
    __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)*p, P == HODLR_E4M3 ? __NV_E4M3 : __NV_E5M2);
    return (W)__half2float(*reinterpret_cast<__half*>(&h));
  }
}

template <typename W, int P>
__device__ __forceinline__ W ldg_fmt(const uint8_t* p) {
  if constexpr (P == HODLR_FP64) {
    return (W)__ldg(reinterpret_cast<const double*>(p));
  } else if constexpr (P == HODLR_FP32) {
    return (W)__ldg(reinterpret_cast<const float*>(p));
  } else if constexpr (P == HODLR_FP16) {
    return (W)__half2float(__ushort_as_half(__ldg(reinterpret_cast<const unsigned short*>(p))));
  } else if constexpr (P == HODLR_BF16) {
    return (W)__uint_as_float(((uint32_t)__ldg(reinterpret_cast<const unsigned short*>(p))) << 16);
  } else {
    const unsigned char b = __ldg(reinterpret_cast<const unsigned char*>(p));
    __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)b, P == HODLR_E4M3 ? __NV_E4M3 : __NV_E5M2);
    return (W)__half2float(*reinterpret_cast<__half*>(&h));
  }
}

// R values of an X row (zeros past R); XV: as 16-byte vectors (R a multiple
// of the vector width, the row 16-byte aligned)
// A row of RB values (a staged X row in shared memory, zeros past R, or a
// row of Y written earlier in this launch: plain loads), as 16-byte vectors
// when the row length allows
template <typename W, int RB>
__device__ __forceinline__ void ld_row(const W* x, W (&xv)[RB]) {
  if constexpr (RB * sizeof(W) % 16 == 0) {
#pragma unroll
    for (int j4 = 0; j4 < RB * (int)sizeof(W) / 16; ++j4) {
      const uint4 t = reinterpret_cast<const uint4*>(x)[j4];
      if constexpr (sizeof(W) == 4) {
        xv[4 * j4] = __uint_as_float(t.x);
        xv[4 * j4 + 1] = __uint_as_float(t.y);
        xv[4 * j4 + 2] = __uint_as_float(t.z);
        xv[4 * j4 + 3] = __uint_as_float(t.w);
      } else {
        xv[2 * j4] = __hiloint2double((int)t.y, (int)t.x);
        xv[2 * j4 + 1] = __hiloint2double((int)t.w, (int)t.z);
      }
    }
  } else {
#pragma unroll
    for (int j = 0; j < RB; ++j) xv[j] = x[j];
  }
}

template <typename W, int RB, bool XV>
__device__ __forceinline__ void ld_xrow(const W* x, int R, W (&xv)[RB]) {
  if constexpr (XV && sizeof(W) == 4 && RB % 4 == 0) {
#pragma unroll
    for (int j4 = 0; j4 < RB / 4; ++j4) {
      const float4 t = 4 * j4 < R ? __ldg(reinterpret_cast<const float4*>(x) + j4) : make_float4(0.f, 0.f, 0.f, 0.f);
      xv[4 * j4] = t.x;
      xv[4 * j4 + 1] = t.y;
      xv[4 * j4 + 2] = t.z;
      xv[4 * j4 + 3] = t.w;
    }
  } else if constexpr (XV && sizeof(W) == 8 && RB % 2 == 0) {
#pragma unroll
    for (int j2 = 0; j2 < RB / 2; ++j2) {
      const double2 t = 2 * j2 < R ? __ldg(reinterpret_cast<const double2*>(x) + j2) : make_double2(0.0, 0.0);
      xv[2 * j2] = (W)t.x;
      xv[2 * j2 + 1] = (W)t.y;
    }
  } else {
#pragma unroll
    for (int j = 0; j < RB; ++j) xv[j] = j < R ? __ldg(x + j) : (W)0;
  }
}

// Row steps unrolled in the V^T X units, V columns per pass and leaf-block
// chunks loaded ahead in the tile pass: more as the rows get narrower (the
// registers they take grow with RB).
template <typename W, int RB>
__host__ __device__ constexpr int batch_unroll() { return RB <= 2 ? 4 : RB <= 4 ? 2 : 1; }
template <typename W, int RB>
__host__ __device__ constexpr int batch_cols() {
  return sizeof(W) == 4 ? (RB <= 8 ? 8 : 4) : (RB <= 2 ? 8 : RB <= 4 ? 4 : RB <= 8 ? 2 : 1);
}
template <int RB>
__host__ __device__ constexpr int batch_dq() { return RB <= 4 ? 8 : 4; }

// One matrix's product by the whole CTA (the three steps above).
// Not inlined: each column block gets its own register allocation (inlined
// into one kernel, the widest block's spills reached every item).
template <typename W, int RB, bool XV>
__device__ __noinline__ void batch_item(const BItem& b) {
  constexpr int es = sizeof(W);
  constexpr int G16 = 16 / es;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const W* X = reinterpret_cast<const W*>(b.X);
    W* Y = reinterpret_cast<W*>(b.Y);
    W* P = reinterpret_cast<W*>(b.P);
    const int R = b.R;
    // ---- 1. V^T X per unit: CG columns of V_q at a time (independent
    //      loads in flight: CG V values and the X row per row step) ----
    for (int u = warp; u < b.nunits; u += nw) {
      const int4 un = b.units[u];
      const NodeDev& nd = b.nodes[un.x];
      auto unit = [&](auto tc) {
        constexpr int TIER = decltype(tc)::value;
        constexpr int eb = TIER == HODLR_FP64 ? 8 : TIER == HODLR_FP32 ? 4 : (TIER == HODLR_E4M3 || TIER == HODLR_E5M2) ? 1 : 2;
        constexpr int CG = batch_cols<W, RB>();
        for (int c0 = 0; c0 < nd.rV; c0 += CG) {
          W acc[CG][RB];
#pragma unroll
          for (int a = 0; a < CG; ++a)
#pragma unroll
            for (int j = 0; j < RB; ++j) acc[a][j] = (W)0;
          for (int l = un.y; l < un.z; ++l) {
            const LeafDev& lf = b.leaves[l];
            const int lm = lf.m, lrow0 = lf.row0;
            const uint8_t* col0 = b.pool + nd.offV + ((int64_t)c0 * nd.pm + (lf.prow0 - nd.prow0)) * eb;
            const int64_t cstride = (int64_t)nd.pm * eb;
            constexpr int kU = batch_unroll<W, RB>();
#pragma unroll kU
            for (int r = lane; r < lm; r += 32) {
              W xv[RB];
              ld_xrow<W, RB, XV>(X + (int64_t)(lrow0 + r) * b.ldx, R, xv);
#pragma unroll
              for (int a = 0; a < CG; ++a) {
                // columns past the rank read the last column (never stored)
                const int cc = min(a, nd.rV - 1 - c0);
                const W v = ldg_fmt<W, TIER>(col0 + cc * cstride + (int64_t)r * eb);
#pragma unroll
                for (int j = 0; j < RB; ++j) acc[a][j] = fma(v, xv[j], acc[a][j]);
              }
            }
          }
#pragma unroll
          for (int a = 0; a < CG; ++a) {
            if (c0 + a >= nd.rV) break;
#pragma unroll
            for (int j = 0; j < RB; ++j) {
              if (j >= R) break;
              const W sm = warp_sum(acc[a][j]);
              if (lane == 0) P[(int64_t)(un.w + c0 + a) * R + j] = sm;
            }
          }
        }
      };
      with_format(nd.tierV, unit);
    }
    __syncthreads();
    // ---- 2. Y_q = scales x (sum of the unit partials in order) ----
    for (int q = warp; q < b.nnodes; q += nw) {
      const NodeDev& nd = b.nodes[q];
      const W sc = (W)(nd.invsV * b.nodes[q ^ 1].invsU);
      const int u0 = b.node_u[q], u1 = b.node_u[q + 1];
      for (int e2 = lane; e2 < nd.rV * RB; e2 += 32) {
        const int c = e2 / RB, j = e2 - c * RB;
        W s = (W)0;
        if (j < R)
          for (int u = u0; u < u1; ++u) s += P[(int64_t)(b.units[u].w + c) * R + j];
        Y[(int64_t)(b.yoff[q] + c) * RB + j] = s * sc;   // rows of RB values, zeros past R
      }
    }
    __syncthreads();
    // ---- 3. B rows = D X + U Y.  Warp w takes leaves w, w + nw, ...: the
    //      leaf's X rows go once into the warp's shared-memory slice (when
    //      they fit), then its tiles, lane = row ----
    W* B = reinterpret_cast<W*>(b.B);
    extern __shared__ __align__(16) uint8_t bsm[];
    W* const xs = reinterpret_cast<W*>(bsm + (size_t)warp * kSlice);
    const uint32_t us = (uint32_t)__cvta_generic_to_shared(bsm + (size_t)warp * kSlice + kXSlice);
    for (int lf = warp; lf < b.nleaves; lf += nw) {
    const int lt0 = b.leaf_t0[lf], lt1 = b.leaf_t0[lf + 1];
    const int lm = b.tiles[lt0].m, lx0 = b.tiles[lt0].xrow0;
    const bool staged = (int64_t)lm * RB * es <= kXSlice;
    if (staged) {
      for (int e2 = lane; e2 < lm * RB; e2 += 32) {
        const int cc = e2 / RB, j = e2 - cc * RB;
        xs[e2] = j < R ? __ldg(X + (int64_t)(lx0 + cc) * b.ldx + j) : (W)0;
      }
    }
    __syncwarp();
    for (int t = lt0; t < lt1; ++t) {
      const P2Tile& tq = b.tiles[t];
      const int r = lane;
      const uint8_t* hdr = b.pool + tq.off;
      // The tile's U columns go through shared memory in pieces (whole
      // columns of one level, at most kUPiece bytes, 16-byte asynchronous
      // copies): the first piece is requested before the leaf-block part,
      // each next one before the current one is used.
      int pk = 1, pc = 0;   // the next piece starts at column pc of level pk
      auto issue = [&](int buf, int& ko, int& co, int& no) {
        ko = 0;
        while (pk <= b.depth) {
          const uint2 hw = __ldg(reinterpret_cast<const uint2*>(hdr) + (pk - 1));
          const int ru = (int)(hw.y & 0xffffu);
          if (pc < ru) {
            const int eb = fmt_bytes((int)(hw.y >> 16));
            const int nc = min(ru - pc, kUPiece / (kTileRows * eb));
            const uint8_t* src = hdr + tq.hbytes + hw.x + (int64_t)pc * kTileRows * eb;
            const int nv = nc * kTileRows * eb / 16;
            for (int v = lane; v < nv; v += 32) bcp16(us + buf * kUPiece + v * 16, src + v * 16);
            ko = pk;
            co = pc;
            no = nc;
            pc += nc;
            break;
          }
          ++pk;
          pc = 0;
        }
        bcp_commit();
      };
      int ck, cc0, cn;
      issue(0, ck, cc0, cn);
      W acc[RB];
#pragma unroll
      for (int j = 0; j < RB; ++j) acc[j] = (W)0;
      const uint8_t* d2 = b.pool + tq.d2off + (int64_t)r * 16;
      const int nchunk = (tq.m + G16 - 1) / G16;
      // DQ chunks of the leaf-block row loaded before any is used (16-byte
      // vectors, consecutive lanes consecutive rows); the X rows are the same
      // on every lane (shared-memory broadcasts when staged)
      constexpr int DQ = batch_dq<RB>();
      // two groups in flight: group q0 + DQ is requested before group q0 is used
      uint4 raw[DQ], nxt[DQ];
#pragma unroll
      for (int qq = 0; qq < DQ; ++qq)
        raw[qq] = qq < nchunk ? __ldg(reinterpret_cast<const uint4*>(d2 + (int64_t)qq * kTileRows * 16))
                              : make_uint4(0u, 0u, 0u, 0u);
      for (int q0 = 0; q0 < nchunk; q0 += DQ) {
#pragma unroll
        for (int qq = 0; qq < DQ; ++qq)
          nxt[qq] = q0 + DQ + qq < nchunk
                        ? __ldg(reinterpret_cast<const uint4*>(d2 + (int64_t)(q0 + DQ + qq) * kTileRows * 16))
                        : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int qq = 0; qq < DQ; ++qq) {
          W d[G16];
          if constexpr (sizeof(W) == 4) {
            d[0] = __uint_as_float(raw[qq].x);
            d[1] = __uint_as_float(raw[qq].y);
            d[2] = __uint_as_float(raw[qq].z);
            d[3] = __uint_as_float(raw[qq].w);
          } else {
            d[0] = __hiloint2double((int)raw[qq].y, (int)raw[qq].x);
            d[1] = __hiloint2double((int)raw[qq].w, (int)raw[qq].z);
          }
#pragma unroll
          for (int g = 0; g < G16; ++g) {
            const int cc = (q0 + qq) * G16 + g;
            if (cc >= tq.m) break;
            W xv[RB];
            if (staged)
              ld_row<W, RB>(xs + cc * RB, xv);
            else
              ld_xrow<W, RB, XV>(X + (int64_t)(tq.xrow0 + cc) * b.ldx, R, xv);
#pragma unroll
            for (int j = 0; j < RB; ++j) acc[j] = fma(d[g], xv[j], acc[j]);
          }
        }
#pragma unroll
        for (int qq = 0; qq < DQ; ++qq) raw[qq] = nxt[qq];
      }
      int buf = 0;
      while (ck) {
        int nk, nc0, nn;
        issue(buf ^ 1, nk, nc0, nn);
        if (nk) bcp_wait<1>(); else bcp_wait<0>();
        __syncwarp();   // every lane's copies of the current piece have landed
        const int tier = (int)(__ldg(reinterpret_cast<const uint2*>(hdr) + (ck - 1)).y >> 16);
        const int sib = node_index(ck, (tq.leaf >> (b.depth - ck)) ^ 1);
        const W* yb = Y + ((int64_t)b.yoff[sib] + cc0) * RB;
        const uint8_t* up = bsm + (size_t)warp * kSlice + kXSlice + buf * kUPiece;
        auto level = [&](auto tc) {
          constexpr int TIER = decltype(tc)::value;
          constexpr int eb = TIER == HODLR_FP64 ? 8 : TIER == HODLR_FP32 ? 4 : (TIER == HODLR_E4M3 || TIER == HODLR_E5M2) ? 1 : 2;
#pragma unroll 8
          for (int c = 0; c < cn; ++c) {
            const W uv = lds_fmt<W, TIER>(up + (c * kTileRows + r) * eb);
            W yv[RB];
            ld_row<W, RB>(yb + c * RB, yv);
#pragma unroll
            for (int j = 0; j < RB; ++j) acc[j] = fma(uv, yv[j], acc[j]);
          }
        };
        with_format(tier, level);
        __syncwarp();   // the piece is read before its buffer is refilled
        ck = nk;
        cc0 = nc0;
        cn = nn;
        buf ^= 1;
      }
      if (r < tq.rows) {
        W* brow = B + (int64_t)(tq.row0 + r) * b.ldb;
#pragma unroll
        for (int j = 0; j < RB; ++j)
          if (j < R) brow[j] = acc[j];
      }
    }
    __syncwarp();   // the slice is read before the next leaf's rows overwrite it
    }
}

template <typename W, int RB>
__device__ __forceinline__ void batch_item_rb(const BItem& b) {
  if (b.xvec)
    batch_item<W, RB, true>(b);
  else
    batch_item<W, RB, false>(b);
}

// Each item runs with its own column block (so one with few right-hand
// sides does no work for the widest item's columns).
template <typename W>
__global__ void __launch_bounds__(512, 1)
batch_kernel(const BItem* __restrict__ items, const int32_t* __restrict__ cta_first, const int32_t* __restrict__ cta_items) {
  for (int e = cta_first[blockIdx.x]; e < cta_first[blockIdx.x + 1]; ++e) {
    const BItem& b = items[cta_items[e]];
    switch (b.rb) {
      case 1: batch_item_rb<W, 1>(b); break;
      case 2: batch_item_rb<W, 2>(b); break;
      case 4: batch_item_rb<W, 4>(b); break;
      case 8: batch_item_rb<W, 8>(b); break;
      default: batch_item_rb<W, 16>(b); break;
    }
    __syncthreads();
  }
}

template <typename W>
cudaError_t launch_batch_w(int grid, int threads, const BItem* items, const int32_t* first, const int32_t* list,
                           cudaStream_t s) {
  const int smem = (threads / 32) * kSlice;
  static int smem_set = 0;   // per instantiation: largest size opted in so far
  if (smem > smem_set) {
    cudaError_t e = cudaFuncSetAttribute(batch_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    smem_set = smem;
  }
  batch_kernel<W><<<grid, threads, smem, s>>>(items, first, list);
  return cudaGetLastError();
}

}  // namespace
}  // namespace hodlr

using namespace hodlr;

struct hodlr_batch_s {
  int count = 0, work = HODLR_FP32, grid = 1, threads = 256, device = 0;
  BItem* d_items = nullptr;
  int32_t* d_first = nullptr;
  int32_t* d_list = nullptr;
  uint8_t* d_meta = nullptr;   // units, node_u, yoff of every item
  void* d_scratch = nullptr;   // Y and P of every item
  ~hodlr_batch_s() {
    cudaFree(d_items);
    cudaFree(d_first);
    cudaFree(d_list);
    cudaFree(d_meta);
    cudaFree(d_scratch);
  }
};

extern "C" hodlr_status hodlr_batch_create(int32_t count, const hodlr_t* hs, const int32_t* nrhs, const void* const* X,
                                           const int64_t* ldx, void* const* B, const int64_t* ldb, int32_t xb_prec,
                                           hodlr_batch_t* out) {
  if (!out) return set_error(HODLR_EINVAL, "null out");
  *out = nullptr;
  if (count < 1 || !hs || !nrhs || !X || !ldx || !B || !ldb) return set_error(HODLR_EINVAL, "bad batch arguments");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_cuda_error(e, "cudaGetDevice");
  if (xb_prec != HODLR_FP32 && xb_prec != HODLR_FP64) return set_error(HODLR_EINVAL, "X/B precision must be fp32 or fp64");
  const int es = prec_bytes(xb_prec);
  for (int i = 0; i < count; ++i) {
    const hodlr_t h = hs[i];
    if (!h) return set_error(HODLR_EINVAL, "null handle in the batch");
    if (h->device != dev) return set_error(HODLR_EINVAL, "a handle lives on another device than the current one");
    if (h->work != xb_prec) return set_error(HODLR_EINVAL, "X/B type must equal every matrix's working precision");
    if (nrhs[i] < 1 || nrhs[i] > kBatchMaxCols) return set_error(HODLR_EINVAL, "nrhs must be in [1, 16]");
    if (!X[i] || !B[i] || ldx[i] < nrhs[i] || ldb[i] < nrhs[i]) return set_error(HODLR_EINVAL, "bad X/B of an item");
  }
  hodlr_batch_s* bt = new hodlr_batch_s();
  bt->count = count;
  bt->work = xb_prec;
  bt->device = dev;
  // work lists: units, node_u, yoff (int32 words) of every item, scratch rows
  std::vector<int32_t> meta;
  std::vector<size_t> meta_units(count), meta_nodeu(count), meta_yoff(count), meta_lt0(count);
  std::vector<int64_t> y_off(count), p_off(count);
  std::vector<BItem> items(count);
  std::vector<int> nunits(count);
  int64_t scratch = 0;
  std::vector<double> cost(count);
  for (int i = 0; i < count; ++i) {
    const hodlr_t h = hs[i];
    const int depth = h->depth, nnodes = (int)h->nodes.size();
    std::vector<int4> units;
    std::vector<int32_t> node_u(nnodes + 1, 0), yoff(std::max(nnodes, 1), 0);
    int poff = 0, yrows = 0;
    for (int k = 1; k <= depth; ++k) {
      const int span = 1 << (depth - k);
      for (int j = 0; j < (1 << k); ++j) {
        const int q = node_index(k, j);
        node_u[q] = (int)units.size();
        yoff[q] = yrows;
        yrows += h->nodes[q].rV;
        if (h->nodes[q].rV == 0) continue;
        for (int l0 = j * span; l0 < (j + 1) * span; l0 += kLeavesPerUnit) {
          const int l1 = std::min(l0 + kLeavesPerUnit, (j + 1) * span);
          units.push_back(make_int4(q, l0, l1, poff));
          poff += h->nodes[q].rV;
        }
      }
    }
    node_u[nnodes] = (int)units.size();   // nodes were visited in index order
    nunits[i] = (int)units.size();
    // align each section to 16 bytes
    while (meta.size() % 4) meta.push_back(0);
    meta_units[i] = meta.size();
    for (const int4& u : units) {
      meta.push_back(u.x);
      meta.push_back(u.y);
      meta.push_back(u.z);
      meta.push_back(u.w);
    }
    meta_nodeu[i] = meta.size();
    meta.insert(meta.end(), node_u.begin(), node_u.end());
    meta_yoff[i] = meta.size();
    meta.insert(meta.end(), yoff.begin(), yoff.end());
    {
      const int nleaves = (int)h->leaves.size();
      std::vector<int32_t> lt0(nleaves + 1, (int)h->p2.size());
      for (int t = (int)h->p2.size() - 1; t >= 0; --t) lt0[h->p2[t].leaf] = t;
      meta_lt0[i] = meta.size();
      meta.insert(meta.end(), lt0.begin(), lt0.end());
    }
    const int rb = nrhs[i] <= 1 ? 1 : nrhs[i] <= 2 ? 2 : nrhs[i] <= 4 ? 4 : nrhs[i] <= 8 ? 8 : 16;
    scratch = (scratch + 16 / es - 1) / (16 / es) * (16 / es);   // Y rows load as 16-byte vectors
    y_off[i] = scratch;
    scratch += (int64_t)std::max(yrows, 1) * rb;
    p_off[i] = scratch;
    scratch += (int64_t)std::max(poff, 1) * nrhs[i];
    BItem& it = items[i];
    memset(&it, 0, sizeof(it));
    it.pool = h->d_pool;
    it.nodes = h->d_nodes;
    it.leaves = h->d_leaves;
    it.tiles = h->d_p2;
    it.X = X[i];
    it.B = B[i];
    it.ldx = ldx[i];
    it.ldb = ldb[i];
    it.depth = depth;
    it.R = nrhs[i];
    it.nnodes = nnodes;
    it.nunits = nunits[i];
    it.ntiles = (int)h->p2.size();
    it.nleaves = (int)h->leaves.size();
    it.rb = rb;
    {
      const int vw = 16 / es;   // elements per 16-byte vector
      it.xvec = nrhs[i] % vw == 0 && ldx[i] % vw == 0 && reinterpret_cast<uintptr_t>(X[i]) % 16 == 0 ? 1 : 0;
    }
    // bytes read and written (measured: dealing by a multiply-add count
    // instead balanced the CTAs worse)
    cost[i] = (double)(h->info.leaf_bytes + h->info.factor_bytes) + 2.0 * h->n * nrhs[i] * es;
  }
  e = cudaMalloc(&bt->d_meta, std::max<size_t>(meta.size(), 4) * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&bt->d_scratch, (size_t)std::max<int64_t>(scratch, 1) * es);
  if (e == cudaSuccess) e = cudaMalloc(&bt->d_items, sizeof(BItem) * count);
  int G = 1;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&G, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    delete bt;
    return set_error(HODLR_ENOMEM, "batch work list");
  }
  G = std::max(1, std::min(G, count));
  bt->grid = G;
  const int32_t* dm = reinterpret_cast<const int32_t*>(bt->d_meta);
  for (int i = 0; i < count; ++i) {
    items[i].units = reinterpret_cast<const int4*>(dm + meta_units[i]);
    items[i].node_u = dm + meta_nodeu[i];
    items[i].yoff = dm + meta_yoff[i];
    items[i].leaf_t0 = dm + meta_lt0[i];
    items[i].Y = (uint8_t*)bt->d_scratch + (size_t)y_off[i] * es;
    items[i].P = (uint8_t*)bt->d_scratch + (size_t)p_off[i] * es;
  }
  // longest first onto the least-loaded CTA (deterministic ties: lower index)
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cost[a] > cost[c]; });
  using Load = std::pair<double, int>;
  std::priority_queue<Load, std::vector<Load>, std::greater<Load>> pq;
  for (int c = 0; c < G; ++c) pq.push({0.0, c});
  std::vector<std::vector<int>> per(G);
  for (int i : order) {
    Load l = pq.top();
    pq.pop();
    per[l.second].push_back(i);
    pq.push({l.first + cost[i], l.second});
  }
  std::vector<int32_t> first(G + 1, 0), list;
  for (int c = 0; c < G; ++c) {
    first[c] = (int)list.size();
    list.insert(list.end(), per[c].begin(), per[c].end());
  }
  first[G] = (int)list.size();
  e = cudaMalloc(&bt->d_first, sizeof(int32_t) * (G + 1));
  if (e == cudaSuccess) e = cudaMalloc(&bt->d_list, sizeof(int32_t) * count);
  if (e == cudaSuccess) e = cudaMemcpy(bt->d_meta, meta.data(), meta.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(bt->d_items, items.data(), sizeof(BItem) * count, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(bt->d_first, first.data(), sizeof(int32_t) * (G + 1), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(bt->d_list, list.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    delete bt;
    return set_cuda_error(e, "hodlr_batch_create");
  }
  *out = bt;
  return HODLR_OK;
}

extern "C" hodlr_status hodlr_batch_run(hodlr_batch_t b, int32_t threads, void* stream) {
  if (!b) return set_error(HODLR_EINVAL, "null batch");
  if (threads == 0) threads = b->threads;
  if (threads != 128 && threads != 256 && threads != 512) return set_error(HODLR_EINVAL, "threads must be 128, 256 or 512");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = b->work == HODLR_FP64
                      ? launch_batch_w<double>(b->grid, threads, b->d_items, b->d_first, b->d_list, s)
                      : launch_batch_w<float>(b->grid, threads, b->d_items, b->d_first, b->d_list, s);
  return e == cudaSuccess ? HODLR_OK : set_cuda_error(e, "hodlr_batch_run");
}

extern "C" hodlr_status hodlr_batch_tune(hodlr_batch_t b, void* stream, int32_t* best_threads, float* best_ms) {
  if (!b) return set_error(HODLR_EINVAL, "null batch");
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return set_error(HODLR_ECUDA, "hodlr_batch_tune: events");
  }
  int best = b->threads;
  float bms = 1e30f;
  hodlr_status st = HODLR_OK;
  for (int th : {128, 256, 512}) {
    for (int w = 0; w < 2 && st == HODLR_OK; ++w) st = hodlr_batch_run(b, th, stream);
    float tot = 0.0f;
    for (int rep = 0; rep < 5 && st == HODLR_OK; ++rep) {
      cudaEventRecord(e0, s);
      st = hodlr_batch_run(b, th, stream);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) st = set_error(HODLR_ECUDA, "hodlr_batch_tune");
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      tot += ms;
    }
    if (st != HODLR_OK) break;
    if (tot / 5 < bms) {
      bms = tot / 5;
      best = th;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != HODLR_OK) return st;
  b->threads = best;
  if (best_threads) *best_threads = best;
  if (best_ms) *best_ms = bms;
  return HODLR_OK;
}

extern "C" void hodlr_batch_destroy(hodlr_batch_t b) { delete b; }
