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
// The same three steps serve a partitioned product (part j of tree level g:
// its leaves' rows), each over the whole grid as its own launch, with the
// summed levels' Y rows in a buffer that the parts add up between steps 2
// and 3.
//
// Included by batch_f32.cu, batch_f64.cu, part_f32.cu and part_f64.cu only
// (one launch family and working precision each, compiled in parallel).
#pragma once
#include "batch.cuh"
#include "dev_common.cuh"

namespace hodlr {
namespace {

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

// Step 1: V^T X per unit, warps w0, w0 + nw, ... of the units: CG columns
// of V_q at a time (independent loads in flight: CG V values and the X row
// per row step).
template <typename W, int RB, bool XV>
__device__ __forceinline__ void item_vtx_x(const BItem& b, const int w0, const int nw) {
  const int lane = threadIdx.x & 31;
  const W* X = reinterpret_cast<const W*>(b.X);
  W* P = reinterpret_cast<W*>(b.P);
  const int R = b.R;
  for (int u = w0; u < b.nunits; u += nw) {
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
            ld_xrow<W, RB, XV>(X + (lrow0 + r - b.row_base) * b.ldx, R, xv);
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
}
// (the X-row load form fixed at compile time: a branch in the unrolled row
// loop would keep its loads from being issued together)
template <typename W, int RB>
__device__ __forceinline__ void item_vtx(const BItem& b, const int w0, const int nw) {
  if (b.xvec)
    item_vtx_x<W, RB, true>(b, w0, nw);
  else
    item_vtx_x<W, RB, false>(b, w0, nw);
}

// Step 2: Y_q = scales x (sum of the unit partials in order), warps w0,
// w0 + nw, ... over the nodes; the summed levels' rows go to Yred.
template <typename W, int RB>
__device__ __forceinline__ void item_y(const BItem& b, const int w0, const int nw) {
  const int lane = threadIdx.x & 31;
  W* Y = reinterpret_cast<W*>(b.Y);
  W* Yr = reinterpret_cast<W*>(b.Yred);
  const W* P = reinterpret_cast<const W*>(b.P);
  const int R = b.R;
  for (int q = w0; q < b.nnodes; q += nw) {
    const NodeDev& nd = b.nodes[q];
    W* const Yq = (b.yoff[q] < b.yred_rows ? Yr : Y) + (int64_t)b.yoff[q] * RB;
    const W sc = (W)(nd.invsV * b.nodes[q ^ 1].invsU);
    const int u0 = b.node_u[q], u1 = b.node_u[q + 1];
    for (int e2 = lane; e2 < nd.rV * RB; e2 += 32) {
      const int c = e2 / RB, j = e2 - c * RB;
      W s = (W)0;
      if (j < R)
        for (int u = u0; u < u1; ++u) s += P[(int64_t)(b.units[u].w + c) * R + j];
      Yq[(int64_t)c * RB + j] = s * sc;   // rows of RB values, zeros past R
    }
  }
}

// Step 3: B rows = D X + U Y of leaves [lf_lo, lf_hi), warps w0, w0 + nw,
// ... over them: the leaf's X rows go once into the warp's shared-memory
// slice (when they fit), then its tiles, lane = row.
template <typename W, int RB>
__device__ __forceinline__ void item_apply(const BItem& b, const int w0, const int nw, const int lf_lo,
                                           const int lf_hi) {
  constexpr int es = sizeof(W);
  constexpr int G16 = 16 / es;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const W* X = reinterpret_cast<const W*>(b.X);
  const W* Y = reinterpret_cast<const W*>(b.Y);
  const W* Yr = reinterpret_cast<const W*>(b.Yred);
  const int R = b.R;
  const bool xvec = b.xvec != 0;
  W* B = reinterpret_cast<W*>(b.B);
  extern __shared__ __align__(16) uint8_t bsm[];
  W* const xs = reinterpret_cast<W*>(bsm + (size_t)warp * kSlice);
  const uint32_t us = (uint32_t)__cvta_generic_to_shared(bsm + (size_t)warp * kSlice + kXSlice);
  for (int lf = lf_lo + w0; lf < lf_hi; lf += nw) {
    const int lt0 = b.leaf_t0[lf], lt1 = b.leaf_t0[lf + 1];
    const int lm = b.tiles[lt0].m, lx0 = b.tiles[lt0].xrow0;
    const bool staged = (int64_t)lm * RB * es <= kXSlice;
    if (staged) {
      for (int e2 = lane; e2 < lm * RB; e2 += 32) {
        const int cc = e2 / RB, j = e2 - cc * RB;
        xs[e2] = j < R ? __ldg(X + (lx0 + cc - b.row_base) * b.ldx + j) : (W)0;
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
            else if (xvec)
              ld_xrow<W, RB, true>(X + (tq.xrow0 + cc - b.row_base) * b.ldx, R, xv);
            else
              ld_xrow<W, RB, false>(X + (tq.xrow0 + cc - b.row_base) * b.ldx, R, xv);
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
        const int ys = b.yoff[sib];
        const W* yb = (ys < b.yred_rows ? Yr : Y) + ((int64_t)ys + cc0) * RB;
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
        W* brow = B + (tq.row0 + r - b.row_base) * b.ldb;
#pragma unroll
        for (int j = 0; j < RB; ++j)
          if (j < R) brow[j] = acc[j];
      }
    }
    __syncwarp();   // the slice is read before the next leaf's rows overwrite it
  }
}

// One matrix's product by the whole CTA (the three steps, CTA barriers
// between them).  Not inlined: each column block gets its own register
// allocation (inlined into one kernel, the widest block's spills reached
// every item).
template <typename W, int RB>
__device__ __noinline__ void batch_item_rb(const BItem& b) {
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  item_vtx<W, RB>(b, warp, nw);
  __syncthreads();
  item_y<W, RB>(b, warp, nw);
  __syncthreads();
  item_apply<W, RB>(b, warp, nw, 0, b.nleaves);
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


// A partitioned product's steps, each over the whole grid (warp g of the
// grid takes units / nodes / leaves g, g + warps, ...).
template <typename W, int RB>
__global__ void __launch_bounds__(512, 1) part_vtx_kernel(const BItem b) {
  const int nwl = blockDim.x >> 5;
  item_vtx<W, RB>(b, (int)blockIdx.x * nwl + (int)(threadIdx.x >> 5), (int)gridDim.x * nwl);
}
template <typename W, int RB>
__global__ void __launch_bounds__(512, 1) part_y_kernel(const BItem b) {
  const int nwl = blockDim.x >> 5;
  item_y<W, RB>(b, (int)blockIdx.x * nwl + (int)(threadIdx.x >> 5), (int)gridDim.x * nwl);
}
template <typename W, int RB>
__global__ void __launch_bounds__(512, 1) part_apply_kernel(const BItem b, int lf0, int lf1) {
  const int nwl = blockDim.x >> 5;
  item_apply<W, RB>(b, (int)blockIdx.x * nwl + (int)(threadIdx.x >> 5), (int)gridDim.x * nwl, lf0, lf1);
}

template <typename W, int RB>
cudaError_t launch_part_rb(int step, const BItem& b, int lf0, int lf1, int grid, int threads, cudaStream_t s) {
  if (step == 0) {
    part_vtx_kernel<W, RB><<<grid, threads, 0, s>>>(b);
  } else if (step == 1) {
    part_y_kernel<W, RB><<<grid, threads, 0, s>>>(b);
  } else {
    const int smem = (threads / 32) * kSlice;
    static int smem_set = 0;
    if (smem > smem_set) {
      cudaError_t e =
          cudaFuncSetAttribute(part_apply_kernel<W, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) return e;
      smem_set = smem;
    }
    part_apply_kernel<W, RB><<<grid, threads, smem, s>>>(b, lf0, lf1);
  }
  return cudaGetLastError();
}

template <typename W>
cudaError_t launch_part_w(int step, const BItem& b, int lf0, int lf1, int grid, int threads, cudaStream_t s) {
  switch (b.rb) {
    case 1: return launch_part_rb<W, 1>(step, b, lf0, lf1, grid, threads, s);
    case 2: return launch_part_rb<W, 2>(step, b, lf0, lf1, grid, threads, s);
    case 4: return launch_part_rb<W, 4>(step, b, lf0, lf1, grid, threads, s);
    case 8: return launch_part_rb<W, 8>(step, b, lf0, lf1, grid, threads, s);
    default: return launch_part_rb<W, 16>(step, b, lf0, lf1, grid, threads, s);
  }
}

}  // namespace
}  // namespace hodlr
