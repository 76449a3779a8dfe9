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

constexpr int kP1Segs = 16;          // leaf segments per V chunk at most (inline)
constexpr int kTileRows = 32;        // rows per product tile
constexpr int kChunkRows = 256;      // padded rows per V chunk at most
constexpr int kConsumerWarps = 16;   // consumer warps of the product kernel

// Bytes of the product's sync buffer (a 64-bit grid counter, padded).
constexpr int kSyncHeadBytes = 256;

// One leaf (or piece of a leaf) of a V chunk.
struct P1Seg {
  int32_t row0, m;                // first real row and valid rows of the segment
  int32_t prel;                   // padded offset of the segment inside the chunk
  int32_t pad_;
};

// V chunk: padded rows [p0, p0 + rows) of all rV columns of V_node (column c
// at byte offset off + c * colbytes of the pool).  The warp that takes it
// writes its part of V_node^T X to partial rows [poff, poff + rV).
struct VChunk {
  int64_t off;                    // byte offset of column 0 at padded row p0
  int32_t colbytes;               // bytes between columns in the pool (pm * eb)
  int32_t bytes;                  // bytes per column segment (rows * eb, multiple of 16)
  int32_t rows, node;             // padded rows; index of the node's NodeRed
  int32_t rV, tier, poff, nseg;   // rank, format, partial rows, segments
  int32_t xrow0, xrows;           // real rows covered (X rows xrow0 .. xrow0 + xrows)
  P1Seg seg[kP1Segs];
};

// Final reduction of one node: Y_node = invs * sum of its chunk partials
// (chunk order), written to its gathered-Y targets.  The rows of every node
// are reduction items (node, row) spread over the whole grid.
struct NodeRed {
  double invs;                    // 1/s of V_node times 1/s of U of the node's sibling
  int32_t rV, poff0, nparts;      // part p has partial rows poff0 + p * rV
  int32_t yscat0, nyscat;         // targets of Y_node in the gathered Y (see HandleDev)
  int32_t pad_;
};

// Product tile: rows [t0, t0 + kTileRows) of a leaf.  Its data sits in three
// areas of the pool, each in tile order (so the parts of consecutive tiles
// are contiguous):
//  * U area: a header of two words per level (byte offset of the level's U
//    block after the header; rank | format << 16), then the ancestors' U rows
//    for these 32 rows (level by level, column by column, 32 rows per
//    column, each level in its own format, each level 16-byte aligned);
//  * D area: the leaf block D[t0:t0+32, :] row by row (row length m rounded
//    up to 4, zero padded, working precision);
//  * V area (streamed product): the ancestors' V rows for these 32 rows,
//    laid out like the U rows (level by level, column by column, 32 rows per
//    column, each level 16-byte aligned, in its format);
//  * D2 area (streamed product): the leaf block D[t0:t0+32, :] once more,
//    in chunks of 16 bytes per row (4 fp32 or 2 fp64 consecutive columns):
//    chunk q of row r at (q * 32 + r) * 16, so that a warp with lane = row
//    reads 512 contiguous bytes per chunk.
struct P2Tile {
  int64_t off;                    // byte offset of the header-and-U region in the pool
  int64_t doff;                   // byte offset of the leaf-block part D[t0:t0+32, :] (128-byte aligned)
  int64_t voff;                   // byte offset of the tile's V part (streamed product)
  int64_t d2off;                  // byte offset of the tile's interleaved leaf-block part (streamed product)
  int32_t d2bytes;                // bytes of the interleaved leaf-block part (multiple of 512)
  int32_t vbytes;                 // bytes of the V part (multiple of 16)
  int32_t bytes, hbytes, dbytes;  // header + U, header and D bytes (multiples of 16)
  int32_t m;                      // leaf rows = D columns
  int32_t rows;                   // valid rows in the tile (<= 32)
  int32_t row0;                   // first real row of the tile
  int32_t xrow0;                  // first real row of the leaf (row of X for column 0)
  int32_t nq;                     // U columns (sum of the ancestors' ranks)
  int32_t yrow;                   // first row of the leaf's block in the gathered Y
  int32_t ubytes;                 // U bytes after the header (multiple of 16)
  int32_t leaf;                   // the tile's leaf
};
static_assert(sizeof(P2Tile) % 8 == 0, "P2Tile records are copied whole (8-byte aligned)");

// Tensor-core products (fp32 work, many right-hand sides).  A leaf group is
// up to 128 consecutive rows of one leaf, i.e. up to four product tiles:
// C = D[rows, :] X[I_i], written to B.  A V group is up to 128 columns of
// fp32 generators V_j restricted to the same rows I (one V chunk of one
// leaf, for several levels): C = V_j[I, :]^T X[I], written to the chunks'
// partial rows; its rows come from the TC row table.
constexpr int kTcMinCols = 16;    // products with at least this many columns use them
constexpr int kTcMaxCols = 64;    // columns per launch at most (MMA N)
constexpr int kTcRows = 128;      // rows per group (MMA M)
struct TcGroup {
  int64_t doff[4];                // leaf group: byte offset of each tile's leaf-block part in the pool
  int32_t ntl;                    // leaf group: tiles in the group (1..4)
  int32_t rows;                   // valid rows (<= 128); in a V group rows 0 .. rows-1 of its table
  int32_t row0;                   // leaf group: first row of the group
  int32_t xrow0;                  // first row of X (K index 0)
  int32_t m;                      // K extent: leaf rows (leaf group) or valid chunk rows (V group)
  int32_t vtab;                   // -1: leaf group; V group g: g * kTcRows (its entries in the row table)
};
// One A row of a group (kTcRows per group, group g at entries g * kTcRows):
// a row of a leaf block, or column c of a V chunk (K contiguous, fp32), and
// in a V group the partial row it produces.
struct TcVRow {
  int64_t off;                    // byte offset in the pool of the row's first element, or -1
  int32_t prow;                   // V group: partial row, or -1
  int32_t pad_;
};

// Streamed product (stream.cu).  Every CTA owns a contiguous range of
// tiles, so of whole leaves except at its ends.  Per tile:
struct StTile {
  int64_t voff, uoff, d2off;      // pool byte offsets of the tile's V part, header + U region, D2 part
  int32_t vbytes, ubytes, d2bytes;   // their bytes (ubytes includes the header)
  int32_t row0, xrow0;            // first row of the tile and of its leaf
  int16_t m, rows;                // leaf rows, tile rows
  int16_t lleaf;                  // the tile's leaf among its CTA's leaves (0, 1, ...)
  int16_t hbytes;                 // header bytes of the U region
  int32_t pad_;
};
// Per (CTA, one of its leaves, level k = 1..depth), entry (l0 + leaf) *
// depth + k - 1 (the same for every tile of the leaf in the CTA):
struct StLev {
  int32_t voff;                   // byte offset of the level's V block inside the tile's V part
  int32_t pslot;                  // first partial row of (ancestor at level k, the tile's CTA), -1 if rank 0
  int32_t yrow;                   // row in the CTA's Y area of Y of the ancestor's sibling, -1 if rank 0
  uint16_t rV;                    // rank of V of the ancestor
  uint8_t tierV, pad_;            // its storage format
};
// Per (CTA, one of its leaves): the leaf's tiles in the CTA and its U
// columns (over the levels 1..depth, level by level) with the storage
// format they all share (-1 if they do not), followed in the CTA's record by
// the columns themselves (StCol).
struct StLeaf {
  int32_t nu;                     // U columns
  int16_t t0, nt;                 // its tiles: CTA-local tiles t0 .. t0 + nt - 1
  int16_t utier, pad0_;           // common format of its U columns, or -1
  int32_t pad1_;
};
// One U column of a tile's U region: byte offset of its row 0 inside the
// region (header included), the row of Y it multiplies in the CTA's Y area,
// its level and format.
struct StCol {
  int32_t off;
  uint16_t idx;
  uint8_t k, tier;
};
// One Y_j a CTA needs for its U Y products: Y_j = invs * (sum of the
// partial slots of node j), the slots of the CTAs that hold rows of j, in CTA
// order.  The sum is split into tasks of at most kRedSlots slots whose
// results go to the CTA's reduction scratch (rows srow + p * rV, task p),
// then added in task order.
constexpr int kRedSlots = 16;
struct YItem {
  int32_t pbase;                  // first partial row of the node's first slot
  int32_t nslots;                 // number of slots
  int32_t rV;                     // rows of Y_j
  int32_t yrow;                   // first row in the CTA's Y area
  double invs;                    // 1/s of V_j times 1/s of U of j's sibling
  int32_t srow;                   // first row of its tasks' results in the reduction scratch
  int32_t ntask;                  // ceil(nslots / kRedSlots)
};
// One reduction task: slots [s0, s1) of item yi (the CTA's yi-th Y item).
struct RTask {
  int32_t yi, s0, s1, srow;       // srow: first row of this task's result
};
// What one CTA of the streamed product owns.  Everything a CTA reads about
// its own work is one record of fixed size (st_blob_stride bytes) that the
// CTA fetches with one bulk copy at the start: this header, then its tiles
// (StTile[nt] at st_off_tile), its leaves' level entries (StLev[nl * depth]
// at st_off_lev), the accumulator offsets (int32[depth + 1] at st_off_acc),
// its reduction tasks (RTask[nk] at st_off_task) and its Y items (YItem[ny]
// at st_off_y), then one column record per leaf (at st_off_leaf, stride
// st_leaf_stride).
struct StCta {
  int64_t voff;                   // first byte of its tiles' V parts (contiguous)
  int64_t uoff;                   // first byte of its tiles' header + U regions (contiguous)
  int32_t ubytes;                 // bytes of its tiles' header + U regions
  int32_t pad0_;
  int32_t t0, nt;                 // its tiles
  int32_t l0, nl;                 // its leaves
  int32_t vbytes;                 // bytes of its tiles' V parts
  int32_t xrow0, xrows;           // the rows of X its tiles cover
  int32_t y0, ny;                 // its Y items
  int32_t k0, nk;                 // its reduction tasks
  int32_t pad_[3];
};

// Device-resident description of a handle (passed by value to kernels).
// The gathered Y: for every leaf, the rows Y_{a_k ^ 1} (k = 1..depth) its
// tiles need, in the order of the tile's U columns, one block per leaf
// (row-major, R values per row).  Phase 1 writes each Y_j into the blocks of
// all leaves below the sibling of j: yscat[yscat0 .. yscat0 + nyscat) hold
// the target rows.
struct HandleDev {
  const NodeDev* nodes;
  const LeafDev* leaves;
  const VChunk* vch;
  const NodeRed* nred;
  const P2Tile* p2;
  const int32_t* yscat;
  const int2* ritems;             // reduction items: (NodeRed index, row of Y_node), all nodes
  const TcGroup* tcg;             // tensor-core groups, CTA c's at tc_first[c] .. tc_first[c + 1] - 1
  const int32_t* tc_first;        // [n_tc_cta + 1]
  const TcVRow* tcv;              // row table of the V groups
  const VChunk* vch_rest;         // V chunks no V group covers (tensor-core mode)
  const uint8_t* pool;
  int* err;                       // device error word (bounded waits that gave up)
  int32_t n, depth, n_nodes, n_leaves;
  int32_t n_vch, n_nred, n_p2, n_ritems, n_tcg;
  int32_t n_tcg_leaf;             // leaf groups among them
  int32_t n_tc_cta;               // CTAs of the tensor-core launch
  int32_t n_vch_rest;
  int32_t chunk_xrows_max;        // largest real-row span of a V chunk
  int32_t y_rows, p_rows;         // rows of the gathered Y and of the partial buffer
  int32_t max_nq;                 // largest U column count of a tile
  int32_t stage_bytes;            // largest tile region (multiple of 128)
  int32_t leaf_pm_max;
  int32_t leaf_m_max;             // largest leaf
  int32_t x_aligned;              // every leaf starts and ends on a multiple of 4 rows
  // streamed product
  const uint8_t* st_blob;         // [st_grid] records of st_blob_stride bytes (see StCta)
  int32_t st_blob_stride;         // bytes per record (a multiple of 16)
  int32_t st_off_tile, st_off_lev, st_off_acc, st_off_task, st_off_y;   // sections of a record
  int32_t st_off_leaf, st_leaf_stride;   // per-leaf column records (StLeaf, StCol[st_max_nu])
  int32_t st_max_nu;              // most U columns of one leaf
  int32_t st_grid;                // CTAs of the launch (one per SM)
  int32_t st_p_rows;              // rows of the partial buffer
  int32_t st_y_rows;              // rows of the largest per-CTA Y area
  int32_t st_red_rows;            // rows of the largest per-CTA reduction scratch
  int32_t st_acc_rows;            // accumulator rows (sum over levels of the largest V rank)
  int32_t st_max_rank;            // largest V rank
  int32_t st_max_tiles;           // most tiles of one CTA
  int32_t st_max_leaves;          // most leaves of one CTA
  int32_t st_max_vbytes;          // largest V part of one tile
  int32_t st_max_cta_v;           // largest V parts of one CTA (bytes) and
  int32_t st_max_cta_xrows;       //   rows of X of one CTA
  int32_t st_max_tile_bytes;      // largest header + U part plus leaf-block part of one tile
  int32_t st_max_cta_u;           // largest header + U regions of one CTA (bytes)
  int32_t st_max_ubytes;          // largest header + U region of one tile
  int32_t st_max_d2bytes;         // largest interleaved leaf-block part of one tile
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
  int64_t dst;             // byte offset of (row 0, column c) in the pool
  int32_t prec;
  int32_t dst_stride;      // bytes between consecutive rows in the pool (0: the element size)
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
cudaError_t launch_put_words(uint8_t* pool, const int64_t* off, const uint32_t* val, int64_t count,
                             cudaStream_t s);
cudaError_t launch_unpack(const uint8_t* pool, const PackTask* tasks, int ntasks,
                          double* staging, cudaStream_t s);

// One product launch (nrhs right-hand sides).  Y: gathered Y (y_rows * nrhs
// values + 4 of slack), partials: p_rows * nrhs values, sync: kSyncHeadBytes
// holding a 64-bit grid counter whose value is `sync_base` when the launch
// starts (the launch adds matvec_sync_step to it).
// ev (may be null): three events, recorded before the launch and twice after.
// skip_leaf: the tensor-core launch before it has written B = D X for every
// leaf and the partials of the V chunks its V groups cover; this launch then
// takes only the other chunks (vch_rest), the reductions and U Y.
cudaError_t launch_matvec(const HandleDev& hd, int work, int nrhs, const void* X, int64_t ldx,
                          void* B, int64_t ldb, void* Y, void* partials,
                          unsigned long long* sync, unsigned long long sync_base,
                          cudaStream_t s, cudaEvent_t* ev, int skip_leaf = 0);
// Tensor-core products (fp32 work, kTcMinCols <= nrhs <= kTcMaxCols):
// B[rows of every leaf group] = D_i X[I_i]; for every V group, the partial
// rows of its chunks = V_chunk^T X[I] (row-major, nrhs values per row).
// One CTA per entry of cta_first but the last; CTA c takes groups
// cta_first[c] .. cta_first[c + 1] - 1.
cudaError_t launch_leaf_tc(const TcGroup* groups, const int32_t* cta_first, int ncta, const TcVRow* vrows,
                           const uint8_t* pool, const float* X, int64_t ldx, int nrhs, float* B, int64_t ldb,
                           float* partials, int* err, cudaStream_t s);
// The streamed product (stream.cu): one launch of nrhs <= kStreamMaxCols
// right-hand sides, any working precision.  partials: st_p_rows * nrhs
// values; sync: a grid counter whose value is sync_base when the launch
// starts (the launch adds stream_sync_step).  ev as in launch_matvec.
constexpr int kStreamMaxCols = 16;
cudaError_t launch_stream(const HandleDev& hd, int work, int nrhs, const void* X, int64_t ldx, void* B,
                          int64_t ldb, void* partials, unsigned long long* sync, unsigned long long sync_base,
                          cudaStream_t s, cudaEvent_t* ev);
unsigned long long stream_sync_step(const HandleDev& hd);
// Widest batch launch_stream takes for this handle (0 when a single column
// does not fit the shared memory).
int stream_max_batch(const HandleDev& hd, int work);

// The grid size launch_matvec uses.
int matvec_grid(const HandleDev& hd);
// How far one launch advances the grid barrier counter (sync_base of the
// next launch on the same counter = this launch's + matvec_sync_step).
unsigned long long matvec_sync_step(const HandleDev& hd);

// Widest batch of right-hand sides one product launch accepts (shared-memory
// stages of phase 2); 0 when even one column does not fit.
int matvec_max_batch(const HandleDev& hd, int work);

cudaError_t launch_dense_kernel_matvec(int n, int dim, const double* pts, int kind, double c,
                                       double len2, double diag, int nrows, const int32_t* rows,
                                       int nrhs, const double* X, int64_t ldx, double* B,
                                       int64_t ldb, cudaStream_t s);

}  // namespace hodlr
