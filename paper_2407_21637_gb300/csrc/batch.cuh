// Work-list records shared by the batched and partitioned products (host
// planning in batch.cu; kernels in batch_kern.cuh, compiled per launch
// family and working precision in batch_f32.cu, batch_f64.cu, part_f32.cu
// and part_f64.cu).
#pragma once
#include <cuda_runtime.h>

#include "hodlr_internal.cuh"

namespace hodlr {

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
  void* Yred;             // rows [0, yred_rows) of Y live here instead (a partitioned product's
  int32_t yred_rows;      //   summed levels); Y itself and 0 for a whole product
  int32_t pad_;
  int64_t row_base;       // X and B hold rows row_base.. (0 for a whole product)
};

constexpr int kXSlice = 8192;       // bytes of shared memory per warp for a leaf's X rows
constexpr int kUPiece = 3072;       // and for each of two pieces of a tile's U columns
constexpr int kSlice = kXSlice + 2 * kUPiece;

// The batched launch: CTA c runs items list[first[c] .. first[c + 1]).
cudaError_t launch_batch_f32(int grid, int threads, const BItem* items, const int32_t* first, const int32_t* list,
                             cudaStream_t s);
cudaError_t launch_batch_f64(int grid, int threads, const BItem* items, const int32_t* first, const int32_t* list,
                             cudaStream_t s);
// One step of a partitioned product over the whole grid: 0 = V^T X of the
// item's units, 1 = Y from the unit partials, 2 = B rows of leaves [lf0, lf1).
cudaError_t launch_part_f32(int step, const BItem& b, int lf0, int lf1, int grid, int threads, cudaStream_t s);
cudaError_t launch_part_f64(int step, const BItem& b, int lf0, int lf1, int grid, int threads, cudaStream_t s);

}  // namespace hodlr
