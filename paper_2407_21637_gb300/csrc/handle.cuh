// Host-side handle of libhodlr and the import pipeline shared by
// hodlr_import (caller-provided generators) and hodlr_build (generators
// computed on the device).
#pragma once

#include <string>
#include <vector>

#include "hodlr_internal.cuh"

using hodlr::NodeDev;
using hodlr::LeafDev;
using hodlr::VChunk;
using hodlr::NodeRed;
using hodlr::P1Seg;
using hodlr::P2Tile;
using hodlr::TcGroup;
using hodlr::TcVRow;
using hodlr::PackTask;
using hodlr::HandleDev;
using hodlr::StLev;
using hodlr::YItem;

namespace hodlr {
struct LuState;                  // HODLR LU factors and solver scratch (lu.cu)
void lu_destroy(LuState* s);
}  // namespace hodlr

struct hodlr_s {
  std::vector<std::vector<std::pair<int, int>>> lv;  // cluster tree (row0, m) per level
  int n = 0, depth = 0, work = HODLR_FP64, per_block = 0, max_nrhs = 64;
  int batch = 64;                      // right-hand sides per product launch
  bool use_stream = true;              // CUDA-core products by the streamed kernel (else the two-barrier one)
  double eps = 0.0;
  uint32_t avail = 0;
  int device = 0;
  std::vector<NodeDev> nodes;
  std::vector<LeafDev> leaves;
  std::vector<VChunk> vch;
  std::vector<VChunk> vch_rest;          // chunks no tensor-core V group covers
  std::vector<NodeRed> nred;
  std::vector<P2Tile> p2;
  std::vector<PackTask> tasks;          // fp64 staging <-> pool, for export
  std::vector<PackTask> tasks_v;        // fp64 staging -> V area of the tiles (packed, never unpacked)
  std::vector<int64_t> st_U, st_V, st_D; // staging offsets (elements)
  int64_t st_count = 0;
  hodlr_info_t info{};
  int build_sketch_max = 0;          // largest sketch hodlr_build used
  bool build_accuracy_short = false;  // some block hit the sketch cap
  int build_rounds = 0, build_redone = 0;   // range-finder rounds, blocks redone
  int64_t build_sketch_cols = 0;      // sum over rounds of the blocks' sketch columns
  uint8_t* d_pool = nullptr;
  size_t pool_bytes = 0;
  NodeDev* d_nodes = nullptr;
  LeafDev* d_leaves = nullptr;
  VChunk* d_vch = nullptr;
  NodeRed* d_nred = nullptr;
  int2* d_ritems = nullptr;
  TcGroup* d_tcg = nullptr;
  TcVRow* d_tcv = nullptr;
  int32_t* d_tc_first = nullptr;
  VChunk* d_vch_rest = nullptr;
  P2Tile* d_p2 = nullptr;
  int32_t* d_yscat = nullptr;
  uint8_t* d_st_blob = nullptr;           // streamed product: one record per CTA
  void* d_spart = nullptr;                // its partial slots
  int* d_err = nullptr;
  void* d_Y = nullptr;
  void* d_partials = nullptr;
  unsigned long long* d_sync = nullptr;   // grid barrier counter of the product kernel
  unsigned long long sync_base = 0;       // its value before the next launch
  bool stall_next = false;                // hodlr_debug_stall_next: next product's barrier unreachable
  // hodlr_load: formats and power-of-two scales restored from a file instead
  // of chosen by the precision rule (empty otherwise)
  std::vector<int> force_tier;
  std::vector<double> force_sU, force_sV;
  size_t scratch_bytes = 0;
  HandleDev hd{};
  cudaEvent_t prof_ev[3] = {nullptr, nullptr, nullptr};
  bool prof_on = false, prof_valid = false;
  hodlr::LuState* lu = nullptr;           // hodlr_lu: the factors

  ~hodlr_s() {
    hodlr::lu_destroy(lu);
    for (cudaEvent_t& e : prof_ev)
      if (e) cudaEventDestroy(e);
    cudaFree(d_pool);
    cudaFree(d_nodes);
    cudaFree(d_leaves);
    cudaFree(d_vch);
    cudaFree(d_nred);
    cudaFree(d_ritems);
    cudaFree(d_tcg);
    cudaFree(d_tcv);
    cudaFree(d_tc_first);
    cudaFree(d_vch_rest);
    cudaFree(d_p2);
    cudaFree(d_yscat);
    cudaFree(d_st_blob);
    cudaFree(d_spart);
    cudaFree(d_err);
    cudaFree(d_Y);
    cudaFree(d_partials);
    cudaFree(d_sync);
  }
};

namespace hodlr {

hodlr_status set_error(hodlr_status s, const std::string& msg);
hodlr_status set_cuda_error(cudaError_t e, const char* where);

// Tree, leaves, nodes (ranks) and the fp64 staging layout; validates sizes.
hodlr_status plan_layout(hodlr_s* h, int n, int depth, const int32_t* ranks, const hodlr_opts* opts);

// From fp64 generators in the device staging (layout of plan_layout): the
// precision rule, packing, work lists and scratch.  ``block_norm2`` (per node
// q = block (k, i)) and ``leaf_norm2`` are the norms of the original matrix
// when known (hodlr_build), else nullptr (norms of the factors are used).
hodlr_status finish_from_staging(hodlr_s* h, const double* d_stage, const double* block_norm2,
                                 const double* leaf_norm2, const hodlr_opts* opts, cudaStream_t s);

}  // namespace hodlr
