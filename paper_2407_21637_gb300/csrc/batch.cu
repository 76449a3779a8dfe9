// Batched and partitioned HODLR products: host planning (work lists,
// scratch, CTA dealing, the measured CTA-size search) and the C ABI; the
// kernels are in batch_kern.cuh.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <queue>
#include <vector>

#include "batch.cuh"
#include "handle.cuh"

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
    items[i].Yred = items[i].Y;   // a whole product: no summed levels
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
                      ? launch_batch_f64(b->grid, threads, b->d_items, b->d_first, b->d_list, s)
                      : launch_batch_f32(b->grid, threads, b->d_items, b->d_first, b->d_list, s);
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

// ---- Partitioned product -----------------------------------------------
// Part j of tree level g owns the rows of node (g, j).  Its V^T X over those
// rows is complete for the nodes below (g, j) and partial for its g
// ancestors; those ancestors' levels (1..g) are the first rows of Y (Y is in
// level order), so summing every part's copy of that prefix (zeros for the
// nodes that are not its ancestors) gives the whole product's Y there.

struct hodlr_part_s {
  int work = HODLR_FP32, device = 0, g = 0, j = 0, lf0 = 0, lf1 = 0;
  int grid_v = 1, grid_y = 1, grid_a = 1;
  int64_t row0 = 0, rows = 0, yred_count = 0;
  BItem item;
  uint8_t* d_meta = nullptr;
  void* d_scratch = nullptr;
  ~hodlr_part_s() {
    cudaFree(d_meta);
    cudaFree(d_scratch);
  }
};

namespace {
constexpr int kPartThreads = 512;

hodlr_status part_launch(hodlr_part_t p, int step, int grid, cudaStream_t s) {
  const cudaError_t e = p->work == HODLR_FP64
                            ? launch_part_f64(step, p->item, p->lf0, p->lf1, grid, kPartThreads, s)
                            : launch_part_f32(step, p->item, p->lf0, p->lf1, grid, kPartThreads, s);
  return e == cudaSuccess ? HODLR_OK : set_cuda_error(e, "hodlr_part");
}

hodlr_status part_operands(hodlr_part_t p, const void* X, int64_t ldx, const void* Yred) {
  if (!p) return set_error(HODLR_EINVAL, "null part");
  if (!X || ldx < p->item.R) return set_error(HODLR_EINVAL, "bad X of the part");
  if (p->yred_count > 0 && !Yred) return set_error(HODLR_EINVAL, "the part needs a buffer for the summed levels");
  int dev = 0;
  const cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_cuda_error(e, "cudaGetDevice");
  if (dev != p->device) return set_error(HODLR_EINVAL, "the part lives on another device than the current one");
  const int vw = 16 / prec_bytes(p->work);
  p->item.X = X;
  p->item.ldx = ldx;
  p->item.Yred = p->yred_count > 0 ? const_cast<void*>(Yred) : p->item.Y;
  p->item.xvec = p->item.R % vw == 0 && ldx % vw == 0 && reinterpret_cast<uintptr_t>(X) % 16 == 0 ? 1 : 0;
  return HODLR_OK;
}
}  // namespace

extern "C" hodlr_status hodlr_part_create(hodlr_t h, int32_t g, int32_t j, int32_t nrhs, hodlr_part_t* out) {
  if (!out) return set_error(HODLR_EINVAL, "null out");
  *out = nullptr;
  if (!h) return set_error(HODLR_EINVAL, "null handle");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_cuda_error(e, "cudaGetDevice");
  if (h->device != dev) return set_error(HODLR_EINVAL, "the handle lives on another device than the current one");
  if (g < 0 || g > h->depth) return set_error(HODLR_EINVAL, "g must be in [0, depth]");
  if (j < 0 || j >= (1 << g)) return set_error(HODLR_EINVAL, "j must be in [0, 2^g)");
  if (nrhs < 1 || nrhs > kBatchMaxCols) return set_error(HODLR_EINVAL, "nrhs must be in [1, 16]");
  const int depth = h->depth, nnodes = (int)h->nodes.size(), nleaves = (int)h->leaves.size();
  const int es = prec_bytes(h->work);
  const int span = 1 << (depth - g), L0 = j * span, L1 = L0 + span;
  const int rb = nrhs <= 1 ? 1 : nrhs <= 2 ? 2 : nrhs <= 4 ? 4 : nrhs <= 8 ? 8 : 16;
  // units: the part's leaves of every node whose rows meet them
  std::vector<int4> units;
  std::vector<int32_t> node_u(nnodes + 1, 0), yoff(std::max(nnodes, 1), 0);
  int poff = 0, yrows = 0, yred_rows = 0;
  for (int k = 1; k <= depth; ++k) {
    const int kspan = 1 << (depth - k);
    for (int i = 0; i < (1 << k); ++i) {
      const int q = node_index(k, i);
      node_u[q] = (int)units.size();
      yoff[q] = yrows;
      yrows += h->nodes[q].rV;
      if (k <= g) yred_rows += h->nodes[q].rV;
      if (h->nodes[q].rV == 0) continue;
      const int a = std::max(i * kspan, L0), z = std::min((i + 1) * kspan, L1);
      for (int l0 = a; l0 < z; l0 += kLeavesPerUnit) {
        units.push_back(make_int4(q, l0, std::min(l0 + kLeavesPerUnit, z), poff));
        poff += h->nodes[q].rV;
      }
    }
  }
  node_u[nnodes] = (int)units.size();
  std::vector<int32_t> lt0(nleaves + 1, (int)h->p2.size());
  for (int t = (int)h->p2.size() - 1; t >= 0; --t) lt0[h->p2[t].leaf] = t;
  std::vector<int32_t> meta;
  for (const int4& u : units) {
    meta.push_back(u.x);
    meta.push_back(u.y);
    meta.push_back(u.z);
    meta.push_back(u.w);
  }
  const size_t m_nodeu = meta.size();
  meta.insert(meta.end(), node_u.begin(), node_u.end());
  const size_t m_yoff = meta.size();
  meta.insert(meta.end(), yoff.begin(), yoff.end());
  const size_t m_lt0 = meta.size();
  meta.insert(meta.end(), lt0.begin(), lt0.end());
  const int64_t yelems = (int64_t)std::max(yrows, 1) * rb;
  const int64_t pstart = (yelems + 16 / es - 1) / (16 / es) * (16 / es);
  const int64_t selems = pstart + (int64_t)std::max(poff, 1) * nrhs;
  hodlr_part_s* p = new hodlr_part_s();
  p->work = h->work;
  p->device = dev;
  p->g = g;
  p->j = j;
  p->lf0 = L0;
  p->lf1 = L1;
  p->row0 = h->leaves[L0].row0;
  p->rows = (int64_t)h->leaves[L1 - 1].row0 + h->leaves[L1 - 1].m - p->row0;
  p->yred_count = (int64_t)yred_rows * rb;
  e = cudaMalloc(&p->d_meta, std::max<size_t>(meta.size(), 4) * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&p->d_scratch, (size_t)selems * es);
  if (e == cudaSuccess && !meta.empty())
    e = cudaMemcpy(p->d_meta, meta.data(), meta.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
  int G = 1;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&G, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    delete p;
    return set_cuda_error(e, "hodlr_part_create");
  }
  const int wpc = kPartThreads / 32;
  auto grid_for = [&](int work) { return std::max(1, std::min(G, (work + wpc - 1) / wpc)); };
  p->grid_v = grid_for((int)units.size());
  p->grid_y = grid_for(nnodes);
  p->grid_a = grid_for(L1 - L0);
  BItem& it = p->item;
  memset(&it, 0, sizeof(it));
  const int32_t* dm = reinterpret_cast<const int32_t*>(p->d_meta);
  it.pool = h->d_pool;
  it.nodes = h->d_nodes;
  it.leaves = h->d_leaves;
  it.tiles = h->d_p2;
  it.units = reinterpret_cast<const int4*>(dm);
  it.node_u = dm + m_nodeu;
  it.yoff = dm + m_yoff;
  it.leaf_t0 = dm + m_lt0;
  it.Y = p->d_scratch;
  it.P = reinterpret_cast<uint8_t*>(p->d_scratch) + pstart * es;
  it.depth = depth;
  it.R = nrhs;
  it.nnodes = nnodes;
  it.nunits = (int)units.size();
  it.ntiles = (int)h->p2.size();
  it.nleaves = nleaves;
  it.rb = rb;
  it.yred_rows = yred_rows;
  it.row_base = p->row0;
  *out = p;
  return HODLR_OK;
}

extern "C" hodlr_status hodlr_part_info(hodlr_part_t p, int64_t* row0, int64_t* rows, int64_t* yred_count) {
  if (!p) return set_error(HODLR_EINVAL, "null part");
  if (row0) *row0 = p->row0;
  if (rows) *rows = p->rows;
  if (yred_count) *yred_count = p->yred_count;
  return HODLR_OK;
}

extern "C" hodlr_status hodlr_part_partial(hodlr_part_t p, const void* X, int64_t ldx, void* Yred, void* stream) {
  hodlr_status st = part_operands(p, X, ldx, Yred);
  if (st != HODLR_OK) return st;
  const cudaStream_t s = (cudaStream_t)stream;
  st = part_launch(p, 0, p->grid_v, s);
  return st == HODLR_OK ? part_launch(p, 1, p->grid_y, s) : st;
}

extern "C" hodlr_status hodlr_part_finish(hodlr_part_t p, const void* X, int64_t ldx, const void* Yred, void* B,
                                          int64_t ldb, void* stream) {
  hodlr_status st = part_operands(p, X, ldx, Yred);
  if (st != HODLR_OK) return st;
  if (!B || ldb < p->item.R) return set_error(HODLR_EINVAL, "bad B of the part");
  p->item.B = B;
  p->item.ldb = ldb;
  return part_launch(p, 2, p->grid_a, (cudaStream_t)stream);
}

extern "C" void hodlr_part_destroy(hodlr_part_t p) { delete p; }
