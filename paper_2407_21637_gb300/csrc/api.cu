// C ABI of libhodlr: handle management, validation, the precision rule of
// Algorithm 3.2 (on device-computed norms), layout planning and launches.
#include <algorithm>
#include <cmath>
#include <map>
#include <memory>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "handle.cuh"

using namespace hodlr;

namespace {

thread_local std::string g_last_error;

hodlr_status fail(hodlr_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

hodlr_status cuda_fail(cudaError_t e, const char* where) {
  g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
  return HODLR_ECUDA;
}

#define CK(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

double unit_roundoff(int p) {
  switch (p) {
    case HODLR_FP64: return std::ldexp(1.0, -53);
    case HODLR_FP32: return std::ldexp(1.0, -24);
    case HODLR_FP16: return std::ldexp(1.0, -11);
    case HODLR_BF16: return std::ldexp(1.0, -8);
    case HODLR_E4M3: return std::ldexp(1.0, -4);
    case HODLR_E5M2: return std::ldexp(1.0, -3);
  }
  return 1.0;
}

// Largest finite value of the formats that get a per-block scale.
double scaled_format_max(int p) {
  switch (p) {
    case HODLR_FP16: return 65504.0;
    case HODLR_E4M3: return 448.0;
    case HODLR_E5M2: return 57344.0;
  }
  return 0.0;
}

// s = 2^floor(log2(x_max / (2 amax))) for fp16/e4m3/e5m2, else 1.
double pow2_scale(double amax, int p) {
  const double xm = scaled_format_max(p);
  if (xm == 0.0 || amax == 0.0) return 1.0;
  int e = 0;
  std::frexp(xm / (2.0 * amax), &e);  // y = f 2^e, f in [0.5, 1)
  return std::ldexp(1.0, e - 1);
}

// u_k = max{u* <= u' : u* in avail}; the most precise format when empty.
int choose_format(double u_prime, uint32_t avail) {
  int best = -1, most_precise = -1;
  for (int p = 0; p < kPrecCount; ++p) {
    if (!(avail >> p & 1u)) continue;
    const double u = unit_roundoff(p);
    if (most_precise < 0 || u < unit_roundoff(most_precise)) most_precise = p;
    if (u <= u_prime && (best < 0 || u > unit_roundoff(best))) best = p;
  }
  return best >= 0 ? best : most_precise;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace


namespace {

struct DevBuf {  // RAII for import-time temporaries
  void* p = nullptr;
  ~DevBuf() { cudaFree(p); }
};

template <typename T>
hodlr_status upload(const std::vector<T>& v, T** dst) {
  if (v.empty()) { *dst = nullptr; return HODLR_OK; }
  CK(cudaMalloc((void**)dst, v.size() * sizeof(T)));
  CK(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return HODLR_OK;
}

// Cluster tree of Def. 2.1 with the ceil-half split of Sect. 4.
void build_tree(int n, int depth, std::vector<std::vector<std::pair<int, int>>>& lv) {
  lv.assign(depth + 1, {});
  lv[0].push_back({0, n});
  for (int k = 0; k < depth; ++k) {
    for (auto& nd : lv[k]) {
      const int left = (nd.second + 1) / 2;
      lv[k + 1].push_back({nd.first, left});
      lv[k + 1].push_back({nd.first + left, nd.second - left});
    }
  }
}

}  // namespace

namespace hodlr {

hodlr_status set_error(hodlr_status s, const std::string& msg) { return fail(s, msg); }
hodlr_status set_cuda_error(cudaError_t e, const char* where) { return cuda_fail(e, where); }

hodlr_status plan_layout(hodlr_s* h, int n, int depth, const int32_t* ranks, const hodlr_opts* opts) {
  if (n < 1) return fail(HODLR_EINVAL, "n must be >= 1");
  if (depth < 0 || depth > HODLR_MAX_DEPTH) return fail(HODLR_EINVAL, "depth out of range");
  if ((int64_t(1) << depth) > n) return fail(HODLR_EINVAL, "2^depth > n (empty leaves)");
  if (!(opts->eps >= 0.0 && opts->eps < 1.0)) return fail(HODLR_EINVAL, "eps must be in [0, 1)");
  if (opts->work != HODLR_FP64 && opts->work != HODLR_FP32)
    return fail(HODLR_EINVAL, "working precision must be FP64 or FP32");
  if (opts->tier_mask >> kPrecCount) return fail(HODLR_EINVAL, "tier_mask has unknown bits");
  if (opts->max_nrhs < 0 || opts->max_nrhs > 4096) return fail(HODLR_EINVAL, "max_nrhs out of range");
  if (depth > 0 && !ranks) return fail(HODLR_EINVAL, "null ranks");
  h->n = n;
  h->depth = depth;
  h->work = opts->work;
  h->per_block = opts->per_block ? 1 : 0;
  h->eps = opts->eps;
  h->avail = opts->tier_mask | (1u << opts->work);
  h->max_nrhs = opts->max_nrhs ? opts->max_nrhs : 64;
  CK(cudaGetDevice(&h->device));
  build_tree(n, depth, h->lv);
  const auto& lv = h->lv;
  const int nleaves = 1 << depth;
  const int nnodes = (1 << (depth + 1)) - 2;

  // leaves: padded row space
  h->leaves.resize(nleaves);
  int prow = 0;
  for (int l = 0; l < nleaves; ++l) {
    LeafDev& lf = h->leaves[l];
    memset(&lf, 0, sizeof(lf));
    lf.row0 = lv[depth][l].first;
    lf.m = lv[depth][l].second;
    if (lf.m > kMaxLeaf) return fail(HODLR_EINVAL, "leaf larger than 1024 rows; increase depth");
    lf.pm = (int)align_up(lf.m, kRowPad);
    lf.prow0 = prow;
    lf.node = depth > 0 ? node_index(depth, l) : -1;
    prow += lf.pm;
  }
  // nodes
  h->nodes.resize(nnodes);
  for (int k = 1; k <= depth; ++k) {
    const int span = 1 << (depth - k);  // leaves per node
    for (int i = 0; i < (1 << k); ++i) {
      NodeDev& nd = h->nodes[node_index(k, i)];
      memset(&nd, 0, sizeof(nd));
      nd.level = k;
      nd.idx = i;
      nd.row0 = lv[k][i].first;
      nd.m = lv[k][i].second;
      nd.prow0 = h->leaves[i * span].prow0;
      const LeafDev& last = h->leaves[i * span + span - 1];
      nd.pm = last.prow0 + last.pm - nd.prow0;
      const int rU = ranks[node_index(k, i)];
      const int rV = ranks[node_index(k, i ^ 1)];
      const int msib = lv[k][i ^ 1].second;
      if (rU < 0 || rU > std::min(nd.m, msib)) return fail(HODLR_EINVAL, "rank out of range");
      nd.rU = rU;
      nd.rV = rV;
    }
  }
  // fp64 staging: the row-major generators back to back, then the leaves
  h->st_U.assign(nnodes, 0);
  h->st_V.assign(nnodes, 0);
  h->st_D.assign(nleaves, 0);
  int64_t off = 0;
  for (int q = 0; q < nnodes; ++q) {
    h->st_U[q] = off; off += (int64_t)h->nodes[q].m * h->nodes[q].rU;
    h->st_V[q] = off; off += (int64_t)h->nodes[q].m * h->nodes[q].rV;
  }
  for (int l = 0; l < nleaves; ++l) { h->st_D[l] = off; off += (int64_t)h->leaves[l].m * h->leaves[l].m; }
  h->st_count = off;
  return HODLR_OK;
}

hodlr_status finish_from_staging(hodlr_s* h, const double* d_stage, const double* block_norm2,
                                 const double* leaf_norm2, const hodlr_opts* opts, cudaStream_t s) {
  const int depth = h->depth, n = h->n;
  const int nleaves = (int)h->leaves.size(), nnodes = (int)h->nodes.size();
  int leaf_pm_max = 0;
  for (const LeafDev& lf : h->leaves) leaf_pm_max = std::max(leaf_pm_max, lf.pm);

  // ---- norms on the device (Algorithm 3.2: nrm, nrmAll) ----
  // tasks: [0, nnodes) V_q sum of squares + amax; [nnodes, 2 nnodes) U_q amax; then leaves.
  std::vector<NormTask> ntasks;
  for (int q = 0; q < nnodes; ++q) ntasks.push_back({h->st_V[q], (int64_t)h->nodes[q].m * h->nodes[q].rV});
  for (int q = 0; q < nnodes; ++q) ntasks.push_back({h->st_U[q], (int64_t)h->nodes[q].m * h->nodes[q].rU});
  for (int l = 0; l < nleaves; ++l) ntasks.push_back({h->st_D[l], (int64_t)h->leaves[l].m * h->leaves[l].m});
  DevBuf d_ntasks, d_sumsq, d_amax;
  const size_t nt = ntasks.size();
  CK(cudaMalloc(&d_ntasks.p, nt * sizeof(NormTask)));
  CK(cudaMalloc(&d_sumsq.p, nt * sizeof(double)));
  CK(cudaMalloc(&d_amax.p, nt * sizeof(double)));
  CK(cudaMemcpyAsync(d_ntasks.p, ntasks.data(), nt * sizeof(NormTask), cudaMemcpyHostToDevice, s));
  CK(launch_norms(d_stage, (const NormTask*)d_ntasks.p, (int)nt, (double*)d_sumsq.p,
                  (double*)d_amax.p, s));
  std::vector<double> sumsq(nt), amax(nt);
  CK(cudaMemcpyAsync(sumsq.data(), d_sumsq.p, nt * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(amax.data(), d_amax.p, nt * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));

  // ---- precision rule (Algorithm 3.2) ----
  // block (k, i) = H(I_i, I_{i^1}) ~ U_i V_{i^1}^T: ||.||_F^2 = ||V_{i^1}||_F^2
  // from the factors, or the original block norm when given.
  std::vector<double> bn(nnodes, 0.0);
  double total = 0.0;
  for (int k = 1; k <= depth; ++k)
    for (int i = 0; i < (1 << k); ++i) {
      const int q = node_index(k, i);
      bn[q] = block_norm2 ? block_norm2[q] : sumsq[node_index(k, i ^ 1)];
      total += bn[q];
    }
  for (int l = 0; l < nleaves; ++l) total += leaf_norm2 ? leaf_norm2[l] : sumsq[2 * nnodes + l];
  hodlr_info_t& inf = h->info;
  memset(&inf, 0, sizeof(inf));
  inf.n = n;
  inf.depth = depth;
  inf.work = h->work;
  inf.per_block = h->per_block;
  inf.n_blocks = nnodes;
  inf.norm2_all = total;
  std::vector<int> block_tier(nnodes, h->work);
  for (int k = 1; k <= depth; ++k) {
    const double lvl_scale = std::pow(2.0, k / 2.0);
    double level_max = 0.0;
    for (int i = 0; i < (1 << k); ++i) level_max = std::max(level_max, bn[node_index(k, i)]);
    const double xi_k = total > 0.0 ? std::sqrt(level_max / total) : 0.0;
    const double up_k = xi_k > 0.0 ? opts->eps / (lvl_scale * xi_k) : INFINITY;
    inf.xi[k] = xi_k;
    inf.u_prime[k] = up_k;
    if (!h->per_block) {
      const int t = choose_format(up_k, h->avail);
      inf.level_tier[k] = t;
      for (int i = 0; i < (1 << k); ++i) block_tier[node_index(k, i)] = t;
    } else {
      int most = -1;
      for (int i = 0; i < (1 << k); ++i) {
        const double xi = total > 0.0 ? std::sqrt(bn[node_index(k, i)] / total) : 0.0;
        const double up = xi > 0.0 ? opts->eps / (lvl_scale * xi) : INFINITY;
        const int t = choose_format(up, h->avail);
        block_tier[node_index(k, i)] = t;
        if (most < 0 || unit_roundoff(t) < unit_roundoff(most)) most = t;
      }
      inf.level_tier[k] = most;
    }
  }

  if (!h->force_tier.empty()) block_tier = h->force_tier;   // hodlr_load

  // ---- formats and scales of every generator ----
  const int ebw = prec_bytes(h->work);
  std::vector<double> sU(nnodes, 1.0), sV(nnodes, 1.0);
  for (int k = 1; k <= depth; ++k)
    for (int i = 0; i < (1 << k); ++i) {
      const int q = node_index(k, i);
      NodeDev& nd = h->nodes[q];
      nd.tierU = block_tier[q];
      nd.tierV = block_tier[node_index(k, i ^ 1)];
      sU[q] = h->force_sU.empty() ? pow2_scale(amax[nnodes + q], nd.tierU) : h->force_sU[q];
      sV[q] = h->force_sV.empty() ? pow2_scale(amax[q], nd.tierV) : h->force_sV[q];
      nd.invsU = 1.0 / sU[q];
      nd.invsV = 1.0 / sV[q];
      inf.max_rank = std::max(inf.max_rank, nd.rU);
      inf.factor_bytes += (int64_t)nd.m * (nd.rU * prec_bytes(nd.tierU) + nd.rV * prec_bytes(nd.tierV));
      inf.u_bytes += (int64_t)nd.m * nd.rU * prec_bytes(nd.tierU);
      inf.v_bytes += (int64_t)nd.m * nd.rV * prec_bytes(nd.tierV);
      inf.bytes_per_tier[nd.tierU] += (int64_t)nd.m * nd.rU * prec_bytes(nd.tierU);
      inf.bytes_per_tier[nd.tierV] += (int64_t)nd.m * nd.rV * prec_bytes(nd.tierV);
      if (sU[q] != 1.0 && nd.rU) inf.scale_bytes += 8;
      if (sV[q] != 1.0 && nd.rV) inf.scale_bytes += 8;
    }
  for (const LeafDev& lf : h->leaves) inf.leaf_bytes += (int64_t)lf.m * lf.m * ebw;

  // ---- pool: V columns per node (phase 1), then one region per leaf tile ----
  size_t pool = 0;
  h->tasks.clear();
  for (int k = 1; k <= depth; ++k) {
    const int span = 1 << (depth - k);
    for (int i = 0; i < (1 << k); ++i) {
      const int q = node_index(k, i);
      NodeDev& nd = h->nodes[q];
      pool = align_up(pool, 256);
      nd.offV = (int64_t)pool;
      const int ebv = prec_bytes(nd.tierV);
      pool += (size_t)nd.rV * nd.pm * ebv;
      for (int l = i * span; l < (i + 1) * span; ++l) {
        const LeafDev& lf = h->leaves[l];
        const int rel = lf.row0 - nd.row0, prel = lf.prow0 - nd.prow0;
        for (int c = 0; c < nd.rV; ++c)
          h->tasks.push_back({h->st_V[q] + (int64_t)rel * nd.rV + c, nd.rV, lf.m, lf.pm,
                              nd.offV + ((int64_t)c * nd.pm + prel) * ebv, nd.tierV, 0, sV[q]});
      }
    }
  }
  // tiles: header and U rows (U area), leaf-block rows (D area) and V rows
  // (V area), each area in tile order so that the parts of consecutive
  // tiles are contiguous
  h->p2.clear();
  std::vector<std::pair<int64_t, uint32_t>> headers;   // (byte offset in pool, word)
  int max_nq = 0, max_region = 0;
  std::vector<int> leaf_nq(nleaves, 0), leaf_yrow(nleaves, 0), leaf_tile0(nleaves + 1, 0);
  std::vector<std::vector<int>> leaf_anc(nleaves), leaf_vseg(nleaves), leaf_useg(nleaves);
  int yrows = 0;
  const int hbytes = (int)align_up((size_t)8 * depth, 16);   // one header entry per level
  pool = align_up(pool, 256);
  for (int l = 0; l < nleaves; ++l) {
    const LeafDev& lf = h->leaves[l];
    // the leaf's U columns: ancestors level 1..depth, columns 0..rU-1
    std::vector<int>& anc = leaf_anc[l];
    anc.assign(depth + 1, 0);
    int nq = 0;
    for (int k = 1; k <= depth; ++k) {
      anc[k] = node_index(k, l >> (depth - k));
      nq += h->nodes[anc[k]].rU;
    }
    leaf_nq[l] = nq;
    leaf_yrow[l] = yrows;
    yrows += (int)align_up(nq, 4);               // 16-byte aligned blocks in fp32 and fp64
    max_nq = std::max(max_nq, nq);
    const int mp = (int)align_up(lf.m, 4);                // D row length (zero padded)
    const int dbytes = mp * kTileRows * ebw;
    // byte offset of each level's U (V) block after the header (inside the V part)
    std::vector<int>& useg = leaf_useg[l];
    useg.assign(depth + 2, 0);
    std::vector<int>& vseg = leaf_vseg[l];
    vseg.assign(depth + 2, 0);
    for (int k = 1; k <= depth; ++k) {
      const NodeDev& a = h->nodes[anc[k]];
      useg[k + 1] = useg[k] + (int)align_up((size_t)a.rU * kTileRows * prec_bytes(a.tierU), 16);
      vseg[k + 1] = vseg[k] + (int)align_up((size_t)a.rV * kTileRows * prec_bytes(a.tierV), 16);
    }
    const int ubytes = useg[depth + 1];
    max_region = std::max(max_region, dbytes);
    leaf_tile0[l] = (int)h->p2.size();
    for (int t0 = 0; t0 < lf.m; t0 += kTileRows) {
      P2Tile tl;
      memset(&tl, 0, sizeof(tl));
      tl.off = (int64_t)pool;
      tl.bytes = hbytes + ubytes;
      tl.hbytes = hbytes;
      tl.ubytes = ubytes;
      tl.dbytes = dbytes;
      tl.vbytes = vseg[depth + 1];
      tl.m = lf.m;
      tl.rows = std::min(kTileRows, lf.m - t0);
      tl.row0 = lf.row0 + t0;
      tl.xrow0 = lf.row0;
      tl.nq = nq;
      tl.yrow = leaf_yrow[l];
      tl.leaf = l;
      h->p2.push_back(tl);
      // header, two words per level k = 1..depth: byte offset of the level's
      // U block after the header; rank | format << 16
      for (int k = 1; k <= depth; ++k) {
        const NodeDev& a = h->nodes[anc[k]];
        headers.push_back({tl.off + 8 * (k - 1), (uint32_t)useg[k]});
        headers.push_back({tl.off + 8 * (k - 1) + 4, (uint32_t)a.rU | ((uint32_t)a.tierU << 16)});
      }
      // U_a[rows of this tile, c] for every ancestor a and column c (column
      // by column: 32 consecutive rows per column)
      for (int k = 1; k <= depth; ++k) {
        const int q = anc[k];
        const NodeDev& a = h->nodes[q];
        const int eb = prec_bytes(a.tierU);
        const int rel = lf.row0 - a.row0 + t0;
        for (int c = 0; c < a.rU; ++c)
          h->tasks.push_back({h->st_U[q] + (int64_t)rel * a.rU + c, a.rU, tl.rows, kTileRows,
                              tl.off + hbytes + useg[k] + (int64_t)c * kTileRows * eb, a.tierU, 0, sU[q]});
      }
      pool += (size_t)tl.bytes;
    }
  }
  leaf_tile0[nleaves] = (int)h->p2.size();
  const int n_tiles = (int)h->p2.size();
  std::vector<int> tile_leaf(n_tiles, 0);
  for (int l = 0; l < nleaves; ++l)
    for (int t = leaf_tile0[l]; t < leaf_tile0[l + 1]; ++t) tile_leaf[t] = l;
  // D area
  pool = align_up(pool, 256);
  for (int l = 0; l < nleaves; ++l) {
    const LeafDev& lf = h->leaves[l];
    const int mp = (int)align_up(lf.m, 4);
    for (int t = leaf_tile0[l]; t < leaf_tile0[l + 1]; ++t) {
      P2Tile& tl = h->p2[t];
      pool = align_up(pool, 128);
      tl.doff = (int64_t)pool;
      const int t0 = tl.row0 - lf.row0;
      // D[t0:t0+32, j] for every column j (row-major, row stride mp)
      for (int j = 0; j < lf.m; ++j)
        h->tasks.push_back({h->st_D[l] + (int64_t)t0 * lf.m + j, lf.m, tl.rows, kTileRows,
                            tl.doff + (int64_t)j * ebw, h->work, mp * ebw, 1.0});
      pool += (size_t)tl.dbytes;
    }
  }
  // V area (streamed product only; the node-ordered V columns above stay the
  // copy that export, save and the tensor-core V groups read): per tile and
  // level a block of 32 rows x rank, column by column, rows past the tile zero
  pool = align_up(pool, 256);
  h->tasks_v.clear();
  for (int l = 0; l < nleaves; ++l) {
    const LeafDev& lf = h->leaves[l];
    for (int t = leaf_tile0[l]; t < leaf_tile0[l + 1]; ++t) {
      P2Tile& tl = h->p2[t];
      tl.voff = (int64_t)pool;
      const int t0 = tl.row0 - lf.row0;
      for (int k = 1; k <= depth; ++k) {
        const int q = leaf_anc[l][k];
        const NodeDev& a = h->nodes[q];
        const int eb = prec_bytes(a.tierV);
        const int rel = lf.row0 - a.row0 + t0;
        for (int c = 0; c < a.rV; ++c)
          h->tasks_v.push_back({h->st_V[q] + (int64_t)rel * a.rV + c, a.rV, tl.rows, kTileRows,
                                tl.voff + leaf_vseg[l][k] + (int64_t)c * kTileRows * eb, a.tierV, 0, sV[q]});
      }
      pool += (size_t)tl.vbytes;
    }
  }
  // D2 area (streamed product): each tile's leaf block once more, in
  // 16-byte chunks of consecutive columns, chunk q of row r at (q * 32 + r) * 16
  pool = align_up(pool, 256);
  {
    const int g16 = 16 / ebw;   // columns per chunk
    for (int l = 0; l < nleaves; ++l) {
      const LeafDev& lf = h->leaves[l];
      for (int t = leaf_tile0[l]; t < leaf_tile0[l + 1]; ++t) {
        P2Tile& tl = h->p2[t];
        tl.d2off = (int64_t)pool;
        tl.d2bytes = (lf.m + g16 - 1) / g16 * kTileRows * 16;
        const int t0 = tl.row0 - lf.row0;
        for (int j = 0; j < lf.m; ++j)
          h->tasks_v.push_back({h->st_D[l] + (int64_t)t0 * lf.m + j, lf.m, tl.rows, kTileRows,
                                tl.d2off + (int64_t)(j / g16) * kTileRows * 16 + (int64_t)(j % g16) * ebw, h->work,
                                16, 1.0});
        pool += (size_t)tl.d2bytes;
      }
    }
  }
  // tensor-core groups: up to four consecutive tiles (128 rows) of a leaf
  std::vector<TcGroup> tcg;
  for (size_t t = 0; t < h->p2.size();) {
    const P2Tile& t0 = h->p2[t];
    TcGroup gr;
    memset(&gr, 0, sizeof(gr));
    gr.row0 = t0.row0;
    gr.xrow0 = t0.xrow0;
    gr.m = t0.m;
    gr.vtab = -1;   // a leaf group
    while (t < h->p2.size() && gr.ntl < 4 && h->p2[t].xrow0 == t0.xrow0) {
      const P2Tile& tt = h->p2[t];
      gr.doff[gr.ntl++] = tt.doff;
      gr.rows += tt.rows;
      ++t;
    }
    tcg.push_back(gr);
  }
  pool = align_up(std::max<size_t>(pool, 256), 256);
  h->pool_bytes = pool;
  if (cudaMalloc((void**)&h->d_pool, pool) != cudaSuccess) return fail(HODLR_ENOMEM, "factor pool");
  CK(cudaMemsetAsync(h->d_pool, 0, pool, s));
  {
    DevBuf d_tasks, d_hoff, d_hval;
    CK(cudaMalloc(&d_tasks.p, std::max<size_t>(h->tasks.size(), 1) * sizeof(PackTask)));
    CK(cudaMemcpyAsync(d_tasks.p, h->tasks.data(), h->tasks.size() * sizeof(PackTask),
                       cudaMemcpyHostToDevice, s));
    CK(launch_pack(d_stage, (const PackTask*)d_tasks.p, (int)h->tasks.size(), h->d_pool, s));
    if (!h->tasks_v.empty()) {
      DevBuf d_tv;
      CK(cudaMalloc(&d_tv.p, h->tasks_v.size() * sizeof(PackTask)));
      CK(cudaMemcpyAsync(d_tv.p, h->tasks_v.data(), h->tasks_v.size() * sizeof(PackTask),
                         cudaMemcpyHostToDevice, s));
      CK(launch_pack(d_stage, (const PackTask*)d_tv.p, (int)h->tasks_v.size(), h->d_pool, s));
      CK(cudaStreamSynchronize(s));
    }
    std::vector<int64_t> hoff(headers.size());
    std::vector<uint32_t> hval(headers.size());
    for (size_t e = 0; e < headers.size(); ++e) { hoff[e] = headers[e].first; hval[e] = headers[e].second; }
    CK(cudaMalloc(&d_hoff.p, std::max<size_t>(hoff.size(), 1) * sizeof(int64_t)));
    CK(cudaMalloc(&d_hval.p, std::max<size_t>(hval.size(), 1) * sizeof(uint32_t)));
    CK(cudaMemcpyAsync(d_hoff.p, hoff.data(), hoff.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(d_hval.p, hval.data(), hval.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    CK(launch_put_words(h->d_pool, (const int64_t*)d_hoff.p, (const uint32_t*)d_hval.p, (int64_t)hoff.size(), s));
    CK(cudaStreamSynchronize(s));
  }

  // ---- phase-1 work items and the scatter table of the gathered Y ----
  // yscat: for node j (level k), one entry per leaf L below the sibling of j:
  // the gathered-Y row of Y_j[0] in L's block.
  std::vector<int32_t> yscat;
  std::vector<int> yscat0(nnodes, 0), nyscat(nnodes, 0);
  for (int k = 1; k <= depth; ++k) {
    const int span = 1 << (depth - k);
    for (int j = 0; j < (1 << k); ++j) {
      const int q = node_index(k, j);
      yscat0[q] = (int)yscat.size();
      const int sib = j ^ 1;
      for (int L = sib * span; L < (sib + 1) * span; ++L) {
        int q0 = 0;   // U columns of L's ancestors above level k
        for (int kk = 1; kk < k; ++kk) q0 += h->nodes[node_index(kk, L >> (depth - kk))].rU;
        yscat.push_back(leaf_yrow[L] + q0);
      }
      nyscat[q] = (int)yscat.size() - yscat0[q];
    }
  }
  // V chunks: runs of whole leaves (or pieces of a leaf) of one node whose
  // rV column segments fit one shared-memory stage of the product kernel.
  int poff = 0, chunk_xrows_max = 0;
  h->vch.clear();
  h->nred.clear();
  for (int k = 1; k <= depth; ++k) {
    const int span = 1 << (depth - k);
    for (int i = 0; i < (1 << k); ++i) {
      const int q = node_index(k, i);
      const NodeDev& nd = h->nodes[q];
      if (nd.rV == 0) continue;
      const int eb = prec_bytes(nd.tierV);
      // at most kChunkRows padded rows (one warp of the product takes a chunk)
      const int cap = kChunkRows;
      NodeRed red;
      memset(&red, 0, sizeof(red));
      // Y_node is only ever multiplied by U of the sibling: fold both
      // power-of-two scales (exact) into the gathered Y
      red.invs = nd.invsV * h->nodes[node_index(k, i ^ 1)].invsU;
      red.rV = nd.rV;
      red.poff0 = poff;
      red.yscat0 = yscat0[q];
      red.nyscat = nyscat[q];
      VChunk ch{};
      bool open = false;
      auto close_chunk = [&]() {
        if (!open) return;
        ch.bytes = ch.rows * eb;
        int xend = ch.xrow0;
        for (int e = 0; e < ch.nseg; ++e)
          if (ch.seg[e].m > 0) xend = std::max(xend, ch.seg[e].row0 + ch.seg[e].m);
        ch.xrows = xend - ch.xrow0;
        chunk_xrows_max = std::max(chunk_xrows_max, ch.xrows);
        h->vch.push_back(ch);
        poff += nd.rV;                           // one partial per chunk
        red.nparts += 1;
        open = false;
      };
      for (int l = i * span; l < (i + 1) * span; ++l) {
        const LeafDev& lf = h->leaves[l];
        for (int o = 0; o < lf.pm;) {
          if (open && (ch.rows >= cap || ch.nseg == kP1Segs)) close_chunk();
          if (!open) {
            memset(&ch, 0, sizeof(ch));
            const int p0 = lf.prow0 - nd.prow0 + o;
            ch.off = nd.offV + (int64_t)p0 * eb;
            ch.colbytes = nd.pm * eb;
            ch.rV = nd.rV;
            ch.node = (int)h->nred.size();
            ch.tier = nd.tierV;
            ch.poff = poff;
            ch.xrow0 = lf.row0 + o;
            open = true;
          }
          const int len = std::min(lf.pm - o, cap - ch.rows);
          P1Seg& sg = ch.seg[ch.nseg++];
          sg.row0 = lf.row0 + o;
          sg.m = std::max(0, std::min(len, lf.m - o));
          sg.prel = ch.rows;
          ch.rows += len;
          o += len;
        }
      }
      close_chunk();
      h->nred.push_back(red);
    }
  }

  // Tensor-core V groups (fp32 work): the fp32 chunks that cover one run of
  // rows (one segment: a leaf or a piece of one), for every level, packed
  // up to kTcRows columns per group in level order.  The other chunks (and
  // every chunk in other working precisions) stay on the CUDA cores.
  // The row table holds kTcRows entries per group, in group order: the
  // byte offset of every A row's first element (-1: no row) and, in V
  // groups, its partial row.
  const int n_tcg_leaf = (int)tcg.size();
  std::vector<TcVRow> tcv;
  TcVRow no_row;
  memset(&no_row, 0, sizeof(no_row));
  no_row.off = -1;
  no_row.prow = -1;
  for (const TcGroup& gr : tcg) {
    const size_t t0 = tcv.size();
    tcv.resize(t0 + kTcRows, no_row);
    const int lmp = (gr.m + 3) & ~3;
    for (int r = 0; r < kTcRows; ++r)
      if ((r >> 5) < gr.ntl) tcv[t0 + r].off = gr.doff[r >> 5] + (int64_t)(r & 31) * lmp * 4;
  }
  h->vch_rest.clear();
  if (h->work == HODLR_FP32) {
    std::map<std::pair<int, int>, std::vector<int>> by_rows;   // (first row, rows) -> chunks
    for (int c = 0; c < (int)h->vch.size(); ++c) {
      const VChunk& ch = h->vch[c];
      const bool ok = ch.tier == HODLR_FP32 && ch.nseg == 1 && ch.seg[0].m > 0 && ch.seg[0].prel == 0 &&
                      ch.rV <= kTcRows && ch.off % 16 == 0 && ch.colbytes % 16 == 0;
      if (ok)
        by_rows[{ch.seg[0].row0, ch.seg[0].m}].push_back(c);
      else
        h->vch_rest.push_back(ch);
    }
    for (const auto& kv : by_rows) {
      TcGroup gr;
      bool open = false;
      for (int c : kv.second) {
        const VChunk& ch = h->vch[c];
        if (open && gr.rows + ch.rV > kTcRows) {
          tcg.push_back(gr);
          open = false;
        }
        if (!open) {
          memset(&gr, 0, sizeof(gr));
          gr.vtab = (int)tcv.size();
          gr.xrow0 = kv.first.first;
          gr.m = kv.first.second;
          tcv.resize(tcv.size() + kTcRows, no_row);
          open = true;
        }
        for (int a = 0; a < ch.rV; ++a) {
          TcVRow& e = tcv[gr.vtab + gr.rows + a];
          e.off = ch.off + (int64_t)a * ch.colbytes;
          e.prow = ch.poff + a;
        }
        gr.rows += ch.rV;
      }
      if (open) tcg.push_back(gr);
    }
  } else {
    h->vch_rest = h->vch;
  }
  // Tensor-core schedule: the groups are dealt to the CTAs of the launch
  // (one per SM) longest first, each to the least loaded CTA, with a cost
  // of (K chunks) x (1 + (32-row quarters of A) / 4) -- X conversion and
  // MMAs per chunk, plus the A rows converted; each CTA's groups then sit
  // together in the group array and the row table.
  std::vector<int32_t> tc_first(1, 0);
  if (!tcg.empty()) {
    int dev = 0, sms = 1;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int G = std::max(1, std::min<int>(sms, (int)tcg.size()));
    std::vector<double> cost(tcg.size());
    std::vector<int> order(tcg.size());
    for (size_t g = 0; g < tcg.size(); ++g) {
      cost[g] = ((tcg[g].m + 31) / 32) * (1.0 + ((tcg[g].rows + 31) / 32) / 4.0);
      order[g] = (int)g;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<std::vector<int>> per(G);
    std::vector<double> load(G, 0.0);
    for (int g : order) {
      const int c = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      per[c].push_back(g);
      load[c] += cost[g];
    }
    std::vector<TcGroup> tcg2;
    std::vector<TcVRow> tcv2;
    tcg2.reserve(tcg.size());
    tcv2.reserve(tcv.size());
    for (int c = 0; c < G; ++c) {
      for (int g : per[c]) {
        TcGroup gr = tcg[g];
        if (gr.vtab >= 0) gr.vtab = (int)tcg2.size() * kTcRows;
        tcv2.insert(tcv2.end(), tcv.begin() + (size_t)g * kTcRows, tcv.begin() + (size_t)(g + 1) * kTcRows);
        tcg2.push_back(gr);
      }
      tc_first.push_back((int32_t)tcg2.size());
    }
    tcg.swap(tcg2);
    tcv.swap(tcv2);
  }

  // ---- streamed product: tiles dealt to the CTAs in contiguous ranges of
  //      about equal bytes, the partial slots of every node (one per CTA
  //      that covers it, in CTA order), the per-(tile, level) table and the
  //      Y items every CTA reduces for itself ----
  int st_grid = 1;
  {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&st_grid, cudaDevAttrMultiProcessorCount, dev));
    st_grid = std::max(st_grid, 1);
  }
  std::vector<int32_t> st_cta_t0(st_grid + 1, 0), cta_of(n_tiles, 0);
  {
    std::vector<int64_t> pre(n_tiles + 1, 0);
    for (int t = 0; t < n_tiles; ++t)
      pre[t + 1] = pre[t] + h->p2[t].vbytes + h->p2[t].bytes + h->p2[t].dbytes;
    for (int c = 1; c < st_grid; ++c) {
      const double target = (double)pre[n_tiles] * c / st_grid;
      int t = (int)(std::lower_bound(pre.begin(), pre.end(), (int64_t)std::ceil(target)) - pre.begin());
      if (t > 0 && target - (double)pre[t - 1] < (double)pre[std::min(t, n_tiles)] - target) --t;
      st_cta_t0[c] = std::min(std::max(t, st_cta_t0[c - 1]), n_tiles);
    }
    st_cta_t0[st_grid] = n_tiles;
    for (int c = 0; c < st_grid; ++c)
      for (int t = st_cta_t0[c]; t < st_cta_t0[c + 1]; ++t) cta_of[t] = c;
  }
  // slot of every (tile, level): the rank of the tile's CTA among the CTAs
  // holding tiles of the level-k ancestor (CTAs without tiles take none)
  std::vector<int> st_nslots(nnodes, 0), st_pslot0(nnodes, -1);
  std::vector<int> tile_slot((size_t)n_tiles * std::max(depth, 1), 0);
  int st_p_rows = 0, st_max_rank = 0;
  for (int k = 1; k <= depth; ++k) {
    const int span = 1 << (depth - k);
    for (int i = 0; i < (1 << k); ++i) {
      const int q = node_index(k, i);
      const NodeDev& nd = h->nodes[q];
      st_max_rank = std::max(st_max_rank, nd.rV);
      int ns = 0, last = -1;
      for (int t = leaf_tile0[i * span]; t < leaf_tile0[(i + 1) * span]; ++t) {
        if (cta_of[t] != last) {
          last = cta_of[t];
          ++ns;
        }
        tile_slot[(size_t)t * depth + (k - 1)] = ns - 1;
      }
      st_nslots[q] = ns;
      if (nd.rV == 0) continue;
      st_pslot0[q] = st_p_rows;
      st_p_rows += ns * nd.rV;
    }
  }
  std::vector<int32_t> st_accoff(depth + 1, 0);
  int st_acc_rows = 0;
  for (int k = 1; k <= depth; ++k) {
    int mx = 0;
    for (int i = 0; i < (1 << k); ++i) mx = std::max(mx, h->nodes[node_index(k, i)].rV);
    st_accoff[k] = st_acc_rows;
    st_acc_rows += mx;
  }
  std::vector<StLev> stlev;   // per (CTA, leaf of the CTA, level)
  std::vector<hodlr::StTile> st_tile(n_tiles);
  std::vector<YItem> st_y;
  std::vector<hodlr::RTask> st_task;
  std::vector<hodlr::StCta> st_cta(st_grid);
  // per CTA: its leaves' records and U columns
  std::vector<std::vector<hodlr::StLeaf>> st_leaf(st_grid);
  std::vector<std::vector<std::vector<hodlr::StCol>>> st_ucol(st_grid);
  int st_max_nu = 0;
  int st_y_rows = 0, st_red_rows = 0, st_max_tiles = 0, st_max_leaves = 0, st_max_vbytes = 0, st_max_cta_v = 0;
  int st_max_cta_xrows = 0, st_max_tile_bytes = 0, st_max_cta_u = 0, st_max_ubytes = 0, st_max_d2bytes = 0;
  for (int c = 0; c < st_grid; ++c) {
    hodlr::StCta& sc = st_cta[c];
    memset(&sc, 0, sizeof(sc));
    sc.t0 = st_cta_t0[c];
    sc.nt = st_cta_t0[c + 1] - st_cta_t0[c];
    if (sc.nt > 0) {
      const P2Tile& a = h->p2[sc.t0];
      const P2Tile& b = h->p2[sc.t0 + sc.nt - 1];
      sc.voff = a.voff;
      sc.vbytes = (int)(b.voff + b.vbytes - a.voff);
      sc.uoff = a.off;
      sc.ubytes = (int)(b.off + b.bytes - a.off);
      sc.xrow0 = a.row0;
      sc.xrows = b.row0 + b.rows - a.row0;
    }
    st_max_tiles = std::max(st_max_tiles, sc.nt);
    st_max_cta_v = std::max(st_max_cta_v, sc.vbytes);
    st_max_cta_xrows = std::max(st_max_cta_xrows, sc.xrows);
    st_max_cta_u = std::max(st_max_cta_u, sc.ubytes);
    sc.y0 = (int32_t)st_y.size();
    std::map<int, int> yrow_of;   // needed node -> its first row in this CTA's Y area
    int ycount = 0;
    std::vector<YItem> items;
    sc.l0 = depth > 0 ? (int32_t)(stlev.size() / depth) : 0;
    int nl = 0, last_leaf = -1;
    for (int t = st_cta_t0[c]; t < st_cta_t0[c + 1]; ++t) {
      const P2Tile& tl = h->p2[t];
      st_max_vbytes = std::max(st_max_vbytes, tl.vbytes);
      st_max_tile_bytes = std::max(st_max_tile_bytes, tl.bytes + tl.d2bytes);
      st_max_ubytes = std::max(st_max_ubytes, tl.bytes);
      st_max_d2bytes = std::max(st_max_d2bytes, tl.d2bytes);
      const int l = tile_leaf[t];
      hodlr::StTile& rec = st_tile[t];
      memset(&rec, 0, sizeof(rec));
      rec.voff = tl.voff;
      rec.uoff = tl.off;
      rec.d2off = tl.d2off;
      rec.vbytes = tl.vbytes;
      rec.ubytes = tl.bytes;
      rec.d2bytes = tl.d2bytes;
      rec.hbytes = (int16_t)tl.hbytes;
      rec.row0 = tl.row0;
      rec.xrow0 = tl.xrow0;
      rec.m = (int16_t)tl.m;
      rec.rows = (int16_t)tl.rows;
      if (l == last_leaf) {
        rec.lleaf = (int16_t)(nl - 1);
        ++st_leaf[c].back().nt;
        continue;   // the leaf's level entries are in place
      }
      last_leaf = l;
      rec.lleaf = (int16_t)nl++;
      {
        hodlr::StLeaf lr;
        memset(&lr, 0, sizeof(lr));
        lr.t0 = (int16_t)(t - sc.t0);
        lr.nt = 1;
        lr.utier = -2;   // no column yet
        st_leaf[c].push_back(lr);
        st_ucol[c].emplace_back();
      }
      stlev.resize(stlev.size() + depth);
      for (int k = 1; k <= depth; ++k) {
        const int a = leaf_anc[l][k];
        const int sib = node_index(k, (l >> (depth - k)) ^ 1);
        const NodeDev& na = h->nodes[a];
        StLev& e = stlev[stlev.size() - depth + (k - 1)];
        memset(&e, 0, sizeof(e));
        e.voff = leaf_vseg[l][k];
        e.rV = (uint16_t)na.rV;
        e.tierV = (uint8_t)na.tierV;
        e.pslot = na.rV ? st_pslot0[a] + tile_slot[(size_t)t * depth + (k - 1)] * na.rV : -1;
        const NodeDev& ns = h->nodes[sib];   // Y_sib multiplies U_a; rank rV(sib) = rU(a)
        if (ns.rV == 0) {
          e.yrow = -1;
          continue;
        }
        auto it = yrow_of.find(sib);
        if (it == yrow_of.end()) {
          YItem y;
          memset(&y, 0, sizeof(y));
          y.pbase = st_pslot0[sib];
          y.nslots = st_nslots[sib];
          y.rV = ns.rV;
          y.yrow = ycount;
          y.invs = ns.invsV * na.invsU;
          y.ntask = (y.nslots + kRedSlots - 1) / kRedSlots;
          items.push_back(y);
          it = yrow_of.emplace(sib, ycount).first;
          ycount += ns.rV;
        }
        e.yrow = it->second;
      }
      // the leaf's U columns, level by level
      hodlr::StLeaf& lr = st_leaf[c].back();
      for (int k = 1; k <= depth; ++k) {
        const NodeDev& na = h->nodes[leaf_anc[l][k]];
        const StLev& e = stlev[stlev.size() - depth + (k - 1)];
        for (int cc = 0; cc < na.rU; ++cc) {
          hodlr::StCol col;
          col.off = tl.hbytes + leaf_useg[l][k] + cc * kTileRows * prec_bytes(na.tierU);
          col.idx = (uint16_t)(e.yrow + cc);
          col.k = (uint8_t)k;
          col.tier = (uint8_t)na.tierU;
          st_ucol[c].back().push_back(col);
          lr.utier = lr.utier == -2 || lr.utier == na.tierU ? (int16_t)na.tierU : (int16_t)-1;
        }
      }
      lr.nu = (int32_t)st_ucol[c].back().size();
      st_max_nu = std::max(st_max_nu, lr.nu);
    }
    sc.nl = nl;
    st_max_leaves = std::max(st_max_leaves, nl);
    // reduction tasks, the heaviest items first (warps take tasks in turn)
    std::stable_sort(items.begin(), items.end(), [](const YItem& x, const YItem& y) {
      return (int64_t)x.nslots * x.rV > (int64_t)y.nslots * y.rV;
    });
    int srow = 0;
    sc.k0 = (int32_t)st_task.size();
    for (size_t q = 0; q < items.size(); ++q) {
      YItem& y = items[q];
      y.srow = srow;
      for (int p = 0; p < y.ntask; ++p) {
        hodlr::RTask tk;
        tk.yi = (int)q;   // the CTA's q-th Y item
        tk.s0 = p * kRedSlots;
        tk.s1 = std::min(y.nslots, (p + 1) * kRedSlots);
        tk.srow = srow + p * y.rV;
        st_task.push_back(tk);
      }
      srow += y.ntask * y.rV;
    }
    sc.nk = (int32_t)st_task.size() - sc.k0;
    st_red_rows = std::max(st_red_rows, srow);
    sc.ny = (int32_t)items.size();
    st_y.insert(st_y.end(), items.begin(), items.end());
    st_y_rows = std::max(st_y_rows, ycount);
  }

  // ---- descriptors and scratch on the device ----
  hodlr_status st;
  if ((st = upload(h->nodes, &h->d_nodes)) != HODLR_OK) return st;
  if ((st = upload(h->leaves, &h->d_leaves)) != HODLR_OK) return st;
  if ((st = upload(h->vch, &h->d_vch)) != HODLR_OK) return st;
  if ((st = upload(h->nred, &h->d_nred)) != HODLR_OK) return st;
  // reduction items, nodes with the most partials first (they take longest)
  std::vector<int2> ritems;
  for (size_t j = 0; j < h->nred.size(); ++j)
    for (int a = 0; a < h->nred[j].rV; ++a) ritems.push_back(make_int2((int)j, a));
  std::stable_sort(ritems.begin(), ritems.end(), [&](const int2& x, const int2& y) {
    return h->nred[x.x].nparts > h->nred[y.x].nparts;
  });
  if ((st = upload(ritems, &h->d_ritems)) != HODLR_OK) return st;
  if ((st = upload(tcg, &h->d_tcg)) != HODLR_OK) return st;
  if ((st = upload(tcv, &h->d_tcv)) != HODLR_OK) return st;
  if ((st = upload(tc_first, &h->d_tc_first)) != HODLR_OK) return st;
  if ((st = upload(h->vch_rest, &h->d_vch_rest)) != HODLR_OK) return st;
  if ((st = upload(h->p2, &h->d_p2)) != HODLR_OK) return st;
  if ((st = upload(yscat, &h->d_yscat)) != HODLR_OK) return st;
  // one fixed-size record per CTA of the streamed product (StCta): its
  // header, tiles, level entries, accumulator offsets, tasks and Y items
  int st_max_nk = 0, st_max_ny = 0;
  for (const hodlr::StCta& sc : st_cta) {
    st_max_nk = std::max(st_max_nk, sc.nk);
    st_max_ny = std::max(st_max_ny, sc.ny);
  }
  const int dl = std::max(depth, 1);
  const int off_tile = (int)align_up(sizeof(hodlr::StCta), 16);
  const int off_lev = off_tile + (int)align_up((size_t)st_max_tiles * sizeof(hodlr::StTile), 16);
  const int off_acc = off_lev + (int)align_up((size_t)st_max_leaves * dl * sizeof(StLev), 16);
  const int off_task = off_acc + (int)align_up((size_t)(depth + 1) * sizeof(int32_t), 16);
  const int off_y = off_task + (int)align_up((size_t)st_max_nk * sizeof(hodlr::RTask), 16);
  const int off_leaf = off_y + (int)align_up((size_t)st_max_ny * sizeof(YItem), 16);
  const int leaf_stride =
      (int)align_up(sizeof(hodlr::StLeaf) + (size_t)st_max_nu * sizeof(hodlr::StCol), 16);
  const int blob_stride = off_leaf + st_max_leaves * leaf_stride;
  std::vector<uint8_t> blob((size_t)blob_stride * st_grid, 0);
  for (int c = 0; c < st_grid; ++c) {
    const hodlr::StCta& sc = st_cta[c];
    uint8_t* b = blob.data() + (size_t)c * blob_stride;
    memcpy(b, &sc, sizeof(sc));
    if (sc.nt) memcpy(b + off_tile, &st_tile[sc.t0], sizeof(hodlr::StTile) * sc.nt);
    if (sc.nl && depth) memcpy(b + off_lev, &stlev[(size_t)sc.l0 * depth], sizeof(StLev) * sc.nl * depth);
    memcpy(b + off_acc, st_accoff.data(), sizeof(int32_t) * (depth + 1));
    if (sc.nk) memcpy(b + off_task, &st_task[sc.k0], sizeof(hodlr::RTask) * sc.nk);
    if (sc.ny) memcpy(b + off_y, &st_y[sc.y0], sizeof(YItem) * sc.ny);
    for (size_t u = 0; u < st_leaf[c].size(); ++u) {
      uint8_t* lb = b + off_leaf + u * leaf_stride;
      memcpy(lb, &st_leaf[c][u], sizeof(hodlr::StLeaf));
      hodlr::StCol* cols = reinterpret_cast<hodlr::StCol*>(lb + sizeof(hodlr::StLeaf));
      if (!st_ucol[c][u].empty()) memcpy(cols, st_ucol[c][u].data(), sizeof(hodlr::StCol) * st_ucol[c][u].size());
    }
  }
  if ((st = upload(blob, &h->d_st_blob)) != HODLR_OK) return st;
  // gathered Y: yrows rows of up to max_nrhs values, plus 16 bytes of slack
  // for the rounded-up tile copies
  const size_t yb = ((size_t)std::max(yrows, 1) * h->max_nrhs + 4) * ebw;
  const size_t pb = (size_t)std::max(poff, 1) * h->max_nrhs * ebw;
  if (cudaMalloc(&h->d_Y, yb) != cudaSuccess) return fail(HODLR_ENOMEM, "Y scratch");
  if (cudaMalloc(&h->d_partials, pb) != cudaSuccess) return fail(HODLR_ENOMEM, "partials scratch");
  // partial slots of the streamed product (batches of up to kStreamMaxCols columns)
  const size_t spb = (size_t)std::max(st_p_rows, 1) * kStreamMaxCols * ebw;
  if (cudaMalloc(&h->d_spart, spb) != cudaSuccess) return fail(HODLR_ENOMEM, "streamed partials scratch");
  // grid counter (starts at zero and only grows)
  const size_t sync_bytes = kSyncHeadBytes;
  if (cudaMalloc((void**)&h->d_sync, sync_bytes) != cudaSuccess) return fail(HODLR_ENOMEM, "grid counter");
  if (cudaMalloc((void**)&h->d_err, sizeof(int)) != cudaSuccess) return fail(HODLR_ENOMEM, "error word");
  CK(cudaMemsetAsync(h->d_sync, 0, sync_bytes, s));
  h->sync_base = 0;
  CK(cudaMemsetAsync(h->d_err, 0, sizeof(int), s));
  CK(cudaMemsetAsync(h->d_Y, 0, yb, s));
  CK(cudaStreamSynchronize(s));
  h->scratch_bytes = yb + pb + spb + sync_bytes;

  HandleDev& hd = h->hd;
  memset(&hd, 0, sizeof(hd));
  hd.nodes = h->d_nodes;
  hd.leaves = h->d_leaves;
  hd.vch = h->d_vch;
  hd.nred = h->d_nred;
  hd.p2 = h->d_p2;
  hd.yscat = h->d_yscat;
  hd.ritems = h->d_ritems;
  hd.n_ritems = (int)ritems.size();
  hd.tcg = h->d_tcg;
  hd.n_tcg = (int)tcg.size();
  hd.n_tcg_leaf = n_tcg_leaf;
  hd.tc_first = h->d_tc_first;
  hd.n_tc_cta = (int)tc_first.size() - 1;
  hd.tcv = h->d_tcv;
  hd.vch_rest = h->d_vch_rest;
  hd.n_vch_rest = (int)h->vch_rest.size();
  hd.pool = h->d_pool;
  hd.err = h->d_err;
  hd.n = n;
  hd.depth = depth;
  hd.n_nodes = nnodes;
  hd.n_leaves = nleaves;
  hd.n_vch = (int)h->vch.size();
  hd.n_nred = (int)h->nred.size();
  hd.n_p2 = (int)h->p2.size();
  hd.chunk_xrows_max = chunk_xrows_max;
  hd.y_rows = yrows;
  hd.p_rows = poff;
  hd.max_nq = max_nq;
  // a stage holds the leaf-block part of one tile
  hd.stage_bytes = (int)align_up((size_t)std::max(max_region, 16), 128);
  hd.leaf_pm_max = leaf_pm_max;
  hd.x_aligned = 1;
  for (const LeafDev& lf : h->leaves) {
    hd.leaf_m_max = std::max(hd.leaf_m_max, lf.m);
    if (lf.row0 % 4 || lf.m % 4) hd.x_aligned = 0;
  }
  hd.st_blob = h->d_st_blob;
  hd.st_blob_stride = blob_stride;
  hd.st_off_tile = off_tile;
  hd.st_off_lev = off_lev;
  hd.st_off_acc = off_acc;
  hd.st_off_task = off_task;
  hd.st_off_y = off_y;
  hd.st_off_leaf = off_leaf;
  hd.st_leaf_stride = leaf_stride;
  hd.st_max_nu = st_max_nu;
  hd.st_max_leaves = st_max_leaves;
  hd.st_grid = st_grid;
  hd.st_p_rows = st_p_rows;
  hd.st_y_rows = st_y_rows;
  hd.st_acc_rows = st_acc_rows;
  hd.st_max_rank = st_max_rank;
  hd.st_red_rows = st_red_rows;
  hd.st_max_tiles = st_max_tiles;
  hd.st_max_vbytes = st_max_vbytes;
  hd.st_max_cta_v = st_max_cta_v;
  hd.st_max_cta_xrows = st_max_cta_xrows;
  hd.st_max_tile_bytes = st_max_tile_bytes;
  hd.st_max_cta_u = st_max_cta_u;
  hd.st_max_ubytes = st_max_ubytes;
  hd.st_max_d2bytes = st_max_d2bytes;
  // CUDA-core products: the streamed kernel when its shared-memory plan fits
  // (every realistic rank), else the two-barrier kernel, which reads U rows
  // that do not fit from global memory
  const int sb = stream_max_batch(hd, h->work);
  h->use_stream = sb > 0;
  const int mb = h->use_stream ? sb : matvec_max_batch(hd, h->work);
  if (mb < 1) return fail(HODLR_EINVAL, "leaf blocks too large for the product's shared-memory stages; increase depth");
  h->batch = std::min(h->max_nrhs, mb);
  inf.device_bytes = (int64_t)(pool + h->scratch_bytes + h->nodes.size() * sizeof(NodeDev) +
                               h->leaves.size() * sizeof(LeafDev) + h->vch.size() * sizeof(VChunk) +
                               h->nred.size() * sizeof(NodeRed) + ritems.size() * sizeof(int2) + tcg.size() * sizeof(TcGroup) + tcv.size() * sizeof(TcVRow) + h->vch_rest.size() * sizeof(VChunk) + h->p2.size() * sizeof(P2Tile) + yscat.size() * sizeof(int32_t) +
                               blob.size());
  return HODLR_OK;
}

}  // namespace hodlr

extern "C" {

const char* hodlr_status_string(hodlr_status s) {
  switch (s) {
    case HODLR_OK: return "ok";
    case HODLR_EINVAL: return "invalid argument";
    case HODLR_ENOMEM: return "out of memory";
    case HODLR_ECUDA: return "CUDA error";
    case HODLR_ETIMEOUT: return "device wait timed out";
    case HODLR_ENOTFACTORED: return "matrix not factored";
    case HODLR_ESINGULAR: return "singular pivot";
    case HODLR_EACCURACY: return "accuracy target not met";
  }
  return "unknown status";
}

const char* hodlr_last_error(void) { return g_last_error.c_str(); }

void hodlr_destroy(hodlr_t h) {
  if (!h) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(h->device);
  cudaDeviceSynchronize();
  delete h;
  cudaSetDevice(cur);
}

hodlr_status hodlr_import(int32_t n, int32_t depth, const int32_t* ranks, const double* const* U,
                          const double* const* V, const double* const* D, const hodlr_opts* opts,
                          void* stream, hodlr_t* out) {
  g_last_error.clear();
  if (!out || !opts) return fail(HODLR_EINVAL, "null out/opts");
  if (depth > 0 && (!ranks || !U || !V)) return fail(HODLR_EINVAL, "null ranks/U/V");
  if (!D) return fail(HODLR_EINVAL, "null D");
  cudaStream_t s = (cudaStream_t)stream;
  auto h = new hodlr_s();
  std::unique_ptr<hodlr_s> guard(h);
  hodlr_status st = plan_layout(h, n, depth, ranks, opts);
  if (st != HODLR_OK) return st;
  const int nnodes = (int)h->nodes.size(), nleaves = (int)h->leaves.size();
  for (int q = 0; q < nnodes; ++q) {
    if (h->nodes[q].rU > 0 && !U[q]) return fail(HODLR_EINVAL, "null U generator");
    if (h->nodes[q].rV > 0 && !V[q]) return fail(HODLR_EINVAL, "null V generator");
  }
  for (int l = 0; l < nleaves; ++l)
    if (!D[l]) return fail(HODLR_EINVAL, "null leaf block");

  std::vector<double> host_stage;
  try { host_stage.resize((size_t)h->st_count); } catch (...) { return fail(HODLR_ENOMEM, "host staging"); }
  for (int q = 0; q < nnodes; ++q) {
    const NodeDev& nd = h->nodes[q];
    if (nd.rU) memcpy(&host_stage[h->st_U[q]], U[q], sizeof(double) * nd.m * nd.rU);
    if (nd.rV) memcpy(&host_stage[h->st_V[q]], V[q], sizeof(double) * nd.m * nd.rV);
  }
  for (int l = 0; l < nleaves; ++l)
    memcpy(&host_stage[h->st_D[l]], D[l], sizeof(double) * h->leaves[l].m * h->leaves[l].m);
  DevBuf d_stage;
  if (cudaMalloc(&d_stage.p, sizeof(double) * std::max<int64_t>(h->st_count, 1)) != cudaSuccess)
    return fail(HODLR_ENOMEM, "device staging");
  CK(cudaMemcpyAsync(d_stage.p, host_stage.data(), sizeof(double) * h->st_count,
                     cudaMemcpyHostToDevice, s));
  st = finish_from_staging(h, (const double*)d_stage.p, nullptr, nullptr, opts, s);
  if (st != HODLR_OK) return st;
  *out = guard.release();
  return HODLR_OK;
}

hodlr_status hodlr_export(hodlr_t h, double* const* U, double* const* V, double* const* D,
                          void* stream) {
  g_last_error.clear();
  if (!h) return fail(HODLR_EINVAL, "null handle");
  cudaStream_t s = (cudaStream_t)stream;
  DevBuf d_stage, d_tasks;
  if (cudaMalloc(&d_stage.p, sizeof(double) * std::max<int64_t>(h->st_count, 1)) != cudaSuccess)
    return fail(HODLR_ENOMEM, "export staging");
  CK(cudaMalloc(&d_tasks.p, std::max<size_t>(h->tasks.size(), 1) * sizeof(PackTask)));
  CK(cudaMemcpyAsync(d_tasks.p, h->tasks.data(), h->tasks.size() * sizeof(PackTask),
                     cudaMemcpyHostToDevice, s));
  CK(launch_unpack(h->d_pool, (const PackTask*)d_tasks.p, (int)h->tasks.size(),
                   (double*)d_stage.p, s));
  std::vector<double> host((size_t)h->st_count);
  CK(cudaMemcpyAsync(host.data(), d_stage.p, sizeof(double) * h->st_count, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const int nnodes = (int)h->nodes.size();
  for (int q = 0; q < nnodes; ++q) {
    const NodeDev& nd = h->nodes[q];
    if (U && U[q] && nd.rU) memcpy(U[q], &host[h->st_U[q]], sizeof(double) * nd.m * nd.rU);
    if (V && V[q] && nd.rV) memcpy(V[q], &host[h->st_V[q]], sizeof(double) * nd.m * nd.rV);
  }
  for (size_t l = 0; l < h->leaves.size(); ++l)
    if (D && D[l])
      memcpy(D[l], &host[h->st_D[l]], sizeof(double) * h->leaves[l].m * h->leaves[l].m);
  return HODLR_OK;
}

// ---- hodlr_save / hodlr_load ----------------------------------------------
// File: SaveHeader, then per node (2^(depth+1) - 2 of them) the rank, the
// block format and the power-of-two scales of U and V, then hodlr_info_t,
// then the stored generators and leaves decoded to fp64 (the export staging
// layout, st_count values).  Host byte order.
namespace {
struct SaveHeader {
  char magic[8];
  int32_t version, n, depth, work, per_block, max_nrhs;
  uint32_t avail;
  int32_t pad_;
  double eps;
  int64_t st_count;
};
constexpr char kSaveMagic[8] = {'H', 'O', 'D', 'L', 'R', 'S', 'V', '1'};

struct File {
  FILE* f = nullptr;
  ~File() { if (f) fclose(f); }
};
}  // namespace

hodlr_status hodlr_save(hodlr_t h, const char* path, void* stream) {
  g_last_error.clear();
  if (!h || !path) return fail(HODLR_EINVAL, "null handle/path");
  const int nnodes = (int)h->nodes.size(), nleaves = (int)h->leaves.size();
  std::vector<double> host;
  try { host.resize((size_t)h->st_count); } catch (...) { return fail(HODLR_ENOMEM, "host staging"); }
  {
    cudaStream_t s = (cudaStream_t)stream;
    DevBuf d_stage, d_tasks;
    if (cudaMalloc(&d_stage.p, sizeof(double) * std::max<int64_t>(h->st_count, 1)) != cudaSuccess)
      return fail(HODLR_ENOMEM, "save staging");
    CK(cudaMalloc(&d_tasks.p, std::max<size_t>(h->tasks.size(), 1) * sizeof(PackTask)));
    CK(cudaMemcpyAsync(d_tasks.p, h->tasks.data(), h->tasks.size() * sizeof(PackTask), cudaMemcpyHostToDevice, s));
    CK(launch_unpack(h->d_pool, (const PackTask*)d_tasks.p, (int)h->tasks.size(), (double*)d_stage.p, s));
    CK(cudaMemcpyAsync(host.data(), d_stage.p, sizeof(double) * h->st_count, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  SaveHeader hd;
  memset(&hd, 0, sizeof(hd));
  memcpy(hd.magic, kSaveMagic, 8);
  hd.version = 1;
  hd.n = h->n;
  hd.depth = h->depth;
  hd.work = h->work;
  hd.per_block = h->per_block;
  hd.max_nrhs = h->max_nrhs;
  hd.avail = h->avail;
  hd.eps = h->eps;
  hd.st_count = h->st_count;
  std::vector<int32_t> rank(nnodes), tier(nnodes);
  std::vector<double> sU(nnodes), sV(nnodes);
  for (int q = 0; q < nnodes; ++q) {
    rank[q] = h->nodes[q].rU;
    tier[q] = h->nodes[q].tierU;
    sU[q] = 1.0 / h->nodes[q].invsU;
    sV[q] = 1.0 / h->nodes[q].invsV;
  }
  (void)nleaves;
  File fl;
  fl.f = fopen(path, "wb");
  if (!fl.f) return fail(HODLR_EINVAL, std::string("cannot open for writing: ") + path);
  bool ok = fwrite(&hd, sizeof(hd), 1, fl.f) == 1;
  if (nnodes) {
    ok = ok && fwrite(rank.data(), sizeof(int32_t), nnodes, fl.f) == (size_t)nnodes;
    ok = ok && fwrite(tier.data(), sizeof(int32_t), nnodes, fl.f) == (size_t)nnodes;
    ok = ok && fwrite(sU.data(), sizeof(double), nnodes, fl.f) == (size_t)nnodes;
    ok = ok && fwrite(sV.data(), sizeof(double), nnodes, fl.f) == (size_t)nnodes;
  }
  ok = ok && fwrite(&h->info, sizeof(hodlr_info_t), 1, fl.f) == 1;
  ok = ok && fwrite(host.data(), sizeof(double), host.size(), fl.f) == host.size();
  ok = (fclose(fl.f) == 0) && ok;
  fl.f = nullptr;
  if (!ok) return fail(HODLR_EINVAL, std::string("write failed: ") + path);
  return HODLR_OK;
}

hodlr_status hodlr_load(const char* path, void* stream, hodlr_t* out) {
  g_last_error.clear();
  if (!path || !out) return fail(HODLR_EINVAL, "null path/out");
  File fl;
  fl.f = fopen(path, "rb");
  if (!fl.f) return fail(HODLR_EINVAL, std::string("cannot open: ") + path);
  SaveHeader hd;
  if (fread(&hd, sizeof(hd), 1, fl.f) != 1 || memcmp(hd.magic, kSaveMagic, 8) != 0 || hd.version != 1)
    return fail(HODLR_EINVAL, "not a hodlr_save file (magic/version)");
  if (hd.depth < 0 || hd.depth > HODLR_MAX_DEPTH || hd.n < 1 || ((int64_t)1 << hd.depth) > hd.n || hd.st_count < 0)
    return fail(HODLR_EINVAL, "corrupt hodlr_save header");
  const int nnodes = (1 << (hd.depth + 1)) - 2;
  std::vector<int32_t> rank(nnodes), tier(nnodes);
  std::vector<double> sU(nnodes), sV(nnodes);
  bool ok = true;
  if (nnodes) {
    ok = fread(rank.data(), sizeof(int32_t), nnodes, fl.f) == (size_t)nnodes;
    ok = ok && fread(tier.data(), sizeof(int32_t), nnodes, fl.f) == (size_t)nnodes;
    ok = ok && fread(sU.data(), sizeof(double), nnodes, fl.f) == (size_t)nnodes;
    ok = ok && fread(sV.data(), sizeof(double), nnodes, fl.f) == (size_t)nnodes;
  }
  hodlr_info_t info;
  ok = ok && fread(&info, sizeof(info), 1, fl.f) == 1;
  if (!ok) return fail(HODLR_EINVAL, "truncated hodlr_save file");
  for (int q = 0; q < nnodes; ++q)
    if (tier[q] < 0 || tier[q] >= kPrecCount || !((hd.avail >> tier[q]) & 1u) || !(sU[q] > 0.0) || !(sV[q] > 0.0))
      return fail(HODLR_EINVAL, "corrupt hodlr_save file (formats/scales)");
  hodlr_opts opts;
  memset(&opts, 0, sizeof(opts));
  opts.eps = hd.eps;
  opts.work = hd.work;
  opts.tier_mask = hd.avail;
  opts.per_block = hd.per_block;
  opts.max_nrhs = hd.max_nrhs;
  auto h = new hodlr_s();
  std::unique_ptr<hodlr_s> guard(h);
  hodlr_status st = plan_layout(h, hd.n, hd.depth, rank.data(), &opts);
  if (st != HODLR_OK) return st;
  if (h->st_count != hd.st_count) return fail(HODLR_EINVAL, "corrupt hodlr_save file (sizes)");
  std::vector<double> host;
  try { host.resize((size_t)h->st_count); } catch (...) { return fail(HODLR_ENOMEM, "host staging"); }
  if (fread(host.data(), sizeof(double), host.size(), fl.f) != host.size())
    return fail(HODLR_EINVAL, "truncated hodlr_save file (values)");
  h->force_tier.assign(tier.begin(), tier.end());
  h->force_sU = sU;
  h->force_sV = sV;
  cudaStream_t s = (cudaStream_t)stream;
  DevBuf d_stage;
  if (cudaMalloc(&d_stage.p, sizeof(double) * std::max<int64_t>(h->st_count, 1)) != cudaSuccess)
    return fail(HODLR_ENOMEM, "device staging");
  CK(cudaMemcpyAsync(d_stage.p, host.data(), sizeof(double) * h->st_count, cudaMemcpyHostToDevice, s));
  st = finish_from_staging(h, (const double*)d_stage.p, nullptr, nullptr, &opts, s);
  if (st != HODLR_OK) return st;
  h->force_tier.clear();
  h->force_sU.clear();
  h->force_sV.clear();
  const int64_t device_bytes = h->info.device_bytes;
  h->info = info;
  h->info.device_bytes = device_bytes;
  *out = guard.release();
  return HODLR_OK;
}

hodlr_status hodlr_matvec(hodlr_t h, int32_t nrhs, const void* X, int64_t ldx, void* B,
                          int64_t ldb, int32_t xb_prec, void* stream) {
  if (!h) return fail(HODLR_EINVAL, "null handle");
  if (nrhs < 0) return fail(HODLR_EINVAL, "nrhs < 0");
  if (nrhs == 0) return HODLR_OK;
  if (!X || !B) return fail(HODLR_EINVAL, "null X/B");
  if (ldx < nrhs || ldb < nrhs) return fail(HODLR_EINVAL, "leading dimension < nrhs");
  if (xb_prec != h->work) return fail(HODLR_EINVAL, "X/B type must equal the working precision");
  const size_t es = prec_bytes(h->work);
  const char* xb = (const char*)X;
  char* bb = (char*)B;
  const size_t span_x = ((size_t)(h->n - 1) * ldx + nrhs) * es, span_b = ((size_t)(h->n - 1) * ldb + nrhs) * es;
  if (!(xb + span_x <= bb || bb + span_b <= xb)) return fail(HODLR_EINVAL, "X and B overlap");
  cudaStream_t s = (cudaStream_t)stream;
  // fp32 work with many right-hand sides: leaf products on the tensor cores
  // (batches of up to kTcMaxCols columns), low-rank part in the product
  // kernel; otherwise the product kernel alone (batches of h->batch)
  const bool tc = h->work == HODLR_FP32 && nrhs >= kTcMinCols && h->hd.n_tcg_leaf > 0;
  // hodlr_debug_stall_next: the first launch of this call waits for grid
  // barrier arrivals that never come (the counter itself advances as usual)
  unsigned long long skew = h->stall_next ? 4ull * (matvec_sync_step(h->hd) + stream_sync_step(h->hd)) : 0ull;
  h->stall_next = false;
  const int step = tc ? std::min(h->max_nrhs, kTcMaxCols) : h->batch;
  for (int c0 = 0; c0 < nrhs; c0 += step) {
    const int nb = std::min(step, nrhs - c0);
    const bool last = c0 + step >= nrhs;
    cudaEvent_t* ev = (h->prof_on && last) ? h->prof_ev : nullptr;
    cudaError_t e = cudaSuccess;
    if (tc && nb >= kTcMinCols) {
      if (ev) cudaEventRecord(ev[0], s);
      e = launch_leaf_tc(h->hd.tcg, h->hd.tc_first, h->hd.n_tc_cta, h->hd.tcv, h->hd.pool, (const float*)(xb + c0 * es), ldx, nb,
                         (float*)(bb + c0 * es), ldb, (float*)h->d_partials, h->d_err, s);
      if (e != cudaSuccess) return cuda_fail(e, "hodlr_matvec leaf launch");
      if (ev) cudaEventRecord(ev[1], s);
      e = launch_matvec(h->hd, h->work, nb, xb + c0 * es, ldx, bb + c0 * es, ldb, h->d_Y, h->d_partials,
                        h->d_sync, h->sync_base + skew, s, nullptr, 1);
      skew = 0;
      if (ev) cudaEventRecord(ev[2], s);
      h->sync_base += matvec_sync_step(h->hd);
    } else {
      // CUDA cores: the streamed product in batches of h->batch columns
      for (int d0 = 0; d0 < nb && e == cudaSuccess; d0 += h->batch) {
        const int nd = std::min(h->batch, nb - d0);
        const bool lastd = d0 + h->batch >= nb;
        // fp64 work is bound by the FP64 multiply-add rate; beyond one column
        // the two-barrier kernel's lane layouts use it better
        if (h->use_stream && (h->work != HODLR_FP64 || nd == 1)) {
          e = launch_stream(h->hd, h->work, nd, xb + (c0 + d0) * es, ldx, bb + (c0 + d0) * es, ldb, h->d_spart,
                            h->d_sync, h->sync_base + skew, s, lastd ? ev : nullptr);
          h->sync_base += stream_sync_step(h->hd);
        } else {
          e = launch_matvec(h->hd, h->work, nd, xb + (c0 + d0) * es, ldx, bb + (c0 + d0) * es, ldb, h->d_Y,
                            h->d_partials, h->d_sync, h->sync_base + skew, s, lastd ? ev : nullptr);
          h->sync_base += matvec_sync_step(h->hd);
        }
        skew = 0;
      }
    }
    if (e != cudaSuccess) return cuda_fail(e, "hodlr_matvec launch");
  }
  if (h->prof_on) h->prof_valid = true;
  return HODLR_OK;
}

hodlr_status hodlr_sync_status(hodlr_t h, void* stream) {
  if (!h) return fail(HODLR_EINVAL, "null handle");
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  int code = 0;
  CK(cudaMemcpy(&code, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (code == 0) return HODLR_OK;
  CK(cudaMemset(h->d_err, 0, sizeof(int)));
  return fail(HODLR_ETIMEOUT, "a device wait gave up (code " + std::to_string(code) + ")");
}

hodlr_status hodlr_debug_stall_next(hodlr_t h) {
  if (!h) return fail(HODLR_EINVAL, "null handle");
  h->stall_next = true;
  return HODLR_OK;
}

hodlr_status hodlr_profile(hodlr_t h, int32_t enable) {
  if (!h) return fail(HODLR_EINVAL, "null handle");
  if (enable && !h->prof_ev[0])
    for (cudaEvent_t& e : h->prof_ev) CK(cudaEventCreate(&e));
  h->prof_on = enable != 0;
  h->prof_valid = false;
  return HODLR_OK;
}

hodlr_status hodlr_profile_read(hodlr_t h, float* ms, int32_t count) {
  if (!h || !ms || count < 2) return fail(HODLR_EINVAL, "null handle/ms or count < 2");
  if (!h->prof_on || !h->prof_valid) return fail(HODLR_EINVAL, "no profiled call");
  CK(cudaEventSynchronize(h->prof_ev[2]));
  CK(cudaEventElapsedTime(&ms[0], h->prof_ev[0], h->prof_ev[1]));
  CK(cudaEventElapsedTime(&ms[1], h->prof_ev[1], h->prof_ev[2]));
  return HODLR_OK;
}

hodlr_status hodlr_info(hodlr_t h, hodlr_info_t* out) {
  if (!h || !out) return fail(HODLR_EINVAL, "null handle/out");
  *out = h->info;
  return HODLR_OK;
}

hodlr_status hodlr_block_tiers(hodlr_t h, int32_t* tiers, int32_t* ranks) {
  if (!h) return fail(HODLR_EINVAL, "null handle");
  for (size_t q = 0; q < h->nodes.size(); ++q) {
    if (tiers) tiers[q] = h->nodes[q].tierU;
    if (ranks) ranks[q] = h->nodes[q].rU;
  }
  return HODLR_OK;
}

hodlr_status hodlr_build_stats(hodlr_t h, int32_t* rounds, int32_t* redone, int64_t* sketch_cols) {
  if (!h) return fail(HODLR_EINVAL, "null handle");
  if (rounds) *rounds = h->build_rounds;
  if (redone) *redone = h->build_redone;
  if (sketch_cols) *sketch_cols = h->build_sketch_cols;
  return HODLR_OK;
}

hodlr_status hodlr_node_sizes(hodlr_t h, int32_t* row0, int32_t* m) {
  if (!h) return fail(HODLR_EINVAL, "null handle");
  for (size_t q = 0; q < h->nodes.size(); ++q) {
    if (row0) row0[q] = h->nodes[q].row0;
    if (m) m[q] = h->nodes[q].m;
  }
  return HODLR_OK;
}

hodlr_status hodlr_dense_kernel_matvec(int32_t n, int32_t dim, const double* points, int32_t kind,
                                       double c, double len2, double diag, int32_t nrows,
                                       const int32_t* rows, int32_t nrhs, const double* X,
                                       int64_t ldx, double* B, int64_t ldb, void* stream) {
  if (n < 1 || dim < 1 || dim > 3 || !points) return fail(HODLR_EINVAL, "bad n/dim/points");
  if (kind < 0 || kind > 3 || (kind == 3 && dim != 1)) return fail(HODLR_EINVAL, "bad kernel kind");
  if (kind == 1 && !(len2 > 0.0)) return fail(HODLR_EINVAL, "len2 must be > 0");
  if (nrows < 0 || nrhs < 0 || (!rows && nrows != n)) return fail(HODLR_EINVAL, "bad rows");
  if (nrows == 0 || nrhs == 0) return HODLR_OK;
  if (!X || !B || ldx < nrhs || ldb < nrhs) return fail(HODLR_EINVAL, "bad X/B");
  cudaError_t e = launch_dense_kernel_matvec(n, dim, points, kind, c, len2, diag, nrows, rows,
                                             nrhs, X, ldx, B, ldb, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "dense kernel matvec");
  return HODLR_OK;
}

}  // extern "C"
