// HODLR_MATVEC (Algorithm 3.3) on sm_103a.
//
// Algorithm 3.3 walks the levels and adds U_{2i-1}(V_{2i}^T x_{2i}) and
// U_{2i}(V_{2i-1}^T x_{2i-1}) into b, then the leaf products D_i x_i.  Here
// the level loop is flattened into one persistent kernel (one CTA per SM,
// cooperative launch so that all CTAs are co-resident) with these stages:
//
//  phase A  every warp of the grid takes V chunks (up to 256 rows of one
//           node V_j) and writes the chunk's part of V_j^T X[I_j] to its
//           partial rows, loading V and X directly;
//  reduce   after a grid counter shows every chunk done: Y_j = the sum of
//           its chunk partials in chunk order, scaled, written into the
//           gathered-Y block of every leaf below the sibling of j (three
//           reducer warps per CTA; the items are dealt across the CTAs);
//  pass 1   for every 32-row tile of a leaf i: D_i[rows, :] X[I_i], which
//           does not depend on phase A (a producer warp streams the tiles'
//           leaf blocks and X rows through a ring of shared-memory stages
//           with cp.async.bulk, completion on mbarriers) -- it overlaps the
//           reductions;
//  pass 2   after a second grid counter: for every tile, B[rows] = (pass 1)
//           + sum_k U_{a_k}[rows, :] Y_{a_k ^ 1}, a_k the level-k ancestor
//           of leaf i (one warp per tile, U rows by a bulk copy into the
//           warp's slice of shared memory).
//
// With fp32 work and 16 or more right-hand sides the leaf products and the
// fp32 V chunks go to the tensor cores first (leaf_tc.cu); this kernel then
// runs with skip_leaf: no pass 1, phase A only for the chunks left over,
// and the consumer warps help with the reductions.
//
// Each output row is written once, with a fixed summation order, so the
// product is bitwise reproducible.  Every wait gives up after two seconds; a
// wait that gives up records an error code in the handle's error word and
// the CTA drains the copies it issued and returns.
#include <algorithm>
#include <type_traits>

#include "dev_common.cuh"

namespace hodlr {

namespace {

constexpr int kCWarps = kConsumerWarps;       // consumer warps of the product kernel
constexpr int kCThreads = 32 * kCWarps;
constexpr int kRedWarps = 3;                  // node-reduction warps
constexpr int kP2Threads = kCThreads + 32 + 32 * kRedWarps;   // consumers, producer, reducers
constexpr int kMaxStages = 6;
constexpr int kMaxColsLane = 16;              // right-hand sides per lane and step of pass 2
constexpr int kP1Rows = 4;                    // pass 1: tile rows per consumer warp
constexpr int kP1Warps = 8;                   // pass 1: warps per tile (kP1Rows * kP1Warps = 32 rows)
constexpr int kP1Groups = 2;                  // pass 1: tiles in work at once per CTA
// ---- the product kernel ----------------------------------------------------
// Phase A: every V chunk of this CTA -> its part of V_node^T X, summed over
//          the CTA in a fixed order.  A node held by one chunk is finished
//          on the spot (Y_node written to its gathered-Y targets); for a
//          node of several chunks each chunk leaves a partial and the CTA
//          that completes the last one adds them in chunk order.  Then the
//          CTA arrives at the grid counter (without waiting).
// Pass 1:  every tile of this CTA -> D[rows, :] X[I_i] (needs no Y), kept
//          in shared memory (or in B when it does not fit).
// Pass 2:  every tile of this CTA -> B[rows] = pass-1 result +
//          U[rows, :] Yg[leaf].
// The producer warp streams V chunks, the tiles' D parts, and, once the grid
// counter shows that every CTA has finished phase A, the tiles' U parts with
// their gathered-Y blocks, through one ring of shared-memory stages.  Only
// the producer waits for the grid; the consumers never do.
//
// Lane layout: LC lanes across right-hand-side columns (CPL consecutive
// columns each) and LK = 32 / LC lanes across the summation index, so that a
// warp-wide load of X, Y or a factor touches LK consecutive rows of up to
// LC * CPL consecutive columns.  Each lane sums its share of the index in
// order, then the LK partial sums are added by a fixed butterfly.

template <int LC, int CPL>
struct Lanes {
  static constexpr int LK = 32 / LC;            // lanes across the summation index
  static constexpr int BW = LC * CPL;           // columns per pass
  static constexpr int RTA = 8;                 // V columns per phase-A pass
};

__device__ __forceinline__ void bar_consumers() {
  asm volatile("bar.sync 1, %0;" ::"r"(kCThreads) : "memory");
}
template <typename W, int LC, int CPL>
__global__ void __launch_bounds__(kP2Threads, 1)
matvec_kernel(const HandleDev hd, const W* __restrict__ X, int64_t ldx, int R, W* __restrict__ Yg,
              W* __restrict__ partials, W* __restrict__ B, int64_t ldb, unsigned long long* sync,
              unsigned long long sync_base, int nstages, int xstage_bytes, int res_smem, int skip_leaf) {
  using L = Lanes<LC, CPL>;
  constexpr int LK = L::LK, BW = L::BW, RTA = L::RTA;
  extern __shared__ __align__(128) uint8_t smem[];
  constexpr int ebw = sizeof(W);
  const int G = gridDim.x;
  const int ntiles = hd.n_p2 > (int)blockIdx.x ? (hd.n_p2 - (int)blockIdx.x + G - 1) / G : 0;   // this CTA's tiles
  const int stage_bytes = hd.stage_bytes;
  uint8_t* stages = smem;                                               // [S][stage_bytes]
  uint8_t* xstages = smem + (size_t)nstages * stage_bytes;              // [S][xstage_bytes] (may be 0)
  W* res = reinterpret_cast<W*>(xstages + (size_t)nstages * xstage_bytes);   // pass-1 results (if res_smem)
  const size_t res_bytes = res_smem ? ((size_t)ntiles * kTileRows * R * ebw + 127) / 128 * 128 : 0;
  uint64_t* full = reinterpret_cast<uint64_t*>(reinterpret_cast<uint8_t*>(res) + res_bytes);
  uint64_t* empty = full + kMaxStages;
  uint64_t* wbarA = empty + kMaxStages;                                 // [kCWarps] pass-2 copies
  P2Tile* s_tile = reinterpret_cast<P2Tile*>(wbarA + kCWarps);          // [S]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < nstages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kP1Warps);
    }
    for (int w = 0; w < kCWarps; ++w) mbar_init(&wbarA[w], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // ---- node reductions: Y_node[a, :] = invs * sum of its chunk partials
  //      (each lane sums the partials lane, lane + 32, ... in order, then a
  //      fixed butterfly), written to the node's gathered-Y targets.  A work
  //      unit is one item (node, row a) and one block of kMaxColsLane
  //      columns, so that the items with the most partials do not hold up
  //      the grid with a long chain of loads.  The items are sorted heaviest
  //      first and the units dealt to the CTAs in turn (warp w of CTA c
  //      starts at unit w * grid + c) so that no SM gets several heavy ones;
  //      a warp takes units first, first + stride, ... ----
  const int ncb = (R + kMaxColsLane - 1) / kMaxColsLane;
  auto reduce_items = [&](int first, int stride) {
    for (int wu = first; wu < hd.n_ritems * ncb; wu += stride) {
      const int it = wu / ncb;
      const int2 ri = __ldg(hd.ritems + it);
      const NodeRed* nrp = hd.nred + ri.x;
      const int P = __ldg(&nrp->nparts), rV = __ldg(&nrp->rV), poff0 = __ldg(&nrp->poff0);
      const int y0 = __ldg(&nrp->yscat0), ny = __ldg(&nrp->nyscat);
      const W invs = (W)__ldg(&nrp->invs);
      const W* pp = partials + (int64_t)(poff0 + ri.y) * R;
      {
        const int c0 = (wu - it * ncb) * kMaxColsLane;
        const int nc = min(kMaxColsLane, R - c0);
        W acc[kMaxColsLane];
#pragma unroll
        for (int j = 0; j < kMaxColsLane; ++j) acc[j] = (W)0;
        if (sizeof(W) == 4 && nc == kMaxColsLane && R % 4 == 0) {
          // 16 columns as four 16-byte loads per partial, two partials in flight
          int q = lane;
          for (; q + 32 < P; q += 64) {
            const float4* r0 = reinterpret_cast<const float4*>(pp + (int64_t)q * rV * R + c0);
            const float4* r1 = reinterpret_cast<const float4*>(pp + (int64_t)(q + 32) * rV * R + c0);
            float4 v0[kMaxColsLane / 4], v1[kMaxColsLane / 4];
#pragma unroll
            for (int j4 = 0; j4 < kMaxColsLane / 4; ++j4) {
              v0[j4] = __ldcg(r0 + j4);
              v1[j4] = __ldcg(r1 + j4);
            }
#pragma unroll
            for (int j4 = 0; j4 < kMaxColsLane / 4; ++j4) {
              acc[4 * j4 + 0] += (W)v0[j4].x;
              acc[4 * j4 + 1] += (W)v0[j4].y;
              acc[4 * j4 + 2] += (W)v0[j4].z;
              acc[4 * j4 + 3] += (W)v0[j4].w;
              acc[4 * j4 + 0] += (W)v1[j4].x;
              acc[4 * j4 + 1] += (W)v1[j4].y;
              acc[4 * j4 + 2] += (W)v1[j4].z;
              acc[4 * j4 + 3] += (W)v1[j4].w;
            }
          }
          if (q < P) {
            const float4* r0 = reinterpret_cast<const float4*>(pp + (int64_t)q * rV * R + c0);
#pragma unroll
            for (int j4 = 0; j4 < kMaxColsLane / 4; ++j4) {
              const float4 v = __ldcg(r0 + j4);
              acc[4 * j4 + 0] += (W)v.x;
              acc[4 * j4 + 1] += (W)v.y;
              acc[4 * j4 + 2] += (W)v.z;
              acc[4 * j4 + 3] += (W)v.w;
            }
          }
        } else {
          for (int q = lane; q < P; q += 32) {
            const W* row = pp + (int64_t)q * rV * R + c0;
            W v[kMaxColsLane];
#pragma unroll
            for (int j = 0; j < kMaxColsLane; ++j) v[j] = j < nc ? __ldcg(row + j) : (W)0;
#pragma unroll
            for (int j = 0; j < kMaxColsLane; ++j) acc[j] += v[j];
          }
        }
#pragma unroll
        for (int j = 0; j < kMaxColsLane; ++j) acc[j] = warp_sum(acc[j]) * invs;
        for (int t = lane; t < ny; t += 32) {
          W* dst = Yg + (int64_t)(__ldg(hd.yscat + y0 + t) + ri.y) * R + c0;
#pragma unroll
          for (int j = 0; j < kMaxColsLane; ++j)
            if (j < nc) dst[j] = acc[j];
        }
      }
    }
  };
  // warps of the CTA that reduce: the reducers, and in skip_leaf mode (no
  // leaf pass to overlap) the consumers as well
  constexpr int kAllRed = kCWarps + kRedWarps;
  constexpr int kRedBar = 32 * kAllRed;   // threads of barrier 3 (skip_leaf mode)

  if (warp > kCWarps) {
    // ================= reducers =================
    // After every CTA's phase A (first stage of the grid counter): node
    // reductions, then the second stage of the grid counter.
    const int rw = warp - kCWarps - 1;
    if (hd.n_ritems > 0) {
      if (lane == 0) grid_wait(sync, sync_base + (unsigned long long)G, hd.err);
      __syncwarp();
      if (skip_leaf)
        reduce_items((kCWarps + rw) * G + blockIdx.x, G * kAllRed);
      else
        reduce_items(rw * G + blockIdx.x, G * kRedWarps);
      __threadfence();
    }
    if (skip_leaf)
      asm volatile("bar.sync 3, %0;" ::"r"(kRedBar) : "memory");
    else
      asm volatile("bar.sync 2, %0;" ::"r"(32 * kRedWarps) : "memory");
    if (rw == 0 && lane == 0) atomicAdd(sync, 1ull);
    return;
  }

  if (warp == kCWarps) {
    // ================= producer: the leaf blocks of this CTA's tiles =================
    if (lane != 0 || skip_leaf) return;
    int i = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < hd.n_p2; tile += G, ++i) {
      const int s = i % nstages;
      if (i >= nstages && !(ok = mbar_wait(&empty[s], ((i / nstages) - 1) & 1, hd.err, 1))) break;
      const P2Tile t = hd.p2[tile];
      s_tile[s] = t;
      const uint32_t xbytes = xstage_bytes ? (uint32_t)t.m * R * ebw : 0u;
      mbar_arrive_expect_tx(&full[s], (uint32_t)t.dbytes + xbytes);
      bulk_g2s(stages + (size_t)s * stage_bytes, hd.pool + t.doff, (uint32_t)t.dbytes,
               &full[s]);
      if (xbytes) bulk_g2s(xstages + (size_t)s * xstage_bytes, X + (int64_t)t.xrow0 * R, xbytes, &full[s]);
    }
    if (!ok) {
      // a wait gave up: let the copies already issued land before the CTA exits
      for (int j = (i > nstages ? i - nstages : 0); j < i; ++j)
        mbar_wait(&full[j % nstages], (j / nstages) & 1, hd.err, 3);
    }
    return;
  }

  // ================= consumers (warps 0 .. kCWarps-1) =================
  const int tid = threadIdx.x;
  const int kl = lane / LC, cl = lane - (lane / LC) * LC;   // lane = kl * LC + cl
  bool alive = true;

  // ---- phase A: every warp of the grid takes V chunks alone, reading V and
  //      X directly (a chunk is at most kChunkRows rows of one node) ----
  // chunks are dealt to the CTAs in turn (warp w of CTA c starts at chunk
  // w * grid + c), so the wide top-level chunks spread over all SMs
  // (with skip_leaf the tensor-core launch has done the chunks its V groups
  // cover: only the rest are left)
  const VChunk* const vchs = skip_leaf ? hd.vch_rest : hd.vch;
  const int n_vchs = skip_leaf ? hd.n_vch_rest : hd.n_vch;
  for (int c = warp * G + blockIdx.x; c < n_vchs; c += G * kCWarps) {
    const VChunk& ch = vchs[c];
    const int rV = __ldg(&ch.rV), poff = __ldg(&ch.poff), nseg = __ldg(&ch.nseg), tier = __ldg(&ch.tier);
    const int colbytes = __ldg(&ch.colbytes);
    const uint8_t* vbase = hd.pool + __ldg(&ch.off);
    for (int c0 = 0; c0 < R; c0 += BW) {
      const int col = c0 + cl * CPL;
      const bool cok = col < R;
      const int kcol = cok ? col : 0;   // lanes past the last column read column 0 and drop it
      for (int r0 = 0; r0 < rV; r0 += RTA) {
        W acc[RTA][CPL];
#pragma unroll
        for (int a = 0; a < RTA; ++a)
#pragma unroll
          for (int j = 0; j < CPL; ++j) acc[a][j] = (W)0;
        auto run = [&](auto tc) {
          constexpr int TIER = decltype(tc)::value;
          constexpr int eb = TIER == HODLR_FP64 ? 8 : TIER == HODLR_FP32 ? 4 : (TIER == HODLR_E4M3 || TIER == HODLR_E5M2) ? 1 : 2;
          for (int li = 0; li < nseg; ++li) {
            const int srow0 = __ldg(&ch.seg[li].row0), sm = __ldg(&ch.seg[li].m), sprel = __ldg(&ch.seg[li].prel);
            const W* xgr = X + (int64_t)srow0 * ldx + kcol;
            const uint8_t* vrow = vbase + (int64_t)r0 * colbytes + (int64_t)sprel * eb;
            // UNR rows per lane at a time: every load of the block is issued
            // before the first multiply-add (no branch between them: rows past
            // the segment read its first row of the block with x = 0, columns
            // past the rank read the last column and are never stored)
            constexpr int UNR = (CPL >= 4 || sizeof(W) == 8) ? 2 : 4;
            const int a_last = rV - 1 - r0;
            for (int pl0 = kl; pl0 < sm; pl0 += UNR * LK) {
              W xv[UNR][CPL];
              W vv[UNR][RTA];
#pragma unroll
              for (int u = 0; u < UNR; ++u) {
                const int pl = pl0 + u * LK;
                const bool rok = pl < sm;
                const int pr = rok ? pl : pl0;
                load_cols<W, CPL>(xgr + (int64_t)pr * ldx, true, xv[u]);
#pragma unroll
                for (int j = 0; j < CPL; ++j) xv[u][j] = rok ? xv[u][j] : (W)0;
                const uint8_t* vp = vrow + (int64_t)pr * eb;
#pragma unroll
                for (int a = 0; a < RTA; ++a) vv[u][a] = gld_fmt<W, TIER>(vp + (int64_t)min(a, a_last) * colbytes);
              }
#pragma unroll
              for (int u = 0; u < UNR; ++u)
#pragma unroll
                for (int a = 0; a < RTA; ++a)
#pragma unroll
                  for (int j = 0; j < CPL; ++j) acc[a][j] = fma(vv[u][a], xv[u][j], acc[a][j]);
            }
          }
        };
        with_format(tier, run);
        // lanes of one column: fixed butterfly; the chunk's partial
#pragma unroll
        for (int a = 0; a < RTA; ++a)
#pragma unroll
          for (int j = 0; j < CPL; ++j) {
#pragma unroll
            for (int o = LC; o < 32; o <<= 1) acc[a][j] += __shfl_xor_sync(0xffffffffu, acc[a][j], o);
          }
        if (kl == 0 && cok) {
#pragma unroll
          for (int a = 0; a < RTA; ++a)
            if (r0 + a < rV) store_cols<W, CPL>(partials + (int64_t)(poff + r0 + a) * R + col, acc[a]);
        }
      }
    }
  }
  // ---- first stage of the grid counter: this CTA's partials are written ----
  __threadfence();
  bar_consumers();
  if (tid == 0) atomicAdd(sync, 1ull);
  if (skip_leaf) {
    // no leaf pass to overlap: help with the node reductions
    if (hd.n_ritems > 0) {
      if (tid == 0) grid_wait(sync, sync_base + (unsigned long long)G, hd.err);
      bar_consumers();
      reduce_items(warp * G + blockIdx.x, G * kAllRed);
      __threadfence();
    }
    asm volatile("bar.sync 3, %0;" ::"r"(kRedBar) : "memory");
  }

  // ---- pass 1: D[rows, :] X[I_i] for every tile.  The consumers work in
  //      kP1Groups groups of kP1Warps warps; group g takes tiles g, g +
  //      kP1Groups, ... and warp w of a group owns rows kP1Rows w ..
  //      kP1Rows w + kP1Rows - 1 of the tile (each X value read from shared
  //      memory serves kP1Rows rows) ----
  static_assert(kP1Rows * kP1Warps == kTileRows && kP1Warps * kP1Groups == kCWarps, "pass-1 warp layout");
  static_assert(kTileRows == 32, "one lane per tile row in pass 2");
  {
    const int grp = warp / kP1Warps, r0w = kP1Rows * (warp - grp * kP1Warps);
    for (int tl = grp; tl < (skip_leaf ? 0 : ntiles); tl += kP1Groups) {
      const int s = tl % nstages;
      if (!mbar_wait(&full[s], (tl / nstages) & 1, hd.err, 4)) {
        alive = false;
        break;
      }
      const P2Tile t = s_tile[s];
      const uint32_t st_a = smem_u32(stages + (size_t)s * stage_bytes);
      const uint32_t xs_a = smem_u32(xstages + (size_t)s * xstage_bytes);
      // pass-1 results of tile tl, column by column (32 rows per column)
      const uint32_t res_t = smem_u32(res) + (uint32_t)((size_t)tl * kTileRows * R * ebw);
      const int mp = (t.m + 3) & ~3;   // D row length
      const uint32_t da = st_a + (uint32_t)(r0w * mp * ebw), drs = (uint32_t)(mp * ebw);
      for (int c0 = 0; c0 < R; c0 += BW) {
        const int col = c0 + cl * CPL;
        const bool cok = col < R;
        const int kcol = cok ? col : 0;   // lanes past the last column read column 0 and drop it
        W acc[kP1Rows][CPL];
#pragma unroll
        for (int i = 0; i < kP1Rows; ++i)
#pragma unroll
          for (int j = 0; j < CPL; ++j) acc[i][j] = (W)0;
        bool done = false;
        if constexpr (LC == 1 && CPL == 1 && sizeof(W) == 4) {
          if (xstage_bytes) {
            // one right-hand side, X staged (m is a multiple of 4): four
            // consecutive columns of D per lane and step
            for (int k = 4 * lane; k < t.m; k += 128) {
              const float4 x4 = sld_v4f32(xs_a + (uint32_t)(k * 4));
#pragma unroll
              for (int i = 0; i < kP1Rows; ++i) {
                const float4 a4 = sld_v4f32(da + i * drs + (uint32_t)(k * 4));
                acc[i][0] = fmaf(a4.x, x4.x, acc[i][0]);
                acc[i][0] = fmaf(a4.y, x4.y, acc[i][0]);
                acc[i][0] = fmaf(a4.z, x4.z, acc[i][0]);
                acc[i][0] = fmaf(a4.w, x4.w, acc[i][0]);
              }
            }
            done = true;
          }
        }
        if (!done) {
          if (xstage_bytes) {
#pragma unroll 4
            for (int k = kl; k < t.m; k += LK) {
              W xv[CPL];
              sld_cols<W, CPL>(xs_a + (uint32_t)((k * R + kcol) * ebw), xv);
#pragma unroll
              for (int i = 0; i < kP1Rows; ++i) {
                const W d = sld<W>(da + i * drs + (uint32_t)(k * ebw));
#pragma unroll
                for (int j = 0; j < CPL; ++j) acc[i][j] = fma(d, xv[j], acc[i][j]);
              }
            }
          } else {
            const W* xg = X + (int64_t)t.xrow0 * ldx + kcol;
#pragma unroll 4
            for (int k = kl; k < t.m; k += LK) {
              W xv[CPL];
              load_cols<W, CPL>(xg + (int64_t)k * ldx, true, xv);
#pragma unroll
              for (int i = 0; i < kP1Rows; ++i) {
                const W d = sld<W>(da + i * drs + (uint32_t)(k * ebw));
#pragma unroll
                for (int j = 0; j < CPL; ++j) acc[i][j] = fma(d, xv[j], acc[i][j]);
              }
            }
          }
        }
#pragma unroll
        for (int i = 0; i < kP1Rows; ++i)
#pragma unroll
          for (int j = 0; j < CPL; ++j) {
#pragma unroll
            for (int o = LC; o < 32; o <<= 1) acc[i][j] += __shfl_xor_sync(0xffffffffu, acc[i][j], o);
          }
        if (kl == 0 && cok) {
#pragma unroll
          for (int i = 0; i < kP1Rows; ++i) {
            const int ra = r0w + i;
            if (res_smem) {
#pragma unroll
              for (int j = 0; j < CPL; ++j) sst<W>(res_t + (uint32_t)(((col + j) * kTileRows + ra) * ebw), acc[i][j]);
            } else if (ra < t.rows) {
              store_cols<W, CPL>(B + (int64_t)(t.row0 + ra) * ldb + col, acc[i]);
            }
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
    }
  }

  // ---- every Y_node is in the gathered Y after the second stage ----
  if (tid == 0 && ntiles) grid_wait(sync, sync_base + 2ull * (unsigned long long)G, hd.err);
  bar_consumers();   // also: pass-1 results are complete for every warp

  // ---- pass 2: warp (tl mod kCWarps) takes tile tl alone, lane r = row r:
  //      B[row] = (pass 1) + sum_q U[row, q] Y[q, :].  The ring is idle now;
  //      each warp copies its tile's header and U rows into its own slice of
  //      the ring's memory and, for every block of up to 16 columns, loads the
  //      block of the leaf's gathered Y beside them ----
  const size_t wslice = ((size_t)nstages * stage_bytes / kCWarps) / 128 * 128;
  uint8_t* wbuf = stages + (size_t)warp * wslice;
  for (int tl = warp, use = 0; tl < ntiles && alive; tl += kCWarps, ++use) {
    const P2Tile* tp = hd.p2 + blockIdx.x + (int64_t)tl * G;
    const int64_t toff = __ldg(&tp->off);
    const int nq = __ldg(&tp->nq), hbytes = __ldg(&tp->hbytes), ubytes = __ldg(&tp->ubytes);
    const int nlev = hd.depth;   // header entries
    const int rows = __ldg(&tp->rows), row0 = __ldg(&tp->row0), yrow = __ldg(&tp->yrow);
    const uint32_t res_t = smem_u32(res) + (uint32_t)((size_t)tl * kTileRows * R * ebw);
    const int r = lane;
    const bool staged = (size_t)(hbytes + ubytes) + (size_t)nq * kMaxColsLane * ebw <= wslice;
    uint32_t hdr_a, ys_a;
    const uint8_t* hdr_g = hd.pool + toff;
    if (staged) {
      hdr_a = smem_u32(wbuf);
      ys_a = hdr_a + (uint32_t)(hbytes + ubytes);
      uint64_t* bar = &wbarA[warp];
      if (lane == 0) {
        // earlier generic reads of this memory (pass 1) before the async copies
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(bar, (uint32_t)(hbytes + ubytes));
        if (hbytes + ubytes) bulk_g2s(wbuf, hdr_g, (uint32_t)(hbytes + ubytes), bar);
      }
      __syncwarp();
      if (!mbar_wait(bar, use & 1, hd.err, 7)) {
        alive = false;
        break;
      }
    }
    for (int c0 = 0; c0 < R; c0 += kMaxColsLane) {
      const int nc = min(kMaxColsLane, R - c0);
      if (staged) {
        // Y[:, c0 .. c0 + nc) of the leaf beside header and U, rows of
        // kMaxColsLane values (coalesced loads, one round trip)
        __syncwarp();
        if (sizeof(W) == 4 && nc == kMaxColsLane && R % 4 == 0) {
          // four values per lane and load
#pragma unroll 4
          for (int e = lane; e < nq * (kMaxColsLane / 4); e += 32) {
            const int q = e / (kMaxColsLane / 4), j4 = e - q * (kMaxColsLane / 4);
            const float4 v = __ldcg(reinterpret_cast<const float4*>(Yg + (int64_t)(yrow + q) * R + c0) + j4);
            sst_v4f32(ys_a + (uint32_t)(e * 16), v);
          }
        } else {
          for (int e = lane; e < nq * kMaxColsLane; e += 32) {
            const int q = e / kMaxColsLane, j = e - q * kMaxColsLane;
            const W v = j < nc ? __ldcg(Yg + (int64_t)(yrow + q) * R + c0 + j) : (W)0;
            sst<W>(ys_a + (uint32_t)(e * ebw), v);
          }
        }
        __syncwarp();
      }
      // the pass-1 part of this row (shared memory, or B when it did not
      // fit there or the leaf products came from the tensor-core kernel),
      // loaded before the U Y loop so the global loads overlap it
      W* brow = B + (int64_t)(row0 + r) * ldb + c0;
      W acc[kMaxColsLane];
      const bool bvec = sizeof(W) == 4 && nc == kMaxColsLane && ldb % 4 == 0 &&
                        (reinterpret_cast<uintptr_t>(brow) & 15) == 0;
      if (r < rows) {
        if (res_smem) {
#pragma unroll
          for (int j = 0; j < kMaxColsLane; ++j)
            acc[j] = j < nc ? sld<W>(res_t + (uint32_t)(((c0 + j) * kTileRows + r) * ebw)) : (W)0;
        } else if (bvec) {
#pragma unroll
          for (int j4 = 0; j4 < kMaxColsLane / 4; ++j4) {
            const float4 v = *reinterpret_cast<const float4*>(brow + 4 * j4);
            acc[4 * j4 + 0] = (W)v.x;
            acc[4 * j4 + 1] = (W)v.y;
            acc[4 * j4 + 2] = (W)v.z;
            acc[4 * j4 + 3] = (W)v.w;
          }
        } else {
#pragma unroll
          for (int j = 0; j < kMaxColsLane; ++j) acc[j] = j < nc ? brow[j] : (W)0;
        }
      } else {
#pragma unroll
        for (int j = 0; j < kMaxColsLane; ++j) acc[j] = (W)0;
      }
      W uy[kMaxColsLane];
#pragma unroll
      for (int j = 0; j < kMaxColsLane; ++j) uy[j] = (W)0;
      // level by level (the format is fixed within a level): one dispatch on
      // the format per level, then a loop over the level's U columns
      int q = 0;
      for (int lv = 0; lv < nlev; ++lv) {
        uint32_t w0, w1;
        if (staged) {
          w0 = sld_u32(hdr_a + 8u * lv);
          w1 = sld_u32(hdr_a + 8u * lv + 4u);
        } else {
          const uint2 w = __ldg(reinterpret_cast<const uint2*>(hdr_g) + lv);
          w0 = w.x;
          w1 = w.y;
        }
        const int rU = (int)(w1 & 0xffffu), tier = (int)(w1 >> 16);
        auto level = [&](auto tc) {
          constexpr int TIER = decltype(tc)::value;
          constexpr int eb = TIER == HODLR_FP64 ? 8 : TIER == HODLR_FP32 ? 4 : (TIER == HODLR_E4M3 || TIER == HODLR_E5M2) ? 1 : 2;
          if (staged) {
            const uint32_t ucol = hdr_a + (uint32_t)hbytes + w0 + (uint32_t)(r * eb);
#pragma unroll 2
            for (int c = 0; c < rU; ++c) {
              const W u = sld_fmt<W, TIER>(ucol + (uint32_t)(c * kTileRows * eb));
              // the staged Y row (zero past nc): vector loads, the same
              // address for every lane
              W yv[kMaxColsLane];
              sld_vec<W, kMaxColsLane>(ys_a + (uint32_t)((q + c) * kMaxColsLane * ebw), yv);
#pragma unroll
              for (int j = 0; j < kMaxColsLane; ++j) uy[j] = fma(u, yv[j], uy[j]);
            }
          } else {
            // too large for the slice: U and Y read directly
            const uint8_t* ucol = hdr_g + hbytes + w0 + r * eb;
            const W* yb = Yg + (int64_t)(yrow + q) * R + c0;
#pragma unroll 2
            for (int c = 0; c < rU; ++c) {
              const W u = gld_fmt<W, TIER>(ucol + (int64_t)c * kTileRows * eb);
#pragma unroll
              for (int j = 0; j < kMaxColsLane; ++j)
                if (j < nc) uy[j] = fma(u, __ldcg(yb + (int64_t)c * R + j), uy[j]);
            }
          }
        };
        with_format(tier, level);
        q += rU;
      }
      if (r < rows) {
        if (bvec) {
#pragma unroll
          for (int j4 = 0; j4 < kMaxColsLane / 4; ++j4)
            *reinterpret_cast<float4*>(brow + 4 * j4) =
                make_float4(acc[4 * j4] + uy[4 * j4], acc[4 * j4 + 1] + uy[4 * j4 + 1],
                            acc[4 * j4 + 2] + uy[4 * j4 + 2], acc[4 * j4 + 3] + uy[4 * j4 + 3]);
        } else {
#pragma unroll
          for (int j = 0; j < kMaxColsLane; ++j)
            if (j < nc) brow[j] = acc[j] + uy[j];
        }
      }
    }
    __syncwarp();   // every lane is done with the slice before the next copy
  }
}

constexpr int kXStageMax = 32 * 1024;   // stage X through shared memory up to this size
constexpr int kResMax = 32 * 1024;      // pass-1 results in shared memory up to this size

// shared memory besides the stages and the pass-1 results: barriers and
// descriptors
size_t kernel_fixed_smem() {
  return (size_t)(2 * kMaxStages + kCWarps) * sizeof(uint64_t) + (size_t)kMaxStages * sizeof(P2Tile) + 128;
}

int n_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  }
  return n;
}

int smem_optin() {
  static int v = 0;
  if (!v) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  }
  return v;
}

template <typename W, int LC, int CPL>
cudaError_t launch_lc(const HandleDev& hd, int nrhs, const W* X, int64_t ldx, W* B, int64_t ldb, W* Y,
                      W* partials, unsigned long long* sync, unsigned long long sync_base, cudaStream_t s,
                      cudaEvent_t* ev, int skip_leaf) {
  // X rows go through shared memory (a bulk copy with each tile) when they
  // are contiguous, 16-byte aligned and small enough
  const int64_t xb = (int64_t)hd.leaf_m_max * nrhs * (int)sizeof(W);
  const bool x_tma = !skip_leaf && hd.x_aligned && ldx == nrhs && ((uintptr_t)X % 16) == 0 && xb <= kXStageMax;
  const int xstage = x_tma ? (int)((xb + 127) / 128 * 128) : 0;
  // pass-1 results of this CTA's tiles in shared memory when small enough
  const int G = n_sms();
  const int64_t tiles_cta = (hd.n_p2 + G - 1) / G;
  const int64_t rb = (tiles_cta * kTileRows * nrhs * (int64_t)sizeof(W) + 127) / 128 * 128;
  const int res_smem = (!skip_leaf && rb <= kResMax) ? 1 : 0;
  const size_t fixed = kernel_fixed_smem() + (res_smem ? rb : 0);
  const size_t per_stage = (size_t)hd.stage_bytes + xstage;
  const int nstages = (int)std::min<size_t>(kMaxStages, ((size_t)smem_optin() - fixed) / per_stage);
  if (nstages < 1) return cudaErrorInvalidConfiguration;   // the host sizes batches so this cannot happen
  const size_t smem = fixed + per_stage * nstages;
  static size_t smem_set = 0;   // per instantiation: largest size opted in so far
  if (smem > smem_set) {
    cudaError_t e = cudaFuncSetAttribute(matvec_kernel<W, LC, CPL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    smem_set = smem;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(kP2Threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (ev) cudaEventRecord(ev[0], s);
  cudaError_t e = cudaLaunchKernelEx(&cfg, matvec_kernel<W, LC, CPL>, hd, X, ldx, nrhs, Y, partials, B, ldb,
                                     sync, sync_base, nstages, xstage, res_smem, skip_leaf);
  if (e != cudaSuccess) return e;
  if (ev) {
    cudaEventRecord(ev[1], s);
    cudaEventRecord(ev[2], s);
  }
  return cudaGetLastError();
}

// Lane layout for nrhs columns: LC = the smallest power of two >= nrhs (at
// most 32); two columns per lane for nrhs > 32 in fp32 when every row of X, B
// and the scratch starts on an 8-byte boundary; four columns per lane on
// two lanes for 8 fp32 columns when they start on a 16-byte
// boundary (fewer shared-memory loads per multiply-add in the leaf pass,
// more lanes over the rows).
template <typename W>
cudaError_t launch_w(const HandleDev& hd, int nrhs, const W* X, int64_t ldx, W* B, int64_t ldb, W* Y,
                     W* partials, unsigned long long* sync, unsigned long long base, cudaStream_t s,
                     cudaEvent_t* ev, int skip_leaf) {
#define HODLR_LAUNCH(LC, CPL) \
  launch_lc<W, LC, CPL>(hd, nrhs, X, ldx, B, ldb, Y, partials, sync, base, s, ev, skip_leaf)
  if (nrhs == 1) return HODLR_LAUNCH(1, 1);
  if (nrhs == 2) return HODLR_LAUNCH(2, 1);
  if (nrhs <= 4) return HODLR_LAUNCH(4, 1);
  if constexpr (sizeof(W) == 4) {
    const bool quads = nrhs <= 8 && nrhs % 4 == 0 && ldx % 4 == 0 && ldb % 4 == 0 && (uintptr_t)X % 16 == 0 &&
                       (uintptr_t)B % 16 == 0;
    if (quads) return HODLR_LAUNCH(2, 4);
  }
  if (nrhs <= 8) return HODLR_LAUNCH(8, 1);
  if (nrhs <= 16) return HODLR_LAUNCH(16, 1);
  if constexpr (sizeof(W) == 4) {
    const bool pairs = nrhs > 32 && nrhs % 2 == 0 && ldx % 2 == 0 && ldb % 2 == 0 &&
                       (uintptr_t)X % 8 == 0 && (uintptr_t)B % 8 == 0;
    if (pairs) return HODLR_LAUNCH(32, 2);
  }
  return HODLR_LAUNCH(32, 1);
#undef HODLR_LAUNCH
}

}  // namespace

int matvec_grid(const HandleDev& hd) {
  (void)hd;
  return n_sms();
}

unsigned long long matvec_sync_step(const HandleDev& hd) {
  return 2ull * (unsigned long long)matvec_grid(hd);   // two arrivals per CTA
}

// Up to kMaxCols columns per launch: X rows of a chunk or a tile then fit
// one shared-memory stage (512 or leaf rows x 16 x 4 bytes <= 32 KiB);
// wider products run in batches of columns.
constexpr int kMaxCols = 16;

int matvec_max_batch(const HandleDev& hd, int work) {
  const int ebw = prec_bytes(work);
  const size_t fixed = kernel_fixed_smem();
  const int64_t room = (int64_t)smem_optin() - (int64_t)fixed - hd.stage_bytes - 256;
  if (room <= 0) return 0;
  (void)ebw;
  return kMaxCols;
}

cudaError_t launch_matvec(const HandleDev& hd, int work, int nrhs, const void* X, int64_t ldx,
                          void* B, int64_t ldb, void* Y, void* partials,
                          unsigned long long* sync, unsigned long long sync_base,
                          cudaStream_t s, cudaEvent_t* ev, int skip_leaf) {
  if (work == HODLR_FP64)
    return launch_w<double>(hd, nrhs, (const double*)X, ldx, (double*)B, ldb, (double*)Y, (double*)partials,
                            sync, sync_base, s, ev, skip_leaf);
  return launch_w<float>(hd, nrhs, (const float*)X, ldx, (float*)B, ldb, (float*)Y, (float*)partials, sync,
                         sync_base, s, ev, skip_leaf);
}

}  // namespace hodlr
