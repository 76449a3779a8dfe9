// The streamed HODLR product (Algorithm 3.3) on sm_103a, CUDA cores.
//
// Algorithm 3.3 forms, for every node j, Y_j = V_j^T x[I_j] and adds
// U_{j^1} Y_j into the rows of the sibling, then the leaf products D_i x_i.
// Every V_j^T x[I_j] is a sum over the rows of I_j, so a row partition of
// the matrix splits it into partial sums (the identity behind the
// row-partitioned product).  Here the rows are dealt to the CTAs of one
// persistent launch (one CTA per SM, cooperative so that all CTAs are
// co-resident) in contiguous ranges of 32-row tiles of about equal bytes.
// Each CTA reads what its rows need once, by bulk copies into shared memory,
// and three groups of warps work at the same time:
//
//  V warps   the V rows of all its tiles (one copy into the V/U area): the
//            CTA's partial sum of V_j^T X for every node j it covers, written
//            to the node's slot for this CTA; the CTA arrives at a grid
//            counter; once every CTA has arrived, the Y_j its tiles need
//            (each the sum of node j's slots in slot order, times the
//            power-of-two scales of V_j and U_{j^1}) into shared memory;
//  D warps   from the first microsecond, the leaf-block rows of its tiles
//            through a ring of stages: D_i[rows, :] X[I_i] (needs no Y),
//            kept in shared memory (or in B when it does not fit);
//  all       at the end, the header and U rows of its tiles (copied into the
//            V/U area once the V phase is done): B[rows] = D X +
//            sum_k U_{a_k}[rows, :] Y_{a_k ^ 1}, a_k the level-k ancestor.
//
// So the leaf blocks, which are most of the bytes, stream while the V
// phase, the single grid-wide dependency and the reduction run.  A producer
// warp issues the leaf-block copies.  The loops run lane = row where the
// summation index is a row (V^T X, over the rows of a tile) and lane = row
// with a broadcast operand where it is a column (D X, U Y), so no lanes are
// added except at the end of a node's rows in the V phase.
//
// Every output row is written once and every sum has a fixed order, so the
// product is bitwise reproducible.  Every wait is bounded (two seconds); a
// wait that gives up records an error code in the handle's error word, the
// warps skip the remaining work but keep the CTA's barrier protocol, and
// every copy issued is waited for before the CTA exits.
#include <algorithm>
#include <cstring>

#include "dev_common.cuh"

namespace hodlr {

namespace {

constexpr int kSWarps = 16;                           // consumer warps: V warps, then D warps
constexpr int kSThreads = 32 * kSWarps;
constexpr int kSAll = kSThreads + 32;                 // consumers and the producer warp
constexpr int kSStagesMax = 8;
constexpr int kSXMax = 32 * 1024;                     // a leaf's X rows staged with its tiles up to this
constexpr int kSInflight = 2;                         // leaf-block copies in flight per CTA at most

// Shared-memory plan of one launch (host computed).
struct SPlan {
  int nstages, stage_bytes;                // the leaf-block ring
  int dmax;                                // leaf-block copies in flight at most
  int nvw;                                 // V warps (V phase, reduction, U Y); the other consumers are D warps
  int wps;                                 // D warps per ring stage (one group per stage)
  int vu_off, vu_bytes;                    // the V/U area
  int res_off, res_smem;                   // D X results of the CTA's tiles (in shared memory when they fit)
  int uy_off, uy_smem;                     // U Y of the CTA's tiles (computed by the V warps when it fits)
  int part_off;                            // partial rows of the D groups' helpers
  int acc_off, ys_off, red_off, bar_off, meta_off;   // byte offsets in dynamic shared memory
  int xstaged;                             // X rows travel with the copies
  int smem;                                // total bytes
};

// ---- shared-memory accesses as plain loads and stores (the compiler keeps
//      them in the shared window and may schedule them ahead of their use;
//      every wait on a barrier is an asm statement with a memory clobber, so
//      no access moves across one) ----
template <typename W, int P>
__device__ __forceinline__ W ldf(const uint8_t* p) {   // one element of storage format P
  if constexpr (P == HODLR_FP64) {
    return (W)*reinterpret_cast<const double*>(p);
  } else if constexpr (P == HODLR_FP32) {
    return (W)*reinterpret_cast<const float*>(p);
  } else if constexpr (P == HODLR_FP16) {
    return (W)__half2float(*reinterpret_cast<const __half*>(p));
  } else if constexpr (P == HODLR_BF16) {
    return (W)__uint_as_float(((uint32_t)*reinterpret_cast<const uint16_t*>(p)) << 16);
  } else {
    __half_raw h = __nv_cvt_fp8_to_halfraw(*reinterpret_cast<const __nv_fp8_storage_t*>(p),
                                           P == HODLR_E4M3 ? __NV_E4M3 : __NV_E5M2);
    return (W)__half2float(*reinterpret_cast<__half*>(&h));
  }
}
// CPL consecutive values (16-byte aligned when CPL = 4, fp32 only)
template <typename W, int CPL>
__device__ __forceinline__ void ldc(const W* p, W (&v)[CPL]) {
  if constexpr (CPL == 4 && sizeof(W) == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
  } else {
#pragma unroll
    for (int j = 0; j < CPL; ++j) v[j] = p[j];
  }
}
template <typename W, int CPL>
__device__ __forceinline__ void stc(W* p, const W (&v)[CPL]) {
  if constexpr (CPL == 4 && sizeof(W) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
#pragma unroll
    for (int j = 0; j < CPL; ++j) p[j] = v[j];
  }
}

// BW consecutive values of a staged row, as 16-byte vectors when VEC
template <typename W, int BW, bool VEC>
__device__ __forceinline__ void ld_row(const W* p, W (&v)[BW]) {
  if constexpr (VEC && sizeof(W) == 4 && BW % 4 == 0) {
#pragma unroll
    for (int j4 = 0; j4 < BW / 4; ++j4) {
      const float4 t4 = reinterpret_cast<const float4*>(p)[j4];
      v[4 * j4 + 0] = (W)t4.x;
      v[4 * j4 + 1] = (W)t4.y;
      v[4 * j4 + 2] = (W)t4.z;
      v[4 * j4 + 3] = (W)t4.w;
    }
  } else {
#pragma unroll
    for (int j = 0; j < BW; ++j) v[j] = p[j];
  }
}

// the metadata copies move 8- and 16-byte words
static_assert(sizeof(StTile) % 8 == 0, "StTile is copied in 8-byte words");
static_assert(sizeof(StLev) % 16 == 0, "StLev is copied in 16-byte words");

template <int LC, int CPL>
struct SLanes {
  static constexpr int LK = 32 / LC;       // V phase: lanes across the rows of a tile
  static constexpr int BW = LC * CPL;      // columns per launch at most
};

__host__ __device__ __forceinline__ int al16(int x) { return (x + 15) & ~15; }

// Named barriers: 0 is __syncthreads, then the V warps, all consumers,
// the D groups (one per ring stage) and two votes.
constexpr int kBarV = 1, kBarCons = 2, kBarGroup0 = 3, kBarVote = kBarGroup0 + kSStagesMax, kBarConsVote = kBarVote + 1;
static_assert(kBarConsVote < 16, "16 named barriers per CTA");
__device__ __forceinline__ void bar_v(int nvw) { asm volatile("bar.sync %0, %1;" ::"r"(kBarV), "r"(32 * nvw) : "memory"); }
__device__ __forceinline__ void bar_cons() { asm volatile("bar.sync %0, %1;" ::"r"(kBarCons), "r"(kSThreads) : "memory"); }
// Barrier id of nthreads threads that also returns whether p held on every
// one of them, so that a wait that gave up in one warp stops them all at the
// same point.
__device__ __forceinline__ bool bar_and(int id, bool p, int nthreads) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred pi, po;\n\t"
      "setp.ne.u32 pi, %1, 0;\n\t"
      "bar.red.and.pred po, %2, %3, pi;\n\t"
      "selp.u32 %0, 1, 0, po;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)p), "r"(id), "r"(nthreads)
      : "memory");
  return r != 0;
}
// A bounded mbarrier wait whose outcome is the same on every lane.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, int* err, int code) {
  const bool ok = mbar_wait(bar, parity, err, code);
  return __all_sync(0xffffffffu, ok);
}

// Tiles [t, result) make the next V chunk: consecutive V parts and their X
// rows (when staged) within cap bytes; at least one tile.
__device__ __forceinline__ int next_v_chunk(const StTile* tl, int t, int nt, int cap, int xrow_bytes) {
  const int64_t v0 = tl[t].voff;
  const int x0 = tl[t].row0;
  int t2 = t + 1;
  while (t2 < nt) {
    const int vb = (int)(tl[t2].voff + tl[t2].vbytes - v0);
    const int xb = (tl[t2].row0 + tl[t2].rows - x0) * xrow_bytes;
    if (al16(vb) + xb > cap) break;
    ++t2;
  }
  return t2;
}
// Tiles [t, result) make the next U chunk (consecutive header + U regions).
__device__ __forceinline__ int next_u_chunk(const StTile* tl, int t, int nt, int cap) {
  const int64_t u0 = tl[t].uoff;
  int t2 = t + 1;
  while (t2 < nt && (int)(tl[t2].uoff + tl[t2].ubytes - u0) <= cap) ++t2;
  return t2;
}
// Bulk copy of V chunk [t, t2) (and its X rows) into the V/U area.
template <typename W>
__device__ __forceinline__ void copy_v_chunk(const HandleDev& hd, const StTile* tl, int t, int t2, const W* X, int R,
                                             int xrow_bytes, uint8_t* area, uint64_t* bar) {
  const int64_t v0 = tl[t].voff;
  const int vb = (int)(tl[t2 - 1].voff + tl[t2 - 1].vbytes - v0);
  const int x0 = tl[t].row0;
  const int xb = (tl[t2 - 1].row0 + tl[t2 - 1].rows - x0) * xrow_bytes;
  mbar_arrive_expect_tx(bar, (uint32_t)(vb + xb));
  if (vb) bulk_g2s(area, hd.pool + v0, (uint32_t)vb, bar);
  if (xb) bulk_g2s(area + al16(vb), X + (int64_t)x0 * R, (uint32_t)xb, bar);
}
// Bulk copy of U chunk [t, t2) into the V/U area.
__device__ __forceinline__ void copy_u_chunk(const HandleDev& hd, const StTile* tl, int t, int t2, uint8_t* area,
                                             uint64_t* bar) {
  const int64_t u0 = tl[t].uoff;
  const int ub = (int)(tl[t2 - 1].uoff + tl[t2 - 1].ubytes - u0);
  mbar_arrive_expect_tx(bar, (uint32_t)ub);
  if (ub) bulk_g2s(area, hd.pool + u0, (uint32_t)ub, bar);
}

// B rows of one tile += sum over levels of U_{a_k}[rows, :] Y_{a_k ^ 1}: the
// tile's header and U columns at st (column-major, 32 rows per column),
// lane = row, Y rows broadcast from the CTA's Y area (read BW values wide:
// values past R are never stored).
template <typename W, int BW>
__device__ __forceinline__ void tile_uy(const uint8_t* st, int hbytes, const StLev* lev, int depth, const W* ys_s,
                                        int R, int r, bool xvec, W (&acc)[BW]) {
  for (int k = 1; k <= depth; ++k) {
    const uint2 hw = reinterpret_cast<const uint2*>(st)[k - 1];
    const uint32_t w0 = hw.x, w1 = hw.y;
    const int ru = (int)(w1 & 0xffffu), tier = (int)(w1 >> 16);
    if (ru == 0) continue;
    const W* const yb = ys_s + lev[k - 1].yrow * R;
    auto level = [&](auto tc) {
      constexpr int TIER = decltype(tc)::value;
      constexpr int eb = TIER == HODLR_FP64 ? 8 : TIER == HODLR_FP32 ? 4 : (TIER == HODLR_E4M3 || TIER == HODLR_E5M2) ? 1 : 2;
      const uint8_t* const ucol = st + hbytes + w0 + r * eb;
      if (xvec) {
#pragma unroll 4
        for (int c = 0; c < ru; ++c) {
          const W u = ldf<W, TIER>(ucol + c * kTileRows * eb);
          W yv[BW];
          ld_row<W, BW, true>(yb + c * R, yv);
#pragma unroll
          for (int j = 0; j < BW; ++j) acc[j] = fma(u, yv[j], acc[j]);
        }
      } else {
#pragma unroll 4
        for (int c = 0; c < ru; ++c) {
          const W u = ldf<W, TIER>(ucol + c * kTileRows * eb);
          W yv[BW];
          ld_row<W, BW, false>(yb + c * R, yv);
#pragma unroll
          for (int j = 0; j < BW; ++j) acc[j] = fma(u, yv[j], acc[j]);
        }
      }
    };
    with_format(tier, level);
  }
}

// Unroll factor of a loop whose step holds one BW-wide row of X or Y: as
// many loads in flight as the registers allow.
template <int BW>
__host__ __device__ constexpr int unroll_for() {
  return BW >= 16 ? 1 : BW >= 8 ? 2 : BW >= 4 ? 4 : 8;
}

// The same sum over the U columns of a leaf whose columns share one format:
// the columns in level order (the order of tile_uy), each a byte offset in
// the tile's U region and the row of Y it multiplies.
template <typename W, int BW, int TIER>
__device__ __forceinline__ void uy_flat(const uint8_t* st, const StCol* uc, int nu, const W* ys_s, int R, int r,
                                        bool xvec, W (&acc)[BW]) {
  constexpr int eb = TIER == HODLR_FP64 ? 8 : TIER == HODLR_FP32 ? 4 : (TIER == HODLR_E4M3 || TIER == HODLR_E5M2) ? 1 : 2;
  const uint8_t* const rowp = st + r * eb;
  constexpr int kUnroll = unroll_for<BW>();
  if (xvec) {
#pragma unroll kUnroll
    for (int i = 0; i < nu; ++i) {
      const StCol e = uc[i];
      const W u = ldf<W, TIER>(rowp + e.off);
      W yv[BW];
      ld_row<W, BW, true>(ys_s + e.idx * R, yv);
#pragma unroll
      for (int j = 0; j < BW; ++j) acc[j] = fma(u, yv[j], acc[j]);
    }
  } else {
#pragma unroll kUnroll
    for (int i = 0; i < nu; ++i) {
      const StCol e = uc[i];
      const W u = ldf<W, TIER>(rowp + e.off);
      W yv[BW];
      ld_row<W, BW, false>(ys_s + e.idx * R, yv);
#pragma unroll
      for (int j = 0; j < BW; ++j) acc[j] = fma(u, yv[j], acc[j]);
    }
  }
}
// U Y of one tile of the leaf whose record is at lrec (StLeaf, then its U
// columns): the flat loop when its U columns share one format, else level by
// level.
template <typename W, int BW>
__device__ __forceinline__ void tile_uy_any(const uint8_t* st, const StTile& tq, const uint8_t* lrec,
                                            const StLev* llev, int depth, const W* ys_s, int R, int r, bool xvec,
                                            W (&acc)[BW]) {
  const StLeaf& lh = *reinterpret_cast<const StLeaf*>(lrec);
  if (lh.nu == 0) return;
  if (lh.utier >= 0) {
    const StCol* const uc = reinterpret_cast<const StCol*>(lrec + sizeof(StLeaf));
    with_format(lh.utier, [&](auto tc) { uy_flat<W, BW, decltype(tc)::value>(st, uc, lh.nu, ys_s, R, r, xvec, acc); });
  } else {
    tile_uy<W, BW>(st, tq.hbytes, llev + tq.lleaf * depth, depth, ys_s, R, r, xvec, acc);
  }
}

// B row r of a tile (tile rows only), as 16-byte vectors where aligned
template <typename W, int BW>
__device__ __forceinline__ void store_brow(W* brow, int R, bool xvec, int64_t ldb, const W (&acc)[BW]) {
  if (xvec && ldb % 4 == 0 && (reinterpret_cast<uintptr_t>(brow) & 15) == 0) {
#pragma unroll
    for (int j4 = 0; j4 < BW / 4; ++j4)
      *reinterpret_cast<float4*>(brow + 4 * j4) = make_float4(acc[4 * j4], acc[4 * j4 + 1], acc[4 * j4 + 2], acc[4 * j4 + 3]);
  } else {
#pragma unroll
    for (int j = 0; j < BW; ++j)
      if (j < R) brow[j] = acc[j];
  }
}

template <typename W, int LC, int CPL>
__global__ void __launch_bounds__(kSAll, 1)
stream_kernel(const HandleDev hd, const W* __restrict__ X, int64_t ldx, int R, W* __restrict__ part,
              W* __restrict__ B, int64_t ldb, unsigned long long* sync, unsigned long long sync_base,
              const SPlan pl) {
  using L = SLanes<LC, CPL>;
  constexpr int LK = L::LK, BW = L::BW;
  constexpr int es = sizeof(W);
  constexpr int G16 = 16 / es;             // leaf-block columns per 16-byte chunk
  extern __shared__ __align__(128) uint8_t smem[];
  const int S = pl.nstages, SB = pl.stage_bytes, WPS = pl.wps, NVW = pl.nvw;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + pl.bar_off);
  uint64_t* empty = full + kSStagesMax;
  uint64_t* vfull = empty + kSStagesMax;       // a V chunk has landed in the V/U area
  uint64_t* ufull = vfull + 1;                 // a U chunk has landed in the V/U area
  uint64_t* mfull = ufull + 1;                 // the CTA's record has landed
  int* s_ok = reinterpret_cast<int*>(mfull + 1);   // the grid counter was reached
  const int G = gridDim.x;
  const int depth = hd.depth;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
  uint8_t* const vu = smem + pl.vu_off;
  const int vcap = pl.vu_bytes;
  uint8_t* const meta = smem + pl.meta_off;
  // the CTA's record (StCta and its sections), one bulk copy before anything else
  if (warp == kSWarps && lane == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);   // a stage is released by its group's first warp
    }
    mbar_init(vfull, 1);
    mbar_init(ufull, 1);
    mbar_init(mfull, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_arrive_expect_tx(mfull, (uint32_t)hd.st_blob_stride);
    bulk_g2s(meta, hd.st_blob + (size_t)blockIdx.x * hd.st_blob_stride, (uint32_t)hd.st_blob_stride, mfull);
  }
  __syncthreads();
  {
    const bool ok = mbar_wait(mfull, 0, hd.err, 7);
    if (__syncthreads_or(ok ? 0 : 1)) {
      // a wait gave up: let the copy land (bounded) before the CTA exits
      if (warp == kSWarps && lane == 0) mbar_wait(mfull, 0, hd.err, 7);
      return;
    }
  }
  const StCta& cta = *reinterpret_cast<const StCta*>(meta);
  const StTile* const tiles = reinterpret_cast<const StTile*>(meta + hd.st_off_tile);
  const StLev* const llev = reinterpret_cast<const StLev*>(meta + hd.st_off_lev);
  const int32_t* const accoff = reinterpret_cast<const int32_t*>(meta + hd.st_off_acc);
  const RTask* const tasks = reinterpret_cast<const RTask*>(meta + hd.st_off_task);
  const YItem* const yitems = reinterpret_cast<const YItem*>(meta + hd.st_off_y);
  const uint8_t* const leafs = meta + hd.st_off_leaf;   // per-leaf column records
  const int nt = cta.nt;
  const int xrow_bytes = pl.xstaged ? R * es : 0;
  // the whole V range of this CTA in one chunk when it fits
  const bool v_one = depth > 0 && nt > 0 && al16(cta.vbytes) + cta.xrows * xrow_bytes <= vcap;

  // chunks of the V phase and of the U phase (every role takes the same)
  int nvch = 0, nuch = 0;
  if (depth > 0)
    for (int t = 0; t < nt; ++nvch) t = next_v_chunk(tiles, t, nt, vcap, xrow_bytes);
  if (cta.ubytes > 0)
    for (int t = 0; t < nt; ++nuch) t = next_u_chunk(tiles, t, nt, vcap);

  if (warp == kSWarps) {
    // ================= producer =================
    if (lane != 0) return;
    // the V bytes first (the V phase, the grid counter and the reduction are
    // the launch's critical path), then the leaf blocks through the ring,
    // at most pl.dmax copies in flight: a longer queue of leaf-block bytes
    // adds its drain time to every critical-path access of this SM
    if (v_one) {
      const int xb = cta.xrows * xrow_bytes;
      mbar_arrive_expect_tx(vfull, (uint32_t)(cta.vbytes + xb));
      if (cta.vbytes) bulk_g2s(vu, hd.pool + cta.voff, (uint32_t)cta.vbytes, vfull);
      if (xb) bulk_g2s(vu + al16(cta.vbytes), X + (int64_t)cta.xrow0 * R, (uint32_t)xb, vfull);
    } else if (nvch > 0) {
      copy_v_chunk(hd, tiles, 0, next_v_chunk(tiles, 0, nt, vcap, xrow_bytes), X, R, xrow_bytes, vu, vfull);
    }
    // (a cap of S or more is the ring's own: copy j - S has been consumed,
    // and the phase of an older copy may already have been reused)
    const int DM = max(pl.dmax, 1);
    bool ok = true;
    int j = 0;
    for (; j < nt && ok; ++j) {
      const int s = j % S;
      if (j >= S && !(ok = mbar_wait(&empty[s], ((j / S) - 1) & 1, hd.err, 1))) break;
      if (DM < S && j >= DM && !(ok = mbar_wait(&full[(j - DM) % S], ((j - DM) / S) & 1, hd.err, 1))) break;
      const StTile& q = tiles[j];
      const int db = q.d2bytes, xb = q.m * xrow_bytes;
      uint8_t* st = smem + (size_t)s * SB;
      mbar_arrive_expect_tx(&full[s], (uint32_t)(db + xb));
      bulk_g2s(st, hd.pool + q.d2off, (uint32_t)db, &full[s]);
      if (xb) bulk_g2s(st + db, X + (int64_t)q.xrow0 * R, (uint32_t)xb, &full[s]);
    }
    if (!ok) {
      // a wait gave up: let the copies already issued land before the CTA exits
      for (int q = (j > S ? j - S : 0); q < j; ++q) mbar_wait(&full[q % S], (q / S) & 1, hd.err, 3);
    }
    return;
  }

  W* const acc_s = reinterpret_cast<W*>(smem + pl.acc_off);
  W* const ys_s = reinterpret_cast<W*>(smem + pl.ys_off);
  W* const red_s = reinterpret_cast<W*>(smem + pl.red_off);
  W* const res_s = reinterpret_cast<W*>(smem + pl.res_off);
  W* const uy_s = reinterpret_cast<W*>(smem + pl.uy_off);
  const bool xvec = sizeof(W) == 4 && BW % 4 == 0 && R % 4 == 0;
  bool alive = true;

  if (warp < NVW) {
    // ================= V warps =================
    const int kl = lane / LC, cl = lane - (lane / LC) * LC;   // lane = kl * LC + cl
    if (nvch > 0) {
      // ---- V phase.  Item (k, p) = V columns kVC p .. kVC p + kVC - 1 of the
      //      level-k ancestors, for all tiles in order; lane (kl, cl) sums
      //      rows kl, kl + LK, ... of every tile (V column by column:
      //      consecutive rows across the lanes) for CPL right-hand sides, so a
      //      warp reads kVC V columns and X once per row.  The sums of a node run on in
      //      registers across its tiles; at the node's last tile in a chunk
      //      the lanes are added (fixed butterfly) and the sum goes to the
      //      node's slot (carried in shared memory across V chunks) ----
      constexpr int kVC = CPL >= 4 ? 4 : 8;   // V columns per item (registers: kVC * CPL sums)
      const int passes = (hd.st_max_rank + kVC - 1) / kVC;
      const int nitems = depth * passes;
      int c_idx = 0;
      for (int t = 0; t < nt; ++c_idx) {
        const int t2 = next_v_chunk(tiles, t, nt, vcap, xrow_bytes);
        if (alive) alive = warp_wait(vfull, c_idx & 1, hd.err, 4);
        if (alive) {
          const int64_t v0 = tiles[t].voff;
          const int x0 = tiles[t].row0;
          const W* const xs = reinterpret_cast<const W*>(vu + al16((int)(tiles[t2 - 1].voff + tiles[t2 - 1].vbytes - v0)));
          for (int it = warp; it < nitems; it += NVW) {
            const int k = it / passes + 1, pc = (it - (k - 1) * passes) * kVC;
            const int col = cl * CPL;
            const bool cok = col < R;
            const int kcol = cok ? col : 0;   // lanes past the last column read column 0 and drop it
            W acc[kVC][CPL];
#pragma unroll
            for (int a = 0; a < kVC; ++a)
#pragma unroll
              for (int q = 0; q < CPL; ++q) acc[a][q] = (W)0;
            int ts = t;   // first tile of the current segment
            for (int tt = t; tt < t2; ++tt) {
              const StLev lv = llev[tiles[tt].lleaf * depth + (k - 1)];
              const int rv = (int)lv.rV;
              if (pc < rv) {
                const int rows = tiles[tt].rows, row0 = tiles[tt].row0;
                const uint8_t* const tv = vu + (tiles[tt].voff - v0) + lv.voff;
                const bool staged = xrow_bytes != 0;
                auto run = [&](auto tc) {
                  constexpr int TIER = decltype(tc)::value;
                  constexpr int eb = TIER == HODLR_FP64 ? 8 : TIER == HODLR_FP32 ? 4 : (TIER == HODLR_E4M3 || TIER == HODLR_E5M2) ? 1 : 2;
                  const uint8_t* vc[kVC];   // columns past the rank read the last column (never stored)
#pragma unroll
                  for (int a = 0; a < kVC; ++a) vc[a] = tv + min(pc + a, rv - 1) * kTileRows * eb;
                  if (staged) {
#pragma unroll
                    for (int r = kl; r < kTileRows; r += LK) {
                      // rows past the tile: V is zero there, X is read from its last row
                      const int xr = r < rows ? r : rows - 1;
                      W xv[CPL];
                      ldc<W, CPL>(xs + ((row0 - x0 + xr) * R + kcol), xv);
#pragma unroll
                      for (int a = 0; a < kVC; ++a) {
                        const W v = ldf<W, TIER>(vc[a] + r * eb);
#pragma unroll
                        for (int q = 0; q < CPL; ++q) acc[a][q] = fma(v, xv[q], acc[a][q]);
                      }
                    }
                  } else {
#pragma unroll
                    for (int r = kl; r < kTileRows; r += LK) {
                      const int xr = r < rows ? r : rows - 1;
                      W xv[CPL];
                      load_cols<W, CPL>(X + (int64_t)(row0 + xr) * ldx + kcol, true, xv);
#pragma unroll
                      for (int a = 0; a < kVC; ++a) {
                        const W v = ldf<W, TIER>(vc[a] + r * eb);
#pragma unroll
                        for (int q = 0; q < CPL; ++q) acc[a][q] = fma(v, xv[q], acc[a][q]);
                      }
                    }
                  }
                };
                with_format(lv.tierV, run);
              }
              const int pstage = tt + 1 < t2 ? llev[tiles[tt + 1].lleaf * depth + (k - 1)].pslot : -2;
              if (lv.pslot == pstage) continue;   // the node goes on in the next tile of this chunk
              // end of a segment: add the lanes, join the node's running sum
              // or write the node's slot
              if (pc < rv) {
#pragma unroll
                for (int a = 0; a < kVC; ++a)
#pragma unroll
                  for (int q = 0; q < CPL; ++q) {
#pragma unroll
                    for (int o = LC; o < 32; o <<= 1) acc[a][q] += __shfl_xor_sync(0xffffffffu, acc[a][q], o);
                  }
                const int pprev = ts > 0 ? llev[tiles[ts - 1].lleaf * depth + (k - 1)].pslot : -1;
                const int pnext = tt + 1 < nt ? llev[tiles[tt + 1].lleaf * depth + (k - 1)].pslot : -1;
                if (kl == 0 && cok) {
#pragma unroll
                  for (int a = 0; a < kVC; ++a) {
                    const int c = pc + a;
                    if (c >= rv) break;
                    W* const slot = acc_s + ((accoff[k] + c) * R + col);
                    if (lv.pslot == pprev) {
                      W old[CPL];
                      ldc<W, CPL>(slot, old);
#pragma unroll
                      for (int q = 0; q < CPL; ++q) acc[a][q] = old[q] + acc[a][q];
                    }
                    if (lv.pslot != pnext)
                      store_cols<W, CPL>(part + (int64_t)(lv.pslot + c) * R + col, acc[a]);
                    else
                      stc<W, CPL>(slot, acc[a]);
                  }
                }
              }
#pragma unroll
              for (int a = 0; a < kVC; ++a)
#pragma unroll
                for (int q = 0; q < CPL; ++q) acc[a][q] = (W)0;
              ts = tt + 1;
            }
          }
        }
        bar_v(NVW);   // every V warp is done with the chunk
        t = t2;
        // the next V chunk into the V/U area
        if (tid == 0 && t < nt)
          copy_v_chunk(hd, tiles, t, next_v_chunk(tiles, t, nt, vcap, xrow_bytes), X, R, xrow_bytes, vu, vfull);
      }
    }
    // ---- this CTA's partials are written: arrive at the grid counter (the
    //      barrier orders every V warp's writes before thread 0's fence);
    //      then the first U chunk into the V/U area (after the fence, which
    //      would otherwise wait for the copy) ----
    bar_v(NVW);
    if (tid == 0) {
      __threadfence();
      atomicAdd(sync, 1ull);
      if (nuch > 0) copy_u_chunk(hd, tiles, 0, next_u_chunk(tiles, 0, nt, vcap), vu, ufull);
    }
    // ---- reduction: once every CTA has arrived, the Y this CTA needs.
    //      Tasks of up to kRedSlots slots (one round of loads per lane),
    //      then the tasks of every item added in order ----
    bool red_ok = true;
    if (cta.ny > 0) {
      if (tid == 0) *s_ok = grid_wait(sync, sync_base + (unsigned long long)G, hd.err) ? 1 : 0;
      bar_v(NVW);
      red_ok = *s_ok != 0;
      if (red_ok) {
        // a task takes LPT lanes (several tasks per warp when they are small)
        const int LPT = R == 1 ? 8 : R == 2 ? 16 : 32;
        const int tpw = 32 / LPT, sub = lane / LPT, sl = lane - sub * LPT;
        for (int k0 = warp * tpw; k0 < cta.nk; k0 += NVW * tpw) {
          const int k = k0 + sub;
          if (k >= cta.nk) continue;
          const RTask& tk = tasks[k];
          const YItem& y = yitems[tk.yi];
          const int E = y.rV * R;
          const W* data = part + (int64_t)y.pbase * R;
          W* const out = red_s + tk.srow * R;
          const int nsl = tk.s1 - tk.s0;
          bool vec = false;
          if constexpr (sizeof(W) == 4) vec = R % 4 == 0;
          if (vec) {
            const int E4 = E / 4;
            const float4* d4 = reinterpret_cast<const float4*>(data) + (int64_t)tk.s0 * E4;
            for (int e = sl; e < E4; e += LPT) {
              float4 v[kRedSlots];
#pragma unroll
              for (int q = 0; q < kRedSlots; ++q)
                v[q] = q < nsl ? __ldcg(d4 + (int64_t)q * E4 + e) : make_float4(0.f, 0.f, 0.f, 0.f);
              float4 a = v[0];
#pragma unroll
              for (int q = 1; q < kRedSlots; ++q) {
                a.x += v[q].x;
                a.y += v[q].y;
                a.z += v[q].z;
                a.w += v[q].w;
              }
              reinterpret_cast<float4*>(out)[e] = a;
            }
          } else {
            const W* d = data + (int64_t)tk.s0 * E;
            for (int e = sl; e < E; e += LPT) {
              W v[kRedSlots];
#pragma unroll
              for (int q = 0; q < kRedSlots; ++q) v[q] = q < nsl ? __ldcg(d + (int64_t)q * E + e) : (W)0;
              W a = v[0];
#pragma unroll
              for (int q = 1; q < kRedSlots; ++q) a += v[q];
              out[e] = a;
            }
          }
        }
      }
      bar_v(NVW);
      if (red_ok) {
        for (int i = warp; i < cta.ny; i += NVW) {
          const YItem& y = yitems[i];
          const int E = y.rV * R;
          const W invs = (W)y.invs;
          for (int e = lane; e < E; e += 32) {
            W a = (W)0;
            for (int p = 0; p < y.ntask; ++p) a += red_s[(y.srow + p * y.rV) * R + e];
            const int c = e / R, r = e - c * R;
            ys_s[(y.yrow + c) * R + r] = a * invs;
          }
        }
      }
      bar_v(NVW);   // the Y area is complete
    }
    // ---- U Y of every tile into the shared-memory buffer while the leaf
    //      blocks still stream (warp w takes the chunk's tiles w, w + NVW, ...;
    //      lane = row); the next U chunk is copied once every V warp is done
    //      with the current one ----
    if (pl.uy_smem && nuch > 0) {
      const bool compute = alive && red_ok;
      int uc = 0;
      for (int t = 0; t < nt; ++uc) {
        const int t2 = next_u_chunk(tiles, t, nt, vcap);
        const bool landed = warp_wait(ufull, uc & 1, hd.err, 6);
        if (landed && compute) {
          const int64_t u0 = tiles[t].uoff;
          for (int tt = t + warp; tt < t2; tt += NVW) {
            const StTile& tq = tiles[tt];
            W acc[BW];
#pragma unroll
            for (int j = 0; j < BW; ++j) acc[j] = (W)0;
            tile_uy_any<W, BW>(vu + (tq.uoff - u0), tq, leafs + (size_t)tq.lleaf * hd.st_leaf_stride,
                               llev, depth, ys_s, R, lane, xvec, acc);
#pragma unroll
            for (int j = 0; j < BW; ++j)
              if (j < R) uy_s[(tt * R + j) * kTileRows + lane] = acc[j];
          }
        }
        t = t2;
        // every V warp is done with the chunk; a wait that gave up in any of
        // them ends the stage (no copy is issued over one still in flight)
        if (!bar_and(kBarVote, landed, 32 * NVW)) {
          if (tid == 0) mbar_wait(ufull, uc & 1, hd.err, 6);
          alive = false;
          break;
        }
        if (tid == 0 && t < nt) copy_u_chunk(hd, tiles, t, next_u_chunk(tiles, t, nt, vcap), vu, ufull);
      }
    }
  } else {
    // ================= D warps: D X of every tile =================
    // Group g (g < S) of WPS warps owns ring stage g and takes the tiles t
    // with t mod S = g; lane = row; warp p of the group sums the 16-byte
    // chunks p * nchunk / WPS .. (p + 1) * nchunk / WPS - 1 of the row of D
    // times the broadcast X rows; the helpers' rows go to the group's
    // buffer (two, alternating by tile) and the group's first warp adds
    // them in order and stores the tile's D X.
    const int dw = warp - NVW;
    const int grp = dw / WPS, role = dw - grp * WPS;
    if (grp < S) {
      const int r = lane;
      W* const pbuf = reinterpret_cast<W*>(smem + pl.part_off) + (size_t)grp * 2 * 3 * kTileRows * R;   // WPS <= 4
      for (int tl = grp; tl < nt && alive; tl += S) {
        const bool landed = warp_wait(&full[grp], (tl / S) & 1, hd.err, 4);
        const StTile& tq = tiles[tl];
        const int m = tq.m;
        const uint8_t* const st = smem + (size_t)grp * SB;
        const uint8_t* const dp = st + r * 16;
        const W* const xs = reinterpret_cast<const W*>(st + tq.d2bytes);
        const W* const xg = X + (int64_t)tq.xrow0 * ldx;
        const int nchunk = (m + G16 - 1) / G16;
        const int qa = role * nchunk / WPS, qb = (role + 1) * nchunk / WPS;
        W acc[BW];
#pragma unroll
        for (int j = 0; j < BW; ++j) acc[j] = (W)0;
        // MODE 0: X staged, 16-byte vectors; 1: staged, scalars (rows read
        // BW values wide: values past R are the next row's and are never
        // stored); 2: X from global memory
        auto dx = [&](auto mode_c) {
          constexpr int MODE = decltype(mode_c)::value;
#pragma unroll 4
          for (int q = qa; q < qb; ++q) {
            W d[G16];
            if constexpr (sizeof(W) == 4) {
              const float4 d4 = *reinterpret_cast<const float4*>(dp + q * kTileRows * 16);
              d[0] = d4.x;
              d[1] = d4.y;
              d[2] = d4.z;
              d[3] = d4.w;
            } else {
              const double2 d2 = *reinterpret_cast<const double2*>(dp + q * kTileRows * 16);
              d[0] = d2.x;
              d[1] = d2.y;
            }
            if constexpr (MODE == 0 && BW == 1) {
              // one column: the chunk's X values are one 16-byte vector
              const float4 x4 = *reinterpret_cast<const float4*>(xs + q * G16);
              acc[0] = fma(d[0], (W)x4.x, acc[0]);
              acc[0] = fma(d[1], (W)x4.y, acc[0]);
              acc[0] = fma(d[2], (W)x4.z, acc[0]);
              acc[0] = fma(d[3], (W)x4.w, acc[0]);
            } else {
#pragma unroll
              for (int g = 0; g < G16; ++g) {
                const int k = q * G16 + g;
                W xv[BW];
                if constexpr (MODE == 0) {
                  ld_row<W, BW, true>(xs + k * R, xv);
                } else if constexpr (MODE == 1) {
                  ld_row<W, BW, false>(xs + k * R, xv);
                } else {
#pragma unroll
                  for (int j = 0; j < BW; ++j) xv[j] = (j < R && k < m) ? __ldg(xg + (int64_t)k * ldx + j) : (W)0;
                }
#pragma unroll
                for (int j = 0; j < BW; ++j) acc[j] = fma(d[g], xv[j], acc[j]);
              }
            }
          }
        };
        if (landed) {
          if (xrow_bytes && (xvec || (BW == 1 && sizeof(W) == 4)))
            dx(std::integral_constant<int, 0>{});
          else if (xrow_bytes)
            dx(std::integral_constant<int, 1>{});
          else
            dx(std::integral_constant<int, 2>{});
        }
        if (WPS > 1) {
          W* const pb = pbuf + (size_t)((tl / S) & 1) * 3 * kTileRows * R;
          if (role > 0) {
#pragma unroll
            for (int j = 0; j < BW; ++j)
              if (j < R) pb[((role - 1) * kTileRows + r) * R + j] = acc[j];
          }
          // the group's rows are in the buffer (or a wait gave up in a warp)
          if (!(alive = bar_and(kBarGroup0 + grp, landed, 32 * WPS))) break;
          if (role > 0) continue;
          for (int h = 0; h < WPS - 1; ++h)
#pragma unroll
            for (int j = 0; j < BW; ++j)
              if (j < R) acc[j] += pb[(h * kTileRows + r) * R + j];
        } else if (!(alive = landed)) {
          break;
        }
        // the stage is free (every warp of the group passed the barrier)
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[grp]);
        if (pl.res_smem) {
#pragma unroll
          for (int j = 0; j < BW; ++j)
            if (j < R) res_s[(tl * R + j) * kTileRows + r] = acc[j];
        } else if (r < tq.rows) {
          W* brow = B + (int64_t)(tq.row0 + r) * ldb;
#pragma unroll
          for (int j = 0; j < BW; ++j)
            if (j < R) brow[j] = acc[j];
        }
      }
    }
  }

  bar_cons();   // every D X and every U Y (or every Y) is in place
  const int r = lane;
  if (pl.uy_smem) {
    // ---- final pass: B[rows] = D X + U Y, warp w takes tiles w, w + 16, ... ----
    const bool have_uy = nuch > 0;
    for (int tt = warp; tt < nt; tt += kSWarps) {
      const StTile& tq = tiles[tt];
      W* brow = B + (int64_t)(tq.row0 + min(r, tq.rows - 1)) * ldb;
      W acc[BW];
#pragma unroll
      for (int j = 0; j < BW; ++j)
        acc[j] = j < R ? (pl.res_smem ? res_s[(tt * R + j) * kTileRows + r] : brow[j]) : (W)0;
      if (have_uy) {
#pragma unroll
        for (int j = 0; j < BW; ++j)
          if (j < R) acc[j] += uy_s[(tt * R + j) * kTileRows + r];
      }
      if (r < tq.rows) store_brow<W, BW>(brow, R, xvec, ldb, acc);
    }
    return;
  }
  // ---- U phase without the buffer: for each U chunk (the header and U
  //      rows of consecutive tiles, in the V/U area), warp w takes the
  //      chunk's tiles w, w + 16, ...: B[row] = D X + U Y ----
  int uc = 0;
  for (int t = 0; t < nt; ++uc) {
    const int t2 = nuch > 0 ? next_u_chunk(tiles, t, nt, vcap) : nt;
    bool landed = true;
    if (nuch > 0) landed = warp_wait(ufull, uc & 1, hd.err, 6);
    if (landed && alive) {
      const int64_t u0 = nuch > 0 ? tiles[t].uoff : 0;
      for (int tt = t + warp; tt < t2; tt += kSWarps) {
        const StTile& tq = tiles[tt];
        W* brow = B + (int64_t)(tq.row0 + min(r, tq.rows - 1)) * ldb;
        W acc[BW];
#pragma unroll
        for (int j = 0; j < BW; ++j)
          acc[j] = j < R ? (pl.res_smem ? res_s[(tt * R + j) * kTileRows + r] : brow[j]) : (W)0;
        if (nuch > 0)
          tile_uy_any<W, BW>(vu + (tq.uoff - u0), tq, leafs + (size_t)tq.lleaf * hd.st_leaf_stride,
                             llev, depth, ys_s, R, r, xvec, acc);
        if (r < tq.rows) store_brow<W, BW>(brow, R, xvec, ldb, acc);
      }
    }
    t = t2;
    if (nuch > 0) {
      // every warp is done with the chunk; a wait that gave up in any warp
      // ends the phase (no copy is issued over one still in flight)
      if (!bar_and(kBarConsVote, landed, kSThreads)) {
        if (tid == 0) mbar_wait(ufull, uc & 1, hd.err, 6);
        break;
      }
      if (tid == 0 && t < nt) copy_u_chunk(hd, tiles, t, next_u_chunk(tiles, t, nt, vcap), vu, ufull);
    }
  }
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  }
  return n;
}

// Dynamic shared memory a launch may use: the opt-in limit per block less a
// reserve for the kernel's own static shared memory.
int smem_limit() {
  static int v = 0;
  if (!v) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    v -= 1024;
  }
  return v;
}

// Shared memory of a launch with R columns of es bytes: the leaf-block ring,
// the V/U area, the D X results and the U Y of the CTA's tiles (when they
// fit), the D groups' partial rows, the V running sums carried across V
// chunks, the Y area, the reduction scratch, the barriers and the CTA's
// record.
SPlan make_plan(const HandleDev& hd, int R, int es, bool xstaged) {
  SPlan p;
  memset(&p, 0, sizeof(p));
  p.xstaged = xstaged ? 1 : 0;
  const int xrow = xstaged ? R * es : 0;
  const int sb = (hd.st_max_d2bytes + al16(hd.leaf_m_max * xrow) + 127) / 128 * 128;   // a D2 part, its leaf's X rows
  p.stage_bytes = sb;
  // V/U area: the largest CTA's V range with its X rows, or its U regions,
  // at least one tile's worth of either
  int vu = std::max(al16(hd.st_max_cta_v) + hd.st_max_cta_xrows * xrow, hd.st_max_cta_u);
  const int vu_min = std::max(al16(hd.st_max_vbytes) + kTileRows * xrow, hd.st_max_ubytes);
  const int res_b = al16(hd.st_max_tiles * kTileRows * R * es);
  const int acc_b = al16(std::max(hd.st_acc_rows, 1) * R * es);
  const int ys_b = al16(std::max(hd.st_y_rows, 1) * R * es);
  const int red_b = al16(std::max(hd.st_red_rows, 1) * R * es);
  const int bar_b = (2 * kSStagesMax + 3) * 8 + 16;   // the barriers and the grid-counter flag
  const int meta_b = al16(hd.st_blob_stride);
  const int part_stage = 2 * 3 * kTileRows * R * es;   // up to three helpers, two buffers (four warps)
  // eight V warps (V phase, reduction, U Y: the critical path), eight D warps
  p.nvw = 8;
  const int ndw = kSWarps - p.nvw;
  const int fixed0 = acc_b + ys_b + red_b + bar_b + meta_b;
  const int room = smem_limit() - fixed0;
  // the V/U area takes what three stages leave, down to one tile's worth;
  // the D X results, then the U Y, stay in shared memory if two stages
  // still fit beside them
  vu = std::max(vu_min, std::min(vu, room - 3 * (sb + part_stage)));
  vu = al16(vu);
  p.res_smem = room - vu - res_b >= 2 * (sb + part_stage) ? 1 : 0;
  p.uy_smem = p.res_smem && room - vu - 2 * res_b >= 2 * (sb + part_stage) ? 1 : 0;
  const int room2 = room - vu - (p.res_smem ? res_b : 0) - (p.uy_smem ? res_b : 0);
  p.nstages = std::min(kSStagesMax, room2 / (sb + part_stage));
  p.wps = std::max(1, std::min(4, ndw / std::max(p.nstages, 1)));
  p.dmax = kSInflight;
  p.vu_bytes = vu;
  const int ring = std::max(p.nstages, 0) * sb;
  p.vu_off = ring;
  p.res_off = al16(p.vu_off + vu);
  p.uy_off = al16(p.res_off + (p.res_smem ? res_b : 0));
  p.part_off = al16(p.uy_off + (p.uy_smem ? res_b : 0));
  p.acc_off = al16(p.part_off + std::max(p.nstages, 0) * part_stage);
  p.ys_off = p.acc_off + acc_b;
  p.red_off = p.ys_off + ys_b;
  p.bar_off = p.red_off + red_b;
  p.meta_off = al16(p.bar_off + bar_b);
  p.smem = p.meta_off + meta_b;
  return p;
}

template <typename W, int LC, int CPL>
cudaError_t launch_s(const HandleDev& hd, int nrhs, const W* X, int64_t ldx, W* B, int64_t ldb, W* part,
                     unsigned long long* sync, unsigned long long sync_base, cudaStream_t s, cudaEvent_t* ev) {
  const int es = sizeof(W);
  const bool xstaged = hd.x_aligned && ldx == nrhs && ((uintptr_t)X % 16) == 0 &&
                       (int64_t)hd.leaf_m_max * nrhs * es <= kSXMax;
  const SPlan pl = make_plan(hd, nrhs, es, xstaged);
  // two ring stages at least (the host sizes batches so that they fit)
  if (pl.nstages < 2 || pl.smem > smem_limit()) return cudaErrorInvalidConfiguration;
  static int smem_set = 0;   // per instantiation: largest size opted in so far
  if (pl.smem > smem_set) {
    cudaError_t e = cudaFuncSetAttribute(stream_kernel<W, LC, CPL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         pl.smem);
    if (e != cudaSuccess) return e;
    smem_set = pl.smem;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(hd.st_grid);
  cfg.blockDim = dim3(kSAll);
  cfg.dynamicSmemBytes = pl.smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (ev) cudaEventRecord(ev[0], s);
  cudaError_t e = cudaLaunchKernelEx(&cfg, stream_kernel<W, LC, CPL>, hd, X, ldx, nrhs, part, B, ldb, sync,
                                     sync_base, pl);
  if (e != cudaSuccess) return e;
  if (ev) {
    cudaEventRecord(ev[1], s);
    cudaEventRecord(ev[2], s);
  }
  return cudaGetLastError();
}

// Lane layout for nrhs <= 16 columns: LC = the smallest power of two >=
// nrhs, one column per lane; four columns per lane (on two or four lanes)
// for 8 or 16 fp32 columns whose rows start on 16-byte boundaries.
template <typename W>
cudaError_t launch_sw(const HandleDev& hd, int nrhs, const W* X, int64_t ldx, W* B, int64_t ldb, W* part,
                      unsigned long long* sync, unsigned long long base, cudaStream_t s, cudaEvent_t* ev) {
#define HODLR_SLAUNCH(LC, CPL) launch_s<W, LC, CPL>(hd, nrhs, X, ldx, B, ldb, part, sync, base, s, ev)
  if (nrhs == 1) return HODLR_SLAUNCH(1, 1);
  if (nrhs == 2) return HODLR_SLAUNCH(2, 1);
  if (nrhs <= 4) return HODLR_SLAUNCH(4, 1);
  if constexpr (sizeof(W) == 4) {
    const bool quads = nrhs % 4 == 0 && ldx % 4 == 0 && ldb % 4 == 0 && (uintptr_t)X % 16 == 0 &&
                       (uintptr_t)B % 16 == 0;
    if (quads && nrhs <= 8) return HODLR_SLAUNCH(2, 4);
    if (quads) return HODLR_SLAUNCH(4, 4);
  }
  if (nrhs <= 8) return HODLR_SLAUNCH(8, 1);
  return HODLR_SLAUNCH(16, 1);
#undef HODLR_SLAUNCH
}

}  // namespace

unsigned long long stream_sync_step(const HandleDev& hd) { return (unsigned long long)hd.st_grid; }

int stream_max_batch(const HandleDev& hd, int work) {
  const int es = prec_bytes(work);
  for (int R = kStreamMaxCols; R >= 1; --R)
    if (make_plan(hd, R, es, true).nstages >= 2 && make_plan(hd, R, es, false).nstages >= 2) return R;
  return 0;
}

cudaError_t launch_stream(const HandleDev& hd, int work, int nrhs, const void* X, int64_t ldx, void* B,
                          int64_t ldb, void* partials, unsigned long long* sync, unsigned long long sync_base,
                          cudaStream_t s, cudaEvent_t* ev) {
  if (hd.st_grid != sm_count()) return cudaErrorInvalidConfiguration;   // planned for another device
  if (work == HODLR_FP64)
    return launch_sw<double>(hd, nrhs, (const double*)X, ldx, (double*)B, ldb, (double*)partials, sync, sync_base,
                             s, ev);
  return launch_sw<float>(hd, nrhs, (const float*)X, ldx, (float*)B, ldb, (float*)partials, sync, sync_base, s,
                          ev);
}

}  // namespace hodlr
