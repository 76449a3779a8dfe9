// HODLR_MATVEC (Algorithm 3.3) on sm_103a CUDA cores.
//
// Algorithm 3.3 walks the levels and adds U_{2i-1}(V_{2i}^T x_{2i}) and
// U_{2i}(V_{2i-1}^T x_{2i-1}) into b, then the leaf products D_i x_i.  Here
// the level loop is flattened into two data-parallel kernels:
//
//  phase 1  Y_j = V_j^T X[I_j] for every node j of every level: one work item
//           per node and group of leaves (up to 4096 rows); partial sums per
//           item, and the last item of a node to finish adds the partials in
//           item order, so the result does not depend on scheduling;
//  phase 2  for every 32-row tile of a leaf i:
//           B[rows] = D_i X[I_i] + sum_k U_{a_k}[rows] Y_{a_k ^ 1}
//           where a_k is the level-k ancestor of leaf i; each output row is
//           written once, by one CTA, with a fixed summation order.
//
// Phase 2 is launched with programmatic dependent launch: its CTAs start
// while phase 1 runs, stream their leaf block D_i (the bulk of the bytes)
// and only then wait for phase 1 (griddepcontrol.wait) before reading Y.
// Phase 1 releases its dependents as soon as it starts.
//
// Both kernels stream their factor bytes once (V in phase 1, U and D in
// phase 2).  Threads run along rows: a thread owns 4 consecutive rows and
// loads the 4 entries of a generator column (16 bytes in fp32) at a time,
// converting the block's storage format to the working precision on the fly.
#include "hodlr_internal.cuh"

namespace hodlr {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kRankTile = 8;
constexpr int kP2Lanes = kP2Rows / 4;              // threads per 4-row column segment
constexpr int kP2Groups = kThreads / kP2Lanes;     // reduction groups over the columns

template <typename W> struct WorkPrec;
template <> struct WorkPrec<float> { static constexpr int value = HODLR_FP32; };
template <> struct WorkPrec<double> { static constexpr int value = HODLR_FP64; };

__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename W>
__device__ __forceinline__ W warp_sum(W v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Dynamic shared memory of phase 2: the rank-column tables first (8-byte
// aligned), then the working-precision arrays from a 16-byte boundary.
__host__ __device__ inline size_t phase2_w_offset(int sum_r_max) {
  return ((size_t)sum_r_max * (sizeof(int64_t) + sizeof(int)) + 15) / 16 * 16;
}

template <typename W, int CT>
size_t phase2_smem_bytes(const HandleDev& hd) {
  return phase2_w_offset(hd.sum_r_max) +
         ((size_t)hd.leaf_pm_max * CT + (size_t)hd.sum_r_max * CT + (size_t)kWarps * kP2Rows * CT) *
             sizeof(W);
}

// ---- phase 1: Y = V^T X ----------------------------------------------------
template <typename W, int CT>
__global__ void __launch_bounds__(kThreads)
phase1_kernel(const HandleDev hd, const W* __restrict__ X, int64_t ldx, int R,
              W* __restrict__ Y, W* __restrict__ partials, unsigned* __restrict__ counters) {
  pdl_launch_dependents();
  __shared__ W s_red[kWarps][kRankTile * CT];
  __shared__ int s_pref[kP1MaxLeaves + 1];   // prefix sums of 4-row groups per leaf
  __shared__ int s_last;
  const P1Item it = hd.p1[blockIdx.x];
  const NodeDev nd = hd.nodes[it.node];
  const int rV = nd.rV;
  const int eb = prec_bytes(nd.tierV);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    int t = 0;
    for (int q = 0; q < it.nleaf; ++q) {
      s_pref[q] = t;
      t += hd.leaves[it.leaf0 + q].pm / 4;
    }
    s_pref[it.nleaf] = t;
  }
  __syncthreads();
  const int ngroups = s_pref[it.nleaf];

  for (int c0 = 0; c0 < R; c0 += CT) {
    const int nc = min(CT, R - c0);
    for (int r0 = 0; r0 < rV; r0 += kRankTile) {
      const int nr = min(kRankTile, rV - r0);
      W acc[kRankTile][CT];
#pragma unroll
      for (int c = 0; c < kRankTile; ++c)
#pragma unroll
        for (int j = 0; j < CT; ++j) acc[c][j] = (W)0;

      int li = 0;
      for (int gq = threadIdx.x; gq < ngroups; gq += kThreads) {
        while (gq >= s_pref[li + 1]) ++li;           // groups are visited in increasing order
        const LeafDev lf = hd.leaves[it.leaf0 + li];
        const int p = 4 * (gq - s_pref[li]);          // padded row within the leaf
        W xv[4][CT];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const bool ok = p + q < lf.m;
          const W* xr = X + (int64_t)(lf.row0 + p + q) * ldx + c0;
#pragma unroll
          for (int j = 0; j < CT; ++j) xv[q][j] = (ok && j < nc) ? xr[j] : (W)0;
        }
        const uint8_t* vb = hd.pool + nd.offV + ((int64_t)r0 * nd.pm + (lf.prow0 - nd.prow0) + p) * eb;
        Vec4<W> v[kRankTile];
#pragma unroll
        for (int c = 0; c < kRankTile; ++c)
          if (c < nr) v[c] = load4<W>(vb + (int64_t)c * nd.pm * eb, nd.tierV);
#pragma unroll
        for (int c = 0; c < kRankTile; ++c) {
          if (c < nr) {
#pragma unroll
            for (int j = 0; j < CT; ++j) {
              W a = acc[c][j];
              a = fma(v[c].x, xv[0][j], a);
              a = fma(v[c].y, xv[1][j], a);
              a = fma(v[c].z, xv[2][j], a);
              a = fma(v[c].w, xv[3][j], a);
              acc[c][j] = a;
            }
          }
        }
      }
      // CTA reduction: warps, then the warp partials in warp order.
#pragma unroll
      for (int c = 0; c < kRankTile; ++c) {
        if (c < nr) {
#pragma unroll
          for (int j = 0; j < CT; ++j) {
            W v = warp_sum(acc[c][j]);
            if (lane == 0) s_red[warp][c * CT + j] = v;
          }
        }
      }
      __syncthreads();
      if (threadIdx.x < nr * CT) {
        const int c = threadIdx.x / CT, j = threadIdx.x % CT;
        W s = (W)0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) s += s_red[w][threadIdx.x];
        if (j < nc) partials[(int64_t)(it.poff + r0 + c) * R + c0 + j] = s;
      }
      __syncthreads();
    }
  }

  // The last item of the node to finish adds the node's partials in item
  // order (classic threadfence reduction; nothing waits on anything).
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(&counters[it.node], 1u);
    s_last = prev == (unsigned)(it.nitems - 1);
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    const int first = blockIdx.x - it.item_in_node;
    const W invs = (W)nd.invsV;
    for (int e = threadIdx.x; e < rV * R; e += kThreads) {
      const int c = e / R, j = e - c * R;
      W s = (W)0;
      for (int q = 0; q < it.nitems; ++q) {
        const int poff = hd.p1[first + q].poff;
        s += __ldcg(partials + (int64_t)(poff + c) * R + j);
      }
      Y[(int64_t)(nd.yoff + c) * R + j] = s * invs;
    }
    if (threadIdx.x == 0) counters[it.node] = 0u;
  }
}

// ---- phase 2: B = D X + sum_k U Y ------------------------------------------
template <typename W, int CT>
__global__ void __launch_bounds__(kThreads)
phase2_kernel(const HandleDev hd, const W* __restrict__ X, int64_t ldx, int R,
              const W* __restrict__ Y, W* __restrict__ B, int64_t ldb) {
  extern __shared__ __align__(16) uint8_t smem[];
  int64_t* qoff = reinterpret_cast<int64_t*>(smem);                // [sum_r_max]
  int* qprec = reinterpret_cast<int*>(qoff + hd.sum_r_max);        // [sum_r_max]
  W* Zx = reinterpret_cast<W*>(smem + phase2_w_offset(hd.sum_r_max));  // [leaf_pm_max][CT]
  W* Zy = Zx + (size_t)hd.leaf_pm_max * CT;                        // [sum_r_max][CT]
  W* red = Zy + (size_t)hd.sum_r_max * CT;                         // [kWarps][kP2Rows][CT]
  __shared__ int s_anc[HODLR_MAX_DEPTH + 1];
  __shared__ int s_q0[HODLR_MAX_DEPTH + 2];

  constexpr int wprec = WorkPrec<W>::value;
  constexpr int ebw = sizeof(W);
  const P2Item it = hd.p2[blockIdx.x];
  const LeafDev lf = hd.leaves[it.leaf];
  const int g = threadIdx.x / kP2Lanes, l = threadIdx.x % kP2Lanes;
  const int rowbase = it.t0 + 4 * l;                  // leaf-local first row of this thread
  const bool active = rowbase < lf.pm;
  const int depth = hd.depth;

  if (threadIdx.x == 0) {
    int q = 0;
    for (int k = 1; k <= depth; ++k) {
      const int a = node_index(k, it.leaf >> (depth - k));
      s_anc[k] = a;
      s_q0[k] = q;
      q += hd.nodes[a].rU;
    }
    s_q0[depth + 1] = q;
  }
  __syncthreads();
  const int totq = s_q0[depth + 1];
  // per rank column: byte offset of (tile row 0) in U's column, and its format
  for (int k = 1; k <= depth; ++k) {
    const NodeDev a = hd.nodes[s_anc[k]];
    const int eb = prec_bytes(a.tierU);
    const int64_t base = a.offU + (int64_t)(lf.prow0 - a.prow0 + it.t0) * eb;
    for (int c = threadIdx.x; c < a.rU; c += kThreads) {
      qoff[s_q0[k] + c] = base + (int64_t)c * a.pm * eb;
      qprec[s_q0[k] + c] = a.tierU;
    }
  }

  for (int c0 = 0; c0 < R; c0 += CT) {
    const int nc = min(CT, R - c0);
    for (int e = threadIdx.x; e < lf.m * CT; e += kThreads) {
      const int j = e / CT, jj = e - j * CT;
      Zx[e] = jj < nc ? X[(int64_t)(lf.row0 + j) * ldx + c0 + jj] : (W)0;
    }
    __syncthreads();

    W acc[4][CT];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int j = 0; j < CT; ++j) acc[q][j] = (W)0;

    // leaf block: does not depend on phase 1
    if (active) {
      const uint8_t* db = hd.pool + lf.offD + (int64_t)rowbase * ebw;
      const int64_t colstride = (int64_t)lf.pm * ebw;
      constexpr int kBatch = 8;
      for (int j0 = g; j0 < lf.m; j0 += kBatch * kP2Groups) {
        Vec4<W> d[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
          const int j = j0 + u * kP2Groups;
          if (j < lf.m) d[u] = load4<W>(db + (int64_t)j * colstride, wprec);
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
          const int j = j0 + u * kP2Groups;
          if (j < lf.m) {
            const W* z = Zx + j * CT;
#pragma unroll
            for (int jj = 0; jj < CT; ++jj) {
              const W zz = z[jj];
              acc[0][jj] = fma(d[u].x, zz, acc[0][jj]);
              acc[1][jj] = fma(d[u].y, zz, acc[1][jj]);
              acc[2][jj] = fma(d[u].z, zz, acc[2][jj]);
              acc[3][jj] = fma(d[u].w, zz, acc[3][jj]);
            }
          }
        }
      }
    }

    // Y comes from phase 1
    pdl_wait();
    for (int k = 1; k <= depth; ++k) {
      const int a = s_anc[k];
      const int ia = it.leaf >> (depth - k);
      const int sib = node_index(k, ia ^ 1);
      const NodeDev na = hd.nodes[a];
      const int yo = hd.nodes[sib].yoff;
      const W invs = (W)na.invsU;
      for (int e = threadIdx.x; e < na.rU * CT; e += kThreads) {
        const int c = e / CT, jj = e - c * CT;
        Zy[(s_q0[k] + c) * CT + jj] = jj < nc ? Y[(int64_t)(yo + c) * R + c0 + jj] * invs : (W)0;
      }
    }
    __syncthreads();

    if (active) {
      for (int q = g; q < totq; q += kP2Groups) {
        const int p = qprec[q];
        const Vec4<W> u = load4<W>(hd.pool + qoff[q] + (int64_t)4 * l * prec_bytes(p), p);
        const W* z = Zy + q * CT;
#pragma unroll
        for (int jj = 0; jj < CT; ++jj) {
          const W zz = z[jj];
          acc[0][jj] = fma(u.x, zz, acc[0][jj]);
          acc[1][jj] = fma(u.y, zz, acc[1][jj]);
          acc[2][jj] = fma(u.z, zz, acc[2][jj]);
          acc[3][jj] = fma(u.w, zz, acc[3][jj]);
        }
      }
    }
    // the 4 groups of a warp (lane bits 3 and 4) first, then the warps in order
    const int warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int jj = 0; jj < CT; ++jj) {
        W v = acc[q][jj];
        v += __shfl_xor_sync(0xffffffffu, v, 8);
        v += __shfl_xor_sync(0xffffffffu, v, 16);
        if ((threadIdx.x & 31) < kP2Lanes) red[((size_t)warp * kP2Rows + 4 * l + q) * CT + jj] = v;
      }
    __syncthreads();
    for (int e = threadIdx.x; e < kP2Rows * CT; e += kThreads) {
      const int row = e / CT, jj = e - row * CT;
      W s = (W)0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) s += red[(size_t)w * kP2Rows * CT + e];
      if (it.t0 + row < lf.m && jj < nc) B[(int64_t)(lf.row0 + it.t0 + row) * ldb + c0 + jj] = s;
    }
    __syncthreads();
  }
}

template <typename W, int CT>
cudaError_t launch_ct(const HandleDev& hd, int nrhs, const W* X, int64_t ldx, W* B, int64_t ldb,
                      W* Y, W* partials, unsigned* counters, cudaStream_t s, cudaEvent_t* ev) {
  if (ev) cudaEventRecord(ev[0], s);
  if (hd.n_p1 > 0) {
    phase1_kernel<W, CT><<<hd.n_p1, kThreads, 0, s>>>(hd, X, ldx, nrhs, Y, partials, counters);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (ev) cudaEventRecord(ev[1], s);
  const size_t smem = phase2_smem_bytes<W, CT>(hd);
  static size_t smem_set = 48 * 1024;   // per instantiation: largest size opted in so far
  if (smem > smem_set) {
    cudaError_t e = cudaFuncSetAttribute(phase2_kernel<W, CT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    smem_set = smem;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(hd.n_p2);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = (hd.n_p1 > 0 && !ev) ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, phase2_kernel<W, CT>, hd, X, ldx, nrhs, (const W*)Y, B, ldb);
  if (e != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[2], s);
  return cudaGetLastError();
}

template <typename W>
cudaError_t launch_w(const HandleDev& hd, int nrhs, const W* X, int64_t ldx, W* B, int64_t ldb,
                     W* Y, W* partials, unsigned* counters, cudaStream_t s, cudaEvent_t* ev) {
  if (nrhs == 1) return launch_ct<W, 1>(hd, nrhs, X, ldx, B, ldb, Y, partials, counters, s, ev);
  if (nrhs == 2) return launch_ct<W, 2>(hd, nrhs, X, ldx, B, ldb, Y, partials, counters, s, ev);
  if (nrhs <= 4) return launch_ct<W, 4>(hd, nrhs, X, ldx, B, ldb, Y, partials, counters, s, ev);
  return launch_ct<W, 8>(hd, nrhs, X, ldx, B, ldb, Y, partials, counters, s, ev);
}

}  // namespace

cudaError_t launch_matvec(const HandleDev& hd, int work, int nrhs, const void* X, int64_t ldx,
                          void* B, int64_t ldb, void* Y, void* partials, unsigned* counters,
                          cudaStream_t s, cudaEvent_t* ev) {
  if (work == HODLR_FP64)
    return launch_w<double>(hd, nrhs, (const double*)X, ldx, (double*)B, ldb, (double*)Y,
                            (double*)partials, counters, s, ev);
  return launch_w<float>(hd, nrhs, (const float*)X, ldx, (float*)B, ldb, (float*)Y,
                         (float*)partials, counters, s, ev);
}

}  // namespace hodlr
