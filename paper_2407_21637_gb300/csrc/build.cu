// GPU construction of the adaptive-precision HODLR format (Algorithm 3.2)
// for kernel matrices whose entries are generated in registers.
//
// Per off-diagonal block A_b = H(I_i, I_{i^1}) (all blocks of all levels are
// independent in HODLR, so they are processed together):
//
//  1. sketch      Y = A_b Omega (m x s), Omega Gaussian; ||A_b||_F^2 in the
//                 same pass (Algorithm 3.2 needs the block norms of H);
//  2. Q = orth(Y) by classical Gram-Schmidt with one re-orthogonalisation
//     per column (CGS2), which stays orthonormal when Y is rank deficient;
//  3. Bt = A_b^T Q (mc x s), the second generated product;
//  4. resid = ||A_b - Q Q^T A_b||_F^2, computed directly from regenerated
//     entries (no cancellation);
//  5. Bt = Q2 R2 (CGS2 again), SVD of R2^T = W S Z^T by one-sided Jacobi;
//     A_b ~ (Q W) S (Q2 Z)^T;
//  6. rank r = the smallest with sum_{j>=r} s_j^2 + resid <= eps^2 ||A_b||_F^2
//     (Def. 2.3 in the Frobenius norm: the sketch residual and the SVD tail
//     are orthogonal); if the sketch residual alone uses more than a quarter
//     of the budget, the block is redone with twice the sketch size;
//  7. U = Q W_r (orthonormal columns, eq. (3.1)), V = Q2 Z_r S_r.
//
// The generators then go through the same precision rule and packing as
// hodlr_import, with the exact block norms of H.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <string>
#include <memory>
#include <vector>

#include "handle.cuh"

namespace hodlr {

namespace {

constexpr int kBT = 256;     // threads per CTA
constexpr int kSmax = 64;    // largest sketch
constexpr int kRT = 64;      // rows per tile
constexpr int kJC = 32;      // reduction chunk of the generated products
constexpr int kMat = kSmax * kSmax;
constexpr int kJacobiSweeps = 40;

struct KDesc {
  const double* pts;
  int n, dim, kind;
  double c, len2, diag;
};

__device__ __forceinline__ double kval(const KDesc& K, int i, int j) {
  return kernel_entry(K.pts, K.dim, i, j, K.kind, K.c, K.len2, K.diag);
}

struct BBlock {
  int32_t r0, m, c0, mc;   // rows I_i and columns I_{i^1}
  int32_t s;               // sketch columns
  int32_t q;               // node index of block (k, i)
  int64_t yoff;            // Y / Q: m x s, row-major, in the Y buffer
  int64_t boff;            // Bt / Q2: mc x s, row-major, in the B buffer
  int64_t moff;            // 6 s x s slots (stride kMat) in the matrix buffer
  int32_t rank, retry;
  double norm2, resid2;
  int64_t uoff, voff;      // staging offsets of U_i and V_{i^1} (final pass)
  int32_t item0y, nitemy;  // tile items over the m rows
  int32_t item0b, nitemb;  // tile items over the mc rows
  int32_t gram0y, ngramy;  // gram items over the m rows
  int32_t gram0b, ngramb;  // gram items over the mc rows
};

enum Slot { kG = 0, kRinv = 1, kRacc = 2, kW = 3, kZS = 4, kTmp = 5 };

struct TItem { int32_t blk, row0; };

// ---- Gaussian Omega: counter-based (splitmix64 hash) + Box-Muller --------
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

__global__ void omega_kernel(double* __restrict__ om, int64_t count, uint64_t seed) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t a = mix64(seed ^ (2 * (uint64_t)i)), b = mix64(seed ^ (2 * (uint64_t)i + 1));
    const double u1 = ((a >> 11) + 1) * 0x1.0p-53;  // (0, 1]
    const double u2 = (b >> 11) * 0x1.0p-53;        // [0, 1)
    om[i] = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
  }
}

// ---- generated products -----------------------------------------------------
// mode 0: Y[r][c]  = sum_{j < mc} A(r0 + r, c0 + j) * Om[(c0 + j) * ldo + c]   (+ ||A||^2)
// mode 1: Bt[r][c] = sum_{j < m}  A(r0 + j, c0 + r) * Q[j * s + c]
template <int MODE>
__global__ void __launch_bounds__(kBT)
gen_product_kernel(const KDesc K, const BBlock* __restrict__ blocks, const TItem* __restrict__ items,
                   const double* __restrict__ in, int64_t ldo, double* __restrict__ out,
                   double* __restrict__ norm_part) {
  __shared__ __align__(16) double As[kJC][kRT + 2];
  __shared__ __align__(16) double Is[kJC][kSmax];
  __shared__ double s_red[kBT / 32];
  const TItem it = items[blockIdx.x];
  const BBlock b = blocks[it.blk];
  const int s = b.s;
  const int nrows = MODE == 0 ? b.m : b.mc;     // output rows
  const int J = MODE == 0 ? b.mc : b.m;         // reduction length
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  double acc[4][4] = {};
  double nrm = 0.0;
  for (int j0 = 0; j0 < J; j0 += kJC) {
    for (int e = threadIdx.x; e < kRT * kJC; e += kBT) {
      const int r = e % kRT, j = e / kRT;
      const int rr = it.row0 + r, jj = j0 + j;
      double a = 0.0;
      if (rr < nrows && jj < J) {
        a = MODE == 0 ? kval(K, b.r0 + rr, b.c0 + jj) : kval(K, b.r0 + jj, b.c0 + rr);
        if (MODE == 0) nrm = fma(a, a, nrm);
      }
      As[j][r] = a;
    }
    for (int e = threadIdx.x; e < kJC * kSmax; e += kBT) {
      const int c = e % kSmax, j = e / kSmax;
      const int jj = j0 + j;
      double v = 0.0;
      if (c < s && jj < J)
        v = MODE == 0 ? in[(int64_t)(b.c0 + jj) * ldo + c] : in[b.yoff + (int64_t)jj * s + c];
      Is[j][c] = v;
    }
    __syncthreads();
#pragma unroll 8
    for (int j = 0; j < kJC; ++j) {
      double a[4], x[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { a[q] = As[j][4 * ty + q]; x[q] = Is[j][4 * tx + q]; }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], x[q], acc[p][q]);
    }
    __syncthreads();
  }
  double* o = out + (MODE == 0 ? b.yoff : b.boff);
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int r = it.row0 + 4 * ty + p;
    if (r >= nrows) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = 4 * tx + q;
      if (c < s) o[(int64_t)r * s + c] = acc[p][q];
    }
  }
  if (MODE == 0) {
    for (int off = 16; off > 0; off >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, off);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = nrm;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < kBT / 32; ++w) t += s_red[w];
      norm_part[blockIdx.x] = t;
    }
  }
}

// ||A_b - Q Bt^T||_F^2 over the rows of one tile (Bt = A_b^T Q before its QR).
constexpr int kRC = 16;  // residual column chunk
__global__ void __launch_bounds__(kBT)
resid_kernel(const KDesc K, const BBlock* __restrict__ blocks, const TItem* __restrict__ items,
             const double* __restrict__ Qbuf, const double* __restrict__ Bbuf,
             double* __restrict__ part) {
  __shared__ double Qs[kRT][kSmax + 1];
  __shared__ double Bs[kRC][kSmax + 1];
  __shared__ double s_red[kBT / 32];
  const TItem it = items[blockIdx.x];
  const BBlock b = blocks[it.blk];
  const int s = b.s;
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;   // rows 4ty..4ty+3, column tx
  for (int e = threadIdx.x; e < kRT * kSmax; e += kBT) {
    const int r = e / kSmax, c = e % kSmax;
    const int rr = it.row0 + r;
    Qs[r][c] = (rr < b.m && c < s) ? Qbuf[b.yoff + (int64_t)rr * s + c] : 0.0;
  }
  double sum = 0.0;
  for (int j0 = 0; j0 < b.mc; j0 += kRC) {
    __syncthreads();
    for (int e = threadIdx.x; e < kRC * kSmax; e += kBT) {
      const int j = e / kSmax, c = e % kSmax;
      const int jj = j0 + j;
      Bs[j][c] = (jj < b.mc && c < s) ? Bbuf[b.boff + (int64_t)jj * s + c] : 0.0;
    }
    __syncthreads();
    const int jj = j0 + tx;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int r = 4 * ty + p, rr = it.row0 + r;
      if (rr < b.m && jj < b.mc) {
        double qb = 0.0;
        for (int c = 0; c < s; ++c) qb = fma(Qs[r][c], Bs[tx][c], qb);
        const double d = kval(K, b.r0 + rr, b.c0 + jj) - qb;
        sum = fma(d, d, sum);
      }
    }
  }
  for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kBT / 32; ++w) t += s_red[w];
    part[blockIdx.x] = t;
  }
}

// Per-block sums of item partials, in item order (deterministic).
__global__ void reduce_parts_kernel(BBlock* __restrict__ blocks, int nblk, const double* __restrict__ part,
                                    int which) {
  const int bi = blockIdx.x * blockDim.x + threadIdx.x;
  if (bi >= nblk) return;
  BBlock& b = blocks[bi];
  double t = 0.0;
  for (int q = 0; q < b.nitemy; ++q) t += part[b.item0y + q];
  if (which == 0) b.norm2 = t; else b.resid2 = t;
}

// ---- CGS2 orthonormalisation, one column j at a time, all blocks at once ----
// Panel items cover up to kPanelRows rows of one block side.  For column j:
//   dot     part[item][c] = sum_{rows} X[r][c] X[r][j]      (c < j)
//   update  coef = sum of the block's partials in item order; X[:, j] -= X[:, :j] coef;
//           R[:j, j] (+)= coef (first item only); ||X[:, j]||^2 partial per item
//   (dot, update) twice, then
//   norm    X[:, j] /= ||X[:, j]||; R[j][j] = ||X[:, j]||.
// A column whose remainder after the two projections is below 1e-12 of its
// original length lies in the span of the previous columns to working
// accuracy: it is set to zero (R[j][j] = 0) instead of normalising rounding
// noise, which two passes cannot orthogonalise.  Zero columns of Q are
// harmless for the range finder (the matching rows of Q^T A vanish).
// Blocks with j >= s skip.  All sums have a fixed order: deterministic.
constexpr int kPanelRows = 2048;

__global__ void __launch_bounds__(kBT)
cgs_dot_kernel(const BBlock* __restrict__ blocks, const TItem* __restrict__ items, int side, int j,
               const double* __restrict__ buf, double* __restrict__ part) {
  __shared__ double red[kBT / kSmax][kSmax];
  const TItem it = items[blockIdx.x];
  const BBlock b = blocks[it.blk];
  if (j >= b.s) return;
  const int s = b.s;
  const int rows = side == 0 ? b.m : b.mc;
  const double* X = buf + (side == 0 ? b.yoff : b.boff);
  const int c = threadIdx.x % kSmax, g = threadIdx.x / kSmax;
  double acc = 0.0;
  const int rend = min(it.row0 + kPanelRows, rows);
  if (c <= j)
    for (int r = it.row0 + g; r < rend; r += kBT / kSmax)
      acc = fma(X[(int64_t)r * s + c], X[(int64_t)r * s + j], acc);
  red[g][c] = acc;
  __syncthreads();
  if (g == 0 && c <= j) {
    double t = 0.0;
    for (int q = 0; q < kBT / kSmax; ++q) t += red[q][c];
    part[(int64_t)blockIdx.x * kSmax + c] = t;
  }
}

__global__ void __launch_bounds__(kBT)
cgs_update_kernel(const BBlock* __restrict__ blocks, const TItem* __restrict__ items, int side, int j,
                  double* __restrict__ buf, const double* __restrict__ part, double* __restrict__ mats,
                  int rslot, int second, double* __restrict__ npart) {
  __shared__ double coef[kSmax];
  __shared__ double red[kBT / 32];
  const TItem it = items[blockIdx.x];
  const BBlock b = blocks[it.blk];
  if (j >= b.s) return;
  const int s = b.s;
  const int rows = side == 0 ? b.m : b.mc;
  const int p0 = side == 0 ? b.gram0y : b.gram0b, np = side == 0 ? b.ngramy : b.ngramb;
  double* X = buf + (side == 0 ? b.yoff : b.boff);
  double* R = mats + b.moff + rslot * kMat;
  const bool first = blockIdx.x == p0;
  for (int c = threadIdx.x; c <= j; c += kBT) {
    double t = 0.0;
    for (int q = 0; q < np; ++q) t += part[(int64_t)(p0 + q) * kSmax + c];
    if (c == j) {   // self dot: the squared length before the projections (pass 0)
      if (first && !second) mats[b.moff + kTmp * kMat + j] = t;
      continue;
    }
    coef[c] = t;
    if (first) R[c * kSmax + j] = second ? R[c * kSmax + j] + t : t;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rend = min(it.row0 + kPanelRows, rows);
  double nrm = 0.0;
  for (int r = it.row0 + warp; r < rend; r += kBT / 32) {
    double t = 0.0;
    for (int c = lane; c < j; c += 32) t = fma(X[(int64_t)r * s + c], coef[c], t);
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) {
      const double y = X[(int64_t)r * s + j] - t;
      X[(int64_t)r * s + j] = y;
      nrm = fma(y, y, nrm);
    }
  }
  if (lane == 0) red[warp] = nrm;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kBT / 32; ++w) t += red[w];
    npart[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(kBT)
cgs_norm_kernel(const BBlock* __restrict__ blocks, const TItem* __restrict__ items, int side, int j,
                double* __restrict__ buf, const double* __restrict__ npart, double* __restrict__ mats,
                int rslot) {
  __shared__ double s_inv;
  const TItem it = items[blockIdx.x];
  const BBlock b = blocks[it.blk];
  if (j >= b.s) return;
  const int s = b.s;
  const int rows = side == 0 ? b.m : b.mc;
  const int p0 = side == 0 ? b.gram0y : b.gram0b, np = side == 0 ? b.ngramy : b.ngramb;
  double* X = buf + (side == 0 ? b.yoff : b.boff);
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < np; ++q) t += npart[p0 + q];
    const double orig2 = mats[b.moff + kTmp * kMat + j];
    const bool keep = t > 1e-24 * orig2 && t > 0.0;
    const double nr = keep ? sqrt(t) : 0.0;
    s_inv = keep ? 1.0 / nr : 0.0;
    if (blockIdx.x == p0) mats[b.moff + rslot * kMat + j * kSmax + j] = nr;
  }
  __syncthreads();
  const double inv = s_inv;
  const int rend = min(it.row0 + kPanelRows, rows);
  for (int r = it.row0 + threadIdx.x; r < rend; r += kBT) X[(int64_t)r * s + j] *= inv;
}

// Out[rows] = In[rows] (rows x s) * M (s x sout) for one 64-row tile.  In
// place is allowed: each CTA owns its rows, and all reads complete (barrier)
// before any write.  final_out selects the staging output of the last pass
// (U = Q W_r for side 0, V = Q2 (Z S)_r for side 1) with sout = rank.
__global__ void __launch_bounds__(kBT)
apply_kernel(const BBlock* __restrict__ blocks, const TItem* __restrict__ items, int side,
             double* __restrict__ buf, const double* __restrict__ mats, int slot, int final_out,
             double* __restrict__ stage) {
  __shared__ double Ms[kSmax][kSmax + 1];
  const TItem it = items[blockIdx.x];
  const BBlock b = blocks[it.blk];
  const int s = b.s;
  const int sout = final_out ? b.rank : s;
  if (final_out && sout == 0) return;
  const int rows = side == 0 ? b.m : b.mc;
  const int64_t off = side == 0 ? b.yoff : b.boff;
  const double* M = mats + b.moff + slot * kMat;
  for (int e = threadIdx.x; e < kSmax * kSmax; e += kBT) {
    const int i = e / kSmax, j = e % kSmax;
    Ms[i][j] = (i < s && j < sout) ? M[i * kSmax + j] : 0.0;
  }
  __syncthreads();
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  double acc[4][4] = {};
  const double* X = buf + off;
  for (int k = 0; k < s; ++k) {
    double x[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int r = it.row0 + 4 * ty + p;
      x[p] = r < rows ? X[(int64_t)r * s + k] : 0.0;
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[p][q] = fma(x[p], Ms[k][4 * tx + q], acc[p][q]);
  }
  __syncthreads();
  double* o;
  int ld;
  if (final_out) {
    o = stage + (side == 0 ? b.uoff : b.voff);
    ld = sout;
  } else {
    o = buf + off;
    ld = s;
  }
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int r = it.row0 + 4 * ty + p;
    if (r >= rows) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = 4 * tx + q;
      if (c < sout) o[(int64_t)r * ld + c] = acc[p][q];
    }
  }
}

// One CTA per block: one-sided Jacobi on M = Racc^T (s x s), M Z = W S.
// Writes W (columns normalised, sorted by decreasing S), Z S (same order)
// and S; a bounded number of sweeps.
__global__ void __launch_bounds__(kBT)
jacobi_kernel(BBlock* __restrict__ blocks, double* __restrict__ mats, double* __restrict__ sig) {
  extern __shared__ double jsm[];
  double (*M)[kSmax + 1] = reinterpret_cast<double (*)[kSmax + 1]>(jsm);               // M[row][col]
  double (*Z)[kSmax + 1] = reinterpret_cast<double (*)[kSmax + 1]>(jsm + kSmax * (kSmax + 1));
  __shared__ double nrm[kSmax];
  __shared__ int order[kSmax];
  __shared__ int s_rot;
  const BBlock b = blocks[blockIdx.x];
  const int s = b.s;
  const int se = s + (s & 1);              // even number of columns (one zero column if odd)
  const double* Racc = mats + b.moff + kRacc * kMat;
  for (int e = threadIdx.x; e < kSmax * kSmax; e += kBT) {
    const int i = e / kSmax, j = e % kSmax;
    M[i][j] = (i < s && j < s) ? Racc[j * kSmax + i] : 0.0;   // transpose
    Z[i][j] = i == j ? 1.0 : 0.0;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int sweep = 0; sweep < kJacobiSweeps; ++sweep) {
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    for (int step = 0; step < se - 1; ++step) {
      // circle method: P[0] = 0 fixed, P[j] = 1 + (j - 1 + step) mod (se - 1);
      // round `step` pairs P[p] with P[se - 1 - p]
      for (int pr = warp; pr < se / 2; pr += kBT / 32) {
        int a = pr == 0 ? 0 : 1 + (pr - 1 + step) % (se - 1);
        int c = 1 + (se - 2 - pr + step) % (se - 1);
        if (a > c) { int t = a; a = c; c = t; }
        if (c >= s) continue;  // the padding column
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int r = lane; r < s; r += 32) {
          const double x = M[r][a], y = M[r][c];
          al = fma(x, x, al); be = fma(y, y, be); ga = fma(x, y, ga);
        }
        for (int o = 16; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        if (fabs(ga) > 1e-15 * sqrt(al * be) && ga != 0.0) {
          const double zeta = (be - al) / (2.0 * ga);
          const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
          for (int r = lane; r < s; r += 32) {
            const double x = M[r][a], y = M[r][c];
            M[r][a] = cs * x - sn * y;
            M[r][c] = sn * x + cs * y;
            const double zx = Z[r][a], zy = Z[r][c];
            Z[r][a] = cs * zx - sn * zy;
            Z[r][c] = sn * zx + cs * zy;
          }
          if (lane == 0) s_rot = 1;
        }
      }
      __syncthreads();
    }
    if (s_rot == 0) break;
    __syncthreads();
  }
  for (int c = threadIdx.x; c < s; c += kBT) {
    double t = 0.0;
    for (int r = 0; r < s; ++r) t = fma(M[r][c], M[r][c], t);
    nrm[c] = t >= 0.0 ? sqrt(t) : 0.0;   // a NaN becomes 0 so the ordering below is total
  }
  __syncthreads();
  for (int c = threadIdx.x; c < s; c += kBT) {   // rank of column c in decreasing order
    int pos = 0;
    for (int d = 0; d < s; ++d) pos += (nrm[d] > nrm[c]) || (nrm[d] == nrm[c] && d < c);
    order[pos] = c;
  }
  __syncthreads();
  double* W = mats + b.moff + kW * kMat;
  double* ZS = mats + b.moff + kZS * kMat;
  for (int e = threadIdx.x; e < s * s; e += kBT) {
    const int r = e / s, p = e % s;
    const int c = min(max(order[p], 0), s - 1);   // order is a permutation; the clamp is a guard
    const double sg = nrm[c];
    W[r * kSmax + p] = sg > 0.0 ? M[r][c] / sg : 0.0;
    ZS[r * kSmax + p] = Z[r][c] * sg;
  }
  for (int p = threadIdx.x; p < s; p += kBT)
    sig[(int64_t)blockIdx.x * kSmax + p] = nrm[min(max(order[p], 0), s - 1)];
}

// Rank by the truncation rule and the retry decision (one thread per block).
__global__ void truncate_kernel(BBlock* __restrict__ blocks, int nblk, const double* __restrict__ sig,
                                double eps) {
  const int bi = blockIdx.x * blockDim.x + threadIdx.x;
  if (bi >= nblk) return;
  BBlock& b = blocks[bi];
  const double budget = eps * eps * b.norm2;
  const double* sg = sig + (int64_t)bi * kSmax;
  const int full = min(b.m, b.mc);
  b.retry = (b.s < full && b.resid2 > 0.25 * budget) ? 1 : 0;
  // tail[r] = sum_{j >= r} s_j^2, accumulated from the smallest term
  int r = b.s;
  double tail = 0.0;
  while (r > 0) {
    const double t = tail + sg[r - 1] * sg[r - 1];
    if (t + b.resid2 > budget) break;
    tail = t;
    --r;
  }
  b.rank = r;
}

// Leaves D_i = A(I_i, I_i) into the staging (row-major).
__global__ void leaf_kernel(const KDesc K, const int2* __restrict__ leaves, const int64_t* __restrict__ st,
                            double* __restrict__ stage) {
  const int2 lf = leaves[blockIdx.x];  // (row0, m)
  double* d = stage + st[blockIdx.x];
  for (int e = threadIdx.x; e < lf.y * lf.y; e += blockDim.x) {
    const int i = e / lf.y, j = e % lf.y;
    d[e] = kval(K, lf.x + i, lf.x + j);
  }
}

struct DevMem {
  std::vector<void*> ptrs;
  ~DevMem() { for (void* p : ptrs) cudaFree(p); }
  template <typename T>
  cudaError_t alloc(T** p, size_t count) {
    cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(count, 1) * sizeof(T));
    if (e == cudaSuccess) ptrs.push_back(*p);
    return e;
  }
};

#define BCK(call)                                                   \
  do {                                                              \
    cudaError_t e_ = (call);                                        \
    if (e_ != cudaSuccess) return set_cuda_error(e_, #call);        \
  } while (0)

// One construction round over `blocks` with their sketch sizes set.
struct Round {
  std::vector<BBlock> blocks;
  BBlock* d_blocks = nullptr;
  std::vector<TItem> ty, tb, gy, gb;
  TItem *d_ty = nullptr, *d_tb = nullptr, *d_gy = nullptr, *d_gb = nullptr;
  double *d_Y = nullptr, *d_B = nullptr, *d_mats = nullptr, *d_sig = nullptr;
};

void cgs2(Round& R, int side, double* buf, int rslot, int smax_round, double* dots, double* npart,
          cudaStream_t st) {
  const TItem* items = side == 0 ? R.d_gy : R.d_gb;
  const int ni = (int)(side == 0 ? R.gy.size() : R.gb.size());
  for (int j = 0; j < smax_round; ++j) {
    for (int pass = 0; pass < 2; ++pass) {
      cgs_dot_kernel<<<ni, kBT, 0, st>>>(R.d_blocks, items, side, j, buf, dots);
      cgs_update_kernel<<<ni, kBT, 0, st>>>(R.d_blocks, items, side, j, buf, dots, R.d_mats, rslot,
                                             pass, npart);
    }
    cgs_norm_kernel<<<ni, kBT, 0, st>>>(R.d_blocks, items, side, j, buf, npart, R.d_mats, rslot);
  }
}

hodlr_status run_round(Round& R, const KDesc& K, const double* om, double eps, DevMem& mem,
                       cudaStream_t st) {
  int64_t yo = 0, bo = 0;
  const int nb = (int)R.blocks.size();
  for (int bi = 0; bi < nb; ++bi) {
    BBlock& b = R.blocks[bi];
    b.yoff = yo; yo += (int64_t)b.m * b.s;
    b.boff = bo; bo += (int64_t)b.mc * b.s;
    b.moff = (int64_t)bi * 6 * kMat;
    b.item0y = (int)R.ty.size();
    for (int r = 0; r < b.m; r += kRT) R.ty.push_back({bi, r});
    b.nitemy = (int)R.ty.size() - b.item0y;
    b.item0b = (int)R.tb.size();
    for (int r = 0; r < b.mc; r += kRT) R.tb.push_back({bi, r});
    b.nitemb = (int)R.tb.size() - b.item0b;
    b.gram0y = (int)R.gy.size();
    for (int r = 0; r < b.m; r += kPanelRows) R.gy.push_back({bi, r});
    b.ngramy = (int)R.gy.size() - b.gram0y;
    b.gram0b = (int)R.gb.size();
    for (int r = 0; r < b.mc; r += kPanelRows) R.gb.push_back({bi, r});
    b.ngramb = (int)R.gb.size() - b.gram0b;
  }
  BCK(mem.alloc(&R.d_blocks, nb));
  BCK(mem.alloc(&R.d_ty, R.ty.size()));
  BCK(mem.alloc(&R.d_tb, R.tb.size()));
  BCK(mem.alloc(&R.d_gy, R.gy.size()));
  BCK(mem.alloc(&R.d_gb, R.gb.size()));
  BCK(mem.alloc(&R.d_Y, yo));
  BCK(mem.alloc(&R.d_B, bo));
  BCK(mem.alloc(&R.d_mats, (size_t)nb * 6 * kMat));
  BCK(mem.alloc(&R.d_sig, (size_t)nb * kSmax));
  double *d_part = nullptr, *d_dots = nullptr, *d_npart = nullptr;
  BCK(mem.alloc(&d_part, std::max(R.ty.size(), R.tb.size())));
  BCK(mem.alloc(&d_dots, std::max(R.gy.size(), R.gb.size()) * (size_t)kSmax));
  BCK(mem.alloc(&d_npart, std::max(R.gy.size(), R.gb.size())));
  BCK(cudaMemsetAsync(R.d_mats, 0, (size_t)nb * 6 * kMat * sizeof(double), st));
  int smax_round = 0;
  for (const BBlock& b : R.blocks) smax_round = std::max(smax_round, b.s);
  BCK(cudaMemcpyAsync(R.d_blocks, R.blocks.data(), nb * sizeof(BBlock), cudaMemcpyHostToDevice, st));
  BCK(cudaMemcpyAsync(R.d_ty, R.ty.data(), R.ty.size() * sizeof(TItem), cudaMemcpyHostToDevice, st));
  BCK(cudaMemcpyAsync(R.d_tb, R.tb.data(), R.tb.size() * sizeof(TItem), cudaMemcpyHostToDevice, st));
  BCK(cudaMemcpyAsync(R.d_gy, R.gy.data(), R.gy.size() * sizeof(TItem), cudaMemcpyHostToDevice, st));
  BCK(cudaMemcpyAsync(R.d_gb, R.gb.data(), R.gb.size() * sizeof(TItem), cudaMemcpyHostToDevice, st));
  const int nty = (int)R.ty.size(), ntb = (int)R.tb.size();
  const int rb = (nb + 127) / 128;

  // 1. sketch + block norms
  gen_product_kernel<0><<<nty, kBT, 0, st>>>(K, R.d_blocks, R.d_ty, om, kSmax, R.d_Y, d_part);
  BCK(cudaGetLastError());
  reduce_parts_kernel<<<rb, 128, 0, st>>>(R.d_blocks, nb, d_part, 0);
  // 2. Q = orth(Y) by CGS2 (R of Y is not needed: slot kG)
  cgs2(R, 0, R.d_Y, kG, smax_round, d_dots, d_npart, st);
  BCK(cudaGetLastError());
  // 3. Bt = A^T Q; 4. sketch residual
  gen_product_kernel<1><<<ntb, kBT, 0, st>>>(K, R.d_blocks, R.d_tb, R.d_Y, 0, R.d_B, nullptr);
  resid_kernel<<<nty, kBT, 0, st>>>(K, R.d_blocks, R.d_ty, R.d_Y, R.d_B, d_part);
  reduce_parts_kernel<<<rb, 128, 0, st>>>(R.d_blocks, nb, d_part, 1);
  BCK(cudaGetLastError());
  // 5. Bt = Q2 R2 (R2 in slot kRacc), SVD of R2^T
  cgs2(R, 1, R.d_B, kRacc, smax_round, d_dots, d_npart, st);
  const int jsmem = 2 * kSmax * (kSmax + 1) * (int)sizeof(double);
  BCK(cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, jsmem));
  jacobi_kernel<<<nb, kBT, jsmem, st>>>(R.d_blocks, R.d_mats, R.d_sig);
  truncate_kernel<<<rb, 128, 0, st>>>(R.d_blocks, nb, R.d_sig, eps);
  BCK(cudaGetLastError());
  BCK(cudaMemcpyAsync(R.blocks.data(), R.d_blocks, nb * sizeof(BBlock), cudaMemcpyDeviceToHost, st));
  BCK(cudaStreamSynchronize(st));
  return HODLR_OK;
}

}  // namespace

}  // namespace hodlr

using namespace hodlr;

extern "C" hodlr_status hodlr_build(int32_t n, int32_t depth, const hodlr_kernel* kernel,
                                    const double* points, const hodlr_opts* opts,
                                    const hodlr_build_opts* bopts, void* stream, hodlr_t* out) {
  if (!out || !opts || !kernel || !points) return set_error(HODLR_EINVAL, "null argument");
  if (kernel->dim < 1 || kernel->dim > 3) return set_error(HODLR_EINVAL, "dim must be 1..3");
  if (kernel->kind < 0 || kernel->kind > 3 || (kernel->kind == 3 && kernel->dim != 1))
    return set_error(HODLR_EINVAL, "bad kernel kind");
  if (kernel->kind == 1 && !(kernel->len2 > 0.0)) return set_error(HODLR_EINVAL, "len2 must be > 0");
  if (n < 1 || depth < 0 || depth > HODLR_MAX_DEPTH || (int64_t(1) << depth) > n)
    return set_error(HODLR_EINVAL, "bad n/depth");
  int s0 = bopts && bopts->sketch > 0 ? bopts->sketch : 16;
  int smax = bopts && bopts->max_sketch > 0 ? bopts->max_sketch : kSmax;
  if (s0 > kSmax || smax > kSmax) return set_error(HODLR_EINVAL, "sketch sizes are limited to 64");
  s0 = std::min(s0, smax);
  const uint64_t seed = bopts ? bopts->seed : 0;
  cudaStream_t st = (cudaStream_t)stream;
  const KDesc K{points, n, kernel->dim, kernel->kind, kernel->c, kernel->len2, kernel->diag};

  std::vector<std::vector<std::pair<int, int>>> lv(depth + 1);
  lv[0].push_back({0, n});
  for (int k = 0; k < depth; ++k)
    for (auto& nd : lv[k]) {
      const int left = (nd.second + 1) / 2;
      lv[k + 1].push_back({nd.first, left});
      lv[k + 1].push_back({nd.first + left, nd.second - left});
    }
  const int nnodes = (1 << (depth + 1)) - 2;

  DevMem mem;
  double* d_om = nullptr;
  BCK(mem.alloc(&d_om, (size_t)n * kSmax));
  omega_kernel<<<1024, 256, 0, st>>>(d_om, (int64_t)n * kSmax, seed);
  BCK(cudaGetLastError());

  // rounds with growing sketches
  std::vector<std::unique_ptr<Round>> rounds;
  std::vector<int> final_round(nnodes, -1), final_idx(nnodes, -1);
  std::vector<double> block_norm2(nnodes, 0.0);
  std::vector<BBlock> pending;
  for (int k = 1; k <= depth; ++k)
    for (int i = 0; i < (1 << k); ++i) {
      BBlock b{};
      b.r0 = lv[k][i].first;
      b.m = lv[k][i].second;
      b.c0 = lv[k][i ^ 1].first;
      b.mc = lv[k][i ^ 1].second;
      b.q = node_index(k, i);
      pending.push_back(b);
    }
  // every block's current sketch: the node's own first sketch when given
  std::vector<int> sk(nnodes, s0);
  if (bopts && bopts->node_sketch)
    for (int q = 0; q < nnodes; ++q) sk[q] = std::max(1, std::min(bopts->node_sketch[q], smax));
  int nrounds = 0, redone = 0;
  int64_t sketch_cols = 0;
  bool accuracy_short = false;
  double worst_ratio = 0.0;
  std::string worst_msg;
  while (!pending.empty()) {
    auto R = std::make_unique<Round>();
    for (BBlock b : pending) {
      b.s = std::min(sk[b.q], std::min(b.m, b.mc));
      sketch_cols += b.s;
      R->blocks.push_back(b);
    }
    if (nrounds++ > 0) redone += (int)pending.size();
    hodlr_status stt = run_round(*R, K, d_om, opts->eps, mem, st);
    if (stt != HODLR_OK) return stt;
    pending.clear();
    const int ri = (int)rounds.size();
    for (int bi = 0; bi < (int)R->blocks.size(); ++bi) {
      const BBlock& b = R->blocks[bi];
      if (b.retry && b.s < std::min(smax, std::min(b.m, b.mc))) {
        sk[b.q] = std::min(2 * sk[b.q], smax);
        pending.push_back(b);
        continue;
      }
      if (b.retry) {
        const double ratio = b.resid2 / (opts->eps * opts->eps * b.norm2);
        if (!accuracy_short || ratio > worst_ratio) {
          worst_ratio = ratio;
          char buf[256];
          snprintf(buf, sizeof(buf),
                   "block node %d (%d x %d) at sketch %d: sketch residual^2 = %.3e, eps^2 ||A_b||^2 = %.3e, "
                   "||A_b||^2 = %.3e", b.q, b.m, b.mc, b.s, b.resid2, opts->eps * opts->eps * b.norm2, b.norm2);
          worst_msg = buf;
        }
        accuracy_short = true;
      }
      final_round[b.q] = ri;
      final_idx[b.q] = bi;
      block_norm2[b.q] = b.norm2;
    }
    rounds.push_back(std::move(R));
  }

  // layout with the final ranks, then U = Q W_r and V = Q2 (Z S)_r into the staging
  std::vector<int32_t> ranks(nnodes, 0);
  for (int q = 0; q < nnodes; ++q) ranks[q] = rounds[final_round[q]]->blocks[final_idx[q]].rank;
  auto h = new hodlr_s();
  std::unique_ptr<hodlr_s> guard(h);
  hodlr_status stt = plan_layout(h, n, depth, ranks.data(), opts);
  if (stt != HODLR_OK) return stt;
  h->build_sketch_max = 0;
  double* d_stage = nullptr;
  BCK(mem.alloc(&d_stage, (size_t)h->st_count));
  for (size_t ri = 0; ri < rounds.size(); ++ri) {
    Round& R = *rounds[ri];
    bool any = false;
    for (BBlock& b : R.blocks) {
      const bool mine = final_round[b.q] == (int)ri;
      if (mine) {
        const int k = 31 - __builtin_clz(b.q + 2);
        const int i = b.q - node_index(k, 0);
        b.uoff = h->st_U[b.q];
        b.voff = h->st_V[node_index(k, i ^ 1)];
        h->build_sketch_max = std::max(h->build_sketch_max, b.s);
        any = true;
      } else {
        b.rank = 0;   // superseded by a later round: writes nothing
      }
    }
    if (!any) continue;
    BCK(cudaMemcpyAsync(R.d_blocks, R.blocks.data(), R.blocks.size() * sizeof(BBlock),
                        cudaMemcpyHostToDevice, st));
    apply_kernel<<<(int)R.ty.size(), kBT, 0, st>>>(R.d_blocks, R.d_ty, 0, R.d_Y, R.d_mats, kW, 1, d_stage);
    apply_kernel<<<(int)R.tb.size(), kBT, 0, st>>>(R.d_blocks, R.d_tb, 1, R.d_B, R.d_mats, kZS, 1, d_stage);
    BCK(cudaGetLastError());
  }
  {
    const int nleaves = 1 << depth;
    std::vector<int2> lf(nleaves);
    for (int l = 0; l < nleaves; ++l) lf[l] = make_int2(lv[depth][l].first, lv[depth][l].second);
    int2* d_lf = nullptr;
    int64_t* d_st = nullptr;
    BCK(mem.alloc(&d_lf, nleaves));
    BCK(mem.alloc(&d_st, nleaves));
    BCK(cudaMemcpyAsync(d_lf, lf.data(), nleaves * sizeof(int2), cudaMemcpyHostToDevice, st));
    BCK(cudaMemcpyAsync(d_st, h->st_D.data(), nleaves * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    leaf_kernel<<<nleaves, 256, 0, st>>>(K, d_lf, d_st, d_stage);
    BCK(cudaGetLastError());
  }
  stt = finish_from_staging(h, d_stage, block_norm2.data(), nullptr, opts, st);
  if (stt != HODLR_OK) return stt;
  h->build_accuracy_short = accuracy_short;
  h->build_rounds = nrounds;
  h->build_redone = redone;
  h->build_sketch_cols = sketch_cols;
  *out = guard.release();
  if (accuracy_short)
    return set_error(HODLR_EACCURACY, "a block needed a sketch larger than max_sketch (its rank is capped); worst: " + worst_msg);
  return HODLR_OK;
}
