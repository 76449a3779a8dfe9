// HODLR LU factorization (Algorithm 3.4, HODLR_LU), its triangular solves,
// and GMRES-based iterative refinement with the factors as preconditioner
// (Sect. 3.4), on the device in fp64.
//
// Generator form.  Block (q, q^1) of the matrix is U_q V_{q^1}^T (node q's U,
// its sibling's V).  At a node with children a, b (Algorithm 3.4):
//
//   L_a, U_a = HODLR_LU(H_aa)
//   U12 = L_a^{-1} H_ab = (L_a^{-1} U_a) V_b^T      -> U_a := L_a^{-1} U_a
//   L21 = H_ba U_a^{-1} = U_b (U_a^{-T} V_a)^T      -> V_a := U_a^{-T} V_a
//   S   = H_bb - L21 U12 = H_bb - U_b C V_b^T,  C = V_a^T U_a (the new ones)
//   S is truncated back to the HODLR format of b (Assumption 3.6): every
//   leaf of b takes the exact update; every off-diagonal block (p, p^1)
//   inside b becomes [U_p | -(U_b C)_p] [V_{p^1} | (V_b)_{p^1}]^T and is
//   recompressed to the relative Frobenius tolerance eps_lu (QR of both
//   bases, SVD of the small core, the truncation rule of the construction);
//   L_b, U_b = HODLR_LU(S).
//
// So L has unit-lower leaves and lower blocks U_b V_a^T, U has upper leaves
// and upper blocks U_a V_b^T, all held in place of the generators.  Leaves
// are factored without pivoting (the leading blocks must be nonsingular; a
// zero pivot is reported as HODLR_ESINGULAR).
//
// The recursion runs on the host in tree order; every step is a device
// kernel over all the rows, columns and blocks the step touches.  Every sum
// has a fixed order, so the factors are reproducible.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "handle.cuh"

namespace hodlr {

namespace {

constexpr int kLT = 256;        // threads of the LU kernels
constexpr int kGemmTile = 16;   // output tile of the small GEMM
constexpr int kSplitK = 2048;   // GEMM reduction length per split at most
constexpr int kJacobiSweeps = 40;
constexpr int kSolveCols = 64;  // right-hand sides per triangular solve at most

__host__ __device__ inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ---- block reductions with a fixed order ------------------------------------
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// Sum over the CTA: lane partials by butterfly, then the warps in order.
__device__ double block_sum(double v, double* red) {
  v = warp_sum_d(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];
  __syncthreads();
  return s;
}

// ---- leaf LU: right-looking, no pivoting, D row-major m x m in place --------
__global__ void __launch_bounds__(kLT) leaf_lu_kernel(double* __restrict__ D, int m, int* err) {
  for (int j = 0; j < m; ++j) {
    const double piv = D[(int64_t)j * m + j];   // the same value on every thread
    if (piv == 0.0 || !isfinite(piv)) {
      if (threadIdx.x == 0) atomicExch(err, 1);
      return;
    }
    for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) D[(int64_t)i * m + j] /= piv;
    __syncthreads();
    const int w = m - j - 1;
    for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
      const int i = j + 1 + e / w, k = j + 1 + e % w;
      D[(int64_t)i * m + k] -= D[(int64_t)i * m + j] * D[(int64_t)j * m + k];
    }
    __syncthreads();
  }
}

// ---- leaf triangular solves on Z (m x p, leading dimension ldz), in place ----
// mode 0: L Z' = Z, L the unit lower part of the leaf; 1: U Z' = Z, U the
// upper part; 2: U^T Z' = Z.  Column-oriented: once row k is final, it is
// removed from the rows it couples to.
__global__ void __launch_bounds__(kLT) leaf_trsm_kernel(const double* __restrict__ D, int m, double* __restrict__ Z,
                                                        int64_t ldz, int p, int mode) {
  if (mode == 1) {
    for (int k = m - 1; k >= 0; --k) {
      const double d = D[(int64_t)k * m + k];
      for (int c = threadIdx.x; c < p; c += blockDim.x) Z[k * ldz + c] /= d;
      __syncthreads();
      for (int e = threadIdx.x; e < k * p; e += blockDim.x) {
        const int i = e / p, c = e % p;
        Z[i * ldz + c] -= D[(int64_t)i * m + k] * Z[k * ldz + c];
      }
      __syncthreads();
    }
    return;
  }
  for (int k = 0; k < m; ++k) {
    if (mode == 2) {
      const double d = D[(int64_t)k * m + k];
      for (int c = threadIdx.x; c < p; c += blockDim.x) Z[k * ldz + c] /= d;
      __syncthreads();
    }
    const int w = m - k - 1;
    for (int e = threadIdx.x; e < w * p; e += blockDim.x) {
      const int i = k + 1 + e / p, c = e % p;
      const double coef = mode == 0 ? D[(int64_t)i * m + k] : D[(int64_t)k * m + i];
      Z[i * ldz + c] -= coef * Z[k * ldz + c];
    }
    __syncthreads();
  }
}

// ---- small fp64 GEMM ----------------------------------------------------------
// C (M x N) = beta C + alpha op(A) op(B), row-major; op(A) is M x K (tA: A is
// K x M), op(B) is K x N (tB: B is N x K).  Split z of the reduction (K in
// ranges of kSplitK) writes its partial to part[z]; gemm_reduce adds the
// splits in order.  One thread per output element.
struct GemmArgs {
  const double* A;
  int64_t lda;
  const double* B;
  int64_t ldb;
  double* C;
  int64_t ldc;
  int M, N, K, tA, tB, nsplit;
  double alpha, beta;
  double* part;
};
__global__ void gemm_kernel(const GemmArgs g) {
  const int i = blockIdx.y * kGemmTile + threadIdx.y, j = blockIdx.x * kGemmTile + threadIdx.x;
  const int z = blockIdx.z;
  if (i >= g.M || j >= g.N) return;
  const int k0 = z * kSplitK, k1 = g.K - k0 < kSplitK ? g.K : k0 + kSplitK;
  double s = 0.0;
  for (int k = k0; k < k1; ++k) {
    const double a = g.tA ? g.A[(int64_t)k * g.lda + i] : g.A[(int64_t)i * g.lda + k];
    const double b = g.tB ? g.B[(int64_t)j * g.ldb + k] : g.B[(int64_t)k * g.ldb + j];
    s = fma(a, b, s);
  }
  if (g.nsplit == 1) {
    double* c = g.C + (int64_t)i * g.ldc + j;
    *c = (g.beta == 0.0 ? 0.0 : g.beta * *c) + g.alpha * s;
  } else {
    g.part[((int64_t)z * g.M + i) * g.N + j] = s;
  }
}
__global__ void gemm_reduce_kernel(const GemmArgs g) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)g.M * g.N) return;
  const int i = (int)(e / g.N), j = (int)(e % g.N);
  double s = 0.0;
  for (int z = 0; z < g.nsplit; ++z) s += g.part[((int64_t)z * g.M + i) * g.N + j];
  double* c = g.C + (int64_t)i * g.ldc + j;
  *c = (g.beta == 0.0 ? 0.0 : g.beta * *c) + g.alpha * s;
}

// ---- Schur update of the leaves of a subtree ------------------------------
// D_i -= GC[rows of i] H[rows of i]^T for the leaves listed (t columns).
struct LeafUpd {
  double* D;
  int m;
  int row;   // first row of the leaf inside the subtree (GC and H rows)
};
__global__ void __launch_bounds__(kLT) schur_leaf_kernel(const LeafUpd* __restrict__ lv, const double* __restrict__ GC,
                                                         int64_t ldgc, const double* __restrict__ H, int64_t ldh, int t) {
  const LeafUpd L = lv[blockIdx.x];
  for (int e = threadIdx.x; e < L.m * L.m; e += blockDim.x) {
    const int r = e / L.m, c = e % L.m;
    const double* g = GC + (int64_t)(L.row + r) * ldgc;
    const double* h = H + (int64_t)(L.row + c) * ldh;
    double s = 0.0;
    for (int l = 0; l < t; ++l) s = fma(g[l], h[l], s);
    L.D[(int64_t)r * L.m + c] -= s;
  }
}

// ---- recompression of one off-diagonal block per CTA ------------------------
// Block = [U | -GC] [V | H]^T: U (m1 x r), GC (m1 x t), V (m2 x r), H (m2 x t).
// QR of both bases by CGS2 (workspace A, B of w = r + t columns), core
// M = R_A R_B^T, one-sided Jacobi on the columns of M (M Z = W S), rank by
// the relative Frobenius rule, then U := Q_A W_r (orthonormal columns) and
// V := Q_B Z_r S_r (the construction's convention).
struct RcBlock {
  double* U;
  int64_t ldu;
  double* V;
  int64_t ldv;
  const double* GC;
  int64_t ldgc;
  const double* H;
  int64_t ldh;
  int m1, m2, r, t, cap;
  double* A;   // m1 x w
  double* B;   // m2 x w
  double* S;   // 4 w^2 + w: R_A, R_B, M, Z, sigma
};

// CGS2 QR of X (m x w, row-major, ld w) in place; R (w x w, row-major) out.
// A column whose remainder is below 1e-13 of its length is set to zero
// (R[j][j] = 0): it lies in the span of the previous ones.
__device__ void cgs2_qr(double* X, int m, int w, double* R, double* coef, double* red) {
  for (int e = threadIdx.x; e < w * w; e += blockDim.x) R[e] = 0.0;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = 0; j < w; ++j) {
    double s0 = 0.0;
    for (int r = threadIdx.x; r < m; r += blockDim.x) s0 += X[(int64_t)r * w + j] * X[(int64_t)r * w + j];
    const double n0 = sqrt(block_sum(s0, red));
    for (int pass = 0; pass < 2; ++pass) {
      for (int l = warp; l < j; l += nw) {
        double s = 0.0;
        for (int r = lane; r < m; r += 32) s += X[(int64_t)r * w + l] * X[(int64_t)r * w + j];
        s = warp_sum_d(s);
        if (lane == 0) coef[l] = s;
      }
      __syncthreads();
      for (int r = threadIdx.x; r < m; r += blockDim.x) {
        double x = X[(int64_t)r * w + j];
        for (int l = 0; l < j; ++l) x -= coef[l] * X[(int64_t)r * w + l];
        X[(int64_t)r * w + j] = x;
      }
      for (int l = threadIdx.x; l < j; l += blockDim.x) R[l * w + j] += coef[l];
      __syncthreads();
    }
    double s1 = 0.0;
    for (int r = threadIdx.x; r < m; r += blockDim.x) s1 += X[(int64_t)r * w + j] * X[(int64_t)r * w + j];
    const double nr = sqrt(block_sum(s1, red));
    const bool zero = !(nr > 1e-13 * n0);
    for (int r = threadIdx.x; r < m; r += blockDim.x) X[(int64_t)r * w + j] = zero ? 0.0 : X[(int64_t)r * w + j] / nr;
    if (threadIdx.x == 0) R[j * w + j] = zero ? 0.0 : nr;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kLT) recompress_kernel(const RcBlock* __restrict__ blocks, double eps,
                                                         int* __restrict__ rank_out, int* err) {
  __shared__ double red[kLT / 32];
  __shared__ double coef[512];
  __shared__ int perm[512];
  __shared__ int s_rank, s_rot;
  const RcBlock bk = blocks[blockIdx.x];
  const int w = bk.r + bk.t;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  // the two bases
  for (int64_t e = threadIdx.x; e < (int64_t)bk.m1 * w; e += blockDim.x) {
    const int i = (int)(e / w), c = (int)(e % w);
    bk.A[e] = c < bk.r ? bk.U[i * bk.ldu + c] : -bk.GC[i * bk.ldgc + (c - bk.r)];
  }
  for (int64_t e = threadIdx.x; e < (int64_t)bk.m2 * w; e += blockDim.x) {
    const int i = (int)(e / w), c = (int)(e % w);
    bk.B[e] = c < bk.r ? bk.V[i * bk.ldv + c] : bk.H[i * bk.ldh + (c - bk.r)];
  }
  __syncthreads();
  double* RA = bk.S;
  double* RB = RA + (int64_t)w * w;
  double* M = RB + (int64_t)w * w;
  double* Z = M + (int64_t)w * w;
  double* sig = Z + (int64_t)w * w;
  cgs2_qr(bk.A, bk.m1, w, RA, coef, red);
  cgs2_qr(bk.B, bk.m2, w, RB, coef, red);
  // M = R_A R_B^T, Z = I
  for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
    const int i = e / w, j = e % w;
    double s = 0.0;
    for (int l = 0; l < w; ++l) s += RA[i * w + l] * RB[j * w + l];
    M[e] = s;
    Z[e] = i == j ? 1.0 : 0.0;
  }
  __syncthreads();
  // one-sided Jacobi on the columns of M, round-robin pairs (W = w rounded up
  // to even; player W-1 fixed, the others rotate), one warp per pair
  const int W = w + (w & 1);
  for (int sweep = 0; sweep < kJacobiSweeps; ++sweep) {
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    for (int round = 0; round < W - 1; ++round) {
      for (int k = warp; k < W / 2; k += nw) {
        int i, j;
        if (k == 0) {
          i = round;
          j = W - 1;
        } else {
          i = (round + k) % (W - 1);
          j = (round - k + (W - 1)) % (W - 1);
        }
        if (i > j) { const int x = i; i = j; j = x; }
        if (j >= w) continue;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int r = lane; r < w; r += 32) {
          const double mi = M[r * w + i], mj = M[r * w + j];
          al += mi * mi;
          be += mj * mj;
          ga += mi * mj;
        }
        al = warp_sum_d(al);
        be = warp_sum_d(be);
        ga = warp_sum_d(ga);
        if (ga == 0.0 || fabs(ga) <= 1e-15 * sqrt(al * be)) continue;
        const double zeta = (be - al) / (2.0 * ga);
        const double tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / sqrt(1.0 + tt * tt), sn = c * tt;
        for (int r = lane; r < w; r += 32) {
          const double mi = M[r * w + i], mj = M[r * w + j];
          M[r * w + i] = c * mi - sn * mj;
          M[r * w + j] = sn * mi + c * mj;
          const double zi = Z[r * w + i], zj = Z[r * w + j];
          Z[r * w + i] = c * zi - sn * zj;
          Z[r * w + j] = sn * zi + c * zj;
        }
        if (lane == 0) s_rot = 1;
      }
      __syncthreads();
    }
    const int any = s_rot;
    __syncthreads();
    if (!any) break;
  }
  // singular values (column norms), their order, the rank
  for (int j = warp; j < w; j += nw) {
    double s = 0.0;
    for (int r = lane; r < w; r += 32) s += M[r * w + j] * M[r * w + j];
    s = warp_sum_d(s);
    if (lane == 0) sig[j] = sqrt(s);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int j = 0; j < w; ++j) perm[j] = j;
    for (int a = 1; a < w; ++a) {   // insertion sort, decreasing (stable)
      const int x = perm[a];
      int b = a - 1;
      while (b >= 0 && sig[perm[b]] < sig[x]) {
        perm[b + 1] = perm[b];
        --b;
      }
      perm[b + 1] = x;
    }
    double total = 0.0;
    for (int j = 0; j < w; ++j) total += sig[perm[j]] * sig[perm[j]];
    int rk = 0;
    if (total > 0.0) {
      // smallest rk with sqrt(sum_{j >= rk} s_j^2) <= eps sqrt(total)
      double tail = 0.0;
      rk = w;
      for (int j = w - 1; j >= 0; --j) {
        tail += sig[perm[j]] * sig[perm[j]];
        if (sqrt(tail) <= eps * sqrt(total)) rk = j;
        else break;
      }
    }
    if (rk > bk.cap) {
      atomicExch(err, 2);
      rk = bk.cap;
    }
    s_rank = rk;
    rank_out[blockIdx.x] = rk;
  }
  __syncthreads();
  const int rk = s_rank;
  // U := Q_A W_r, W_j = M[:, perm j] / s; V := Q_B Z[:, perm j] s
  for (int64_t e = threadIdx.x; e < (int64_t)bk.m1 * rk; e += blockDim.x) {
    const int i = (int)(e / rk), j = (int)(e % rk), pj = perm[j];
    const double sj = sig[pj];
    double s = 0.0;
    for (int l = 0; l < w; ++l) s += bk.A[(int64_t)i * w + l] * M[l * w + pj];
    bk.U[i * bk.ldu + j] = sj > 0.0 ? s / sj : 0.0;
  }
  for (int64_t e = threadIdx.x; e < (int64_t)bk.m2 * rk; e += blockDim.x) {
    const int i = (int)(e / rk), j = (int)(e % rk), pj = perm[j];
    double s = 0.0;
    for (int l = 0; l < w; ++l) s += bk.B[(int64_t)i * w + l] * Z[l * w + pj];
    bk.V[i * bk.ldv + j] = s * sig[pj];
  }
}

// ---- vectors (GMRES) ----------------------------------------------------------
// Strided column copy / scale: Y[i * ldy] = a X[i * ldx] + b Y[i * ldy].
__global__ void axpby_kernel(int n, double a, const double* __restrict__ X, int64_t ldx, double b, double* __restrict__ Y,
                             int64_t ldy) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) Y[i * ldy] = a * X[i * ldx] + (b == 0.0 ? 0.0 : b * Y[i * ldy]);
}
// out[0] = sum_i X[i * ldx] Y[i * ldy], one CTA, fixed order.
__global__ void __launch_bounds__(1024) dot_kernel(int n, const double* __restrict__ X, int64_t ldx,
                                                   const double* __restrict__ Y, int64_t ldy, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s = fma(X[i * ldx], Y[i * ldy], s);
  s = block_sum(s, red);
  if (threadIdx.x == 0) *out = s;
}

// Copy U/V generators or leaves between the staging (m x r, ld r) and the
// factor pool (ld cap).
__global__ void copy2d_kernel(const double* __restrict__ src, int64_t lds, double* __restrict__ dst, int64_t ldd, int rows,
                              int cols) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)rows * cols) return;
  const int64_t i = e / cols, c = e % cols;
  dst[i * ldd + c] = src[i * lds + c];
}

}  // namespace

// ---- the factorization state of a handle ----------------------------------
struct LuState {
  int depth = 0, n = 0;
  std::vector<int> m, row0;        // per node q (tree order of node_index) and per leaf via lnode
  std::vector<int> rU, rV, cap;    // current ranks, capacity (columns) of U_q and V_q
  std::vector<int64_t> offU, offV, offD;
  double* pool = nullptr;          // generators (ld cap) and leaves (ld m)
  double* work = nullptr;          // recompression workspace
  size_t work_n = 0;
  double* gc = nullptr;            // U_b C (m_b x t) and C (t x t)
  double* cm = nullptr;
  double* gpart = nullptr;         // GEMM split partials
  size_t gpart_n = 0;
  double* vec = nullptr;           // GMRES vectors and scalars
  size_t vec_n = 0;
  RcBlock* d_rc = nullptr;
  int* d_rank = nullptr;
  LeafUpd* d_lu = nullptr;
  int max_blocks = 0;
  int* d_err = nullptr;
  double eps_lu = 0.0;
  bool factored = false;
  cudaStream_t s = nullptr;
  ~LuState() {
    cudaFree(pool);
    cudaFree(work);
    cudaFree(gc);
    cudaFree(cm);
    cudaFree(gpart);
    cudaFree(vec);
    cudaFree(d_rc);
    cudaFree(d_rank);
    cudaFree(d_lu);
    cudaFree(d_err);
  }
  double* U(int q) { return pool + offU[q]; }
  double* V(int q) { return pool + offV[q]; }
  double* D(int l) { return pool + offD[l]; }
};

void lu_destroy(LuState* s) { delete s; }

namespace {

cudaError_t gemm(LuState& L, const double* A, int64_t lda, int tA, const double* B, int64_t ldb, int tB, double* C,
                 int64_t ldc, int M, int N, int K, double alpha, double beta) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  GemmArgs g{A, lda, B, ldb, C, ldc, M, N, K, tA, tB, 1, alpha, beta, nullptr};
  g.nsplit = (int)std::max<int64_t>(1, cdiv(K, kSplitK));
  if (g.nsplit > 1) {
    const size_t need = (size_t)g.nsplit * M * N;
    if (need > L.gpart_n) {
      cudaFree(L.gpart);
      L.gpart = nullptr;
      L.gpart_n = 0;
      cudaError_t e = cudaMalloc(&L.gpart, need * sizeof(double));
      if (e != cudaSuccess) return e;
      L.gpart_n = need;
    }
    g.part = L.gpart;
  }
  dim3 grid((unsigned)cdiv(N, kGemmTile), (unsigned)cdiv(M, kGemmTile), (unsigned)g.nsplit);
  gemm_kernel<<<grid, dim3(kGemmTile, kGemmTile), 0, L.s>>>(g);
  if (g.nsplit > 1) gemm_reduce_kernel<<<(unsigned)cdiv((int64_t)M * N, 256), 256, 0, L.s>>>(g);
  return cudaGetLastError();
}

int child(int k, int i) { return node_index(k, i); }

// ---- recursive triangular solves on Z (rows of node (k, i)), p columns -----
// Node (0, 0) is the root (the whole matrix); below it node_index numbers
// the tree.  lev(k, i) returns the node's rows and leaf.
struct Tree {
  const hodlr_s* h;
  int row0(int k, int i) const { return k == 0 ? 0 : h->nodes[node_index(k, i)].row0; }
  int m(int k, int i) const { return k == 0 ? h->n : h->nodes[node_index(k, i)].m; }
};

cudaError_t tri_solve(LuState& L, const Tree& T, int k, int i, double* Z, int64_t ldz, int p, int mode);

// mode 0: L, 1: U, 2: U^T (see leaf_trsm_kernel)
cudaError_t tri_solve(LuState& L, const Tree& T, int k, int i, double* Z, int64_t ldz, int p, int mode) {
  cudaError_t e;
  if (k == L.depth) {
    const int leaf = i;
    leaf_trsm_kernel<<<1, kLT, 0, L.s>>>(L.D(leaf), T.m(k, i), Z, ldz, p, mode);
    return cudaGetLastError();
  }
  const int a = child(k + 1, 2 * i), b = child(k + 1, 2 * i + 1);
  const int ma = T.m(k + 1, 2 * i), mb = T.m(k + 1, 2 * i + 1);
  double* Za = Z;
  double* Zb = Z + (int64_t)ma * ldz;
  if (mode == 1) {
    // U Z = B: Z_b = U_bb^{-1} B_b; Z_a = U_aa^{-1} (B_a - U_a (V_b^T Z_b))
    if ((e = tri_solve(L, T, k + 1, 2 * i + 1, Zb, ldz, p, 1)) != cudaSuccess) return e;
    const int r = L.rU[a];
    if (r > 0) {
      if ((e = gemm(L, L.V(b), L.cap[b], 1, Zb, ldz, 0, L.cm, p, r, p, mb, 1.0, 0.0)) != cudaSuccess) return e;
      if ((e = gemm(L, L.U(a), L.cap[a], 0, L.cm, p, 0, Za, ldz, ma, p, r, -1.0, 1.0)) != cudaSuccess) return e;
    }
    return tri_solve(L, T, k + 1, 2 * i, Za, ldz, p, 1);
  }
  if ((e = tri_solve(L, T, k + 1, 2 * i, Za, ldz, p, mode)) != cudaSuccess) return e;
  if (mode == 0) {
    // L: Z_b -= U_b (V_a^T Z_a)
    const int r = L.rV[a];
    if (r > 0) {
      if ((e = gemm(L, L.V(a), L.cap[a], 1, Za, ldz, 0, L.cm, p, r, p, ma, 1.0, 0.0)) != cudaSuccess) return e;
      if ((e = gemm(L, L.U(b), L.cap[b], 0, L.cm, p, 0, Zb, ldz, mb, p, r, -1.0, 1.0)) != cudaSuccess) return e;
    }
  } else {
    // U^T: Z_b -= V_b (U_a^T Z_a)
    const int r = L.rU[a];
    if (r > 0) {
      if ((e = gemm(L, L.U(a), L.cap[a], 1, Za, ldz, 0, L.cm, p, r, p, ma, 1.0, 0.0)) != cudaSuccess) return e;
      if ((e = gemm(L, L.V(b), L.cap[b], 0, L.cm, p, 0, Zb, ldz, mb, p, r, -1.0, 1.0)) != cudaSuccess) return e;
    }
  }
  return tri_solve(L, T, k + 1, 2 * i + 1, Zb, ldz, p, mode);
}

// Subtract G C H^T (G = U_b, H = V_b, C = the small core in L.cm) from the
// HODLR matrix of node b = (kb, ib): the leaves exactly, every block inside
// recompressed.
hodlr_status schur_update(LuState& L, const Tree& T, int kb, int ib, int b) {
  const int mb = T.m(kb, ib), rb0 = T.row0(kb, ib);
  const int s = L.rU[b], t = L.rV[b];
  if (s == 0 || t == 0) return HODLR_OK;
  cudaError_t e;
  // GC = U_b C (mb x t), C (s x t) in L.cm
  if ((e = gemm(L, L.U(b), L.cap[b], 0, L.cm, t, 0, L.gc, t, mb, t, s, 1.0, 0.0)) != cudaSuccess)
    return set_cuda_error(e, "hodlr_lu: Schur product");
  // leaves of b
  std::vector<LeafUpd> lu;
  const int span = 1 << (L.depth - kb);
  for (int j = ib * span; j < (ib + 1) * span; ++j) {
    LeafUpd u;
    u.D = L.D(j);
    u.m = T.m(L.depth, j);
    u.row = T.row0(L.depth, j) - rb0;
    lu.push_back(u);
  }
  if ((e = cudaMemcpyAsync(L.d_lu, lu.data(), lu.size() * sizeof(LeafUpd), cudaMemcpyHostToDevice, L.s)) != cudaSuccess)
    return set_cuda_error(e, "hodlr_lu: leaf list");
  schur_leaf_kernel<<<(unsigned)lu.size(), kLT, 0, L.s>>>(L.d_lu, L.gc, t, L.V(b), L.cap[b], t);
  if ((e = cudaGetLastError()) != cudaSuccess) return set_cuda_error(e, "hodlr_lu: leaf update");
  // blocks (p, p^1) inside b
  std::vector<RcBlock> rc;
  std::vector<int> rc_p;
  size_t wneed = 0;
  for (int k = kb + 1; k <= L.depth; ++k) {
    const int sp = 1 << (k - kb);
    for (int j = ib * sp; j < (ib + 1) * sp; ++j) {
      const int p = node_index(k, j), p1 = node_index(k, j ^ 1);
      RcBlock r;
      memset(&r, 0, sizeof(r));
      r.U = L.U(p);
      r.ldu = L.cap[p];
      r.V = L.V(p1);
      r.ldv = L.cap[p1];
      r.GC = L.gc + (int64_t)(T.row0(k, j) - rb0) * t;
      r.ldgc = t;
      r.H = L.V(b) + (int64_t)(T.row0(k, j ^ 1) - rb0) * L.cap[b];
      r.ldh = L.cap[b];
      r.m1 = T.m(k, j);
      r.m2 = T.m(k, j ^ 1);
      r.r = L.rU[p];
      r.t = t;
      r.cap = std::min(L.cap[p], L.cap[p1]);
      const int w = r.r + t;
      if (w > 512) return set_error(HODLR_EACCURACY, "hodlr_lu: Schur block rank above 512");
      wneed += (size_t)(r.m1 + r.m2) * w + 4 * (size_t)w * w + w;
      rc.push_back(r);
      rc_p.push_back(p);
    }
  }
  if (rc.empty()) return HODLR_OK;
  if (wneed > L.work_n) {
    cudaFree(L.work);
    L.work = nullptr;
    L.work_n = 0;
    if (cudaMalloc(&L.work, wneed * sizeof(double)) != cudaSuccess) return set_error(HODLR_ENOMEM, "hodlr_lu workspace");
    L.work_n = wneed;
  }
  double* wp = L.work;
  for (RcBlock& r : rc) {
    const int w = r.r + r.t;
    r.A = wp;
    wp += (size_t)r.m1 * w;
    r.B = wp;
    wp += (size_t)r.m2 * w;
    r.S = wp;
    wp += 4 * (size_t)w * w + w;
  }
  if ((e = cudaMemcpyAsync(L.d_rc, rc.data(), rc.size() * sizeof(RcBlock), cudaMemcpyHostToDevice, L.s)) != cudaSuccess)
    return set_cuda_error(e, "hodlr_lu: block list");
  recompress_kernel<<<(unsigned)rc.size(), kLT, 0, L.s>>>(L.d_rc, L.eps_lu, L.d_rank, L.d_err);
  if ((e = cudaGetLastError()) != cudaSuccess) return set_cuda_error(e, "hodlr_lu: recompression");
  std::vector<int> rk(rc.size());
  if ((e = cudaMemcpyAsync(rk.data(), L.d_rank, rk.size() * sizeof(int), cudaMemcpyDeviceToHost, L.s)) != cudaSuccess)
    return set_cuda_error(e, "hodlr_lu: ranks");
  if ((e = cudaStreamSynchronize(L.s)) != cudaSuccess) return set_cuda_error(e, "hodlr_lu");
  for (size_t q = 0; q < rc.size(); ++q) {
    const int p = rc_p[q];
    const int p1 = (p % 2 == 0) ? p + 1 : p - 1;   // node_index keeps siblings adjacent (2j, 2j + 1)
    L.rU[p] = rk[q];
    L.rV[p1] = rk[q];
  }
  return HODLR_OK;
}

hodlr_status lu_node(LuState& L, const Tree& T, int k, int i) {
  cudaError_t e;
  if (k == L.depth) {
    leaf_lu_kernel<<<1, kLT, 0, L.s>>>(L.D(i), T.m(k, i), L.d_err);
    if ((e = cudaGetLastError()) != cudaSuccess) return set_cuda_error(e, "hodlr_lu: leaf");
    return HODLR_OK;
  }
  const int a = node_index(k + 1, 2 * i), b = node_index(k + 1, 2 * i + 1);
  const int ma = T.m(k + 1, 2 * i);
  hodlr_status st;
  if ((st = lu_node(L, T, k + 1, 2 * i)) != HODLR_OK) return st;
  // U_a := L_a^{-1} U_a (upper block), V_a := U_a^{-T} V_a (lower block)
  if (L.rU[a] > 0 && (e = tri_solve(L, T, k + 1, 2 * i, L.U(a), L.cap[a], L.rU[a], 0)) != cudaSuccess)
    return set_cuda_error(e, "hodlr_lu: L solve");
  if (L.rV[a] > 0 && (e = tri_solve(L, T, k + 1, 2 * i, L.V(a), L.cap[a], L.rV[a], 2)) != cudaSuccess)
    return set_cuda_error(e, "hodlr_lu: U^T solve");
  // C = V_a^T U_a (rV_a x rU_a = rU_b x rV_b)
  if (L.rV[a] > 0 && L.rU[a] > 0) {
    if ((e = gemm(L, L.V(a), L.cap[a], 1, L.U(a), L.cap[a], 0, L.cm, L.rU[a], L.rV[a], L.rU[a], ma, 1.0, 0.0)) !=
        cudaSuccess)
      return set_cuda_error(e, "hodlr_lu: core");
    if ((st = schur_update(L, T, k + 1, 2 * i + 1, b)) != HODLR_OK) return st;
  }
  return lu_node(L, T, k + 1, 2 * i + 1);
}

cudaError_t lu_apply(LuState& L, const Tree& T, double* Z, int64_t ldz, int p) {
  cudaError_t e = tri_solve(L, T, 0, 0, Z, ldz, p, 0);
  if (e != cudaSuccess) return e;
  return tri_solve(L, T, 0, 0, Z, ldz, p, 1);
}

hodlr_status check_err(LuState& L) {
  int err = 0;
  cudaError_t e = cudaMemcpyAsync(&err, L.d_err, sizeof(int), cudaMemcpyDeviceToHost, L.s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(L.s);
  if (e != cudaSuccess) return set_cuda_error(e, "hodlr_lu");
  if (err == 1) return set_error(HODLR_ESINGULAR, "hodlr_lu: zero pivot in a leaf factorization");
  if (err == 2) return set_error(HODLR_EACCURACY, "hodlr_lu: a Schur block needs more columns than its capacity");
  return HODLR_OK;
}

}  // namespace
}  // namespace hodlr

using namespace hodlr;

extern "C" hodlr_status hodlr_lu(hodlr_t h, double eps_lu, void* stream) {
  if (!h) return set_error(HODLR_EINVAL, "null handle");
  if (!(eps_lu >= 0.0) || eps_lu >= 1.0) return set_error(HODLR_EINVAL, "eps_lu must be in [0, 1)");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_cuda_error(e, "cudaGetDevice");
  if (dev != h->device) return set_error(HODLR_EINVAL, "the current device differs from the handle's device");
  if (h->lu) {
    lu_destroy(h->lu);
    h->lu = nullptr;
  }
  LuState* Lp = new LuState();
  h->lu = Lp;
  LuState& L = *Lp;
  L.s = (cudaStream_t)stream;
  L.depth = h->depth;
  L.n = h->n;
  L.eps_lu = eps_lu;
  const int nnodes = (int)h->nodes.size(), nleaves = (int)h->leaves.size();
  // capacities: the stored rank, room for growth by the recompression
  int rmax = 0;
  for (const NodeDev& nd : h->nodes) rmax = std::max(rmax, std::max(nd.rU, nd.rV));
  const int grow = std::max(64, 4 * rmax + 32);
  L.rU.resize(nnodes);
  L.rV.resize(nnodes);
  L.cap.resize(nnodes);
  L.offU.resize(nnodes);
  L.offV.resize(nnodes);
  L.offD.resize(nleaves);
  int64_t off = 0;
  for (int q = 0; q < nnodes; ++q) {
    const NodeDev& nd = h->nodes[q];
    L.rU[q] = nd.rU;
    L.rV[q] = nd.rV;
    L.cap[q] = std::max(std::min(nd.m, grow), std::max(nd.rU, nd.rV));
    L.offU[q] = off;
    off += (int64_t)nd.m * L.cap[q];
    L.offV[q] = off;
    off += (int64_t)nd.m * L.cap[q];
  }
  for (int l = 0; l < nleaves; ++l) {
    L.offD[l] = off;
    off += (int64_t)h->leaves[l].m * h->leaves[l].m;
  }
  int tmax = 0, mmax = 0;
  for (int q = 0; q < nnodes; ++q) {
    tmax = std::max(tmax, L.cap[q]);
    mmax = std::max(mmax, h->nodes[q].m);
  }
  int max_blocks = 1;
  for (int k = 1; k <= h->depth; ++k) max_blocks += 1 << k;
  if (cudaMalloc(&L.pool, sizeof(double) * std::max<int64_t>(off, 1)) != cudaSuccess ||
      cudaMalloc(&L.gc, sizeof(double) * (size_t)std::max(mmax, 1) * std::max(tmax, 1)) != cudaSuccess ||
      cudaMalloc(&L.cm, sizeof(double) * (size_t)std::max(tmax, 1) * std::max(tmax, kSolveCols)) != cudaSuccess ||
      cudaMalloc(&L.d_rc, sizeof(RcBlock) * max_blocks) != cudaSuccess ||
      cudaMalloc(&L.d_rank, sizeof(int) * max_blocks) != cudaSuccess ||
      cudaMalloc(&L.d_lu, sizeof(LeafUpd) * std::max(nleaves, 1)) != cudaSuccess ||
      cudaMalloc(&L.d_err, sizeof(int)) != cudaSuccess) {
    lu_destroy(h->lu);
    h->lu = nullptr;
    return set_error(HODLR_ENOMEM, "hodlr_lu: factor storage");
  }
  // the stored generators and leaves, decoded to fp64, into the factor pool
  {
    double* stage = nullptr;
    PackTask* tasks = nullptr;
    if (cudaMalloc(&stage, sizeof(double) * std::max<int64_t>(h->st_count, 1)) != cudaSuccess ||
        cudaMalloc(&tasks, std::max<size_t>(h->tasks.size(), 1) * sizeof(PackTask)) != cudaSuccess) {
      cudaFree(stage);
      lu_destroy(h->lu);
      h->lu = nullptr;
      return set_error(HODLR_ENOMEM, "hodlr_lu: staging");
    }
    e = cudaMemcpyAsync(tasks, h->tasks.data(), h->tasks.size() * sizeof(PackTask), cudaMemcpyHostToDevice, L.s);
    if (e == cudaSuccess) e = launch_unpack(h->d_pool, tasks, (int)h->tasks.size(), stage, L.s);
    for (int q = 0; q < nnodes && e == cudaSuccess; ++q) {
      const NodeDev& nd = h->nodes[q];
      if (nd.rU) {
        copy2d_kernel<<<(unsigned)cdiv((int64_t)nd.m * nd.rU, 256), 256, 0, L.s>>>(stage + h->st_U[q], nd.rU, L.U(q),
                                                                                    L.cap[q], nd.m, nd.rU);
      }
      if (nd.rV) {
        copy2d_kernel<<<(unsigned)cdiv((int64_t)nd.m * nd.rV, 256), 256, 0, L.s>>>(stage + h->st_V[q], nd.rV, L.V(q),
                                                                                    L.cap[q], nd.m, nd.rV);
      }
      e = cudaGetLastError();
    }
    for (int l = 0; l < nleaves && e == cudaSuccess; ++l)
      e = cudaMemcpyAsync(L.D(l), stage + h->st_D[l], sizeof(double) * h->leaves[l].m * h->leaves[l].m,
                          cudaMemcpyDeviceToDevice, L.s);
    if (e == cudaSuccess) e = cudaMemsetAsync(L.d_err, 0, sizeof(int), L.s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(L.s);
    cudaFree(stage);
    cudaFree(tasks);
    if (e != cudaSuccess) return set_cuda_error(e, "hodlr_lu: decode");
  }
  Tree T{h};
  hodlr_status st = lu_node(L, T, 0, 0);
  if (st == HODLR_OK) st = check_err(L);
  L.factored = st == HODLR_OK;
  return st;
}

extern "C" hodlr_status hodlr_lu_solve(hodlr_t h, int32_t nrhs, const double* B, int64_t ldb, double* X, int64_t ldx,
                                       void* stream) {
  if (!h) return set_error(HODLR_EINVAL, "null handle");
  if (!h->lu || !h->lu->factored) return set_error(HODLR_ENOTFACTORED, "hodlr_lu_solve before hodlr_lu");
  if (nrhs < 0) return set_error(HODLR_EINVAL, "nrhs < 0");
  if (nrhs == 0) return HODLR_OK;
  if (!B || !X) return set_error(HODLR_EINVAL, "null B/X");
  if (ldb < nrhs || ldx < nrhs) return set_error(HODLR_EINVAL, "leading dimension < nrhs");
  LuState& L = *h->lu;
  L.s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (X != B) e = cudaMemcpy2DAsync(X, ldx * sizeof(double), B, ldb * sizeof(double), nrhs * sizeof(double), h->n,
                                    cudaMemcpyDeviceToDevice, L.s);
  // columns in batches that the solves' small temporaries hold
  const int pb = std::max(1, kSolveCols);
  for (int c0 = 0; c0 < nrhs && e == cudaSuccess; c0 += pb) {
    Tree T{h};
    e = lu_apply(L, T, X + c0, ldx, std::min(pb, nrhs - c0));
  }
  return e == cudaSuccess ? HODLR_OK : set_cuda_error(e, "hodlr_lu_solve");
}

namespace hodlr {
namespace {

// GMRES for one column, left preconditioned by the LU factors, modified
// Gram-Schmidt Arnoldi and Givens rotations on the host (the oracle's
// algorithm); the matrix products and preconditioner solves on the device.
// x (device, stride ldx) starts at zero; stops when the preconditioned
// residual is at most tol times its initial norm.
hodlr_status gmres_col(hodlr_t h, LuState& L, const Tree& T, const double* b, int64_t ldb, double* x, int64_t ldx,
                       double tol, int restart, int max_steps, int* steps_out) {
  const int n = h->n;
  double* Q = L.vec;                          // n x (restart + 1), column j at Q + j * n
  double* w = Q + (size_t)n * (restart + 1);  // n
  double* sc = w + n;                         // device scalars
  cudaStream_t s = L.s;
  const unsigned nb = (unsigned)cdiv(n, 256);
  auto dot = [&](const double* a, int64_t la, const double* c, int64_t lc, double* out) -> hodlr_status {
    dot_kernel<<<1, 1024, 0, s>>>(n, a, la, c, lc, sc);
    cudaError_t e = cudaMemcpyAsync(out, sc, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? HODLR_OK : set_cuda_error(e, "hodlr_solve: dot");
  };
  // r = M^{-1} (b - A x) into column 0 of Q (x = 0 at the start)
  auto resid = [&](double* dst) -> hodlr_status {
    hodlr_status st = hodlr_matvec(h, 1, x, ldx, w, 1, HODLR_FP64, s);
    if (st != HODLR_OK) return st;
    axpby_kernel<<<nb, 256, 0, s>>>(n, 1.0, b, ldb, -1.0, w, 1);
    cudaError_t e = lu_apply(L, T, w, 1, 1);
    if (e != cudaSuccess) return set_cuda_error(e, "hodlr_solve: preconditioner");
    axpby_kernel<<<nb, 256, 0, s>>>(n, 1.0, w, 1, 0.0, dst, 1);
    return HODLR_OK;
  };
  hodlr_status st;
  axpby_kernel<<<nb, 256, 0, s>>>(n, 0.0, b, ldb, 0.0, x, ldx);
  if ((st = resid(Q)) != HODLR_OK) return st;
  double beta0 = 0.0;
  if ((st = dot(Q, 1, Q, 1, &beta0)) != HODLR_OK) return st;
  beta0 = std::sqrt(beta0);
  int steps = 0;
  if (beta0 == 0.0) {
    *steps_out = 0;
    return HODLR_OK;
  }
  double beta = beta0;
  std::vector<double> Hh((size_t)(restart + 1) * restart), cs(restart), sn(restart), g(restart + 1);
  while (steps < max_steps) {
    std::fill(Hh.begin(), Hh.end(), 0.0);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    axpby_kernel<<<nb, 256, 0, s>>>(n, 1.0 / beta, Q, 1, 0.0, Q, 1);
    int j = 0, kdim = 0;
    for (j = 0; j < restart; ++j) {
      double* qj = Q + (size_t)j * n;
      double* qn = Q + (size_t)(j + 1) * n;
      if ((st = hodlr_matvec(h, 1, qj, 1, w, 1, HODLR_FP64, s)) != HODLR_OK) return st;
      cudaError_t e = lu_apply(L, T, w, 1, 1);
      if (e != cudaSuccess) return set_cuda_error(e, "hodlr_solve: preconditioner");
      for (int i = 0; i <= j; ++i) {
        double hij;
        if ((st = dot(Q + (size_t)i * n, 1, w, 1, &hij)) != HODLR_OK) return st;
        Hh[(size_t)i * restart + j] = hij;
        axpby_kernel<<<nb, 256, 0, s>>>(n, -hij, Q + (size_t)i * n, 1, 1.0, w, 1);
      }
      double nw2;
      if ((st = dot(w, 1, w, 1, &nw2)) != HODLR_OK) return st;
      const double hn = std::sqrt(nw2);
      Hh[(size_t)(j + 1) * restart + j] = hn;
      axpby_kernel<<<nb, 256, 0, s>>>(n, hn > 0.0 ? 1.0 / hn : 0.0, w, 1, 0.0, qn, 1);
      for (int i = 0; i < j; ++i) {
        const double a = Hh[(size_t)i * restart + j], c = Hh[(size_t)(i + 1) * restart + j];
        Hh[(size_t)i * restart + j] = cs[i] * a + sn[i] * c;
        Hh[(size_t)(i + 1) * restart + j] = -sn[i] * a + cs[i] * c;
      }
      const double a = Hh[(size_t)j * restart + j], c = Hh[(size_t)(j + 1) * restart + j];
      const double den = std::hypot(a, c);
      cs[j] = den > 0.0 ? a / den : 1.0;
      sn[j] = den > 0.0 ? c / den : 0.0;
      Hh[(size_t)j * restart + j] = den;
      Hh[(size_t)(j + 1) * restart + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++steps;
      kdim = j + 1;
      if (std::fabs(g[j + 1]) <= tol * beta0 || steps >= max_steps || hn == 0.0) break;
    }
    // y = H^{-1} g (upper triangular kdim x kdim), x += Q y
    std::vector<double> y(kdim);
    for (int i = kdim - 1; i >= 0; --i) {
      double v = g[i];
      for (int l = i + 1; l < kdim; ++l) v -= Hh[(size_t)i * restart + l] * y[l];
      y[i] = Hh[(size_t)i * restart + i] != 0.0 ? v / Hh[(size_t)i * restart + i] : 0.0;
    }
    for (int i = 0; i < kdim; ++i) axpby_kernel<<<nb, 256, 0, s>>>(n, y[i], Q + (size_t)i * n, 1, 1.0, x, ldx);
    if ((st = resid(Q)) != HODLR_OK) return st;
    double b2;
    if ((st = dot(Q, 1, Q, 1, &b2)) != HODLR_OK) return st;
    beta = std::sqrt(b2);
    if (beta <= tol * beta0 || beta == 0.0) break;
  }
  *steps_out = steps;
  return HODLR_OK;
}

}  // namespace
}  // namespace hodlr

extern "C" hodlr_status hodlr_solve(hodlr_t h, int32_t nrhs, const double* B, int64_t ldb, double* X, int64_t ldx,
                                    double tol, int32_t max_it, hodlr_solve_stats* stats, void* stream) {
  if (!h) return set_error(HODLR_EINVAL, "null handle");
  if (!h->lu || !h->lu->factored) return set_error(HODLR_ENOTFACTORED, "hodlr_solve before hodlr_lu");
  if (h->work != HODLR_FP64) return set_error(HODLR_EINVAL, "hodlr_solve needs fp64 working precision (fp64 residuals)");
  if (nrhs < 0 || max_it < 0) return set_error(HODLR_EINVAL, "nrhs < 0 or max_it < 0");
  if (!(tol > 0.0)) return set_error(HODLR_EINVAL, "tol must be positive");
  if (nrhs == 0) return HODLR_OK;
  if (!B || !X) return set_error(HODLR_EINVAL, "null B/X");
  if (ldb < nrhs || ldx < nrhs) return set_error(HODLR_EINVAL, "leading dimension < nrhs");
  LuState& L = *h->lu;
  L.s = (cudaStream_t)stream;
  const int n = h->n;
  const int restart = 60;
  const size_t need = (size_t)n * (restart + 2) + 16 + (size_t)n * (2 * (size_t)nrhs + 1);
  if (need > L.vec_n) {
    cudaFree(L.vec);
    L.vec = nullptr;
    L.vec_n = 0;
    if (cudaMalloc(&L.vec, need * sizeof(double)) != cudaSuccess) return set_error(HODLR_ENOMEM, "hodlr_solve vectors");
    L.vec_n = need;
  }
  double* R = L.vec + (size_t)n * (restart + 2) + 16;   // n x nrhs residual
  double* Dx = R + (size_t)n * nrhs;                    // n x nrhs correction
  double* sc = L.vec + (size_t)n * (restart + 2);
  cudaStream_t s = L.s;
  Tree T{h};
  const double normA = std::sqrt(std::max(h->info.norm2_all, 0.0));
  auto fro = [&](const double* A, int64_t lda, double* out) -> hodlr_status {
    double acc = 0.0;
    for (int c = 0; c < nrhs; ++c) {
      dot_kernel<<<1, 1024, 0, s>>>(n, A + c, lda, A + c, lda, sc);
      double v = 0.0;
      cudaError_t e = cudaMemcpyAsync(&v, sc, sizeof(double), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return set_cuda_error(e, "hodlr_solve: norm");
      acc += v;
    }
    *out = std::sqrt(acc);
    return HODLR_OK;
  };
  // X_0 = (LU)^{-1} B
  hodlr_status st = hodlr_lu_solve(h, nrhs, B, ldb, X, ldx, stream);
  if (st != HODLR_OK) return st;
  double be = 0.0;
  int it = 0, inner_total = 0;
  for (;; ++it) {
    // R = B - H X (fp64 product), backward error ||R||_F / (||H||_F ||X||_F)
    if ((st = hodlr_matvec(h, nrhs, X, ldx, R, nrhs, HODLR_FP64, stream)) != HODLR_OK) return st;
    for (int c = 0; c < nrhs; ++c) axpby_kernel<<<(unsigned)cdiv(n, 256), 256, 0, s>>>(n, 1.0, B + c, ldb, -1.0, R + c, nrhs);
    double nr, nx;
    if ((st = fro(R, nrhs, &nr)) != HODLR_OK) return st;
    if ((st = fro(X, ldx, &nx)) != HODLR_OK) return st;
    be = nx > 0.0 && normA > 0.0 ? nr / (normA * nx) : (nr == 0.0 ? 0.0 : INFINITY);
    if (be <= tol || it >= max_it) break;
    // correction: GMRES on H D = R per column, preconditioned, to 1e-4
    int inner_max = 0;
    for (int c = 0; c < nrhs; ++c) {
      int steps = 0;
      if ((st = gmres_col(h, L, T, R + c, nrhs, Dx + c, nrhs, 1e-4, restart, 600, &steps)) != HODLR_OK) return st;
      inner_max = std::max(inner_max, steps);
    }
    inner_total += inner_max;
    for (int c = 0; c < nrhs; ++c) axpby_kernel<<<(unsigned)cdiv(n, 256), 256, 0, s>>>(n, 1.0, Dx + c, nrhs, 1.0, X + c, ldx);
  }
  if (stats) {
    stats->iterations = it;
    stats->gmres_steps = inner_total;
    stats->backward_error = be;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_cuda_error(e, "hodlr_solve");
  return be <= tol ? HODLR_OK : set_error(HODLR_EACCURACY, "hodlr_solve: tolerance not reached within max_it");
}

extern "C" hodlr_status hodlr_lu_export(hodlr_t h, int32_t* ranks_u, int32_t* ranks_v, double* const* U,
                                        double* const* V, double* const* D, void* stream) {
  if (!h) return set_error(HODLR_EINVAL, "null handle");
  if (!h->lu || !h->lu->factored) return set_error(HODLR_ENOTFACTORED, "hodlr_lu_export before hodlr_lu");
  LuState& L = *h->lu;
  cudaStream_t s = (cudaStream_t)stream;
  const int nnodes = (int)h->nodes.size();
  for (int q = 0; q < nnodes; ++q) {
    if (ranks_u) ranks_u[q] = L.rU[q];
    if (ranks_v) ranks_v[q] = L.rV[q];
  }
  cudaError_t e = cudaSuccess;
  for (int q = 0; q < nnodes && e == cudaSuccess; ++q) {
    const int m = h->nodes[q].m;
    if (U && U[q] && L.rU[q])
      e = cudaMemcpy2DAsync(U[q], L.rU[q] * sizeof(double), L.U(q), L.cap[q] * sizeof(double), L.rU[q] * sizeof(double),
                            m, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && V && V[q] && L.rV[q])
      e = cudaMemcpy2DAsync(V[q], L.rV[q] * sizeof(double), L.V(q), L.cap[q] * sizeof(double), L.rV[q] * sizeof(double),
                            m, cudaMemcpyDeviceToHost, s);
  }
  for (size_t l = 0; l < h->leaves.size() && e == cudaSuccess; ++l)
    if (D && D[l])
      e = cudaMemcpyAsync(D[l], L.D((int)l), sizeof(double) * h->leaves[l].m * h->leaves[l].m, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? HODLR_OK : set_cuda_error(e, "hodlr_lu_export");
}
