/*
 * hodlr.h -- C ABI of the GB300 (sm_103a) adaptive-precision HODLR library.
 *
 * The method is that of Carson, Chen and Liu, "Mixed Precision HODLR
 * Matrices" (arXiv 2407.21637).  A HODLR matrix on the cluster tree of
 * Def. 2.1 stores, for every level k = 1..depth and every sibling pair of
 * nodes (i, i^1), the low-rank generators of the off-diagonal block
 * H(I_i, I_{i^1}) ~ U_i V_{i^1}^T (eq. (2.1), eq. (3.1)), and the dense leaf
 * blocks D_i.  Algorithm 3.2 stores each generator in the precision its
 * level (or block) admits; Algorithm 3.3 multiplies by the result.
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 * - Indices are in tree order: the caller has already permuted its points.
 * - Tree: the root is {0..n-1}; a node of size m splits into a left child of
 *   size ceil(m/2) and a right child of size m - ceil(m/2) (the practical
 *   split of Sect. 4).  Level k has 2^k nodes numbered i = 0..2^k-1 from
 *   left to right; the sibling of node i is i^1.
 * - Node tables ("per node") list the nodes of level 1, then level 2, ...,
 *   then level depth: 2^(depth+1) - 2 entries; node (k, i) is entry
 *   2^k - 2 + i.
 * - Matrices passed as host arrays are fp64, row-major, dense.
 * - X and B of a product are DEVICE arrays, row-major (n, nrhs) with a
 *   leading dimension in elements; the right-hand sides are the fastest
 *   index.  They are owned by the caller.  The library owns the handle and
 *   every byte it allocates; hodlr_destroy frees them.
 * - Every call that launches GPU work takes a CUDA stream (cudaStream_t
 *   passed as void*; NULL = legacy default stream), enqueues on it and
 *   returns without waiting unless stated otherwise.
 * - Errors are returned as hodlr_status.  Arguments are validated before
 *   anything is launched; nothing aborts or exits, and there is no CPU
 *   fallback: a call that cannot run on the GPU returns an error.
 * - A handle may be used from one host thread at a time.
 */
#ifndef HODLR_H
#define HODLR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hodlr_s* hodlr_t;

typedef enum {
  HODLR_OK = 0,
  HODLR_EINVAL = 1,       /* bad argument (null pointer, size, rank, stride, precision) */
  HODLR_ENOMEM = 2,       /* device or host allocation failed */
  HODLR_ECUDA = 3,        /* a CUDA runtime call failed */
  HODLR_ETIMEOUT = 4,     /* a device-side bounded wait gave up */
  HODLR_ENOTFACTORED = 5, /* solve before factorisation */
  HODLR_ESINGULAR = 6,    /* zero pivot */
  HODLR_EACCURACY = 7     /* a requested tolerance could not be met */
} hodlr_status;

/* Storage / arithmetic formats (Table 1.1; E5M2 is the paper's q52, E4M3 is
 * the OCP FP8 "fn" format).  The value is the bit index used in tier_mask. */
typedef enum {
  HODLR_FP64 = 0,
  HODLR_FP32 = 1,
  HODLR_FP16 = 2,
  HODLR_BF16 = 3,
  HODLR_E4M3 = 4,
  HODLR_E5M2 = 5
} hodlr_prec;

/* Options of the adaptive-precision format (Algorithm 3.2 inputs). */
typedef struct {
  double eps;          /* truncation parameter epsilon of Def. 2.3 (0 < eps < 1) */
  int32_t work;        /* working precision u: HODLR_FP64 or HODLR_FP32.  The leaves
                          are stored in it and the products are computed in it
                          (Algorithm 3.2 step "store in u", Algorithm 3.3). */
  uint32_t tier_mask;  /* the set calU of available storage formats: bit p set for
                          hodlr_prec p.  The working precision is always added. */
  int32_t per_block;   /* 0: xi_k = max over the level (Algorithm 3.2 as printed);
                          1: xi_ij per block (same Thm 3.1 bound) */
  int32_t max_nrhs;    /* widest product one launch sequence handles (scratch size);
                          wider products are split into column batches.  0 -> 64 */
} hodlr_opts;

/* Summary of a stored HODLR matrix.  Arrays are indexed by level k = 1..depth
 * (entry 0 unused); depth <= HODLR_MAX_DEPTH. */
#define HODLR_MAX_DEPTH 24
typedef struct {
  int32_t n, depth, work, per_block;
  int32_t max_rank;                 /* largest off-diagonal rank */
  int32_t n_blocks;                 /* 2^(depth+1) - 2 off-diagonal blocks */
  int64_t factor_bytes;             /* algorithmic bytes of U and V (no padding) */
  int64_t u_bytes, v_bytes;         /* the U and the V part of factor_bytes */
  int64_t leaf_bytes;               /* algorithmic bytes of the leaves */
  int64_t scale_bytes;              /* 8 bytes per block with a power-of-two scale */
  int64_t device_bytes;             /* bytes the handle holds on the device */
  int64_t bytes_per_tier[6];        /* factor bytes per hodlr_prec */
  double norm2_all;                 /* ||H||_F^2 estimate used for xi (from the factors) */
  double xi[HODLR_MAX_DEPTH + 1];   /* xi_k (per_block: the level maximum of xi_ij) */
  double u_prime[HODLR_MAX_DEPTH + 1]; /* u'_k = eps / (2^{k/2} xi_k) */
  int32_t level_tier[HODLR_MAX_DEPTH + 1]; /* u_k as hodlr_prec (per_block: most precise
                                              tier used on the level) */
} hodlr_info_t;

/* ---------------------------------------------------------------------- */
/* hodlr_import -- store given fp64 generators in the adaptive-precision
 * format (Algorithm 3.2, steps after the compression).
 *
 *  n, depth      matrix size and tree depth; 1 <= 2^depth <= n, depth <= 24.
 *  ranks         host, per node: ranks[node(k,i)] = rank of block (i, i^1).
 *  U             host, per node: U[node(k,i)] -> m_i x ranks[node(k,i)] fp64,
 *                row-major; the left generator of block (i, i^1), with
 *                orthonormal columns (eq. (3.1)).  May be NULL when the rank is 0.
 *  V             host, per node: V[node(k,j)] -> m_j x ranks[node(k,j^1)] fp64,
 *                row-major; the right generator of block (j^1, j), so that
 *                H(I_{j^1}, I_j) ~ U[node(k,j^1)] V[node(k,j)]^T.
 *  D             host, per leaf i = 0..2^depth-1: m_i x m_i fp64 row-major.
 *  opts          see hodlr_opts.
 *  stream        work is enqueued here; the call synchronises this stream
 *                before returning (it reads the block norms back).
 *  out           receives the new handle (unchanged on error).
 *
 * The precision of every block is chosen on the device-computed norms of the
 * fp64 generators: ||U_i V_{i^1}^T||_F = ||V_{i^1}||_F because U_i has
 * orthonormal columns, and ||H||_F^2 is estimated by the sum of the block
 * norms plus the leaves' (the O(eps) estimate allowed in Sect. 3.2).
 * u'_k = eps / (2^{k/2} xi_k); u_k = the largest available u* <= u'_k, or the
 * most precise available format when none qualifies.  fp16/E4M3/E5M2
 * generators carry a per-block power-of-two scale s = 2^floor(log2(x_max /
 * (2 amax))); rounding is to nearest, ties to even.
 * Errors: HODLR_EINVAL for bad sizes/ranks/precisions, HODLR_ENOMEM,
 * HODLR_ECUDA. */
hodlr_status hodlr_import(int32_t n, int32_t depth, const int32_t* ranks,
                          const double* const* U, const double* const* V,
                          const double* const* D, const hodlr_opts* opts,
                          void* stream, hodlr_t* out);

/* Kernel matrix A_ij = f(x_i, x_j) + diag * delta_ij (eq. (4.1) kernels and
 * the synthetic workloads).  f at i == j is f(0) where finite, else 0.
 *   kind 0  f = 1/(r + c)           kind 1  f = exp(-r^2 / len2)
 *   kind 2  f = log(r + c)          kind 3  f = 1/(x_i - x_j)  (dim 1 only)
 * r = ||x_i - x_j||_2 over dim in {1, 2, 3} coordinates. */
typedef struct {
  int32_t kind, dim;
  double c, len2, diag;
} hodlr_kernel;

/* Randomized range finder settings of hodlr_build. */
typedef struct {
  int32_t sketch;      /* first sketch size per block (0 -> 16) */
  int32_t max_sketch;  /* largest sketch size, <= 64 (0 -> 64) */
  uint64_t seed;       /* seed of the Gaussian test matrix */
  const int32_t* node_sketch;  /* NULL, or host int32[2^(depth+1) - 2]: the
                                  first sketch of block (k, i) at node
                                  2^k - 2 + i (clamped to [1, max_sketch]),
                                  e.g. from a rank predictor; a block whose
                                  sketch falls short is redone with twice its
                                  sketch as always */
} hodlr_build_opts;

/* hodlr_build -- construct the adaptive-precision HODLR matrix of a kernel
 * matrix on the GPU (Algorithm 3.2): every off-diagonal block is compressed
 * to relative Frobenius accuracy eps (Def. 2.3) by a randomized range finder
 * whose matrix entries are generated in registers (never stored): sketch
 * Y = A_b Omega, Q = orth(Y) (classical Gram-Schmidt applied twice),
 * B = Q^T A_b, the sketch residual ||A_b - Q Q^T A_b||_F computed from
 * regenerated entries, and a one-sided Jacobi SVD of B's triangular factor;
 * the rank is the smallest r whose SVD tail plus sketch residual is within
 * eps ||A_b||_F.  A block whose sketch residual exceeds a quarter of that
 * budget is redone with a doubled sketch.  The block norms ||A_b||_F and
 * ||A||_F of Algorithm 3.2 are exact (computed from the generated entries).
 * Then the precision rule and storage of hodlr_import apply.
 *
 *  points  device, (n, kernel->dim) fp64 row-major, in tree order.
 *  bopts   may be NULL (defaults).
 *  stream  used for all work; the call synchronises it.
 * Returns HODLR_EACCURACY (with a valid handle in *out) when some block still
 * exceeded its budget at the largest sketch; its rank is then the sketch
 * size.  Other errors leave *out unchanged. */
hodlr_status hodlr_build(int32_t n, int32_t depth, const hodlr_kernel* kernel,
                         const double* points, const hodlr_opts* opts,
                         const hodlr_build_opts* bopts, void* stream, hodlr_t* out);

/* hodlr_build_stats -- how the last hodlr_build of this handle went:
 * rounds of the range finder, blocks redone with a larger sketch (summed over
 * the rounds after the first), and the sum over rounds of the sketch columns
 * of the blocks in the round.  Any output may be NULL; zeros for a handle
 * from hodlr_import or hodlr_load. */
hodlr_status hodlr_build_stats(hodlr_t h, int32_t* rounds, int32_t* redone, int64_t* sketch_cols);

/* hodlr_export -- read the stored generators back, decoded to fp64 (the
 * values Algorithm 3.3 multiplies by: stored / scale).  Same layouts as
 * hodlr_import; any of U, V, D may be NULL to skip it.  Synchronous. */
hodlr_status hodlr_export(hodlr_t h, double* const* U, double* const* V,
                          double* const* D, void* stream);

/* hodlr_matvec -- B = H-hat X by Algorithm 3.3 (HODLR_MATVEC), all levels
 * and the leaves, for nrhs right-hand sides.
 *
 *  X       device, (n, nrhs) row-major, leading dimension ldx >= nrhs,
 *          element type = the working precision (double for HODLR_FP64,
 *          float for HODLR_FP32).
 *  B       device, (n, nrhs) row-major, ldb >= nrhs, same type; overwritten.
 *          B must not overlap X.
 *  xb_prec the element type of X and B; must equal the handle's working
 *          precision (HODLR_EINVAL otherwise).
 * Low-precision generators are cast to the working precision as they are
 * loaded (Sect. 3.3); every product and sum is in the working precision.
 * Each output entry is written exactly once, by a fixed summation order, so
 * results are bitwise reproducible run to run.  nrhs = 0 is a no-op.
 * Calls on one handle must not overlap in time (they share its scratch);
 * enqueue them on one stream.  Errors: HODLR_EINVAL, HODLR_ECUDA. */
hodlr_status hodlr_matvec(hodlr_t h, int32_t nrhs, const void* X, int64_t ldx,
                          void* B, int64_t ldb, int32_t xb_prec, void* stream);

/* hodlr_matvec_noalloc -- the same product as hodlr_matvec, for callers that
 * cannot allocate device memory when they multiply: for example a process
 * whose device memory is already fully reserved by another allocator (a
 * framework's caching allocator or a pre-partitioned pool), or code on a
 * latency-critical path that must not enter the driver's allocator.  The
 * paper has no counterpart; this is a library convenience.
 *
 * It allocates nothing (no cudaMalloc, cudaFree or allocating library call)
 * and does not use the handle's own scratch: its scratch is one 256 KiB
 * device array inside this library, which every GPU that loads the library
 * holds until the process exits.  Arguments and results are those of
 * hodlr_matvec.  It always runs the CUDA-core product, in batches of columns
 * that fit the array (at most as many as hodlr_matvec takes per launch).
 * Where hodlr_matvec runs the same kernel with the same batches (fp32 work
 * with fewer than 16 columns, fp64 work with one column) and the array
 * holds a whole batch, B is bitwise the same; other products (fp32 with 16
 * or more columns, which hodlr_matvec runs on the tensor cores, fp64 with
 * more columns, which it runs on its two-barrier kernel, and products split
 * into narrower batches) agree within the rounding bound of the products.  A matrix whose
 * per-column scratch (its partial V^T X sums: one value per rank column, per
 * node and per SM that holds rows of the node) does not fit at all, or
 * whose ranks are too large for the streamed product's shared-memory stages
 * (hodlr_matvec then takes its other CUDA-core kernel), is rejected with
 * HODLR_EINVAL before anything is enqueued.
 *
 * The current device must be the handle's device (HODLR_EINVAL otherwise):
 * the array's device address is looked up on the current device on every
 * call.  Every call on every handle shares the array and the array keeps
 * the last call's contents: the call clears what must start at zero itself,
 * and calls that overlap in time on the GPU (different streams, threads or
 * handles) race on the array and must be serialised by the caller. */
hodlr_status hodlr_matvec_noalloc(hodlr_t h, int32_t nrhs, const void* X, int64_t ldx,
                                  void* B, int64_t ldb, int32_t xb_prec, void* stream);

/* hodlr_save -- write the stored matrix to `path`: sizes and options, every
 * block's rank, format and power-of-two scales, the hodlr_info_t summary and
 * the stored generators and leaves decoded to fp64 (exact).  Host byte order;
 * the file is meant for the same library on the same kind of host.  Waits
 * for `stream`.  Errors: HODLR_EINVAL (null arguments, file not writable),
 * HODLR_ENOMEM, HODLR_ECUDA. */
hodlr_status hodlr_save(hodlr_t h, const char* path, void* stream);

/* hodlr_load -- a new handle from a hodlr_save file, stored exactly as the
 * saved one (the same formats and scales, bitwise the same stored values, so
 * bitwise the same products; the precision rule is not applied again).  The
 * file is checked (magic, version, sizes, formats) before any device work.
 * Waits for `stream`.  Errors: HODLR_EINVAL (unreadable, truncated or corrupt
 * file), HODLR_ENOMEM, HODLR_ECUDA. */
hodlr_status hodlr_load(const char* path, void* stream, hodlr_t* out);

/* hodlr_sync_status -- wait for `stream`, then report whether a kernel of
 * this handle gave up on a device-side wait since the last check.  Every
 * wait in the library's kernels (a grid barrier, an mbarrier of a copy or of
 * the tensor cores) is bounded: after two seconds the kernel records a code
 * in the handle's device error word, finishes without further waiting and
 * leaves the context usable; the results of that call are then undefined.
 * Returns HODLR_ETIMEOUT (and clears the word; hodlr_last_error names the
 * code) when a wait gave up, HODLR_OK otherwise; HODLR_ECUDA when the
 * stream reports an error. */
hodlr_status hodlr_sync_status(hodlr_t h, void* stream);

/* hodlr_debug_stall_next -- test hook for the timeout path: the next
 * hodlr_matvec call on this handle launches its first product kernel with
 * grid-barrier targets that are never reached, so every CTA's barrier waits
 * give up after their two-second limit (about four seconds in all) and
 * hodlr_sync_status then returns HODLR_ETIMEOUT.  Nothing faults and no
 * memory outside the call's own buffers is touched; later calls are
 * unaffected. */
hodlr_status hodlr_debug_stall_next(hodlr_t h);

/* hodlr_profile -- enable (1) or disable (0) CUDA-event timing of the
 * kernels launched by the following hodlr_matvec calls on this handle (events
 * are recorded on the call's stream around each kernel of its last column
 * batch; recording costs a few microseconds of host time per call). */
hodlr_status hodlr_profile(hodlr_t h, int32_t enable);

/* hodlr_profile_read -- device time in ms of the last column batch of the
 * last profiled hodlr_matvec call.  On the CUDA cores alone (fewer than 16
 * columns, or fp64 work): ms[0] = the product kernel (all of Algorithm 3.3 in
 * one persistent launch), ms[1] = 0.  With the tensor cores (fp32 work, 16
 * or more columns): ms[0] = the tensor-core kernel (leaf products D_i X and
 * V_j^T X of the fp32 chunks), ms[1] = the product kernel that follows (the
 * other chunks, the node reductions and U Y).  count >= 2.  Waits for that
 * call's events.  HODLR_EINVAL when profiling is off or nothing was profiled
 * yet. */
hodlr_status hodlr_profile_read(hodlr_t h, float* ms, int32_t count);

/* hodlr_info -- sizes, bytes per tier and the precision rule's quantities. */
hodlr_status hodlr_info(hodlr_t h, hodlr_info_t* out);

/* hodlr_block_tiers -- per node (layout as ranks in hodlr_import): the storage
 * format (hodlr_prec) and rank of block (i, i^1).  Either output may be NULL. */
hodlr_status hodlr_block_tiers(hodlr_t h, int32_t* tiers, int32_t* ranks);

/* ---- block-rank predictor ---------------------------------------------------- */
/* A 11-64-64-64-1 multilayer perceptron (relu hidden layers, fp16 weights,
 * fp32 arithmetic) that predicts y = log2(rank + 1) of an off-diagonal block
 * from cheap features, to size each block's first sketch in hodlr_build
 * (hodlr_build_opts.node_sketch).  The paper has no learned component; the
 * adaptive rule still decides every rank.  Parameter vector (P =
 * hodlr_mlp_num_params() = 9153 values): W1 (64 x 11, row-major), b1 (64),
 * W2 (64 x 64), b2, W3 (64 x 64), b3, W4 (1 x 64), b4 (1).  All arrays are
 * device arrays; calls are enqueued on `stream` unless stated. */
int32_t hodlr_mlp_num_params(void);

/* hodlr_mlp_features -- the 11 features of every off-diagonal block of the
 * kernel matrix of `points` (device, (n, dim) fp64, tree order) with depth
 * levels, in node order (feat: fp32 [2^(depth+1) - 2][11]): k / 12,
 * log2(m) / 20, log10(eps) / 10, and log10 of eight row norms of the block
 * (rows (2j + 1) m / 16, all columns; entries generated in registers) over
 * the largest of them, / 10.  Synchronous.  Errors: HODLR_EINVAL,
 * HODLR_ENOMEM, HODLR_ECUDA. */
hodlr_status hodlr_mlp_features(const hodlr_kernel* kernel, const double* points, int32_t n,
                                int32_t depth, double eps, float* feat, void* stream);

/* hodlr_mlp_forward -- y[s] for S samples X (fp32 [S][11]) with the fp16
 * parameters w16; act (fp32 [S][192], or NULL) receives the pre-activations
 * of the three hidden layers for hodlr_mlp_backward. */
hodlr_status hodlr_mlp_forward(const uint16_t* w16, int32_t S, const float* X, float* y,
                               float* act, void* stream);

/* hodlr_mlp_loss -- mean squared error of y against targets t (written to
 * *loss, device) and dy = 2 (y - t) / S. */
hodlr_status hodlr_mlp_loss(int32_t S, const float* y, const float* t, float* dy, float* loss,
                            void* stream);

/* hodlr_mlp_backward -- grad (fp32 [P]) = dL/dparameters for the samples of
 * the last forward (X, act) and dy, by the chain rule; work: fp32 [S][192]
 * scratch.  Every sum runs over the samples in order (reproducible). */
hodlr_status hodlr_mlp_backward(const uint16_t* w16, int32_t S, const float* X, const float* act,
                                const float* dy, float* grad, float* work, void* stream);

/* hodlr_mlp_adam -- one Adam step (beta1 0.9, beta2 0.999, eps 1e-8; step
 * counts from 1) on the fp32 master parameters w32 with moments m, v; w16
 * receives the updated parameters rounded to fp16. */
hodlr_status hodlr_mlp_adam(float* w32, uint16_t* w16, float* m, float* v, const float* grad,
                            int32_t step, float lr, void* stream);

/* ---- batched products ------------------------------------------------------ */

/* A planned batch: many stored matrices (any sizes, ranks and formats; one
 * working precision), each with its own X and B, computed by one persistent
 * launch.  Each matrix's product (Algorithm 3.3) runs inside one CTA (V^T X
 * per node in fixed-order partial sums, then D X + U Y per 32-row tile), so
 * the launch has no grid-wide dependency; the matrices are dealt to the CTAs
 * longest first by their bytes.  Results equal hodlr_matvec's within the
 * rounding bound of the product (the sums are ordered differently). */
typedef struct hodlr_batch_s* hodlr_batch_t;

/* hodlr_batch_create -- plan a batch of `count` products B_i = H_i X_i:
 * hs[i] (handles on the current device, all with working precision
 * xb_prec), nrhs[i] in [1, 16], X[i] / B[i] device arrays (n_i, nrhs[i])
 * row-major with ldx[i], ldb[i] >= nrhs[i].  Uploads the work list and
 * allocates the scratch (Y and the partial sums of every item); the handles
 * and X/B buffers must outlive the batch (their contents may change between
 * runs).  One handle may appear in several items.  Synchronous.
 * Errors: HODLR_EINVAL, HODLR_ENOMEM, HODLR_ECUDA. */
hodlr_status hodlr_batch_create(int32_t count, const hodlr_t* hs, const int32_t* nrhs,
                                const void* const* X, const int64_t* ldx,
                                void* const* B, const int64_t* ldb, int32_t xb_prec,
                                hodlr_batch_t* out);

/* hodlr_batch_run -- one launch of the planned products on `stream`; threads
 * per CTA 128, 256 or 512, or 0 for the batch's current choice (256 until
 * hodlr_batch_tune).  Allocates nothing and copies nothing from the host, so
 * it can be captured in a CUDA graph.  Two runs of one batch that overlap on
 * the GPU race on its scratch.  Errors: HODLR_EINVAL, HODLR_ECUDA. */
hodlr_status hodlr_batch_run(hodlr_batch_t b, int32_t threads, void* stream);

/* hodlr_batch_tune -- measured search over the CTA size (128, 256, 512
 * threads; two warm-up and five timed runs each, CUDA events on `stream`):
 * keeps the fastest as the batch's choice and returns it with its mean time
 * in ms (either output may be NULL).  Runs the batch 21 times (B is
 * overwritten).  Errors: HODLR_EINVAL, HODLR_ECUDA. */
hodlr_status hodlr_batch_tune(hodlr_batch_t b, void* stream, int32_t* best_threads, float* best_ms);

/* hodlr_batch_destroy -- free the plan (synchronises its device work).  NULL
 * is a no-op. */
void hodlr_batch_destroy(hodlr_batch_t b);

/* ---- Partitioned product (Algorithm 3.3 split by rows) ------------------ */

/* A row-partitioned product B = H X over P = 2^g parts (one per GPU, or one
 * per stream): part j owns the rows of node (g, j) of the cluster tree
 * (Def. 2.1), i.e. its 2^(depth-g) leaves.  In Algorithm 3.3 the products
 * V^T x of the levels k > g inside (g, j) need only the part's rows; those of
 * levels k <= g sum over the parts.  So each part computes, from its own X
 * rows only:
 *   1. hodlr_part_partial: V_q^T X over its rows for every node q, the
 *      levels 1..g into the caller's buffer Yred (zeros for the nodes that
 *      are not its ancestors), the rest into the part's scratch;
 *   2. the caller sums Yred over the P parts (an all-reduce: sum) -- the
 *      only exchange, yred_count values (sum over levels k <= g of the
 *      ranks, times R rounded up to 1, 2, 4, 8 or 16);
 *   3. hodlr_part_finish: its B rows = D X + sum_k U_k Y_k, the levels <= g
 *      from the summed Yred.
 * No X or factor bytes cross parts.  The handle is shared (each part reads
 * only its rows' data).  g = 0 is one part: the whole product. */
typedef struct hodlr_part_s* hodlr_part_t;

/* hodlr_part_create -- plan part j (0 <= j < 2^g, 0 <= g <= depth) of h for
 * nrhs in [1, 16] right-hand sides: uploads its work list, allocates its
 * scratch.  The handle must outlive the part.  Synchronous.
 * Errors: HODLR_EINVAL, HODLR_ECUDA. */
hodlr_status hodlr_part_create(hodlr_t h, int32_t g, int32_t j, int32_t nrhs, hodlr_part_t* out);

/* hodlr_part_info -- the part's first row and rows (X and B of the part hold
 * rows row0 .. row0 + rows - 1 of the whole product) and the length of Yred
 * in elements of the working precision (0 when g = 0).  Outputs may be NULL. */
hodlr_status hodlr_part_info(hodlr_part_t p, int64_t* row0, int64_t* rows, int64_t* yred_count);

/* hodlr_part_partial -- step 1 on `stream`.  X: device (rows, nrhs) of the
 * working precision, row-major, ldx >= nrhs (the part's rows only).  Yred:
 * device, yred_count elements, overwritten (may be NULL when yred_count is
 * 0).  Allocates nothing.  Steps 1 and 3 of one part use its scratch: run
 * them in order, one product at a time.  Errors: HODLR_EINVAL, HODLR_ECUDA. */
hodlr_status hodlr_part_partial(hodlr_part_t p, const void* X, int64_t ldx, void* Yred, void* stream);

/* hodlr_part_finish -- step 3 on `stream`: B (device (rows, nrhs), ldb >=
 * nrhs) = the part's rows of H X, from the same X and from Yred holding the
 * sum over all parts.  Allocates nothing.  Errors: HODLR_EINVAL,
 * HODLR_ECUDA. */
hodlr_status hodlr_part_finish(hodlr_part_t p, const void* X, int64_t ldx, const void* Yred, void* B, int64_t ldb,
                               void* stream);

/* hodlr_part_destroy -- free the part (its scratch; cudaFree waits for its
 * device work).  NULL is a no-op. */
void hodlr_part_destroy(hodlr_part_t p);

/* hodlr_tree_order -- host function (no device work): the order in which
 * to pass points in 1 to 3 dimensions so that every node of the cluster tree
 * (Def. 2.1, ceiling split of Sect. 4) of the given depth is a spatial
 * cluster -- a kd-tree on the tree's ranges.  Going down the tree, the
 * points of each node are sorted by the coordinate along which they spread
 * most (max - min; the lowest such coordinate on a tie), ties by original
 * index; the node's left child is its first ceil(m/2) positions.  For 1D
 * points (depth >= 1) this is a stable sort.
 *  points  host, (n, dim) fp64 row-major, finite; not modified.
 *  perm    host int32[n], written: perm[t] = the original index of the point
 *          at tree position t (pass points[perm[t]] to hodlr_build).
 * Errors: HODLR_EINVAL (n < 1, dim outside 1..3, 2^depth > n, a non-finite
 * coordinate, NULL arrays); perm is unspecified then. */
hodlr_status hodlr_tree_order(int32_t n, int32_t dim, const double* points, int32_t depth, int32_t* perm);

/* hodlr_node_sizes -- per node (layout as ranks in hodlr_import: node
 * q = 2^k - 2 + i is (k, i), k = 1..depth) its first row and its rows, the
 * ceil-half cluster tree of Def. 2.1 (the leaves are the level-depth nodes;
 * with depth 0 the one leaf is rows [0, n)).  Either output may be NULL. */
hodlr_status hodlr_node_sizes(hodlr_t h, int32_t* row0, int32_t* m);

/* hodlr_dense_kernel_matvec -- on-the-fly FP64 dense product b = A x for a
 * kernel matrix A_ij = f(x_i, x_j) + diag * delta_ij, used to check HODLR
 * products at sizes where A cannot be stored (its entries are generated in
 * registers, never stored).  Kinds: 0 1/(r+c), 1 exp(-r^2/len2), 2 log(r+c),
 * 3 1/(x_i - x_j) (1D) -- the test kernels of eq. (4.1) and the synthetic
 * workloads; at i == j, f is f(0) where finite and 0 otherwise.
 *
 *  points  device, (n, dim) fp64 row-major, dim in {1, 2, 3}.
 *  rows    device int32[nrows]: the rows of A to compute (any subset, any
 *          order); NULL means all n rows in order (nrows must equal n).
 *          An entry outside [0, n) gives a row of NaN.
 *  X       device fp64 (n, nrhs) row-major, ldx >= nrhs.
 *  B       device fp64 (nrows, nrhs) row-major, ldb >= nrhs; overwritten.
 * Errors: HODLR_EINVAL, HODLR_ECUDA. */
hodlr_status hodlr_dense_kernel_matvec(int32_t n, int32_t dim, const double* points,
                                       int32_t kind, double c, double len2, double diag,
                                       int32_t nrows, const int32_t* rows,
                                       int32_t nrhs, const double* X, int64_t ldx,
                                       double* B, int64_t ldb, void* stream);

/* ---- HODLR LU and solves (Sect. 3.4) ------------------------------------- */

/* hodlr_lu -- HODLR_LU (Algorithm 3.4) of the stored matrix H-hat (its
 * generators and leaves decoded to fp64), in fp64 on the device, kept in
 * the handle (a previous factorization is replaced).  At every node with
 * children a, b: the LU of H_aa, U12 = L_aa^{-1} H_ab and L21 = H_ba U_aa^{-1}
 * on the generators, and the Schur complement H_bb - L21 U12 truncated back
 * to the HODLR format (Assumption 3.6): every off-diagonal block inside b is
 * recompressed with the per-block relative Frobenius tolerance eps_lu (the
 * truncation rule of the construction, Def. 2.3); leaves are updated
 * exactly.  eps_lu = 0 keeps every nonzero singular value.  Leaves are
 * factored without pivoting (the block LU needs nonsingular leading blocks,
 * as for the diagonally dominant kernel matrices of Sect. 4).  Waits for
 * `stream`.  The current device must be the handle's.
 * Errors: HODLR_EINVAL (eps_lu outside [0, 1), another device),
 * HODLR_ESINGULAR (zero pivot in a leaf), HODLR_EACCURACY (a recompressed
 * block needs more columns than the factor storage holds: at least
 * max(64, 4 r + 32), r the largest stored rank), HODLR_ENOMEM, HODLR_ECUDA. */
hodlr_status hodlr_lu(hodlr_t h, double eps_lu, void* stream);

/* hodlr_lu_solve -- X = U^{-1} L^{-1} B with the factors of hodlr_lu
 * (forward substitution with L, back substitution with U, both recursive
 * over the tree).  B, X device fp64 (n, nrhs) row-major, ldb, ldx >= nrhs;
 * X == B solves in place.  Enqueued on `stream`.
 * Errors: HODLR_ENOTFACTORED, HODLR_EINVAL, HODLR_ECUDA. */
hodlr_status hodlr_lu_solve(hodlr_t h, int32_t nrhs, const double* B, int64_t ldb,
                            double* X, int64_t ldx, void* stream);

typedef struct {
  int32_t iterations;     /* refinement steps taken */
  int32_t gmres_steps;    /* GMRES steps, summed over the refinement steps
                             (the most of any column in each) */
  double backward_error;  /* ||B - H X||_F / (||H||_F ||X||_F) of the result */
} hodlr_solve_stats;

/* hodlr_solve -- H-hat X = B by GMRES-based iterative refinement with the
 * factors of hodlr_lu as preconditioner (Sect. 3.4): X_0 = (LU)^{-1} B;
 * then, while the normwise backward error ||B - H X||_F / (||H||_F ||X||_F)
 * (residual in fp64 by hodlr_matvec) exceeds tol and fewer than max_it steps
 * were taken: per column, GMRES (restart 60, modified Gram-Schmidt Arnoldi,
 * left preconditioned by the LU solve) on H D = R to a relative
 * preconditioned residual of 1e-4, and X += D.  The handle's working
 * precision must be fp64.  B, X device fp64 (n, nrhs) row-major.  stats may
 * be NULL.  Waits for `stream` (the Arnoldi scalars go to the host).
 * Errors: HODLR_ENOTFACTORED, HODLR_EINVAL, HODLR_EACCURACY (tol not reached
 * within max_it; X holds the last iterate), HODLR_ENOMEM, HODLR_ECUDA. */
hodlr_status hodlr_solve(hodlr_t h, int32_t nrhs, const double* B, int64_t ldb,
                         double* X, int64_t ldx, double tol, int32_t max_it,
                         hodlr_solve_stats* stats, void* stream);

/* hodlr_lu_export -- the factors of hodlr_lu on the host, in the layout of
 * hodlr_import: ranks_u[q], ranks_v[q] = the columns of U_q and V_q now;
 * U[q] (m_q x ranks_u[q]) and V[q] (m_q x ranks_v[q]) row-major, where for a
 * left child a of children (a, b) U_a holds L_aa^{-1} U_a (so the upper block
 * of U is U_a V_b^T) and V_a holds U_aa^{-T} V_a (the lower block of L is
 * U_b V_a^T); D[l] (m_l x m_l) the leaf's LU (unit lower L below the
 * diagonal, U on and above it).  Any output pointer may be NULL (ranks first,
 * then buffers of the right size).  Waits for `stream`.
 * Errors: HODLR_ENOTFACTORED, HODLR_EINVAL, HODLR_ECUDA. */
hodlr_status hodlr_lu_export(hodlr_t h, int32_t* ranks_u, int32_t* ranks_v,
                             double* const* U, double* const* V, double* const* D,
                             void* stream);

/* hodlr_destroy -- free the handle and its device memory (synchronises the
 * device work the handle owns).  NULL is a no-op. */
void hodlr_destroy(hodlr_t h);

/* hodlr_status_string -- static, human-readable text of a status code. */
const char* hodlr_status_string(hodlr_status s);

/* hodlr_last_error -- text of the last error on this host thread (e.g. the
 * CUDA error string or which argument was invalid); static storage. */
const char* hodlr_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HODLR_H */
