/*
 * ffc.h - C ABI of libffc: far-field compression by sampled-row interpolative
 * decomposition (March & Biros, "Far-field compression for fast kernel
 * summation methods in high dimensions").
 *
 * Problem statement (§1, eq. e:sum): u_i = sum_j K(y_i, x_j) q_j, u = K q with
 * rows of K indexed by targets y_i and columns by sources x_j. The outgoing
 * representation of a source set is an interpolative decomposition K ~ C P
 * (§2.1.3): C = K(:, J) for a skeleton J of r source columns and P (r x n)
 * containing I_r. The method (§2.2) computes the ID of a sampled block
 * K'(rows, :) of s far-field target rows instead of the whole m x n block.
 *
 * Conventions for every entry point:
 *  - Pointers named *_dev are device pointers owned by the caller; pointers
 *    named *_host are host pointers owned by the caller. No entry point keeps
 *    a pointer after it returns, except where stated (ffc_tree_result).
 *  - Points are row-major (point i, coordinate k at [i*d + k]); kernel blocks
 *    are column-major with a leading dimension (entry (i, j) at [i + j*ld]).
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream). Work is
 *    enqueued on it. Calls that return device-computed scalars through *_host
 *    pointers, or a device-detected status, synchronise that stream before
 *    they return; this is stated per call.
 *  - Every call returns an ffc_status. Arguments are validated before any
 *    launch; on FFC_E_INVALID nothing was enqueued. Nothing is thrown across
 *    the ABI. ffc_last_error() gives a one-line message for the calling thread.
 *  - Device waits inside the library are bounded: a wait that runs out sets
 *    FFC_E_TIMEOUT instead of hanging the GPU.
 */
#ifndef FFC_H
#define FFC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FFC_OK = 0,
  FFC_E_INVALID = 1,            /* bad argument; nothing enqueued */
  FFC_E_NOMEM = 2,              /* device allocation failed */
  FFC_E_CUDA = 3,               /* a CUDA runtime call failed */
  FFC_E_TIMEOUT = 4,            /* a bounded device wait gave up */
  FFC_E_FARFIELD_TOO_SMALL = 5, /* soft: fewer far-field rows than requested; outputs valid */
  FFC_E_SINGULAR = 6,           /* Laplace kernel at coincident points */
  FFC_E_TOL_NOT_REACHED = 7     /* soft: tolerance not met within the rank cap; outputs valid */
} ffc_status;

typedef enum { FFC_GAUSSIAN = 0, FFC_LAPLACE = 1, FFC_POLYNOMIAL = 2 } ffc_kernel_kind;
typedef enum { FFC_F64 = 0, FFC_F32 = 1 } ffc_dtype;
/* FFC_FP64: every step in FP64. FFC_MIXED: reduced-precision block and QR
 * updates with FP64 column norms and FP64 triangular solve. */
typedef enum { FFC_FP64 = 0, FFC_MIXED = 1 } ffc_precision;

/*
 * Kernel function (§4.2-§4.4):
 *   FFC_GAUSSIAN   K(y,x) = exp(-||x-y||^2 / (2 h^2))        (h > 0)
 *   FFC_LAPLACE    K(y,x) = ||x-y||^(2-d), d != 2 (d = 2 is rejected)
 *   FFC_POLYNOMIAL K(y,x) = (x.y / h + c)^p                  (h != 0, p >= 1)
 * Laplace blocks are returned divided by their largest entry: the call also
 * returns log_scale with K_true = exp(log_scale) * K_returned. A scalar
 * factor changes neither the ID nor any relative error.
 */
typedef struct {
  int32_t kind;   /* ffc_kernel_kind */
  int32_t p;      /* polynomial degree */
  double h;       /* Gaussian bandwidth / polynomial scale */
  double c;       /* polynomial constant */
} ffc_kernel;

/* One-line message describing the last failure on the calling thread. */
const char* ffc_last_error(void);

/* Library version string. */
const char* ffc_version(void);

/*
 * ffc_set_wait_limit - how many times a bounded device wait polls before it
 * gives up (the pivoted QR's group barrier of ffc_id, ffc_id_noalloc and
 * ffc_compress_tree). The paper has no counterpart: this is the control of the
 * library's failure detection. A wait that runs out ends its QR with
 * FFC_E_TIMEOUT (returned by ffc_id, per node in ffc_compress_tree) and leaves
 * the device usable. polls < 0 restores the default (2e7 polls, a second or
 * more); 0 makes every wait that is not already satisfied give up at once.
 * Applies to launches enqueued after the call, process-wide. Always FFC_OK.
 */
ffc_status ffc_set_wait_limit(int64_t polls);

/* Evaluation paths of the mixed-precision Gaussian and polynomial blocks (the
 * same arithmetic: three BF16 parts per FP32 coordinate, six partial
 * products, FP32 accumulation; they differ in summation order only):
 * FFC_EVAL_DEFAULT: tcgen05 for d >= 64, SIMT below;
 * FFC_EVAL_SIMT: FP32 direct differences (no tensor cores), any d;
 * FFC_EVAL_MMA_SYNC: mma.sync m16n8k16, 128 x 128 tiles, synchronous staging;
 * FFC_EVAL_TCGEN05: tcgen05.mma with TMEM accumulators and TMA staging, the
 *   library's tile; FFC_EVAL_TCGEN05_TILE0 + v, v < FFC_EVAL_TCGEN05_TILES: the
 *   same with tile variant v (targets x sources per tile, coordinates per
 *   stage, stages): 0: 128 x 256, 32, 3; 1: 128 x 128, 64, 2;
 *   2: 128 x 128, 32, 4; 3: 128 x 256, 16, 6; 4: 128 x 128, 16, 8. */
#define FFC_EVAL_DEFAULT 0
#define FFC_EVAL_SIMT 1
#define FFC_EVAL_MMA_SYNC 2
#define FFC_EVAL_TCGEN05 3
#define FFC_EVAL_TCGEN05_TILE0 4
#define FFC_EVAL_TCGEN05_TILES 5

/* Triangular solve T = R11^-1 R12 of the mixed-precision path (the FP64 path always solves in FP64):
 * FFC_SOLVE_DEFAULT: FP32 solves refined once (T1 with R11 rounded to FP32; the residual
 *   R12 - R11 T1 from exact products summed in double-float, the diagonal term in FP64; its FP32
 *   solve added to T1 in FP64), about the FP64 solve's accuracy at the FP32 rate;
 * FFC_SOLVE_FP64: FP64 back-substitution. */
#define FFC_SOLVE_DEFAULT 0
#define FFC_SOLVE_FP64 1

/*
 * ffc_set_eval_path - the evaluation path FFC_EVAL_DEFAULT stands for, for
 * ffc_eval_block and for ffc_compress_tree calls whose params.eval_path is
 * FFC_EVAL_DEFAULT (the project's autotuner compares them). Process-wide,
 * for calls made after it. FFC_E_INVALID for an unknown path.
 */
ffc_status ffc_set_eval_path(int32_t path);

/*
 * ffc_far_field - list the far field of a source set (§4.1, setup step 3):
 *   T = { j in [0, M) \ [ex_begin, ex_end) : ||Y_j - x_c|| >= xi * radius }.
 * Y_dev: M x d points (dtype). x_c_dev: d doubles, or NULL for "no distance
 * test" (every non-excluded candidate is far). idx_dev: receives the far
 * indices in ascending order (capacity M int64). count_host: |T|.
 * Synchronises `stream`.
 */
ffc_status ffc_far_field(const void* Y_dev, int32_t dtype, int64_t M, int32_t d,
                         const double* x_c_dev, double radius, double xi,
                         int64_t ex_begin, int64_t ex_end,
                         int64_t* idx_dev, int64_t* count_host, void* stream);

/*
 * ffc_sample_rows - uniform sample of s far-field rows without replacement
 * (§2.2; §4.1.3 "Uniform sampling"). Far field as in ffc_far_field.
 * Randomness: draw t of the stream (seed, stream_id) is word t mod 4 of
 * Philox4x64-10(counter = (t/4, stream_id, 0, 0), key = (seed, 0)).
 * Phase A: for t < 64 s, candidate j = floor(w_t M / 2^64) is accepted if it
 * is far and new, until s rows are accepted (rows in acceptance order, so a
 * size-s sample is a prefix of the size-2s sample). Phase B, only if phase A
 * ran out: the not-yet-taken far rows T' in ascending order are appended
 * whole if |T'| <= s - k, else picked by a partial Fisher-Yates shuffle with
 * draws t = 64 s, 64 s + 1, ...
 * rows_dev: capacity s int64. s_out_host: rows written, min(s, |T|).
 * far_count_host (may be NULL): |T|. Requires M <= 1,500,000.
 * Returns FFC_E_FARFIELD_TOO_SMALL (soft) when |T| < s. Synchronises `stream`.
 */
ffc_status ffc_sample_rows(const void* Y_dev, int32_t dtype, int64_t M, int32_t d,
                           const double* x_c_dev, double radius, double xi,
                           int64_t ex_begin, int64_t ex_end,
                           int64_t s, uint64_t seed, uint64_t stream_id,
                           int64_t* rows_dev, int64_t* s_out_host, int64_t* far_count_host,
                           void* stream);

/*
 * ffc_eval_block - evaluate the sampled block K'_ij = K(Y[rows_i], X_j)
 * (§2.2: the s x n matrix K~ of the sampled targets against the sources).
 * Y_dev: candidate targets (M x d, dtype); rows_dev: s int64 indices into Y.
 * X_dev: n x d sources (dtype). K_dev: column-major s x n, leading dim
 * ldk >= s, double for FFC_FP64 and float for FFC_MIXED. center_dev: d
 * doubles (the source centre) or NULL; FFC_MIXED forms distances of centred
 * coordinates. log_scale_host: ln of the factor removed from a Laplace block
 * (0 for the other kernels). Synchronises `stream` (Laplace: to return the
 * scale). Returns FFC_E_SINGULAR for a Laplace block with a zero distance.
 * FFC_MIXED arithmetic:
 *   Gaussian, polynomial, d < 64: FP32 direct differences (inner products).
 *   Gaussian, polynomial, d >= 64: tensor cores, each FP32 coordinate split
 *     into three BF16 parts, FP32 accumulation; Gaussian D2 recomputed from
 *     FP32 differences where ||y||^2 + ||x||^2 - 2 y.x cancels. By default the
 *     tcgen05 path (TMA-staged BF16 planes, TMEM accumulators, 128 x 256
 *     tiles; device scratch of about 6 (s + n) d bytes, allocated and freed on
 *     `stream`); ffc_set_eval_path selects another.
 *   Laplace: FP32 distances; FP64 where they cancel and for every entry at or
 *     above 1e-6 of the largest. The block is scaled by the minimum of those
 *     distances: the same block as FP64's up to a constant factor within
 *     FP32 rounding (J, T and relative errors do not depend on it), and
 *     log_scale_host is that scale.
 */
ffc_status ffc_eval_block(ffc_kernel kernel, const void* Y_dev, int32_t dtype,
                          const int64_t* rows_dev, int64_t s,
                          const void* X_dev, int64_t n, int32_t d,
                          const double* center_dev, int32_t precision,
                          void* K_dev, int64_t ldk, double* log_scale_host, void* stream);

/*
 * ffc_id - interpolative decomposition of K' (§2.1.3, Appendix A.1) by
 * Businger-Golub column-pivoted Householder QR: at step k the pivot is the
 * remaining column of largest residual norm (lowest index on ties); the
 * reflector follows LAPACK dlarfg (beta = -sign(alpha) ||x||, sign(0) = +).
 * Then T = R11^-1 R12 by back-substitution.
 * K_dev: s x n column-major (ld ldk; double for FFC_FP64, float for
 * FFC_MIXED); OVERWRITTEN. Stop rule: tol > 0 -> the smallest r <= r_max
 * with ||R22||_F <= tol ||K'||_F; tol <= 0 -> r = r_max (earlier only if the
 * remaining columns are exactly zero).
 * Outputs: skel_perm_dev (n int32): [0, r) the skeleton in pivot order,
 * [r, n) the other columns ascending. T_dev (double, column-major, ld ldt >=
 * max(r_max, 1), capacity ldt * n): T(:, c) expresses column skel_perm[r + c]
 * in the skeleton columns, so P = [I_r T] Pi^T. rank_host: r.
 * r22_rel_host: ||R22||_F / ||K'||_F. Synchronises `stream`.
 * Returns FFC_E_TOL_NOT_REACHED (soft) if tol > 0 was not met at r_max.
 */
ffc_status ffc_id(void* K_dev, int64_t s, int64_t n, int64_t ldk, int32_t precision,
                  int64_t r_max, double tol,
                  int32_t* skel_perm_dev, double* T_dev, int64_t ldt,
                  int64_t* rank_host, double* r22_rel_host, void* stream);

/*
 * ffc_id_noalloc - ffc_id without any device allocation. The paper has no
 * counterpart: this is an interface variant for callers that cannot call
 * cudaMalloc (or cudaMallocAsync) at call time, for example code running
 * inside a framework whose caching allocator already owns the device memory
 * (a raw allocation can fail or fragment its pool), latency-critical loops
 * that cannot afford an allocation's implicit synchronisation, and
 * deployments that fix their device memory budget up front.
 *
 * Arguments, outputs, statuses and results are those of ffc_id (FFC_FP64).
 * Instead of allocating, the call keeps its QR scratch (column norms, pivot
 * and reflector data, group slots, R11) in one fixed array of about 0.8 MB
 * that every GPU loading the library holds until the process exits. Limits:
 * n <= FFC_NOALLOC_MAX_COLS, min(r_max, s, n) <= FFC_NOALLOC_MAX_RANK,
 * s <= 2048; larger problems return FFC_E_INVALID before anything is
 * enqueued. The first call on a device looks up the array's device address
 * (once per device, with that device current). All calls share the one
 * array and the next call overwrites it: calls that overlap on the GPU
 * (other streams, other host threads on the same device) race. Synchronises
 * `stream`.
 */
#define FFC_NOALLOC_MAX_COLS 16384
#define FFC_NOALLOC_MAX_RANK 256
ffc_status ffc_id_noalloc(void* K_dev, int64_t s, int64_t n, int64_t ldk, int32_t precision,
                          int64_t r_max, double tol,
                          int32_t* skel_perm_dev, double* T_dev, int64_t ldt,
                          int64_t* rank_host, double* r22_rel_host, void* stream);

/*
 * ffc_id_error - relative Frobenius error of an ID on a full block
 * (§4.1.3, step 4): ||K - K(:, J) P||_F / ||K||_F with K_ij = K(Y[rows_i], X_j)
 * over m target rows (rows_dev NULL = rows 0..m-1 of Y). skel_perm_dev, T_dev,
 * ldt, r: as returned by ffc_id for these n sources. The block is streamed
 * in tiles and never stored; all arithmetic is FP64. err_host: the error.
 * Synchronises `stream`.
 */
ffc_status ffc_id_error(ffc_kernel kernel, const void* Y_dev, int32_t dtype,
                        const int64_t* rows_dev, int64_t m,
                        const void* X_dev, int64_t n, int32_t d,
                        const int32_t* skel_perm_dev, const double* T_dev, int64_t ldt, int64_t r,
                        double* err_host, void* stream);

/* ---------------- the outgoing representation (§2.1.3) ------------------ */

/*
 * ffc_skeleton_charges - the skeleton charges of an ID, q~ = P q (§2.1.3,
 * after eq. e:id-error: the n source charges q of a node become r charges on
 * its skeleton points, u = K q ~ C P q = C q~). With P = [I_r T] Pi^T as
 * ffc_id returns it: q~ = q[skel_perm[0:r]] + T q[skel_perm[r:n]].
 * skel_perm_dev: n int32; T_dev: r x (n - r) doubles, column c at T + c ldt
 * (ldt >= max(r, 1); may be NULL when r = n); q_dev: n x nrhs doubles, column
 * j at q + j ldq (ldq >= n); qt_dev: r x nrhs, column j at qt + j ldqt
 * (ldqt >= r). FP64. Asynchronous.
 */
ffc_status ffc_skeleton_charges(const int32_t* skel_perm_dev, const double* T_dev, int64_t ldt, int64_t r, int64_t n,
                                const double* q_dev, int64_t ldq, int64_t nrhs, double* qt_dev, int64_t ldqt,
                                void* stream);

/*
 * ffc_potential - u_i = exp(-log_scale) sum_c K(Y[rows_i], X[cols_c]) w_c:
 * the kernel sum of §1 (eq. e:sum) over a subset of the sources. With cols =
 * the skeleton skel_perm[0:r] and w = q~ it is the potential of the outgoing
 * representation, u ~ C q~ (§2.1.3); with cols_dev = NULL (nc = n) and w = q
 * it is the direct sum u = K q it approximates. Y_dev: targets (M x d, dtype),
 * rows_dev: m int64 indices into Y or NULL (rows 0..m-1); X_dev: n x d sources
 * (dtype); cols_dev: nc int32 indices into X or NULL; w_dev: nc doubles;
 * u_dev: m doubles. log_scale shifts every kernel value by exp(-log_scale)
 * (the Laplace kernel's range; 0 for none). FP64 arithmetic. A Laplace
 * target that coincides with a source gives an infinite value.
 * Asynchronous.
 */
ffc_status ffc_potential(ffc_kernel kernel, const void* Y_dev, int32_t dtype, const int64_t* rows_dev, int64_t m,
                         const void* X_dev, int64_t n, int32_t d, const int32_t* cols_dev, int64_t nc,
                         const double* w_dev, double log_scale, double* u_dev, void* stream);

/* ----------------------------- trees ---------------------------------- */

/*
 * Binary PCA tree (the space-partitioning tree of §2 that defines each
 * node's far field). Depth D = smallest D with ceil(N / 2^D) <= leaf_size;
 * 2^(D+1) - 1 nodes in heap order (children of i: 2i+1, 2i+2); a node holds
 * positions [begin, begin + count) of `perm`, its left child the first
 * floor(count / 2). Each node's points are ordered by (projection on the
 * principal direction of its centred points, original index); the principal
 * direction comes from 32 power iterations from (1,..,1)/sqrt(d), signed so
 * that its largest-magnitude component is positive. Node geometry (§4.1):
 * centroid x_c = mean, radius = max ||x - x_c||.
 */
int32_t ffc_tree_depth(int64_t N, int64_t leaf_size);

/*
 * ffc_build_tree - build the tree above on the GPU.
 * points_dev: N x d (dtype). perm_dev: N int64 (position -> point index).
 * begin_dev, count_dev: n_nodes int64. centroid_dev: n_nodes x d doubles.
 * radius_dev: n_nodes doubles; n_nodes = 2^(depth+1) - 1.
 * Synchronises `stream`.
 */
ffc_status ffc_build_tree(const void* points_dev, int32_t dtype, int64_t N, int32_t d,
                          int64_t leaf_size, int64_t* perm_dev, int64_t* begin_dev,
                          int64_t* count_dev, double* centroid_dev, double* radius_dev,
                          void* stream);

/* Tree as consumed by ffc_compress_tree (all device pointers). */
typedef struct {
  int32_t depth;
  int64_t n_nodes;
  const int64_t* begin_dev;
  const int64_t* count_dev;
  const double* centroid_dev;
  const double* radius_dev;
} ffc_tree;

typedef struct {
  ffc_kernel kernel;
  int32_t precision;   /* ffc_precision */
  int32_t min_level;   /* compress nodes at levels >= min_level (2) */
  int32_t s0;          /* first sample size (128) */
  int32_t s_max;       /* largest sample size (2048); the rank cap is s_max / 2 */
  double tol;          /* relative tolerance on ||R22||_F / ||K'||_F (1e-6) */
  double xi;           /* far-field separation (1.0) */
  uint64_t seed;       /* sampling seed; the stream id of a node is its heap id */
  int32_t sampler;     /* ffc_sampler */
  int32_t pool_rows;   /* learned: 0 = the whole far field is the candidate pool, else a
                          uniform pool of pool_rows >= s_max rows */
  const double* proj_dev;   /* learned: 8 x d random directions of the projection features */
  const float* mlp_dev;     /* learned: FFC_MLP_PARAMS network parameters (FP32 master copy) */
  /* launch shape of the pivoted QR (no effect on what is computed beyond FP32 summation order;
   * 0 = the library's defaults, which the project's autotuner measures against):
   * qr_big_min_s: mixed precision, rounds with s >= this use the register-resident variant
   *   (2 CTAs per SM, 128 registers; default 1024); > s_max disables it;
   * qr_l2_budget_mb: bytes of sampled blocks per cooperative QR launch, in MB (default 96) */
  int32_t qr_big_min_s;
  int32_t qr_l2_budget_mb;
  /* qr_panel: panel width of the pivoted QR. 0 or 1 = unblocked, the library's default (every step
   *   updates the trailing matrix); 2..8 = the blocked form with that width (the trailing matrix is
   *   only read at each step and updated once per panel; a panel also ends early once the pivot norm
   *   falls below a quarter of the panel's first; rounds whose CTAs own more than 128 columns each
   *   stay unblocked). Same pivots and outputs up to rounding. */
  int32_t qr_panel;
  /* nested: 0 = every node's ID has all of the node's points as its columns; 1 = nested skeletonization
   *   (the upward pass of a treecode, §2; ASKIT, §1): levels are compressed from the deepest up, a leaf's
   *   columns are its points and a node's columns are its children's skeleton points (left child's,
   *   then right child's, each in pivot order; a child without an ID of status FFC_OK or
   *   FFC_E_TOL_NOT_REACHED contributes all of its points). Rows are the node's own far-field sample
   *   either way. */
  int32_t nested;
  /* eval_path: FFC_EVAL_* evaluation path of the sampled blocks (mixed precision, Gaussian and
   *   polynomial); FFC_EVAL_DEFAULT (0) = the process default (ffc_set_eval_path) */
  int32_t eval_path;
  /* graphs: 0 = each sample-size round's memsets and launches are captured into a CUDA graph the first
   *   time that round (same items, sizes, workspace and parameters) runs on this result, and replayed as
   *   one graph launch whenever it recurs, e.g. in every later call on the same tree; 1 = every kernel is
   *   launched directly. Identical results either way. */
  int32_t graphs;
  /* qr_defer: write-back depth of the pivoted QR's lazy form, for mixed-precision rounds that run the
   *   register-resident variant (s of 1,024 or 2,048) unblocked. A step still reads every trailing
   *   column, applies the reflectors not yet written back (kept on chip) and the new one, but writes
   *   the columns back only every qr_defer steps. 0 = the library's default, 1 = every step (the plain
   *   form), 2..4 = that depth. Every depth >= 2 gives bitwise the same outputs; against 1 they differ
   *   by FP32 summation order only. */
  int32_t qr_defer;
  /* solve: FFC_SOLVE_* of the mixed-precision triangular solve (FFC_SOLVE_DEFAULT = 0) */
  int32_t solve;
} ffc_params;

/* Row sampler of a tree compression: uniform (§2.2), the learned proposal
 * (ffc_propose_rows, same seed and stream id), or one of the paper's samplers
 * of §4.1.3 over the node's whole far field (ffc_sample_paper with the far
 * field in ascending order as the candidates, same seed, stream id = node):
 * distance, inverse distance, nearest neighbours. */
typedef enum {
  FFC_SAMPLE_UNIFORM = 0,
  FFC_SAMPLE_LEARNED = 1,
  FFC_SAMPLE_DISTANCE = 2,
  FFC_SAMPLE_INV_DISTANCE = 3,
  FFC_SAMPLE_NEAREST = 4
} ffc_sampler;

/*
 * Compression of every node at level >= min_level. For a node with
 * centroid x_c, radius rho and positions [b, b + n): far field = positions
 * outside [b, b + n) at distance >= xi rho from x_c; s = s0; sample s rows
 * (ffc_sample_rows with stream_id = node id, or ffc_propose_rows with the
 * learned sampler), evaluate K' (s x n), run the pivoted QR in tolerance mode
 * for at most s/2 steps (min(s, n) when the sample already holds the whole
 * far field); if the tolerance is not met, double s (both samplers are
 * prefix consistent: the learned draw's keys do not depend on s, so its
 * s_max best rows are drawn once) while s <= s_max; else keep the last ID
 * with status FFC_E_TOL_NOT_REACHED.
 */
typedef struct ffc_tree_result ffc_tree_result;   /* opaque; owns device memory */

/*
 * ffc_compress_tree - run the compression above on points_perm_dev (N x d,
 * rows in tree order, i.e. points[perm]). *result: NULL on the first call
 * (allocated here and returned), or a result from an earlier call on the
 * same tree shape and params, whose memory is reused. Synchronises `stream`
 * once per sample-size round (at most log2(s_max / s0) + 1 rounds).
 */
ffc_status ffc_compress_tree(const void* points_perm_dev, int32_t dtype, int64_t N, int32_t d,
                             const ffc_tree* tree, const ffc_params* params,
                             ffc_tree_result** result, void* stream);

/* Per-node outputs, in the order of the compressed nodes (increasing heap id). */
typedef struct {
  int64_t n_out;                 /* number of compressed nodes */
  int32_t rounds;                /* sample-size rounds the last call ran */
  const int32_t* node_dev;       /* heap id */
  const int32_t* rank_dev;       /* r */
  const int32_t* s_dev;          /* rows sampled */
  const int32_t* status_dev;     /* ffc_status of the node */
  const double* r22_rel_dev;     /* ||R22||_F / ||K'||_F */
  const double* log_scale_dev;   /* Laplace block scale (0 otherwise) */
  const int64_t* far_count_dev;  /* |T| */
  const int64_t* rows_off_dev;   /* node i's rows start at rows_dev[rows_off[i]] */
  const int64_t* rows_dev;       /* sampled positions (tree order), s entries per node */
  const int64_t* skel_off_dev;   /* node i's skel_perm starts at skel_dev[skel_off[i]] (n entries) */
  const int32_t* skel_dev;       /* node-local column indices, as ffc_id */
  const int64_t* T_off_dev;      /* node i's T starts at T_dev[T_off[i]], ld = rank */
  const double* T_dev;
  const int32_t* ncols_dev;      /* number of ID columns of node i (its point count unless nested) */
  const int32_t* cols_dev;       /* node i's columns (node-local point indices) at cols_dev[skel_off[i]];
                                    skel indexes these: skeleton point k is cols[skel[k]] */
} ffc_tree_view;

ffc_status ffc_tree_result_view(const ffc_tree_result* result, ffc_tree_view* view);
void ffc_tree_result_free(ffc_tree_result* result);

/*
 * ffc_tree_apply - the potential at every point of a compressed tree from the
 * nodes' outgoing representations (§2.1.3; the far-field criterion of the
 * §4.1 setup, per node). Charges q_dev: N doubles in tree order (the same
 * order as points_perm_dev). For every target y (every point, tree order):
 *   u(y) = sum over b in IL(y) of sum_j K(y, x~_j) q~_j   (far field)
 *        + sum over the near leaves of y of K(y, x) q(x), x != y  (near field,
 *          only with near_field != 0)
 * where IL(y) holds each node b at level >= min_level whose far field
 * contains y while no ancestor at level >= min_level has y in its far field;
 * a leaf reached with no such node on its path is a near leaf. Every source
 * other than y is counted once. mode FFC_APPLY_SKELETON uses each node's ID
 * (q~ = P q_cols, x~ its skeleton points; q_cols = the charges of the ID's
 * columns: its points' charges, or for a nested compression the children's
 * skeleton charges, computed from the leaves up; a node whose status is
 * neither FFC_OK nor FFC_E_TOL_NOT_REACHED, or without rows, is summed from
 * its sources); FFC_APPLY_DIRECT sums
 * every far node from its sources: the exact value the representation
 * approximates. The kernel, xi, min_level and s_max are those of the
 * compression that produced `result` (same tree, same points). qt_dev:
 * skeleton charges, output node i's r_i values at qt + i (s_max / 2)
 * (capacity n_out (s_max / 2) doubles; written in skeleton mode, may be NULL
 * in direct mode). u_dev: N doubles. log_scale as in ffc_potential. FP64
 * arithmetic. Requires 2^min_level + 2 depth + 2 <= 96. Skeleton mode
 * allocates (cudaMallocAsync) and frees a buffer of one double per ID column
 * and synchronises `stream` once; direct mode is asynchronous.
 */
typedef enum { FFC_APPLY_SKELETON = 0, FFC_APPLY_DIRECT = 1 } ffc_apply_mode;
ffc_status ffc_tree_apply(const void* points_perm_dev, int32_t dtype, int64_t N, int32_t d, const ffc_tree* tree,
                          const ffc_tree_result* result, const double* q_dev, int32_t mode, int32_t near_field,
                          double log_scale, double* qt_dev, double* u_dev, void* stream);

/*
 * Phase timing of ffc_compress_tree (tracing). When enabled on a result,
 * each later ffc_compress_tree call records CUDA events on its stream around
 * every phase of every round and adds the elapsed times (milliseconds) into
 * the profile; ffc_tree_profile_reset zeroes it. Phases: 0 sampling,
 * 1 block evaluation, 2 pivoted QR, 3 finalize + triangular solve,
 * 4 bookkeeping (size patch, epilogue, table uploads). `launches` counts
 * the library's kernels launched (directly or as nodes of a round's CUDA
 * graph), `qr_flops` the algorithmic flops of the QR
 * steps taken, sum over steps k of 4 (s - k)(n - k) (one dot product and
 * one update per remaining element), `eval_flops` 3 s n d per block
 * (difference, square, add per coordinate; 2 s n d for the polynomial).
 */
typedef struct {
  int32_t enabled;
  int32_t calls;        /* ffc_compress_tree calls accumulated */
  int32_t rounds;       /* sample-size rounds accumulated */
  int32_t pad;
  int64_t launches;     /* kernel launches accumulated */
  int64_t qr_launches;  /* of which QR launches */
  double ms[5];         /* per phase, accumulated */
  double qr_flops;      /* accumulated */
  double eval_flops;    /* accumulated */
  double qr_bytes;      /* one read + one write of every QR block, accumulated */
  double qr_ms_round[8];      /* QR time of sample-size round i (s = s0 2^i), accumulated */
  int64_t items_round[8];     /* nodes that round i processed, accumulated */
  int64_t graph_launches;     /* rounds run as one CUDA graph launch (params.graphs = 0), accumulated */
  int64_t graph_captures;     /* rounds captured into a new graph, accumulated */
} ffc_tree_profile;

ffc_status ffc_tree_profile_enable(ffc_tree_result* result, int32_t enabled);
ffc_status ffc_tree_profile_reset(ffc_tree_result* result);
ffc_status ffc_tree_profile_get(const ffc_tree_result* result, ffc_tree_profile* out);


/* ------------------------------------------------------------------------
 * Learned row proposal and its training (the leverage-score distribution of
 * §3, Def. "Statistical Leverage", and §4.1.3 "Leverage sampling", predicted
 * by a small network from per-row features).
 *
 * Network: 12 features -> 128 (GELU) -> 128 (GELU) -> 1 logit, GELU(z) =
 * z Phi(z) (erf form). Parameters: an FP32 master vector of FFC_MLP_PARAMS
 * floats, matrices row-major with W[j][k] = weight from input k to unit j:
 *   W1 128x12 at 0 | b1 128 at 1536 | W2 128x128 at 1664 | b2 128 at 18048 |
 *   w3 128 at 18176 | b3 at 18304.
 * Every pass uses the parameters rounded to FP16 (nearest even) and
 * accumulates in FP32.
 */
#define FFC_MLP_PARAMS 18305
#define FFC_N_FEATURES 12
#define FFC_MAX_DRAW 8192    /* largest number of rows of one weighted draw */

/*
 * ffc_features - the 12 features of targets Y[rows[i]] for a node with
 * centroid x_c and radius rho (rho <= 0 is taken as 1), with
 * delta = y - x_c, r = ||delta||:
 *   f0 = r / rho
 *   f1 = K(y, x_c) normalised: Gaussian exp(-r^2/(2h^2)); Laplace
 *        (rho/r)^(d-2); polynomial (y.x_c/h + c)^p / (||y|| ||x_c||/h + c)^p
 *   f2 = ||y|| / rho;  f3 = rho / h (h = 1 for Laplace)
 *   f4..f11 = <g_k, delta> / rho for the rows g_k of proj_dev (8 x d FP64).
 * Computed in FP32 (coordinates, centroid and directions rounded to FP32);
 * stored as FP32 row-major R x 12 in feats_dev. d <= 5000.
 * rows_dev: R indices in [0, M). x_c_dev: d doubles. Asynchronous.
 */
ffc_status ffc_features(ffc_kernel k, const void* Y_dev, int32_t dtype, int64_t M, int32_t d,
                        const int64_t* rows_dev, int64_t R, const double* x_c_dev, double radius,
                        const double* proj_dev, float* feats_dev, void* stream);

/* ffc_mlp_forward - logits_dev[i] (R floats) of the feature rows feats_dev
 * (R x 12 FP32): the proposal's inference pass. Its 128 x 128 product runs on
 * the tensor cores with FP32 accumulation: the FP16 weights times the FP32
 * first-layer activations, each split into two FP16 parts (hi + lo), so the
 * activations keep about 2^-22 relative precision. Asynchronous. */
ffc_status ffc_mlp_forward(const float* params_dev, const float* feats_dev, int64_t R, float* logits_dev,
                           void* stream);

/*
 * ffc_sample_weighted - s of the P pool rows without replacement, row i with
 * weight w'_i = 0.9 w_i / mean(w) + 0.1, w_i = exp(o_i - max o), by the keys
 * of Efraimidis & Spirakis (2006): key_i = ln(u_i) / w'_i with u_i the unit
 * double (top 53 bits + 1/2) * 2^-53 of draw i of stream (seed, stream_id,
 * domain 2) (Philox layout as in ffc_sample_rows). The min(s, P) largest keys
 * win (ties: lower pool position) and are written in decreasing key order,
 * so a size-s draw is a prefix of the size-2s draw. Keys are formed in FP64
 * from the FP32 logits; pools above 16,384 rows are first ranked by FP32
 * keys within a proven relative error of 2^-18 of the FP64 ones, and only
 * the rows that can be among the selection get their FP64 key, so the result
 * is the FP64 keys' selection. min(s, P) <= FFC_MAX_DRAW; any P.
 * rows_dev: capacity min(s, P). Allocates 8 P + 256 bytes of stream-ordered
 * device memory for the call (the draw's item and a key buffer). Asynchronous.
 */
ffc_status ffc_sample_weighted(const int64_t* pool_dev, const float* logits_dev, int64_t P, int64_t s,
                               uint64_t seed, uint64_t stream_id, int64_t* rows_dev, void* stream);

/*
 * ffc_propose_rows - the learned proposal of s far-field rows: the candidate
 * pool is the whole far field in ascending order (pool_rows = 0; the
 * leverage distribution the network predicts is over every row) or a
 * uniform pool of pool_rows rows (ffc_sample_rows with s = pool_rows, same
 * seed and stream); then the features and logits of every pool row and
 * ffc_sample_weighted over the pool. s <= FFC_MAX_DRAW. rows_dev: capacity
 * s. Outputs and statuses as in ffc_sample_rows (FFC_E_FARFIELD_TOO_SMALL
 * when fewer than s rows exist). Synchronises.
 */
ffc_status ffc_propose_rows(ffc_kernel k, const void* Y_dev, int32_t dtype, int64_t M, int32_t d,
                            const double* x_c_dev, double radius, double xi, int64_t ex_begin, int64_t ex_end,
                            const double* proj_dev, const float* params_dev, int64_t pool_rows, int64_t s,
                            uint64_t seed, uint64_t stream_id, int64_t* rows_dev, int64_t* s_out_host,
                            int64_t* far_count_host, void* stream);

/*
 * The paper's other row samplers (§4.1.3, compared there with uniform
 * sampling; the heuristics of §3), for comparison with the learned proposal.
 *   FFC_DRAW_DISTANCE      probability proportional to ||y - x_c||
 *   FFC_DRAW_INV_DISTANCE  probability proportional to 1 / ||y - x_c|| (rows
 *                          near the sources carry the block, §3)
 *   FFC_DRAW_NEAREST       deterministic: the candidates closest to the
 *                          node's sources (squared distance to the nearest
 *                          source, FP64; ties to the lower position)
 * The weighted draws are without replacement by Efraimidis & Spirakis' keys
 * ln(u_i) / w_i, u_i the unit double (top 53 bits + 1/2) 2^-53 of draw i
 * (i = candidate position) of stream (seed, stream_id, domain 3), Philox
 * layout as in ffc_sample_rows; the min(s, P) largest keys win, in key order,
 * ties to the lower position (a size-s draw is a prefix of the size-2s draw).
 */
typedef enum { FFC_DRAW_DISTANCE = 0, FFC_DRAW_INV_DISTANCE = 1, FFC_DRAW_NEAREST = 2 } ffc_paper_sampler;

/*
 * ffc_sample_paper - s of the P candidates cand_dev (int64 rows of Y_dev,
 * M x d, dtype) by one of the samplers above. x_c_dev: d doubles (distance
 * samplers); X_dev: the node's n sources (n x d, dtype; nearest neighbours).
 * rows_dev: capacity min(s, P). min(s, P) <= FFC_MAX_DRAW when P > 16384.
 * Distances in FP64. Asynchronous.
 */
ffc_status ffc_sample_paper(int32_t sampler, const void* Y_dev, int32_t dtype, int32_t d, const int64_t* cand_dev,
                            int64_t P, const double* x_c_dev, const void* X_dev, int64_t n, int64_t s, uint64_t seed,
                            uint64_t stream_id, int64_t* rows_dev, void* stream);

/*
 * ffc_sample_leverage - leverage sampling (§4.1.3 "Leverage sampling"; §3,
 * Def. "Statistical Leverage"): s rows of the full far-field block K (m x n
 * FP64, column-major, ld ldk; row i stands for candidate cand_dev[i], or i
 * when cand_dev is NULL) drawn with probabilities proportional to their
 * leverage scores at the eps-rank of K (ffc_leverage), over the rows with a
 * positive score; Efraimidis-Spirakis keys as above, i = the row's position
 * among the rows with a positive score. n <= 1024. rows_dev: capacity
 * min(s, m). s_out_host: rows drawn; rank_host: the eps-rank.
 * FFC_E_TOL_NOT_REACHED (soft) if the eigen-solver did not converge.
 * Synchronises.
 */
ffc_status ffc_sample_leverage(const double* K_dev, int64_t m, int64_t n, int64_t ldk, const int64_t* cand_dev,
                               double eps, int64_t s, uint64_t seed, uint64_t stream_id, int64_t* rows_dev,
                               int64_t* s_out_host, int64_t* rank_host, void* stream);

/*
 * ffc_mlp_loss_grad - loss and gradient of the proposal on a batch of nodes:
 * rows [node_off[b], node_off[b+1]) of feats_dev / targets_dev belong to
 * node b (node_off_dev: n_nodes + 1 int64 on the device, non-decreasing,
 * node_off[0] = 0, node_off[n_nodes] = R). Targets t >= 0 (FP64, e.g. the
 * leverage scores of ffc_leverage) are normalised per node, q = t / sum_b t,
 * and the loss is the mean cross-entropy between q and the proposal:
 *   L = (1/B) sum_b -sum_{i in b} q_i log softmax_b(o)_i
 * (a node whose targets sum to zero contributes nothing).
 * grad_dev: FFC_MLP_PARAMS floats (dL/dparameter, taken at the FP16 values).
 * loss_host: L (FP64 sums). Deterministic for a fixed device. Synchronises.
 */
ffc_status ffc_mlp_loss_grad(const float* params_dev, const float* feats_dev, const double* targets_dev,
                             const int64_t* node_off_dev, int32_t n_nodes, int64_t R, double* loss_host,
                             float* grad_dev, void* stream);

/*
 * ffc_adam_step - one Adam update (Kingma & Ba 2015, Algorithm 1; step >= 1)
 * of n FP32 parameters with FP32 moments m, v, computed in FP64:
 *   m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 *   theta -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).
 * Asynchronous.
 */
ffc_status ffc_adam_step(float* params_dev, const float* grad_dev, float* m_dev, float* v_dev, int64_t n,
                         int64_t step, double lr, double beta1, double beta2, double eps, void* stream);

/*
 * ffc_leverage - statistical leverage scores of the rows of K (m x n FP64,
 * column-major, ld ldk) with respect to rank r (§3, Def. "Statistical
 * Leverage"): l_i = ||U_r(i, :)||^2 for K = U Sigma V^T. r = r_fixed when
 * r_fixed > 0, else the eps-rank (number of sigma_k >= eps sigma_1, §4.1.3).
 * Route: G = K^T K, Jacobi eigen-decomposition of G, l_i = ||K(i,:) V_r
 * Sigma_r^-1||^2, all FP64; singular values below about 1e-7 sigma_1 are not
 * resolved. lev_dev: m doubles (sum = r). sigma_dev: n doubles, decreasing.
 * n <= 1024. FFC_E_TOL_NOT_REACHED (soft) if Jacobi did not converge.
 * Synchronises.
 */
ffc_status ffc_leverage(const double* K_dev, int64_t m, int64_t n, int64_t ldk, double eps, int64_t r_fixed,
                        double* lev_dev, double* sigma_dev, int64_t* rank_host, void* stream);

/*
 * ffc_spectrum - the singular values of K (m x n FP64, column-major, ld ldk;
 * §4.2 "Singular values of K") and its eps-rank, the smallest r with
 * sigma_{r+1} / sigma_1 < eps (§4.1.3 step 1): the route of ffc_leverage
 * without the scores (G = K^T K, Jacobi eigenvalues, FP64), so singular
 * values below about 1e-7 sigma_1 are not resolved. sigma_dev: n doubles,
 * decreasing. n <= 1024. FFC_E_TOL_NOT_REACHED (soft) if Jacobi did not
 * converge. Synchronises.
 */
ffc_status ffc_spectrum(const double* K_dev, int64_t m, int64_t n, int64_t ldk, double eps, double* sigma_dev,
                        int64_t* rank_host, void* stream);

/*
 * ffc_leverage_batched - ffc_leverage of B blocks at once (the eigen-
 * decompositions run concurrently, one CTA per block). Host arrays of B
 * entries: K_dev[b] (m[b] x n[b], ld ldk[b]), lev_dev[b] (m[b]),
 * sigma_dev[b] (n[b]); rank_host[b] receives r. Synchronises; returns the
 * first non-OK status (FFC_E_TOL_NOT_REACHED if some Jacobi did not converge).
 */
ffc_status ffc_leverage_batched(int32_t B, const double* const* K_dev, const int64_t* m, const int64_t* n,
                                const int64_t* ldk, double eps, int64_t r_fixed, double* const* lev_dev,
                                double* const* sigma_dev, int64_t* rank_host, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FFC_H */
