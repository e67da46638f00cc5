/*
 * tlr.h -- C ABI of the GB300 tile low-rank (TLR) Matérn likelihood library.
 *
 * The library evaluates the Gaussian log-likelihood of eq. 1 (Sec. III),
 *     l(theta) = -n/2 log(2 pi) - 1/2 log|Sigma(theta)| - 1/2 z^T Sigma(theta)^{-1} z,
 * for the Matérn covariance of eq. 5 (Sec. IV) over n irregular 2-D locations,
 * with Sigma held in the tile low-rank format of Sec. V: nb x nb tiles, dense
 * diagonal tiles, off-diagonal tiles U V^T truncated at an absolute threshold
 * eps.  It also gives the gradient of l in theta (not in the paper) and the
 * kriging predictor of eq. 4 on the same factor.
 *
 * Conventions shared by every entry point
 *  - All array arguments are DEVICE pointers to contiguous float64 data unless
 *    stated otherwise; the caller owns them and keeps them alive until the work
 *    enqueued on `stream` has finished.  The library never frees caller memory.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *    stream.  Calls enqueue work on it and return without synchronising, except
 *    tlr_create / tlr_destroy / tlr_status / tlr_rank_stats / tlr_memory, which
 *    synchronise, and tlr_compress / tlr_potrf / tlr_loglik_grad, which
 *    synchronise once to check that the low-rank storage sufficed.
 *  - Vectors indexed by point (z, e, outputs) are in the CALLER's point order;
 *    the internal Morton permutation is applied and undone inside.
 *  - Return value: TLR_OK (0); -i when argument i (1-based) is invalid (nothing
 *    is enqueued); a positive TLR_ERR_* code otherwise.  Failures that happen on
 *    the device (non-SPD pivot, rank cap overflow, wait time-out) are recorded in
 *    the handle and reported by tlr_status after the stream has drained.
 *  - The library owns its tile storage, allocated with cudaMalloc in tlr_create.
 *    The low-rank factors live in rank-packed arenas (each tile a block of about
 *    1.25 times its rank in columns, a new block when its rank outgrows it): an
 *    arena that runs out is enlarged and the operation repeated inside
 *    tlr_compress, tlr_potrf (from regenerated tiles) or tlr_loglik_grad.  The
 *    gradient's inverse L^{-1} (its own arena and dense tiles) and a second
 *    stream with its workspace are allocated by the first tlr_loglik_grad; a
 *    dense pool grows in tlr_compress when more tiles turn dense.  TLR_ERR_OOM
 *    when an allocation fails.  Everything is released by tlr_destroy.
 */
#ifndef TLR_H_
#define TLR_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tlr_ctx* tlr_handle;
typedef void* tlr_stream_t; /* a cudaStream_t */

/* theta = (theta1, theta2, theta3) of eq. 5: variance, range, smoothness. */
typedef struct {
  double sigma2;
  double beta;
  double nu;
} tlr_theta;

/* Options.  nb: tile size (Sec. V); eps: absolute truncation threshold of the
 * off-diagonal tiles (a singular value s of a tile is kept iff s > eps; eps < 0
 * selects dense mode, every tile dense, the exact full-tile comparator);
 * rank_cap: largest rank an off-diagonal tile may take (0 = nb/2);
 * truncate_at_cap: 0 = exceeding rank_cap is an error (TLR_ERR_RANK_CAP),
 * 1 = keep the rank_cap largest terms; order: 1 = Morton (Z-curve) ordering of
 * the points before tiling, 0 = keep the caller's order; dense_rank: an
 * off-diagonal tile whose eps-rank exceeds it is stored and updated dense
 * (0 = max(16, nb/9)); tiles are also made dense where a dense x dense
 * product would land on them during the factorization; inv_scale: the
 * gradient's inverse keeps L^{-1} in tile low-rank form truncated at
 * inv_scale * eps * zeta^(1/2), zeta = the largest 1 / L_aa^2 (0 = 1: the same
 * truncation relative to the size of L^{-1} as eps is to Sigma);
 * Sigma^{-1} = L^{-T} L^{-1} is then formed densely tile by tile, a batch of
 * tiles at a time, each batch reduced into the gradient and overwritten by a
 * later one (with tensor cores; the double-float path keeps every tile).
 * metric: 0 = Euclidean distance; 1 = great-circle distance of eq. 6 (Sec. IV,
 * haversine) with x = longitude and y = latitude in degrees (also for the new
 * points of tlr_predict / tlr_predict_var) on a sphere of the given radius
 * (radius <= 0 = 1: distances in radians); beta is in the units of the distance.
 * precision: arithmetic of the gradient's inverse's batched tile contractions of
 * depth >= 256 (dense x dense and dense x thin updates, the triangular transforms
 * with the diagonal inverses, the stacked-panel products of Sigma^{-1}): 0 =
 * default, bf16 tensor cores (tcgen05) on 6 digit slices of every float64
 * operand, about 1e-12 of the operands' scale (see tlr_gemm_tc); 1 = double-float
 * on the CUDA cores (about 2^-44), no tensor cores; 4, 5, 6 = mixed precision:
 * tensor cores with that many slices (4: about 1e-9) in the gradient's inverse
 * and also in the Cholesky factorization's contractions of depth >= 256 (the
 * triangular transforms with L_kk^{-1} and the dense-target updates).  With
 * precision 0 and 1 the Cholesky uses double-float; dense mode (eps < 0) always
 * does. */
typedef struct {
  int nb;
  double eps;
  int rank_cap;
  int truncate_at_cap;
  int order;
  int dense_rank;
  double inv_scale;
  int metric;
  double radius;
  int precision;
} tlr_opts;

enum {
  TLR_OK = 0,
  TLR_ERR_NOT_SPD = 1,  /* a diagonal pivot <= 0; tlr_status gives the column (1-based, sorted order) */
  TLR_ERR_RANK_CAP = 2, /* an off-diagonal rank exceeded rank_cap */
  TLR_ERR_OOM = 3,      /* cudaMalloc failed */
  TLR_ERR_CUDA = 4,     /* a CUDA launch or runtime call failed */
  TLR_ERR_TIMEOUT = 5,  /* a device-side wait gave up */
  TLR_ERR_STATE = 6,    /* call out of order (e.g. tlr_loglik before tlr_potrf) */
  TLR_ERR_NUMERIC = 7   /* a non-finite value met in a low-rank recompression (tile index in info) */
};

/* Create a handle for n points (x[i], y[i]) (device pointers, length n).
 * Copies and (opts->order) Morton-orders the locations and allocates the tile
 * storage for n, opts->nb and opts->rank_cap.  Synchronises `stream`. */
int tlr_create(int64_t n, const double* x, const double* y, const tlr_opts* opts,
               tlr_stream_t stream, tlr_handle* out);

/* Release every device buffer of the handle.  Synchronises the device. */
int tlr_destroy(tlr_handle h);

/* Sec. IV eq. 5: build the device Bessel-K table for theta and generate the
 * dense diagonal tiles Sigma_kk (in dense mode every tile).  Restarts the
 * pipeline: compress and factor must follow. */
int tlr_matern_generate(tlr_handle h, tlr_theta theta, tlr_stream_t stream);

/* Sec. V: generate and compress every off-diagonal tile to U V^T with the
 * absolute threshold eps (adaptive cross approximation on generated rows and
 * columns, then Householder QR of both factors and a column-pivoted QR of the
 * small core, truncated where the trailing part's Frobenius norm is <= eps).
 * A tile whose cross approximation needs more than dense_rank terms is kept
 * dense.  No-op in dense mode. */
int tlr_compress(tlr_handle h, double eps, tlr_stream_t stream);

/* In-place TLR Cholesky Sigma = L L^T (dense POTRF on diagonal tiles,
 * TRSM/SYRK/low-rank GEMM with recompression off the diagonal; Sec. III
 * "Cholesky factorization", Sec. VIII-C "TLR matrix-matrix multiplication").
 * A non-positive pivot sets TLR_ERR_NOT_SPD in the handle. */
int tlr_potrf(tlr_handle h, tlr_stream_t stream);

/* Eq. 1 on the factor: d_out3[0] = l, d_out3[1] = log|Sigma|,
 * d_out3[2] = z^T Sigma^{-1} z (device pointer to 3 doubles).  z: length n. */
int tlr_loglik(tlr_handle h, const double* z, double* d_out3, tlr_stream_t stream);

/* l and dl/dtheta = 1/2 a^T (dSigma/dtheta) a - 1/2 tr(Sigma^{-1} dSigma/dtheta),
 * a = Sigma^{-1} z (not in the paper).  d_ll: 1 double; d_grad3: 3 doubles
 * (sigma2, beta, nu).  dSigma tiles are regenerated, never stored. */
int tlr_loglik_grad(tlr_handle h, const double* z, double* d_ll, double* d_grad3,
                    tlr_stream_t stream);

/* Eq. 4: z_new = Sigma_12 Sigma_22^{-1} z_obs at m new locations (x_new, y_new),
 * Sigma_22 being the factored handle's matrix.  z_obs: length n; z_new: length m. */
int tlr_predict(tlr_handle h, const double* z_obs, int64_t m, const double* x_new,
                const double* y_new, double* z_new, tlr_stream_t stream);

/* Prediction variance of eq. 4's predictor (Sec. III: the conditional
 * covariance Sigma_11 - Sigma_12 Sigma_22^{-1} Sigma_21, its diagonal):
 * var_new[i] = sigma2 - |L^{-1} sigma_i|^2 with sigma_i the covariances between
 * new point i and the observed points, L the handle's factor.  x_new, y_new:
 * m doubles each; var_new: m doubles (device).  Up to 1,024 new points at a
 * time: their covariance columns are generated and L^{-1} applied to all of
 * them by one batched tile forward solve (three batched GEMM launches per
 * tile column, workspace from the handle). */
int tlr_predict_var(tlr_handle h, int64_t m, const double* x_new, const double* y_new,
                    double* var_new, tlr_stream_t stream);

/* Synthetic measurements of Sec. VIII-D: z = L e on the factored handle (in
 * dense mode L is the exact Cholesky factor: a draw from the model itself).
 * e, z: n doubles (device, caller's order). */
int tlr_sample(tlr_handle h, const double* e, double* z, tlr_stream_t stream);

/* Independent regions (exact likelihood of many unrelated problems, e.g. the
 * regions of a large field, Sec. VII-VIII): l and dl/dtheta of R problems.
 * n, x, y, z, theta, opts are host arrays of length R; x[r], y[r], z[r] are
 * device arrays of n[r] doubles; opts[r] may differ per region (tile size,
 * threshold; eps < 0 is dense).  d_ll (device, R doubles) and d_grad (device,
 * 3R doubles, sigma2/beta/nu per region) receive the results; status (host,
 * R ints) each region's TLR status.  nworkers host threads (0 = 8), each with
 * its own stream, take regions in turn and keep one handle per tile size,
 * allocated once at the capacity of the largest region using it and rebound
 * to each region's points.  Returns when every region is done; `stream` is
 * ordered after the work.  Returns the first worker failure, else TLR_OK. */
int tlr_loglik_grad_batched(int R, const int64_t* n, const double* const* x, const double* const* y,
                            const double* const* z, const tlr_theta* theta, const tlr_opts* opts, double* d_ll,
                            double* d_grad, int* status, int nworkers, tlr_stream_t stream);

/* Synchronise the handle's last stream and report the first device-side
 * failure (TLR_OK if none); *info gets the failing column for
 * TLR_ERR_NOT_SPD, the offending tile index for TLR_ERR_RANK_CAP. */
int tlr_status(tlr_handle h, int64_t* info);

/* Rank statistics of the off-diagonal tiles of the current factor (or of the
 * compressed matrix before tlr_potrf) and the bytes the TLR factor occupies
 * (dense diagonal tiles + U, V columns actually used).  Synchronises. */
int tlr_rank_stats(tlr_handle h, int* kmin, double* kmean, int* kmax, int64_t* bytes);

/* Number of tiles per side (nt) and the tile size of the handle. */
int tlr_shape(tlr_handle h, int* nt, int* nb);

/* Copy tile (i, j), i >= j, of the handle's current matrix (after
 * tlr_matern_generate / tlr_compress) or factor (after tlr_potrf) into caller
 * device buffers, rows and columns in the handle's sorted point order
 * (tlr_get_perm).  i == j or a dense tile: the dense nb x nb tile into U
 * (column-major, ld nb; U must hold nb * nb doubles), *k = nb.  A low-rank
 * tile: U and V (nb x k each, column-major, ld nb) with k the tile's rank;
 * U and V must hold nb * rank_cap doubles.
 * *k and *dense are host ints (*dense = 1 for a dense tile).  Synchronises
 * `stream`. */
int tlr_get_tile(tlr_handle h, int i, int j, double* U, double* V, int* k, int* dense, tlr_stream_t stream);

/* Number of off-diagonal tiles stored low rank and dense in the current
 * plan (after tlr_compress, or tlr_matern_generate in dense mode). */
int tlr_tile_counts(tlr_handle h, int64_t* n_lowrank, int64_t* n_dense);

/* perm[s] = caller index of the s-th point in the handle's sorted order
 * (device buffer of n int32).  Synchronises `stream`. */
int tlr_get_perm(tlr_handle h, int* perm, tlr_stream_t stream);

/* Allocation-free variant (the paper has no counterpart).  The Gaussian
 * log-likelihood of n <= 1024 points with Euclidean distances (the Matérn
 * covariance generated, Cholesky-factored, the log-determinant and the
 * quadratic form z^T Sigma^{-1} z taken), evaluated as one dense tile with every
 * piece of workspace in a static device array of the library (about 8.5 MB per
 * GPU).  For callers that cannot call cudaMalloc, e.g. because their process
 * has handed all device memory to another allocator or may not allocate after
 * start-up.  x, y, z: device arrays of n doubles (caller's order); d_out3:
 * device array of 3 doubles (l, log|Sigma|, z^T Sigma^{-1} z).  Makes no
 * allocation of its own, on the device or on the host heap.  The static array
 * is reserved on a device when the library's code for it is loaded there: with
 * CUDA's default lazy module loading that is the first call on the device, which
 * can then fail with TLR_ERR_CUDA under memory pressure, so make that first call
 * at start-up (or set CUDA_MODULE_LOADING=EAGER to reserve it when the library
 * is loaded); the device holds it until the process exits.  The first call on a
 * device also looks up the array's address.  Every call synchronises `stream`
 * (it reads the points' bounding box and the status back to the host), so it
 * must not be called while `stream` is being captured into a graph.  All calls
 * share the array: calls that overlap on the GPU race.
 * Returns TLR_OK; -1 for n outside 1..1024; -2, -3, -4 for a null x, y, z; -5 for
 * a theta entry that is not positive and finite; -6 for a null d_out3;
 * TLR_ERR_NOT_SPD when the covariance is not positive definite (e.g. repeated
 * points; d_out3 then holds no valid likelihood); TLR_ERR_CUDA for a failed CUDA
 * call, or a device ordinal >= 128. */
int tlr_loglik_dense_noalloc(int64_t n, const double* x, const double* y, const double* z, tlr_theta theta,
                             double* d_out3, tlr_stream_t stream);

/* Diagnostics (no counterpart in the paper). */

/* The float64-accurate tensor-core GEMM used for the dense tile contractions,
 * as one call: C = beta C + alpha op(A) op(B) with op(X) = X^T when tX != 0,
 * op(A) m x k, op(B) k x n, column-major A (lda), B (ldb), C (ldc), device
 * pointers.  Each row of op(A) and column of op(B) is scaled by a power of two
 * and cut into `slices` (4..6) bf16 digits of 8 bits (error-free splitting,
 * Ozaki et al. 2012); the digit products run on tcgen05 with exact float32
 * accumulation of the leading groups.  |error| <= |alpha| k 2^sa_i 2^sb_j
 * ((slices + 4) 2^(-8 slices) + 2^-38) with 2^sa_i, 2^sb_j the powers of two
 * above the largest magnitude of row i of op(A) and column j of op(B).
 * Allocates and frees its own workspace (cudaMalloc) and synchronises `stream`.
 * Returns -i for an invalid argument i, TLR_ERR_OOM, TLR_ERR_CUDA, or
 * TLR_ERR_TIMEOUT when a device-side wait gave up. */
int tlr_gemm_tc(int m, int n, int k, const double* A, int lda, int tA, const double* B, int ldb, int tB, double* C,
                int ldc, double alpha, double beta, int slices, tlr_stream_t stream);

/* Device memory held by the handle, in bytes: *total (everything it has
 * allocated), *arenas (the rank-packed low-rank arenas of L and of the
 * inverse), *arena_used (the part of them handed out to tiles) and *workspace
 * (batched-kernel, update and gradient workspaces).  Any output may be NULL.
 * Synchronises. */
int tlr_memory(tlr_handle h, int64_t* total, int64_t* arenas, int64_t* arena_used, int64_t* workspace);

/* Rank statistics of the low-rank tiles of the inverse Sigma^{-1} built by the
 * last tlr_loglik_grad, and its number of dense off-diagonal tiles.
 * Synchronises. */
int tlr_inverse_stats(tlr_handle h, int* kmin, double* kmean, int* kmax, int64_t* n_dense);

/* While profiling is enabled (tlr_profile), device time of each phase of the
 * path (generate, compress, chol.*, trtri.*, lauum.*, solves, grad_fused,
 * update.*) is recorded with CUDA events.  Writes a JSON object
 * {"phase": [ms, count, launches], ...} into buf (len bytes, host memory):
 * device time, times entered, and kernel launches issued inside it.
 * Synchronises the device. */
int tlr_profile_phases(char* buf, int64_t len);

/* Total kernel launches issued by the library in this process. */
int tlr_launch_count(int64_t* count);

/* enable != 0: from now on time every launch of the low-rank update kernel
 * (the TLR GEMM with recompression, the dominant kernel) with CUDA events on
 * its stream and accumulate its algorithmic float64 flops on the device
 * (Householder QR, core product and its pivoted QR, applying Q, forming the
 * product); enable == 0 stops.  Either call resets the counters
 * and synchronises the device. */
int tlr_profile(int enable);

/* Launches timed, their summed device time (ms) and flops since tlr_profile.
 * Synchronises the device. */
int tlr_profile_read(int64_t* launches, double* ms, double* flops);

/* The same for the tensor-core GEMM (k_oz_gemm, every launch while profiling
 * is enabled): launches, summed device time (ms) and the bf16 tensor-core
 * flops issued (2 M N K of every slice-pair MMA).  Synchronises the device. */
int tlr_profile_read_tc(int64_t* launches, double* ms, double* flops);

#ifdef __cplusplus
}
#endif
#endif /* TLR_H_ */
