/*
 * hdf.h -- C ABI of the GB300 Harmonic Decomposition Factorization library (libhdf.so).
 *
 * Method: Ryan & Damle, "Linear Time Kernel Matrix Approximation via Hyperspherical
 * Harmonics", ICML 2022.  For points x_1..x_n in R^d and an isotropic kernel k(|x - y|)
 * the library builds K ~= U diag(S) U^T (Algorithm 1 in the symmetric form of Remark 1)
 * with a relative error target tol (the abstract: the method takes the tolerance, not
 * the rank, as input), then applies K~ V = U (S (U^T V)) (Sec. 3.6) and solves
 * (lambda I + K~) X = B (the system of Eq. opt, via Sherman-Morrison-Woodbury, Sec. 1).
 *
 * Conventions for every entry point below:
 *  - Every call returns an hdf_status; nothing throws across the ABI.  On error the
 *    output buffers are left untouched and hdf_last_error() (thread-local) describes it.
 *  - "_dev" pointers are CUDA device pointers, "_host" pointers host memory.  The caller
 *    owns every buffer it passes; the library owns the opaque hdf_factor and the device
 *    memory inside it (U, S and work space), released by hdf_free.
 *  - Points are row-major n x d FP64 (x[i*d + j]).  Vector blocks V, Y, B, X are
 *    column-major n x ncols with a leading dimension >= n, in the factor's bulk type
 *    (double for HDF_FP64, float for HDF_FP32).
 *  - Work is ordered on the given stream (NULL = legacy default stream).  hdf_build
 *    synchronises the stream (host planning needs device reductions); hdf_matvec is
 *    asynchronous; hdf_solve synchronises (its small core is solved on the host).
 *  - Supported: 3 <= d <= 8, n >= 1, tol in (0, 1), lengthscale > 0, p_max <= 128.
 */
#ifndef HDF_H
#define HDF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hdf_factor hdf_factor;       /* opaque, owned by the library */
typedef void* hdf_stream;                    /* a cudaStream_t; NULL = default stream */

typedef enum {
    HDF_OK = 0,
    HDF_EINVAL = 1,           /* bad argument (message in hdf_last_error) */
    HDF_ENOMEM = 2,           /* device or host allocation failed */
    HDF_ECUDA = 3,            /* a CUDA call failed */
    HDF_ETOL_UNREACHABLE = 4, /* degree cap p_max hit: the factor is built at p = p_max and
                                 hdf_factor_info reports the Chebyshev tail achieved */
    HDF_ENOTFINITE = 5,       /* NaN or Inf in the input points */
    HDF_ESINGULAR = 6,        /* the solve core is singular */
    HDF_ETIMEOUT = 7,         /* a bounded device wait expired */
    HDF_ETOOBIG = 8           /* a size exceeds a documented limit */
} hdf_status;

/* Isotropic kernels of Sec. 4.1 with lengthscale l (the Gaussian in the exp(-r^2/(2 l^2))
 * convention; the paper's exp(-(r/sigma)^2) is the same family with sigma = sqrt(2) l). */
typedef enum {
    HDF_GAUSSIAN = 0,   /* exp(-r^2 / (2 l^2)) */
    HDF_CAUCHY = 1,     /* 1 / (1 + r^2 / l^2) */
    HDF_MATERN32 = 2,   /* (1 + sqrt3 r/l) exp(-sqrt3 r/l) */
    HDF_MATERN52 = 3    /* (1 + sqrt5 r/l + 5 r^2/(3 l^2)) exp(-sqrt5 r/l) */
} hdf_kernel;

/* Bulk precision: the type of U, of the harmonics and of the matvec GEMMs.  The radial
 * basis, its Gram matrix, the cores and every small factorisation stay FP64. */
typedef enum {
    HDF_FP64 = 0,
    HDF_FP32 = 1
} hdf_precision;

typedef struct {
    int p_max;      /* cap on the Chebyshev degree p (even; default 64, max 128) */
    double eta;     /* share of tol given to eigenpair truncation (default 1) */
    int flags;      /* HDF_FLAG_* bits, 0 for defaults */
} hdf_options;

/* Run the matvec GEMMs of an FP32 factor on the CUDA cores instead of the tensor cores. */
#define HDF_FLAG_CUDA_CORES 1
/* Build the matrix-free form (d >= 4): U is not stored.  Every harmonic of degree k with chain
 * (m = mu_1, mu_2, ...) is P_0(m, k - m) times a harmonic Z_m of degree m in d - 1 dimensions
 * (the product form of the chain construction), so per point the factor keeps the Z row
 * (sum_m |H_m^(d-1)| values) and the row of P_0(m, k - m) F[k, s] (sum_k s_k (k + 1) values)
 * instead of the U row (sum_k s_k |H_k| values), and hdf_matvec / hdf_matvec_transpose /
 * hdf_matvec_adjoint form U^T V and U W from them.  hdf_build selects this form by itself
 * (for d >= 4) when U would take more than 80% of the device's memory -- the cost that
 * Sec. 3.6 counts and Sec. 3.7 names as the method's limit.  A matrix-free factor has no
 * solve (HDF_EINVAL), no hdf_matvec_noalloc (HDF_EINVAL), hdf_factor_device gives U_dev = NULL
 * and hdf_factor_export accepts U_host = NULL only.  hdf_info.matrix_free reports the form. */
#define HDF_FLAG_MATRIX_FREE 2

#define HDF_MAX_D 8
#define HDF_MAX_L 64
#define HDF_NPHASE 8

typedef struct {
    int64_t n;
    int d;
    int precision;          /* hdf_precision */
    int p;                  /* Chebyshev degree chosen (Remark 3) */
    int L;                  /* p / 2, the highest harmonic degree */
    int reached;            /* 1 if the tail budget was met at p <= p_max */
    int64_t rank;           /* r = sum_k |H_k| s_k (Sec. 3.6) */
    int64_t ldu;            /* leading dimension of the row-major n x r U */
    int64_t nharm;          /* number of harmonics evaluated per point */
    double center[HDF_MAX_D];
    double radius;          /* R = max |x_i - c|; x' = (x - c) / (2R) */
    double mu2;             /* mean of K_ij^2 used for |K|_F = n sqrt(mu2) */
    double cheb_tail;       /* estimated Chebyshev tail epsilon_c(p) (Sec. 3.5) */
    double tail_budget;     /* tol sqrt(mu2) / 2 */
    double drop_budget;     /* eta tol n sqrt(mu2) / 2 */
    double dropped_cost;    /* sum over dropped eigenpairs of |lambda| |H_k| / |S^{d-1}| */
    double err_bound;       /* (n cheb_tail + dropped_cost) / (n sqrt(mu2)): a-priori bound
                               on |K - K~|_F / |K|_F */
    int s_k[HDF_MAX_L + 1]; /* kept radial rank per harmonic degree k (Sec. 3.4) */
    double t_ms[HDF_NPHASE];/* build phase times in ms: 0 centre/radius/mu2 reductions,
                               1 Chebyshev + degree + radial cores (host, while the device
                               sums the radial moments), 2 rest of the moments + radial-basis
                               Gram, 3 basis factor + eigendecompositions + truncation (host),
                               4 radial factors (device), 5 harmonics + U (device), 6 the
                               Gram U^T U of the first hdf_solve (device; 0 before it),
                               7 whole build */
    int64_t n_y;            /* cross factor (hdf_build_cross): points of the second set Y, the
                               rows of its factor V; 0 for a symmetric factor U S U^T */
    int matrix_free;        /* 1 if U is not stored (HDF_FLAG_MATRIX_FREE) */
    int64_t mf_row;         /* matrix-free form: stored values per point (Z and P_0 F rows) */
    double lu_ms;           /* time of the last factorization of the solve's core (ms; 0 before) */
} hdf_info;

/* ---------------------------------------------------------------- factorization ---- */

/* Build K ~= U S U^T for the points x_dev (row-major n x d FP64, device) -- Algorithm 1,
 * symmetric form (Remark 1).  Steps: centre and scale to |x'| <= 1/2 (Sec. 3.3 footnote),
 * Chebyshev coefficients and degree (Sec. 3.3, Remark 3), radial cores (Eq. rdef,
 * App. A), radial-basis QR (Eq. svd), eigendecomposition and truncation (Sec. 3.4,
 * Remark 2), harmonics times radial factors into U (Algorithm 1's inner loops).
 * opt may be NULL.  *out receives a new factor on HDF_OK or HDF_ETOL_UNREACHABLE (the
 * latter still returns a usable factor at p = p_max); otherwise *out is set to NULL.
 * Synchronises the stream. */
hdf_status hdf_build(const double* x_dev, int64_t n, int d, hdf_kernel kernel,
                     double lengthscale, double tol, hdf_precision prec,
                     const hdf_options* opt, hdf_stream stream, hdf_factor** out);

/* Build K(X, Y) ~= U S V^T for two point sets -- Algorithm 1 in its general form: X = x_dev
 * (row-major m x d FP64, device) and Y = y_dev (row-major n x d).  Both sets are centred and
 * scaled by one map (centre = mean of the union, R = the largest distance of a point of
 * either set from it) so that every |x' - y'| <= 1 (Sec. 3.3); mu2 is the mean of
 * k(x_i, y_j)^2 over cross pairs (strided 512-point samples of each set), the degree
 * budget is tol sqrt(mu2) / 2 and the truncation budget eta tol sqrt(m n mu2) / 2.  The
 * radial bases of X and Y are factored separately (the two QRs of Eq. svd), each block
 * R_X Gamma_k R_Y^T is split by an SVD, and singular triples are dropped by the rule of the
 * symmetric build with sigma in place of |lambda|.  S holds the kept singular values; U
 * (m rows) and V (n rows) share the column order (k, s, h) of hdf_build.  The factor
 * answers hdf_matvec (K~ V for blocks of n rows, results of m rows), hdf_matvec_transpose,
 * hdf_factor_info (n = m, n_y = n), hdf_factor_export (U, S), hdf_factor_export_y (V) and
 * hdf_free; hdf_solve, hdf_matvec_adjoint and hdf_matvec_noalloc return HDF_EINVAL for it.
 * Limits, statuses and synchronisation as hdf_build. */
hdf_status hdf_build_cross(const double* x_dev, int64_t m, const double* y_dev, int64_t n, int d,
                           hdf_kernel kernel, double lengthscale, double tol, hdf_precision prec,
                           const hdf_options* opt, hdf_stream stream, hdf_factor** out);

/* Y = K~ V = U (S (U^T V)) (Sec. 3.6: O(n r) per column).  V_dev and Y_dev are column-major
 * n x ncols blocks (leading dimensions ldv, ldy >= n) of the factor's bulk type; they must
 * not overlap.  1 <= ncols <= 1024.  Asynchronous on the stream.  For a cross factor
 * Y = U (S (V^T V_dev)): V_dev has n_y rows (ldv >= n_y) and Y_dev has n rows. */
hdf_status hdf_matvec(const hdf_factor* f, const void* V_dev, int64_t ldv, int ncols,
                      void* Y_dev, int64_t ldy, hdf_stream stream);

/* Y = K~^T V.  For a cross factor Y = V (S (U^T V_dev)): V_dev has n rows (ldv >= n), Y_dev
 * has n_y rows (ldy >= n_y).  For a symmetric factor the same product as hdf_matvec.
 * Otherwise as hdf_matvec. */
hdf_status hdf_matvec_transpose(const hdf_factor* f, const void* V_dev, int64_t ldv, int ncols,
                                void* Y_dev, int64_t ldy, hdf_stream stream);

/* K~ V as hdf_matvec computes it, for callers that cannot allocate device memory during the
 * call: code whose device memory belongs to another allocator's pool (a raw cudaMalloc may
 * fail while that pool holds the free memory), or loops that reserve all memory up front and
 * must not enter the CUDA allocator.  The paper has no counterpart; this is a library
 * convenience.  The partial sums live in a fixed 32 MiB array inside the library (held on
 * every device that loads it until the process exits) instead of memory obtained per call; no
 * cudaMalloc, cudaFree or allocating library routine is called.  Limit: ldu (the padded width
 * of U that hdf_factor_info reports) * min(ncols, 64) * (8 + element size) bytes <= 32 MiB,
 * otherwise HDF_ETOOBIG.  The products run on the CUDA-core kernels: for an FP64 factor the
 * result equals hdf_matvec's, for an FP32 factor (where hdf_matvec may use the tensor cores) it
 * agrees to FP32 rounding.  The first call on each device looks up the array's device address
 * with that device current; make that first call before any stream capture.  All calls share
 * the one array (each call overwrites every entry it reads), so calls whose executions overlap
 * on the GPU -- on different streams or from different threads -- race and must be serialised
 * by the caller.  Arguments and layout as hdf_matvec. */
hdf_status hdf_matvec_noalloc(const hdf_factor* f, const void* V_dev, int64_t ldv, int ncols,
                              void* Y_dev, int64_t ldy, hdf_stream stream);

/* X = (lambda I + K~)^{-1} B (Eq. opt with the Woodbury identity of Sec. 1), followed by
 * refine_steps steps of iterative refinement X += (lambda I + K~)^{-1} (B - lambda X - K~ X).
 * lambda > 0.  U^T U is formed on the device on the first call (tensor cores for FP32 factors)
 * and kept; the r x r core lambda S^-1 + U^T U (indefinite: S has eigenvalues of both signs) is
 * factored in FP64 by a blocked LU with partial pivoting -- each 64-column panel on the host
 * threads, the interchanges and the trailing updates on the device -- and its factors are kept
 * on the device per lambda; the triangular solves run on the device.  The padded rank (ldu) must
 * be <= 32768 (HDF_ETOOBIG); device memory for two r x r FP64 matrices is needed.  HDF_ESINGULAR
 * if the core is singular.  Synchronises. */
hdf_status hdf_solve(hdf_factor* f, double lambda, const void* B_dev, int64_t ldb, int ncols,
                     void* X_dev, int64_t ldx, int refine_steps, hdf_stream stream);

/* Adjoint of f = sum_j w_j^T K~ v_j (j < ncols <= 64) with respect to the points and the
 * lengthscale.  The paper does not differentiate the factorization; the semantics are
 * "frozen structure": the build's scaling (c, R), degree p, radial-basis factor and kept
 * eigenvectors stay fixed, so row i of U is a smooth function of x_i and S depends on l
 * only through the radial cores (Eq. rdef).  x_dev must be the points the factor was
 * built from (row-major n x d FP64).  V_dev, W_dev: column-major n x ncols blocks of the
 * bulk type.  Output: grad_x_dev (row-major n x d, bulk type, overwritten), and on the
 * host grad_l_host (d f / d l) and value_host (f) when non-NULL.  Harmonics, radial factors
 * and their derivatives are recomputed per point; U's Jacobian is never stored.
 * Synchronises the stream. */
hdf_status hdf_matvec_adjoint(hdf_factor* f, const double* x_dev, const void* V_dev, int64_t ldv,
                              const void* W_dev, int64_t ldw, int ncols, void* grad_x_dev,
                              double* grad_l_host, double* value_host, hdf_stream stream);

/* ------------------------------------------------------------------ batches ---- */
typedef struct hdf_batch hdf_batch;          /* opaque, owned by the library */

/* Factor nsets independent point sets in one pass: set s is rows offsets[s]..offsets[s+1]-1
 * of x_dev (row-major FP64, d columns; offsets_host[0] = 0, every set non-empty) with its own
 * lengthscale lengthscales_host[s].  Each set is factored exactly as hdf_build would
 * factor it alone (Algorithm 1, symmetric form, same tol, kernel and options); the batch only
 * schedules the work together: segmented device reductions, per-set host planning on
 * threads, and one persistent kernel that builds the radial factors and U of every set.
 * Returns HDF_ETOL_UNREACHABLE (with a usable batch) if any set was capped at p_max.
 * Synchronises the stream. */
hdf_status hdf_build_batched(int nsets, const int64_t* offsets_host, const double* x_dev, int d,
                             hdf_kernel kernel, const double* lengthscales_host, double tol,
                             hdf_precision prec, const hdf_options* opt, hdf_stream stream,
                             hdf_batch** out);

/* Y_s = K~_s V_s for every set at once: V_dev, Y_dev are column-major (sum n) x ncols blocks of
 * the bulk type whose rows follow the concatenated points; 1 <= ncols <= 64.  The kernels are
 * recorded in a CUDA graph on the first call for a given (V, Y, ldv, ldy, ncols) and replayed
 * on later calls.  Asynchronous on the stream. */
hdf_status hdf_batch_matvec(hdf_batch* b, const void* V_dev, int64_t ldv, int ncols,
                            void* Y_dev, int64_t ldy, hdf_stream stream);

/* Metadata of set s (as hdf_factor_info). */
hdf_status hdf_batch_info(const hdf_batch* b, int set, hdf_info* info);

/* Phase times of the batched build in ms (layout of hdf_info.t_ms; index 5 is the CUDA graph of
 * the radial-factor phase and the U phases of every size class, index 4 is 0). */
hdf_status hdf_batch_timings(const hdf_batch* b, double* t_ms);

/* *flag = 1 if a kernel of hdf_batch_matvec on this batch gave up a bounded wait since the last
 * call (the outputs of that product are then invalid), else 0; clears the flag.  Synchronises
 * the device. */
hdf_status hdf_batch_device_errors(const hdf_batch* b, int* flag);

/* Copy set s's U (n_s x rank_s, packed row-major, bulk type) and S (FP64) to the host. */
hdf_status hdf_batch_export(const hdf_batch* b, int set, void* U_host, double* S_host);

void hdf_batch_free(hdf_batch* b);

/* ------------------------------------------------------ kernel ridge regression ---- */
/* Sec. 4.2 of the paper: the regularised system (lambda I + K) w = y of Eq. (opt) for the
 * training points, with K replaced by K^ = the HDF factors of its diagonal blocks K_{C_i C_i}
 * (clusters C_i of the points) plus the exact off-diagonal blocks, solved by conjugate
 * gradients preconditioned by the inverses of the exact blocks lambda I + K_{C_i C_i}.
 * Predictions y* = K(x*, x) w use the exact kernel (hdf_kernel_matvec). */
typedef struct hdf_krr hdf_krr;              /* opaque, owned by the library */

/* k-means clustering by Lloyd's iteration (the clusters of Sec. 4.2): from the centres
 * x[init_host[c]] (c < k; the caller draws them), assign every point to its nearest centre
 * (squared distance, lowest index on ties) and move each centre to the mean of its points (a
 * centre without points stays), until no assignment changes or max_iter assignment passes.
 * x_dev: row-major n x d FP64.  Output labels_dev (n ints, device), optionally centres_dev
 * (k x d FP64, device) and *iterations (assignment passes made).  1 <= d <= 8, 1 <= k <= n,
 * k d <= 6144.  Synchronises. */
hdf_status hdf_kmeans(const double* x_dev, int64_t n, int d, int k, const int64_t* init_host, int max_iter,
                      int* labels_dev, double* centres_dev, int* iterations, hdf_stream stream);

/* out[i] = sum_j k(|xq_i - x_j|) w_j for all m query points (the predictions of Sec. 4.2):
 * direct evaluation with coordinates shifted by x_0 and rounded to FP32 and FP32 kernel values
 * (relative error ~1e-7 per value); the products with w and their sums are formed in
 * double-float arithmetic within tiles of 128 points and in FP64 across tiles, so the result is
 * linear in w to ~1e-14.  xq_dev (m x d), x_dev (n x d) row-major FP64; w_dev (n), out_dev (m)
 * FP64.  Asynchronous. */
hdf_status hdf_kernel_matvec(const double* xq_dev, int64_t m, const double* x_dev, int64_t n, int d,
                             hdf_kernel kernel, double lengthscale, const double* w_dev, double* out_dev,
                             hdf_stream stream);

/* Build the operator of Sec. 4.2 for the points x_dev (row-major n x d FP64) grouped by
 * labels_dev (n non-negative ints, device; empty labels are skipped): the points are permuted
 * cluster by cluster, the diagonal blocks are factored by one hdf_build_batched call (kernel,
 * lengthscale, tol, prec, opt as there), the exact blocks lambda I + K_{C_i C_i} are formed on
 * the device and inverted on the host (Cholesky, FP64), and the off-diagonal blocks are
 * evaluated on the fly in every product (as hdf_kernel_matvec, pairs within one cluster
 * skipped).  lambda > 0.  Limit: sum of squared cluster sizes <= 2^28 (HDF_ETOOBIG).  Returns
 * HDF_ETOL_UNREACHABLE (with a usable operator) if a block was capped at p_max; HDF_ESINGULAR
 * if a block lambda I + K_cc is not positive definite.  Synchronises. */
hdf_status hdf_krr_build(const double* x_dev, int64_t n, int d, const int* labels_dev, hdf_kernel kernel,
                         double lengthscale, double lambda, double tol, hdf_precision prec,
                         const hdf_options* opt, hdf_stream stream, hdf_krr** out);

/* out = (lambda I + K^) v (v_dev, out_dev: n FP64 in the caller's point order).  Asynchronous. */
hdf_status hdf_krr_apply(hdf_krr* K, const double* v_dev, double* out_dev, hdf_stream stream);

/* z = M r with M the block-diagonal preconditioner (inverses of lambda I + K_{C_i C_i}).
 * Asynchronous. */
hdf_status hdf_krr_precond(hdf_krr* K, const double* r_dev, double* z_dev, hdf_stream stream);

/* w = (lambda I + K^)^{-1} y by preconditioned CG from w_0 = 0, stopped when the recurrence
 * residual |r| / |y| <= rtol or after max_iter iterations (then HDF_ETOL_UNREACHABLE with the
 * last iterate in w_dev).  y_dev, w_dev: n FP64 in the caller's order.  *iterations and
 * *relres (may be NULL) receive the count and the final relative residual.  Synchronises
 * once per iteration (the CG scalars are formed on the host). */
hdf_status hdf_krr_solve(hdf_krr* K, const double* y_dev, double rtol, int max_iter, double* w_dev,
                         int* iterations, double* relres, hdf_stream stream);

/* Number of clusters, total HDF rank of the diagonal blocks and build times in ms (t_ms2[0]:
 * permutation + batched factorization, t_ms2[1]: block preconditioner).  Pointers may be NULL. */
hdf_status hdf_krr_info(const hdf_krr* K, int* nclusters, int64_t* rank_total, double* t_ms2);

void hdf_krr_free(hdf_krr* K);

/* Metadata of a factor (sizes, scaling, degree, ranks, error budget and bound). */
hdf_status hdf_factor_info(const hdf_factor* f, hdf_info* info);

/* Device pointers to U (row-major n x ldu, bulk type) and S (rank entries, bulk type). */
hdf_status hdf_factor_device(const hdf_factor* f, const void** U_dev, const void** S_dev);

/* Copy U (n x rank, row-major, bulk type, packed: leading dimension rank) and S (FP64) to
 * host buffers the caller allocated.  Either pointer may be NULL.  Synchronises. */
hdf_status hdf_factor_export(const hdf_factor* f, void* U_host, double* S_host);

/* Copy the second factor V of a cross factor (n_y x rank, row-major, bulk type, packed) to a
 * host buffer.  HDF_EINVAL for a symmetric factor.  Synchronises. */
hdf_status hdf_factor_export_y(const hdf_factor* f, void* V_host);

/* Device times (ms, CUDA events on the launching stream) of the most recent hdf_matvec on
 * this factor, first column group: ms3[0] U^T V, ms3[1] partial reduction and scaling by S,
 * ms3[2] U W.  Waits for those events.  HDF_EINVAL if no matvec has run yet. */
hdf_status hdf_matvec_timings(const hdf_factor* f, double* ms3);

/* *flag = 1 if a device kernel working on this factor gave up a bounded wait (its results
 * are then invalid), else 0; clears the flag.  Synchronises the device.  The synchronising
 * calls (hdf_solve, hdf_matvec_adjoint) make the same check themselves and return
 * HDF_ETIMEOUT, with their outputs invalid, when a wait of theirs ran out. */
hdf_status hdf_device_errors(const hdf_factor* f, int* flag);

/* ------------------------------------------------------------- failure detection ---- */
/* Not part of the method (the paper has no failure model): hooks that let a caller or a test
 * drive the library's failure paths without faulting the GPU. */

/* Limit, in clock cycles of the current device, of every wait of the tensor-core kernels on
 * work (a tile, a buffer, an accumulator); cycles <= 0 restores the default (4e9, about 2 s).
 * A kernel whose wait runs out sets its factor's error flag, lets every copy and MMA it issued
 * finish (those drains keep the default limit), frees its tensor memory and returns; the
 * factor stays usable.  *previous (may be NULL) receives the old limit.  Applies to every
 * later launch on the current device until changed; synchronous. */
hdf_status hdf_set_wait_limit(long long cycles, long long* previous);

/* Self-check of the operand rounding of the tensor-core products (3xTF32, FP32 bulk): each FP32
 * operand x is split into hi = x rounded to TF32 (10 mantissa bits, nearest, ties away from
 * zero) and lo = x - hi; the library forms hi with integer operations on the bit pattern.  Runs
 * one kernel over all 2^32 bit patterns and compares that rounding with the device's own
 * conversion instruction on every finite value; mismatches[0] receives the count below 2^127 in
 * magnitude, mismatches[1] the count in the top binade (where rounding up overflows).  Both
 * are 0 on a correct build.  Synchronous; needs a device. */
hdf_status hdf_check_tf32_rounding(unsigned long long* mismatches);

/* Host-side fault injection: the device allocation `after` allocations from now (0 = the next
 * one) made by the library reports out-of-memory without allocating, once; a negative value
 * cancels a pending injection.  The call that meets it returns HDF_ENOMEM with its output
 * buffers untouched (hdf_build and friends set *out = NULL).  Process-wide. */
void hdf_debug_fail_alloc(long long after);

/* Release a factor (NULL is ignored). */
void hdf_free(hdf_factor* f);

/* --------------------------------------------------------- host planner (no GPU) ---- */
/* These run on the host only and need no device; they expose the planning steps so
 * that they can be checked on their own. */

/* Number of DCT nodes used for the Chebyshev coefficients: 4 (p_max + 2). */
int hdf_cheb_nodes(int p_max);

/* a[0..M-1]: Chebyshev coefficients of kappa(|r|) = k(two_r |r|; l) on [-1, 1] by the DCT
 * at M first-kind nodes (Sec. 3.3, Eq. chebtrunc); odd entries are exactly 0. */
hdf_status hdf_cheb_coeffs(hdf_kernel kernel, double lengthscale, double two_r, int M,
                           double* a_host);

/* Smallest even p <= p_max whose estimated tail sum_{p<i<M}|a_i| + sum_{i>=M/2}|a_i| is
 * <= budget (Remark 3).  *p gets the degree, *tail its tail, *reached 0 if capped. */
hdf_status hdf_choose_degree(const double* a_host, int M, double budget, int p_max,
                             int* p, double* tail, int* reached);

/* Radial cores Gamma_k, k = 0..p/2, of r^(k)(a, b) (Eq. rdef) in the basis
 * rho^(k mod 2) T_l(8 rho^2 - 1), l < nb_k, with nb_k = p/2 + 1 (even k) or p/2 (odd k).
 * cores_host receives the row-major nb_k x nb_k blocks one after another (total
 * sum_k nb_k^2 doubles; pass NULL to query the size in *count). */
hdf_status hdf_radial_cores(const double* a_host, int p, int d, double* cores_host,
                            int64_t* count);

/* ----------------------------------------------------------------------- errors ---- */
const char* hdf_status_string(hdf_status s);
/* Number of CUDA kernels this library has launched in the process so far (all threads). */
long long hdf_launch_count(void);
const char* hdf_last_error(void);           /* thread-local message of the last failure */

#ifdef __cplusplus
}
#endif
#endif /* HDF_H */
