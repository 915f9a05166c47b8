/*
 * kl.h - C ABI of the GB300 matrix-free Karhunen-Loeve library.
 *
 * The library computes the M largest eigenpairs of the discretised Fredholm
 * problem of Sec. 2 (Eq. hilbert_schmidt, Eq. fredholm) in the generalized
 * matrix form A v = lambda Z v of Sec. 1 (Eq. matrix_equations), by one of the
 * two matrix-free methods of Sec. 3:
 *
 *   KL_GALERKIN_IBQ  Sec. 3.1: trial space B_i / sqrt(det DF) (Eq. trialspace),
 *                    Z = Z_d x ... x Z_1 (Kronecker mass matrix), and the
 *                    interpolation-based quadrature factorisation
 *                    A = M^T B~^-1 J Gamma J B~^-T M, applied matrix-free with
 *                    Gamma evaluated on the fly over all pairs of Greville
 *                    points of the interpolation space.
 *   KL_COLLOCATION   Sec. 3.2: NURBS trial space collocated at the Greville
 *                    abscissae, A_ij = int Gamma(x_i, x') R_j(x') dx' and
 *                    Z_ij = R_j(x_i) (Eq. colloc system matrices), applied by
 *                    Algorithm 1 with (p+1)^3 Gauss points per element and the
 *                    Kronecker structure of Z (Sec. 3.3, Remark).
 *   KL_GALERKIN_STD  Sec. 3.1 (the standard method the IBQ replaces): the
 *                    trial space of KL_GALERKIN_IBQ with both integrals of
 *                    Eq. galerkin_system_matrices evaluated by the Gauss-Legendre
 *                    rule of (p+1)^3 points per element,
 *                    A = N_q^T W Gamma W N_q with N_q the trial functions at the
 *                    points and W their weights times det DF; Gamma over all
 *                    pairs of Gauss points (O(N_e^2 (p+1)^6) per application).
 *                    Z as for KL_GALERKIN_IBQ. Reference solutions (Sec. 4).
 *
 * Conventions used by every entry point:
 *   - Dofs and points are ordered lexicographically with parametric
 *     direction 1 varying fastest (Sec. 3.1: Z = Z_d x ... x Z_1).
 *   - A block of k vectors of length n is column-major: element (i, c) is at
 *     X[i + c * ldx], ldx >= n.
 *   - Device pointers are CUDA device (or managed) memory of the device that
 *     was current when the handle was created. The caller owns every buffer it
 *     passes; the handle owns its tables and workspaces and frees them in
 *     kl_destroy.
 *   - Every device operation is enqueued on the handle's CUDA stream (the
 *     stream given to kl_create). kl_apply_* return without synchronising;
 *     kl_eigs synchronises that stream.
 *   - Every call returns a kl_status and never aborts the process. On error
 *     kl_last_error(h) returns a one-line message. An asynchronous device
 *     error surfaces as KL_ERR_CUDA on the next call that synchronises.
 *   - Handles are not thread-safe: one host thread at a time per handle.
 */
#ifndef KL_H
#define KL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kl_solver kl_solver;

typedef enum {
    KL_OK = 0,
    KL_ERR_ARG = -1,          /* invalid argument or parameter combination   */
    KL_ERR_CUDA = -2,         /* a CUDA runtime call failed                    */
    KL_ERR_OOM = -3,          /* device allocation failed                      */
    KL_ERR_NOCONV = -4,       /* eigensolver hit its iteration limit; the best
                                 available pairs are still returned            */
    KL_ERR_NUMERIC = -5,      /* NaN/Inf met, or a factorisation broke down    */
    KL_ERR_TIMEOUT = -6,      /* a bounded device wait gave up                 */
    KL_ERR_UNSUPPORTED = -7,  /* feature not available on this device/build    */
    KL_WARN_COMPLEX = 1       /* collocation: a returned pair had an imaginary
                                 part above max(1e-8, tol) |lambda_1| (real
                                 parts are returned)                           */
} kl_status;

/* Domains (single NURBS patches, Sec. 3.1):
 *   KL_GEOM_CUBE             the unit cube (unit square / interval for dim < 3)
 *   KL_GEOM_QUARTER_ANNULUS  quarter annular cylinder: direction 1 the angle
 *                            (exact quadratic NURBS arc), 2 the radius, 3 the
 *                            height
 *   KL_GEOM_HALF_ANNULUS     half annular cylinder (the shape of the Sec. 4
 *                            benchmark): two quarter arcs joined C^0 at the
 *                            angle parameter 1/2; elems[0] counts both halves
 *                            (even). The trial space is C^0 at the join, the
 *                            Galerkin interpolation space C^-1 (Sec. 4.1).
 *   KL_GEOM_PROJECTIVE_CUBE  the unit cube mapped by x = x^ / (1 + c . x^),
 *                            c = geo[0..2] with 1 + sum_d min(c_d, 0) > 0: a
 *                            hexahedron with planar faces, the trilinear NURBS
 *                            volume with corner weights 1 + c . v. Its weight
 *                            function 1 + c . x^ is not a product of
 *                            one-parameter functions, so the collocation
 *                            matrix Z = (R_j(x_i)) is not a Kronecker product
 *                            (Sec. 3.2); it is applied as
 *                            Z^-1 = diag(1 / w) (B-spline Z)^-1 diag(W(x_i)),
 *                            exact for any NURBS weights w_j, W = sum w_j B_j. */
enum { KL_GEOM_CUBE = 0, KL_GEOM_QUARTER_ANNULUS = 1, KL_GEOM_HALF_ANNULUS = 2, KL_GEOM_PROJECTIVE_CUBE = 3 };

/* Covariance kernels Gamma(x, x'), r = |x - x'| (Euclidean):
 *   KL_KERNEL_GAUSS     sigma^2 exp(-r^2 / L^2)
 *   KL_KERNEL_EXP_SEP   sigma^2 exp(-sum_d |x_d - x'_d| / L)
 *   KL_KERNEL_EXP       sigma^2 exp(-r / L)
 *   KL_KERNEL_MATERN32  sigma^2 (1 + sqrt(3) r / L) exp(-sqrt(3) r / L)
 *   KL_KERNEL_CONST     sigma^2 (rank-one test kernel)                    */
enum { KL_KERNEL_GAUSS = 0, KL_KERNEL_EXP_SEP = 1, KL_KERNEL_EXP = 2,
       KL_KERNEL_MATERN32 = 3, KL_KERNEL_CONST = 4 };

enum { KL_GALERKIN_IBQ = 0, KL_COLLOCATION = 1, KL_GALERKIN_STD = 2 };

/* Arithmetic of the pairwise product Gamma * X (the O(N~^2) / O(N N_e N_q)
 * step; Sec. 3.3). Everything else (sum factorisation, Z solves,
 * orthogonalisation, Rayleigh-Ritz) is FP64; with the reduced precisions the
 * small eigenproblems of the early Rayleigh-Ritz steps (and, for the
 * symmetric Galerkin problems, the one that finds all wanted residuals below
 * the tolerance) are solved in FP32, and the returned pairs come from the
 * FP64 Rayleigh-Ritz refinement (`refine`).
 *   KL_FP64        FP64 kernel evaluation and products (CUDA cores).
 *   KL_FP32        FP32 kernel evaluation and FP32 products (CUDA cores).
 *   KL_MIXED_BF16  FP32 kernel tiles written to tensor memory and multiplied
 *                  on tcgen05 tensor cores as split (hi + lo) BF16 products
 *                  with FP32 accumulation.
 *   KL_MIXED_TF32  as KL_MIXED_BF16 with split TF32 products.               */
enum { KL_FP64 = 0, KL_FP32 = 1, KL_MIXED_BF16 = 2, KL_MIXED_TF32 = 3 };

typedef struct kl_params {
    int dim;                 /* 1, 2 or 3 parametric directions (annulus: 3)  */
    int geometry;            /* KL_GEOM_*                                     */
    double geo[3];           /* annulus: r_in, r_out, height (> 0, r_out >
                                r_in); projective cube: c_1, c_2, c_3;
                                ignored for the cube                          */
    int degree;              /* p, 1 <= p <= 8 (trial and interpolation)      */
    int elems[3];            /* elements per direction (>= 1); direction 1 of
                                the annulus is the angle, 2 the radius, 3 the
                                height                                        */
    int kernel;              /* KL_KERNEL_*                                   */
    double sigma;            /* standard deviation (> 0)                      */
    double L;                /* correlation length (> 0)                      */
    int method;              /* KL_GALERKIN_IBQ, KL_COLLOCATION or
                                KL_GALERKIN_STD                               */
    int interp_continuity;   /* Galerkin interpolation space continuity:
                                -2 = rule of Sec. 4 (C^0 for the exponential
                                kernels, C^{p-1} otherwise), else 0 .. p-1    */
    int precision;           /* KL_FP64, KL_FP32, KL_MIXED_BF16, KL_MIXED_TF32 */
    int block_k;             /* eigensolver block size = vectors per operator
                                application, 1..64 (0: 8)                     */
    int refine;              /* final Rayleigh-Ritz refinement when precision
                                is not FP64: 0 none, 1 FP64 Rayleigh-Ritz on
                                the mixed operator, 2 FP64 Rayleigh-Ritz on an
                                FP64 application of the operator (-1: 1)      */
    int max_restarts;        /* restart cycles before KL_ERR_NOCONV (0: 200)  */
    unsigned long long seed; /* start block of the eigensolver                */
} kl_params;

/* Fills *p with: cube, dim 3, p = 2, 4x4x4 elements, Gaussian kernel,
 * sigma = 1, L = 0.5, Galerkin, rule continuity, FP64, block 8, refine -1,
 * max_restarts 0, seed 2101. */
void kl_default_params(kl_params* p);

/* Sec. 3.1 / Sec. 3.2 set-up (negligible cost next to the solve, Sec. 3.3): knot
 * vectors, Greville points, 1D mass / collocation / mixed mass matrices and
 * their factorisations (host, FP64), then the point tables and geometry
 * factors on the device. `stream` is a cudaStream_t (NULL: legacy default
 * stream). On success *out owns all device memory of the solver.
 * Errors: KL_ERR_ARG (bad params or out == NULL), KL_ERR_OOM, KL_ERR_CUDA,
 * KL_ERR_UNSUPPORTED (no sm_100-class device for the tcgen05 precisions). */
int kl_create(const kl_params* params, void* stream, kl_solver** out);

/* Frees every resource of the handle (synchronises its stream). NULL is OK. */
int kl_destroy(kl_solver* h);

/* N = trial dofs; n_src = number of pairwise source points (Galerkin: N~ =
 * interpolation dofs; collocation: N_e N_q quadrature points); n_tgt =
 * pairwise target points (Galerkin: N~; collocation: N). Any pointer may be
 * NULL. */
int kl_dims(const kl_solver* h, int64_t* N, int64_t* n_src, int64_t* n_tgt);

/* Y = A X for k vectors (1 <= k <= 256), X and Y device FP64 blocks of
 * length N (ldx, ldy >= N). A is the generalized matrix in the coefficient
 * basis: Galerkin  M^T B~^-1 J Gamma J B~^-T M  (Sec. 3.1),
 *           collocation  Gamma (J .* W .* (R X))  (Algorithm 1 without the
 *                        final Z^-1).
 * Arithmetic of the pairwise step per params.precision. X and Y must not
 * overlap. Errors: KL_ERR_ARG, KL_ERR_CUDA, KL_ERR_OOM. */
int kl_apply_A(kl_solver* h, const double* X, int64_t ldx, double* Y, int64_t ldy, int k);

/* Y = Z^-1 X (device FP64 blocks as above). Galerkin: Z^-1 = L^-T L^-1 with
 * the Kronecker Cholesky factor L = L_d x ... x L_1 (Sec. 3.1). Collocation:
 * the Kronecker pivoted-LU solve Z^-1 = Q U^-1 L^-1 P per direction
 * (Sec. 3.2, Sec. 3.3 Remark). X and Y may be the same buffer. */
int kl_apply_Zinv(kl_solver* h, const double* X, int64_t ldx, double* Y, int64_t ldy, int k);

/* Y = A' X with the standard-form operator of Eq. standard:
 * Galerkin A' = L^-1 A L^-T (the nine-step product of Sec. 3.1, with the
 * Kronecker factors of each side folded per direction); collocation
 * A' = Z^-1 A (Algorithm 1). Device FP64 blocks, X and Y must not overlap. */
int kl_apply_Aprime(kl_solver* h, const double* X, int64_t ldx, double* Y, int64_t ldy, int k);

typedef struct kl_solve_info {
    int restarts;            /* restart cycles used                           */
    int applies;             /* operator applications (blocks)                */
    int vectors_applied;     /* sum of block widths over all applications    */
    int converged;           /* eigenpairs meeting tol                         */
    double max_resid;        /* max relative residual of the returned pairs   */
    double max_imag;         /* collocation: max |Im lambda| / |lambda_1|     */
    double seconds;          /* wall time of the call                          */
} kl_solve_info;

/* The M largest eigenpairs (1 <= M <= N, M <= 512) of A v = lambda Z v.
 *   tol        stop when every ||A' y - theta y|| <= tol * |theta_1| (<= 0:
 *              1e-10 for KL_FP64, 1e-6 otherwise). A reduced-precision
 *              solve also stops when its largest wanted residual has not
 *              decreased for 10 restarts while within 10 * tol: the rounding
 *              of the split pairwise operands bounds how far the residuals
 *              can fall (resid and info report the residuals reached).
 *   lambda     host array of M doubles, descending (collocation: real parts
 *              in descending order of the real part).
 *   V          N x M column-major (ldv >= N), host memory if v_on_device == 0,
 *              device memory otherwise; NULL to skip the vectors. Galerkin
 *              vectors are Z-orthonormal (v^T Z v = 1: unit L2 norm of the
 *              eigenfunction, Sec. 2); collocation vectors have unit L2 norm of
 *              sum_j v_j R_j under the collocation Gauss rule. The largest-
 *              magnitude entry of each vector is positive.
 *   resid      host array of M relative residuals ||A' y - theta y|| /
 *              |theta_1|, or NULL.
 *   info       optional statistics, or NULL.
 * Synchronises the handle's stream. Returns KL_OK, KL_WARN_COMPLEX,
 * KL_ERR_NOCONV (best pairs still written), or an error. */
int kl_eigs(kl_solver* h, int M, double tol, double* lambda, double* V, int64_t ldv,
            int v_on_device, double* resid, kl_solve_info* info);

/* Per-kernel-class device time measured with CUDA events recorded on the
 * handle's stream around every launch while profiling is on. `units` is the
 * algorithmic work the launches performed: kernel evaluations (pairs) for the
 * pairwise classes, bytes for the sum-factorisation class. */
typedef struct kl_kernel_stats {
    char name[32];
    long long launches;
    double ms;
    double units;
} kl_kernel_stats;

/* Turns event timing on (1) or off (0) and clears the counters. */
int kl_profile_enable(kl_solver* h, int on);
/* Copies up to `cap` entries; *n receives the number of classes. Synchronises
 * the stream to read the events. */
int kl_profile_read(kl_solver* h, kl_kernel_stats* out, int cap, int* n);
/* Number of kernels this handle launched since creation (all classes). */
long long kl_launch_count(const kl_solver* h);

/* Bytes copied host -> device during kl_create (tables and point sets) and
 * bytes of device memory the handle holds. */
int kl_memory(const kl_solver* h, int64_t* h2d_bytes, int64_t* device_bytes);

/* Measured throughput of the arithmetic units that bound the pairwise kernel
 * evaluation on the current device, in operations per second: FP32 FMA, the
 * special-function base-2 exponential (ex2) and FP64 FMA. Used as the
 * denominator of the pairwise kernels' roofline. No paper passage: the
 * paper's computations ran on one CPU core (Sec. 4). Any pointer may be NULL.
 * Errors: KL_ERR_CUDA, KL_ERR_OOM. */
int kl_measure_peaks(double* fp32_fma_per_s, double* ex2_per_s, double* fp64_fma_per_s);

/* Y = sigma^2 Gamma(targets, sources) X with FP64 kernel evaluation on the
 * CUDA cores, allocating no device memory. No paper passage: the paper has no
 * counterpart; this entry point exists for callers that cannot allocate --
 * code inside CUDA graph capture, applications with fixed memory pools, or
 * hosts that hand out one pre-sized arena and forbid cudaMalloc/cudaFree.
 *   kernel, sigma, L  as in kl_params (KL_KERNEL_*, sigma > 0, L > 0).
 *   tgt               device FP64, 3*T values: all x, then all y, then all z.
 *   src               device FP64, 3*S values, same layout.
 *   X                 device FP64, S x k column-major (ldx >= S).
 *   Y                 device FP64, T x k column-major (ldy >= T), written.
 *   stream            cudaStream_t (NULL: legacy default stream).
 * Its partial sums live in one static device array of 2^21 doubles (16 MiB)
 * that every device loading the library holds until the process exits; the
 * call requires k * T <= 2^21 and returns KL_ERR_ARG beyond that. The first
 * call on a device looks up that array's device address (set-up, with the
 * device current); make the first call before any stream capture. All calls
 * on a device share the array: calls that overlap on the GPU (other streams,
 * other host threads) race and must be serialised by the caller. Nothing in
 * the array needs clearing between calls. No cudaMalloc or cudaFree is made.
 * Asynchronous on `stream`. Errors: KL_ERR_ARG, KL_ERR_CUDA; the message is
 * kl_last_error(NULL). */
int kl_pairwise_noalloc(int kernel, double sigma, double L, const double* tgt, int64_t T,
                        const double* src, int64_t S, const double* X, int64_t ldx, double* Y,
                        int64_t ldy, int k, void* stream);

/* ------------------------------------------------------------------------
 * Sampling the truncated K-L expansion (Sec. 2, the expansion of the random
 * field): realisations alpha_M(x, xi) = sum_m sqrt(lambda_m) xi_m phi_m(x)
 * of the centred field, phi_m(x) = sum_j V(j, m) N_j(x) in the method's
 * trial basis N_j (B_j / sqrt(det DF) for Galerkin, Sec. 3.1; the rational
 * basis R_j for collocation, Sec. 3.2), evaluated at the tensor Gauss grid of
 * the parametric domain
 * (p + 1 points per element and direction, lexicographic, direction 1
 * fastest; kl_sample_size points).
 * ------------------------------------------------------------------------ */
int64_t kl_sample_size(const kl_solver* h);
/* Physical coordinates of that grid: device xyz, 3 * kl_sample_size values
 * (all x, then y, then z). Asynchronous on the handle's stream. */
int kl_sample_points(kl_solver* h, double* xyz);
/* lambda: host, M values (negative values count as 0); V: device N x M
 * (ldv >= N), eigenvectors as returned by kl_eigs; xi: device M x ns (ldxi >=
 * M), the standard normal variables (the caller draws them); out: device
 * kl_sample_size x ns (ldo >= kl_sample_size). The sample scratch grows on
 * demand (the only allocation). Errors: KL_ERR_ARG, KL_ERR_CUDA. */
int kl_sample(kl_solver* h, int M, const double* lambda, const double* V, int64_t ldv, const double* xi,
              int64_t ldxi, int ns, double* out, int64_t ldo);

/* CUDA graphs of operator applications (default on): the second application
 * with the same operator, precision, block width and buffers is captured into
 * a graph on the handle's stream and later ones replay it (one launch instead
 * of ~10). While profiling, the sum-factorisation parts are two graphs and the
 * pairwise product runs eagerly between its timing events. Not used for
 * handles run by a server. Turning it off drops the captured graphs.
 * Synchronises the stream. */
int kl_set_graphs(kl_solver* h, int on);
/* SMs the handle's tensor-core pairwise product leaves free (0 <= n < SM
 * count; 0 at creation): its persistent grid of two CTAs per SM spans the
 * other SMs. For solves that run concurrently with other work on the same
 * GPU (several handles on their own streams): a grid over every SM holds all
 * of them for the length of the product, so the short kernels of the other
 * streams wait for its end; a few free SMs let them run beside it. Results
 * are bitwise the same for every n (the work units and their reduction order
 * do not depend on the grid). Synchronises the stream and drops captured
 * graphs. Errors: KL_ERR_ARG (h NULL or n out of range), KL_ERR_CUDA. */
int kl_set_shared_sms(kl_solver* h, int n);
/* Block size (vectors per operator application) the handle uses: params'
 * block_k, or the autotuned value for block_k = 0 (see kl_autotune). */
int kl_block_size(const kl_solver* h);

/* Block-size autotuner: times complete solves (kl_eigs, M pairs, tol) for
 * block sizes 8, 16 and 32 on `stream` (each solved twice, the second timed;
 * sizes the basis limit or convergence rule out are skipped), returns the
 * fastest in *best_k and the times in seconds[3] (or NULL; -1 when skipped),
 * and appends "<problem key> <k> <seconds>" to cache_path (or NULL). A handle
 * created with block_k = 0 takes, at each kl_eigs, the last cached block size
 * for its parameters and M from the file named by the environment variable
 * KL_TUNE_CACHE (8 when there is none). The tuning itself is not meant to be
 * timed: run it once and keep the cache. */
int kl_autotune(const kl_params* params, int M, double tol, void* stream, const char* cache_path, int* best_k,
                double* seconds);

/* ------------------------------------------------------------------------
 * Memory estimate (host only, no GPU needed)
 * ------------------------------------------------------------------------
 * Upper estimate of the device bytes a handle with these parameters holds
 * while kl_eigs(M) runs (tables, point sets, operator workspaces, pairwise
 * scratch for block_k vectors, eigensolver workspace). Used by the serving
 * loop to admit requests by HBM budget. KL_ERR_ARG for invalid parameters. */
int kl_estimate_bytes(const kl_params* params, int M, int64_t* bytes);

/* ------------------------------------------------------------------------
 * Serving: continuous batching of K-L solves on one GPU
 * ------------------------------------------------------------------------
 * No paper passage: the paper solves one problem at a time on one CPU core
 * (Sec. 4). A server owns max_slots worker threads. A submitted request waits
 * in a FIFO queue until a slot is free and its kl_estimate_bytes fits in what
 * is left of hbm_budget_bytes (the first 8 queued requests are scanned, so a
 * large request does not block smaller ones behind it indefinitely: it keeps
 * its place and is admitted as soon as memory frees up); it then gets its own
 * handle, stream and device state (tables, Krylov basis) for the whole solve,
 * and is freed when it completes. While several solves run, the tensor-core
 * pairwise products of all of them that are ready within batch_window_us go
 * into ONE persistent kernel launch (uneven instances: different meshes,
 * degrees, kernels; grouped by precision and block width). The rest of each
 * solve (sum factorisation, orthogonalisation, Rayleigh-Ritz) runs on its own
 * stream and overlaps on the device. FP64/FP32 requests run unbatched. */
typedef struct kl_server kl_server;

typedef struct kl_serve_config {
    int64_t hbm_budget_bytes; /* 0: 80% of the free device memory at open    */
    int max_slots;            /* concurrent solves, 1..64 (0: 8)               */
    int batch_window_us;      /* wait for more ready products (0: 300)        */
} kl_serve_config;

typedef struct kl_serve_result {
    int64_t request_id;
    int status;          /* kl_eigs status (KL_OK, KL_WARN_COMPLEX, ...)  */
    int M;
    int applies, restarts;
    double max_resid;
    double queue_ms;     /* submit -> admitted                           */
    double solve_ms;     /* admitted -> finished (create + eigs + free)  */
    double latency_ms;   /* submit -> finished                           */
    int64_t est_bytes;   /* admission estimate                           */
} kl_serve_result;

typedef struct kl_serve_stats {
    long long submitted, completed;
    long long batches;           /* batched tensor-core launches           */
    long long batched_products;  /* products (instances) in those launches */
    int max_batch;               /* most instances in one launch           */
    int max_concurrent;          /* most solves admitted at once           */
    int64_t peak_est_bytes;      /* most admitted estimate at once         */
    int64_t budget_bytes;
} kl_serve_stats;

/* Starts the worker threads on the current device. */
int kl_serve_open(const kl_serve_config* cfg, kl_server** out);
/* Queues a solve of M eigenpairs (tol as in kl_eigs). lambda_out (host, M
 * doubles) and V_out (host, N x M, ldv >= N, or NULL) are written by the
 * worker before the result is reported by kl_serve_poll and must stay valid
 * until then. Thread-safe. KL_ERR_ARG for invalid parameters or a request
 * whose estimate exceeds the whole budget. */
int kl_serve_submit(kl_server* s, const kl_params* params, int M, double tol, int64_t request_id,
                    double* lambda_out, double* V_out, int64_t ldv);
/* Copies up to cap finished results (completion order) into out, *n of them;
 * waits up to wait_ms for at least one when none is ready. */
int kl_serve_poll(kl_server* s, kl_serve_result* out, int cap, int* n, int wait_ms);
int kl_serve_get_stats(kl_server* s, kl_serve_stats* out);
/* Waits for every queued and running solve, stops the workers, frees. */
int kl_serve_close(kl_server* s);

/* Failure injection on the host, for tests of the error paths (no paper
 * passage). Nothing here faults, traps or hangs the GPU:
 *   KL_DEBUG_WAIT_LIMIT  (handle) clock cycles each pipeline wait of the
 *                        tcgen05 pairwise kernel may take before it gives up
 *                        (0: the default, about a second). A short limit
 *                        makes the waits give up: the kernel records the
 *                        timeout in the handle's error word, always lets its
 *                        issued MMAs and copies finish (default bound), frees
 *                        its tensor memory and returns; kl_eigs then returns
 *                        KL_ERR_TIMEOUT.
 *   KL_DEBUG_FAIL_ALLOC  (h may be NULL; process-wide) the value-th device
 *                        allocation of the library from now on fails as if
 *                        the device were out of memory (KL_ERR_OOM); 0
 *                        cancels a pending failure.
 *   KL_DEBUG_NAN_START   (handle) value != 0 plants a NaN in the
 *                        eigensolver's start block (kl_eigs returns
 *                        KL_ERR_NUMERIC).
 *   KL_DEBUG_PAIR_DENSE  (handle) value != 0 makes the split-BF16 Galerkin
 *                        pairwise product evaluate every pair (the dense
 *                        form, as for collocation) instead of each symmetric
 *                        pair once; for comparisons of the two forms.
 * Errors: KL_ERR_ARG. */
enum { KL_DEBUG_WAIT_LIMIT = 1, KL_DEBUG_FAIL_ALLOC = 2, KL_DEBUG_NAN_START = 3, KL_DEBUG_PAIR_DENSE = 4 };
int kl_debug_set(kl_solver* h, int what, long long value);

/* 1 if the library was built with KL_CHECK_BOUNDS (every kernel launch first
 * checks, on the host, that each device range it will touch lies inside one
 * live device allocation, and the small eigensolver checks its
 * data-dependent indices; a failed check fails the call with KL_ERR_CUDA and
 * a message on stderr instead of launching), 0 for the regular build. No
 * paper passage: a debugging aid of this library. */
int kl_bounds_checked(void);

/* Last error message of the handle (h may be NULL: last kl_create error). */
const char* kl_last_error(const kl_solver* h);
const char* kl_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* KL_H */
