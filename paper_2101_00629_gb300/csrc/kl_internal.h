// Internal declarations shared by the translation units of the library.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/kl.h"

namespace kl {

// ---------------------------------------------------------------------------
// Host dense matrices (column-major, FP64) used only during set-up.
// ---------------------------------------------------------------------------
struct Mat {
    int rows = 0, cols = 0;
    std::vector<double> a;
    Mat() = default;
    Mat(int r, int c) : rows(r), cols(c), a(size_t(r) * c, 0.0) {}
    double& operator()(int i, int j) { return a[size_t(i) + size_t(j) * rows]; }
    double operator()(int i, int j) const { return a[size_t(i) + size_t(j) * rows]; }
};

Mat identity(int n);
Mat transpose(const Mat& A);
Mat matmul(const Mat& A, const Mat& B);
// In-place lower Cholesky (upper part zeroed). False if not positive definite.
bool cholesky(Mat& A);
// Inverse of a lower-triangular matrix.
Mat lower_inverse(const Mat& L);
// Solve A X = B with partial pivoting. False if singular.
bool lu_solve(const Mat& A, const Mat& B, Mat& X);

// ---------------------------------------------------------------------------
// Set-up of one parametric direction (Sec. 3.1, Sec. 3.2), host FP64.
// ---------------------------------------------------------------------------
struct Dir1D {
    int nel = 1, p = 1;
    int N = 1;     // trial dofs
    // Galerkin
    int Nt = 1;                 // interpolation dofs
    std::vector<double> xg;     // Greville points of the interpolation space (Nt)
    Mat Q;                      // B~^-T M             (Nt x N)
    Mat P;                      // B~^-T M L^-T        (Nt x N)
    Mat LinvT;                  // L^-T                (N x N)
    Mat Zinv_gal;               // Z^-1 = L^-T L^-1    (N x N)
    // Collocation
    int nq = 1;                 // quadrature points of this direction
    std::vector<double> xq, wq; // Gauss points / weights (nq)
    std::vector<double> xc;     // Greville points of the trial space (N)
    Mat R;                      // rational basis at quadrature points (nq x N)
    // Both methods: Gauss points of the elements and the trial basis there
    // (B-splines for Galerkin, the rational basis for collocation), for the
    // evaluation of fields sum_j v_j N_j at the tensor Gauss grid.
    int ne = 1;                 // Gauss points of this direction (p + 1 per element)
    std::vector<double> xe;     // their parameters (ne)
    std::vector<double> we;     // their Gauss weights (ne)
    Mat E;                      // trial basis at them (ne x N)
    Mat Zinv_col;               // (R_j(xc_i))^-1      (N x N)
};

// Both Galerkin forms (IBQ and standard quadrature): the trial space
// B_i / sqrt(det DF), a symmetric operator in standard form A' = L^-1 A L^-T.
inline bool galerkin_form(int method) { return method == KL_GALERKIN_IBQ || method == KL_GALERKIN_STD; }

// Builds the direction's tables. `arc`: 0 polynomial direction; 1 direction 1
// of the quarter annulus, 2 of the half annulus (NURBS weights from the
// quadratic arc; the half arc has a C^0 geometry join at 1/2, where the trial
// space is C^0 and the interpolation space C^-1). `present` = false gives the
// 1-dof identity direction used for dim < 3. Returns an empty string on success.
std::string setup_direction(Dir1D& d, bool present, int nel, int p, int interp_cont,
                            int arc, bool need_galerkin, bool need_collocation);

// Bounds-checking build: every launcher checks, before it launches, that each
// device range its kernel reads or writes lies inside one live allocation
// (bounds.cpp). KL_RANGE(p, count, type, what) checks count elements of type
// from p (skipped for NULL p or count <= 0) and returns cudaErrorInvalidValue
// from the launcher on failure; it compiles to nothing in the regular build.
#ifdef KL_CHECK_BOUNDS
cudaError_t check_range(const void* p, int64_t bytes, const char* what);
#define KL_RANGE(p, count, type, what)                                                              \
    do {                                                                                             \
        if ((p) != nullptr && int64_t(count) > 0) {                                                  \
            const cudaError_t kl_range_e = ::kl::check_range((p), int64_t(count) * int64_t(sizeof(type)), (what)); \
            if (kl_range_e != cudaSuccess) return kl_range_e;                                        \
        }                                                                                            \
    } while (0)
#else
#define KL_RANGE(p, count, type, what) \
    do {                               \
    } while (0)
#endif
// Extent (elements) of a column-major block of `rows` x `cols` with leading
// dimension ld: the last column's last row + 1.
inline int64_t block_extent(int64_t rows, int64_t cols, int64_t ld) {
    return (rows <= 0 || cols <= 0) ? 0 : (cols - 1) * ld + rows;
}

// cudaMalloc of the library's device memory, with the allocation-failure
// injection of kl_debug_set (KL_DEBUG_FAIL_ALLOC) in front of it.
cudaError_t device_alloc(void** p, size_t bytes);

// Streaming multiprocessors of the current device, cached per device; 152
// (GB300) when no device is visible (host-only estimates). Grid sizes and the
// split heuristics of the launchers scale with it.
int device_sm_count();

// ---------------------------------------------------------------------------
// Device-side launchers (defined in the .cu files). All take the stream.
// ---------------------------------------------------------------------------
struct KernelSpec {
    int kind;       // KL_KERNEL_*
    double sigma2;  // sigma^2
    double a;       // scale of the argument (see pair kernels)
};

// Geometry factors at a tensor grid of parametric points.
// out_x/y/z: physical coordinates; out_w: weight(i1)*weight(i2)*weight(i3) *
// |det DF|^power (power 0.5 for J = sqrt(det DF), 1 for collocation, -0.5 for
// the Galerkin trial functions B / sqrt(det DF); 0: no Jacobian factor).
cudaError_t launch_tensor_points(int geometry, const double* geo, const double* t1, const double* t2,
                                 const double* t3, int n1, int n2, int n3, const double* w1,
                                 const double* w2, const double* w3, double jac_power, double* out_x,
                                 double* out_y, double* out_z, double* out_w, cudaStream_t s);

// A banded m x n table: row i has its nonzero entries in columns
// start[i] .. start[i] + w - 1 (start[i] + w <= n), values vals[i * w + j].
struct Band {
    const double* vals = nullptr;
    const int* start = nullptr;
    int w = 0;
};
// Y(a, m, b, c) = sum_j vals(i, j) X(a, start[i] + j, b, c): the mode product
// of launch_modeprod with a banded table (same scalings).
cudaError_t launch_modeprod_band(const Band& A, int m, int n, const double* X, int64_t ldx, double* Y,
                                 int64_t ldy, int64_t a, int64_t b, int k, const double* post,
                                 const double* pre, cudaStream_t s);
// Y(a, m, b, c) = sum_l A(i, l) X(a, l, b, c) (+ optional scaling of the
// output rows by post[a + A*(i + m*b)] and of the input rows by
// pre[a + A*(l + n*b)]).
cudaError_t launch_modeprod(const double* A, int m, int n, const double* X, int64_t ldx, double* Y,
                            int64_t ldy, int64_t a, int64_t b, int k, const double* post,
                            const double* pre, cudaStream_t s);
// w_inv <- 1 / w_inv (W at the Gauss points), scale_out = scale * (1 / W).
cudaError_t launch_rational_scales(double* w_inv, const double* scale, double* scale_out, int64_t n,
                                   cudaStream_t s);

// Pairwise products W = Gamma(targets, sources) X, FP64 or FP32 on CUDA cores.
struct PairArgs {
    const double *tx, *ty, *tz;  // targets (T), FP64
    const float *tx32, *ty32, *tz32;
    const double *sx, *sy, *sz;  // sources (S), FP64
    const float *sx32, *sy32, *sz32;
    int64_t T, S;
    const double* X;  // S x k (ldx)
    int64_t ldx;
    double* Y;  // T x k (ldy)
    int64_t ldy;
    int k;
    const double* post;  // optional per-target scale
    KernelSpec ks;
    double* scratch;  // splits * k * T doubles
    int splits;
};
int64_t pair_scratch_doubles(int64_t T, int k, int splits);
int pair_choose_splits(int64_t T, int64_t S, int sm_count);
cudaError_t launch_pair_simt(const PairArgs& a, bool fp32, cudaStream_t s);

// ---------------------------------------------------------------------------
// Small dense FP64 linear algebra on the device (Sec. 3: standard form and
// the outer eigensolver).
// ---------------------------------------------------------------------------
// C(m x n) = alpha * A^T B + beta * C, A: K x m (lda), B: K x n (ldb), K long.
cudaError_t launch_gemm_tn(const double* A, int64_t lda, const double* B, int64_t ldb, double* C,
                           int64_t ldc, int m, int n, int64_t K, double alpha, double beta,
                           double* scratch, int64_t scratch_doubles, cudaStream_t s);
// Scratch (doubles) of launch_gemm_tn for every m' <= m, n' <= n at this K.
int64_t gemm_tn_scratch_doubles(int m, int n, int64_t K);
// C(K x n) = alpha * A(K x m) B(m x n) + beta * C.
cudaError_t launch_gemm_nn(const double* A, int64_t lda, const double* B, int64_t ldb, double* C,
                           int64_t ldc, int64_t K, int m, int n, double alpha, double beta,
                           cudaStream_t s);
// Lower Cholesky of the n x n SPD G (in place) and Rinv = L^-T (upper), flags
// columns whose pivot collapsed (rank deficiency) in bad[n] (0/1).
cudaError_t launch_chol_rinv(double* G, int n, double* Rinv, int* bad, cudaStream_t s);
// Symmetric eigen-decomposition of the n x n H (Hessenberg/tridiagonal
// reduction + Francis QR), eigenvalues descending in w, orthonormal
// eigenvectors in V (n x n). status[0]: 0 ok, 1 no convergence.
// fp32: the whole decomposition in FP32 arithmetic (inputs and outputs stay
// FP64; accuracy ~1e-7 ||H||), for the restarts of the outer solver.
// dfloat (with fp32 false): the QR path in double-float arithmetic (~1e-13
// ||H||), for the FP64-grade problems of reduced-precision solves.
cudaError_t launch_sym_eig(const double* H, int n, double* w, double* V, double* work,
                           int* status, cudaStream_t s, bool fp32 = false, bool dfloat = false);
// Arithmetic of the small eigensolver: FP64, FP32 (accuracy ~1e-7 ||H||) or
// double-float (pairs of FP32 numbers, ~1e-14 ||H||, several times faster
// than FP64 on GB300's small FP64 unit).
enum EigArith { kEigFP64 = 0, kEigFP32 = 1, kEigDF = 2 };
// Real non-symmetric eigen-decomposition (Hessenberg + Francis QR + ordering
// of the real Schur form + back substitution). wr/wi eigenvalues by real part
// descending; Q (optional, n x n) the Schur vectors in the same order, so its
// leading columns span the invariant subspace of the leading eigenvalues; V
// the unit-norm eigenvectors of the leading nvec eigenvalues (complex pairs as
// Re, Im columns; one more column when nvec splits a pair; nvec <= 0: all).
// status[0]: 0 ok, 1 no convergence.
cudaError_t launch_nonsym_eig(const double* H, int n, double* wr, double* wi, double* V, double* Q,
                              double* work, int* status, cudaStream_t s, int nvec = 0, int arith = kEigFP64);
int64_t nonsym_eig_work_doubles(int n);
int64_t sym_eig_work_doubles(int n);
// Symmetric eigenproblems of order n <= jacobi_max_n() by parallel Jacobi
// (FP32, or FP32 refined in FP64); workspace of the FP64 form in doubles.
int jacobi_max_n();
int64_t jacobi_work_doubles(int n);
cudaError_t launch_sym_eig_jacobi(const double* H, int n, double* w, double* V, double* work, int* status,
                                  cudaStream_t s, bool fp32);
// Column 2-norms of X (K x n).
cudaError_t launch_col_norms(const double* X, int64_t ldx, int64_t K, int n, double* out,
                             cudaStream_t s);
// Standard normal block by a counter-based generator (seed, stream offset).
cudaError_t launch_randn(double* X, int64_t ldx, int64_t K, int n, unsigned long long seed,
                         unsigned long long offset, cudaStream_t s);
// Y(:, j) = X(:, j) * scale[j]  (scale on device).
cudaError_t launch_scale_cols(double* X, int64_t ldx, int64_t K, int n, const double* scale,
                              int invert, cudaStream_t s);
// X(i, j) *= scale[i] for the K x n block X (rows scaled).
cudaError_t launch_scale_rows(double* X, int64_t ldx, int64_t K, int n, const double* scale, cudaStream_t s);
// Copy a K x n block between leading dimensions.
cudaError_t launch_copy_block(const double* X, int64_t ldx, double* Y, int64_t ldy, int64_t K,
                              int n, cudaStream_t s);
// Weighted column norms sqrt(sum_i w_i X_ij^2) and signed argmax fix-up.
cudaError_t launch_weighted_norms(const double* X, int64_t ldx, int64_t K, int n, const double* w,
                                  double* out, cudaStream_t s);
cudaError_t launch_sign_fix(double* X, int64_t ldx, int64_t K, int n, cudaStream_t s);
// Residual norms ||AV s_i - theta_i V s_i|| for i < n given Y = V S, AY = AV S.
cudaError_t launch_resid_norms(const double* Y, int64_t ldy, const double* AY, int64_t lday,
                               const double* theta, int64_t K, int n, double* out,
                               cudaStream_t s);

}  // namespace kl
