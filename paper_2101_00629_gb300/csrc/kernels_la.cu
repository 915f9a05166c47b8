// Dense FP64 linear algebra of the outer eigensolver (Sec. 3: the standard
// form A' v' = lambda v' is solved iteratively; Sec. 3.3: N_iter matvecs).
//
//   gemm_tn    C = alpha A^T B + beta C for tall A, B (projections V^T W,
//              Gram matrices, Rayleigh-Ritz matrices). The long dimension is
//              split over CTAs; partial tiles are summed in a fixed order.
//   gemm_nn    C = alpha A B + beta C for tall A and small B (basis updates).
//   chol_rinv  Cholesky of a small SPD Gram matrix and the inverse of its
//              transpose (CholQR), flagging collapsed pivots.
// The small eigenproblem of the Rayleigh-Ritz step is in kernels_eig.cu.
#include <cfloat>
#include <algorithm>
#include <cmath>
#include <mutex>

#include "kl_internal.h"

namespace kl {

namespace {

// ------------------------------- gemm_tn ----------------------------------
constexpr int TN_T = 32;
constexpr int TN_NARROW = 8;   // products with n <= 8 use 32 x 8 tiles
constexpr int TN_KMIN = 64;    // shortest K chunk of one CTA
// about four CTAs per SM
inline int tn_ctas() { return 4 * device_sm_count(); }

inline int tn_tiles(int m, int n) {
    const int tm = (m + TN_T - 1) / TN_T;
    return n <= TN_NARROW ? tm : tm * ((n + TN_T - 1) / TN_T);
}

inline int tn_splits(int m, int n, int64_t K) {
    // the long dimension is cut into chunks of >= 64 rows until about four
    // CTAs per SM exist: every CTA is bound by the SM's FP64 rate (~1.7
    // DFMA/clock on GB300), so the work must reach every SM
    int64_t s = (K + TN_KMIN - 1) / TN_KMIN;
    int64_t cap = tn_ctas() / tn_tiles(m, n);
    if (cap < 1) cap = 1;
    if (s > cap) s = cap;
    if (s < 1) s = 1;
    return int(s);
}

__global__ void __launch_bounds__(256) gemm_tn_kernel(const double* __restrict__ A, int64_t lda,
                                                      const double* __restrict__ B, int64_t ldb,
                                                      int m, int n, int64_t K, int64_t kchunk,
                                                      double* __restrict__ part) {
    __shared__ double As[TN_T][TN_T + 1];
    __shared__ double Bs[TN_T][TN_T + 1];
    const int i0 = blockIdx.x * TN_T, j0 = blockIdx.y * TN_T;
    const int64_t k0 = int64_t(blockIdx.z) * kchunk;
    const int64_t k1 = min(K, k0 + kchunk);
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // ty in 0..7
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t kb = k0; kb < k1; kb += TN_T) {
        for (int e = threadIdx.x; e < TN_T * TN_T; e += 256) {
            const int kk = e & 31, c = e >> 5;
            const int64_t kg = kb + kk;
            As[kk][c] = (kg < k1 && i0 + c < m) ? A[kg + int64_t(i0 + c) * lda] : 0.0;
            Bs[kk][c] = (kg < k1 && j0 + c < n) ? B[kg + int64_t(j0 + c) * ldb] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < TN_T; ++kk) {
            const double b = Bs[kk][tx];
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[r] = fma(As[kk][ty + 8 * r], b, acc[r]);
        }
        __syncthreads();
    }
    const int j = j0 + tx;
    if (j < n) {
        for (int r = 0; r < 4; ++r) {
            const int i = i0 + ty + 8 * r;
            if (i < m) part[(int64_t(blockIdx.z) * n + j) * m + i] = acc[r];
        }
    }
}

// n <= 8: a 32 x 8 tile, one output per thread (the 32 x 32 tile would spend
// three quarters of its FP64 work on zero columns).
__global__ void __launch_bounds__(256) gemm_tn_narrow_kernel(const double* __restrict__ A, int64_t lda,
                                                             const double* __restrict__ B, int64_t ldb,
                                                             int m, int n, int64_t K, int64_t kchunk,
                                                             double* __restrict__ part) {
    __shared__ double As[TN_T][TN_T + 1];
    __shared__ double Bs[TN_T][TN_NARROW + 1];
    const int i0 = blockIdx.x * TN_T;
    const int64_t k0 = int64_t(blockIdx.z) * kchunk;
    const int64_t k1 = min(K, k0 + kchunk);
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // row in the tile, column 0..7
    double acc = 0.0;
    for (int64_t kb = k0; kb < k1; kb += TN_T) {
        for (int e = threadIdx.x; e < TN_T * TN_T; e += 256) {
            const int kk = e & 31, c = e >> 5;
            const int64_t kg = kb + kk;
            As[kk][c] = (kg < k1 && i0 + c < m) ? A[kg + int64_t(i0 + c) * lda] : 0.0;
        }
        {
            const int kk = threadIdx.x & 31, c = threadIdx.x >> 5;
            const int64_t kg = kb + kk;
            Bs[kk][c] = (kg < k1 && c < n) ? B[kg + int64_t(c) * ldb] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < TN_T; ++kk) acc = fma(As[kk][tx], Bs[kk][ty], acc);
        __syncthreads();
    }
    const int i = i0 + tx;
    if (i < m && ty < n) part[(int64_t(blockIdx.z) * n + ty) * m + i] = acc;
}

// C = alpha * (sum of the splits' partial products) + beta * C. A block
// takes 32 outputs (one per lane, coalesced) and its 8 warps take every 8th
// split, each with four partial sums, so that the dependent chain of FP64
// additions (GB300: a dependent FP64 add waits about 63 cycles) and of loads
// is splits / 32 long; the partial sums are added in a fixed order.
__global__ void __launch_bounds__(256) gemm_tn_reduce(const double* __restrict__ part, int splits, int m, int n,
                                                      double alpha, double beta, double* C, int64_t ldc) {
    __shared__ double red[8][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int total = m * n;
    for (int base = blockIdx.x * 32; base < total; base += gridDim.x * 32) {
        const int e = base + tx;
        double s = 0.0;
        if (e < total) {
            // four independent loads and partial sums per step
            double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
            int sp = ty;
            for (; sp + 24 < splits; sp += 32) {
                s0 += part[int64_t(sp) * total + e];
                s1 += part[int64_t(sp + 8) * total + e];
                s2 += part[int64_t(sp + 16) * total + e];
                s3 += part[int64_t(sp + 24) * total + e];
            }
            for (; sp < splits; sp += 8) s0 += part[int64_t(sp) * total + e];
            s = (s0 + s1) + (s2 + s3);
        }
        red[ty][tx] = s;
        __syncthreads();
        if (ty == 0 && e < total) {
            double t = red[0][tx];
            for (int w = 1; w < 8; ++w) t += red[w][tx];
            const int i = e % m, j = e / m;
            double v = alpha * t;
            if (beta != 0.0) v += beta * C[i + j * ldc];
            C[i + j * ldc] = v;
        }
        __syncthreads();
    }
}

// ------------------------------- gemm_nn ----------------------------------
constexpr int NN_C = 8;     // columns of C per block
constexpr int NN_R = 32;    // rows of C per block
constexpr int NN_G = 8;     // threads sharing one row (the inner dimension split)
constexpr int NN_MB = 128;  // rows of B staged per pass

// C(K x n) = alpha A(K x m) B(m x n) + beta C: 32-row blocks so that the FP64
// work (bound by each SM's FP64 rate) reaches every SM for K of a few thousand;
// the 8 threads of a row take every 8th inner index and add up in shared memory.
__global__ void __launch_bounds__(256) gemm_nn_kernel(const double* __restrict__ A, int64_t lda,
                                                      const double* __restrict__ B, int64_t ldb,
                                                      double* C, int64_t ldc, int64_t K, int m,
                                                      int n, double alpha, double beta) {
    __shared__ double Bs[NN_MB][NN_C];
    __shared__ double red[NN_G][NN_R][NN_C + 1];
    const int r = threadIdx.x % NN_R, g = threadIdx.x / NN_R;
    const int64_t i = int64_t(blockIdx.x) * NN_R + r;
    const int c0 = blockIdx.y * NN_C;
    const int nc = min(NN_C, n - c0);
    double acc[NN_C];
#pragma unroll
    for (int c = 0; c < NN_C; ++c) acc[c] = 0.0;
    for (int m0 = 0; m0 < m; m0 += NN_MB) {
        const int mm = min(NN_MB, m - m0);
        __syncthreads();
        for (int e = threadIdx.x; e < mm * NN_C; e += 256) {
            const int j = e / NN_C, c = e % NN_C;
            Bs[j][c] = c < nc ? B[(m0 + j) + int64_t(c0 + c) * ldb] : 0.0;
        }
        __syncthreads();
        if (i < K) {
            for (int j = g; j < mm; j += NN_G) {
                const double a = A[i + int64_t(m0 + j) * lda];
#pragma unroll
                for (int c = 0; c < NN_C; ++c) acc[c] = fma(a, Bs[j][c], acc[c]);
            }
        }
    }
#pragma unroll
    for (int c = 0; c < NN_C; ++c) red[g][r][c] = acc[c];
    __syncthreads();
    if (g == 0 && i < K) {
        for (int c = 0; c < nc; ++c) {
            double v = 0.0;
            for (int q = 0; q < NN_G; ++q) v += red[q][r][c];
            double* p = C + i + int64_t(c0 + c) * ldc;
            v *= alpha;
            if (beta != 0.0) v += beta * (*p);
            *p = v;
        }
    }
}

// ------------------------------ chol_rinv ---------------------------------
__global__ void __launch_bounds__(256) chol_rinv_kernel(double* G, int n, double* Rinv, int* bad) {
    __shared__ double s_d;
    __shared__ int s_bad;
    __shared__ double s_maxd;
    extern __shared__ double g0[];  // original diagonal (n)
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        g0[j] = G[j + int64_t(j) * n];
        bad[j] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int j = 0; j < n; ++j) m = fmax(m, g0[j]);
        s_maxd = m;
    }
    __syncthreads();
    for (int j = 0; j < n; ++j) {
        if (threadIdx.x == 0) {
            const double d2 = G[j + int64_t(j) * n];
            const bool b = !(d2 > 1e-28 * s_maxd) || !(d2 > 1e-14 * g0[j]) || !isfinite(d2);
            s_bad = b ? 1 : 0;
            s_d = b ? 1.0 : sqrt(d2);
            if (b) bad[j] = 1;
        }
        __syncthreads();
        const double d = s_d;
        const int bj = s_bad;
        for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x)
            G[i + int64_t(j) * n] = bj ? 0.0 : G[i + int64_t(j) * n] / d;
        if (threadIdx.x == 0) G[j + int64_t(j) * n] = d;
        __syncthreads();
        const int r = n - j - 1;
        for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
            const int ii = j + 1 + e % r, ll = j + 1 + e / r;
            if (ii >= ll) G[ii + int64_t(ll) * n] -= G[ii + int64_t(j) * n] * G[ll + int64_t(j) * n];
        }
        __syncthreads();
    }
    // Rinv = L^-T : row c of Rinv is column c of L^-1 (forward substitution)
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        for (int i = 0; i < c; ++i) Rinv[c + int64_t(i) * n] = 0.0;
        for (int i = c; i < n; ++i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int l = c; l < i; ++l) s -= G[i + int64_t(l) * n] * Rinv[c + int64_t(l) * n];
            Rinv[c + int64_t(i) * n] = s / G[i + int64_t(i) * n];
        }
    }
}

// Shared-memory form for n <= kCholSmemN: L and X = L^-1 in shared memory,
// one division per column (its reciprocal scales the column) and X by
// column-oriented forward substitution, whose dependent chain is one
// multiply-subtract per column of L instead of a dot product per entry.
constexpr int kCholSmemN = 96;

size_t chol_smem_bytes(int n) { return (2 * size_t(n) * n + 3 * size_t(n)) * sizeof(double); }

// 1 / sqrt(x) for x > 0 finite: x = m 4^e with m in [1, 4) (exact, from the
// exponent bits), an FP32 approximate reciprocal square root of m refined by
// three Newton steps y <- y (3 - m y^2) / 2 in FP64 (each squares the relative
// error: 2^-22 -> about 2^-52), then scaled by 2^-e.
__device__ inline double rsqrt_newton(double x) {
    const long long bits = __double_as_longlong(x);
    const int ex = int((bits >> 52) & 0x7ff) - 1023;  // x = f 2^ex, f in [1, 2)
    if (ex == -1023) return 1.0 / sqrt(x);            // subnormal x
    const int e = ex >> 1;                            // floor(ex / 2)
    const double m = __longlong_as_double(bits - (static_cast<long long>(2 * e) << 52));  // in [1, 4)
    float yf;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(float(m)));
    double y = yf;
    for (int it = 0; it < 3; ++it) y = y * fma(-0.5 * m, y * y, 1.5);
    return y * __longlong_as_double(static_cast<long long>(1023 - e) << 52);
}

__global__ void __launch_bounds__(256) chol_rinv_smem_kernel(double* G, int n, double* Rinv, int* bad) {
    extern __shared__ double sm[];
    double* L = sm;                       // n x n, column-major
    double* X = L + int64_t(n) * n;       // L^-1, column-major
    double* g0 = X + int64_t(n) * n;      // original diagonal
    double* inv = g0 + n;                 // 1 / L(j, j)
    double* s_misc = inv + n;             // [0]: largest original diagonal entry
    __shared__ double s_inv;
    __shared__ int s_bad;
    const int tid = threadIdx.x;
    const int nn = n * n;
    for (int e = tid; e < nn; e += blockDim.x) {
        L[e] = G[e];
        X[e] = (e % n == e / n) ? 1.0 : 0.0;
    }
    for (int j = tid; j < n; j += blockDim.x) {
        g0[j] = G[j + int64_t(j) * n];
        bad[j] = 0;
    }
    __syncthreads();
    if (tid == 0) {
        double m = 0.0;
        for (int j = 0; j < n; ++j) m = fmax(m, g0[j]);
        s_misc[0] = m;
    }
    __syncthreads();
    const double maxd = s_misc[0];
    for (int j = 0; j < n; ++j) {
        if (tid == 0) {
            const double d2 = L[j + j * n];
            const bool b = !(d2 > 1e-28 * maxd) || !(d2 > 1e-14 * g0[j]) || !isfinite(d2);
            // 1 / sqrt(d2) by Newton steps from an FP32 seed, sqrt(d2) = d2 / sqrt(d2):
            // the pivot's chain is a few dependent FP64 FMAs (each waits about 63
            // cycles on GB300) instead of a square root and a division
            const double y = b ? 1.0 : rsqrt_newton(d2);
            s_bad = b ? 1 : 0;
            s_inv = y;
            inv[j] = y;
            L[j + j * n] = b ? 1.0 : d2 * y;
            if (b) bad[j] = 1;
        }
        __syncthreads();
        const double r = s_inv;
        const int bj = s_bad;
        for (int i = j + 1 + tid; i < n; i += blockDim.x) L[i + j * n] = bj ? 0.0 : L[i + j * n] * r;
        __syncthreads();
        const int rr = n - j - 1;
        for (int e = tid; e < rr * rr; e += blockDim.x) {
            const int ii = j + 1 + e % rr, ll = j + 1 + e / rr;
            if (ii >= ll) L[ii + ll * n] -= L[ii + j * n] * L[ll + j * n];
        }
        __syncthreads();
    }
    // X = L^-1 (lower): row l of X is final once scaled; it then updates the
    // rows below it (only columns c <= l are nonzero)
    for (int l = 0; l < n; ++l) {
        const double r = inv[l];
        for (int c = tid; c <= l; c += blockDim.x) X[l + c * n] *= r;
        __syncthreads();
        const int rows = n - l - 1, cols = l + 1;
        for (int e = tid; e < rows * cols; e += blockDim.x) {
            const int i = l + 1 + e % rows, c = e / rows;
            X[i + c * n] -= L[i + l * n] * X[l + c * n];
        }
        __syncthreads();
    }
    // Rinv = L^-T (upper): Rinv(c, i) = X(i, c); L back into G
    for (int e = tid; e < nn; e += blockDim.x) {
        const int c = e % n, i = e / n;
        Rinv[e] = (i >= c) ? X[i + c * n] : 0.0;
        G[e] = L[e];
    }
}

}  // namespace

// Enough for every product with m' <= m, n' <= n and this K: a smaller
// product may take more splits (fewer tiles), but splits * m' * n' never
// exceeds min(ceil(K / TN_KMIN) m n, tn_ctas() * TN_T^2) (at least m n; a tile
// holds at most TN_T^2 outputs).
int64_t gemm_tn_scratch_doubles(int m, int n, int64_t K) {
    const int64_t s = std::max<int64_t>(1, (K + TN_KMIN - 1) / TN_KMIN);
    const int64_t bound = std::min<int64_t>(s * m * n, int64_t(tn_ctas()) * TN_T * TN_T);
    return std::max<int64_t>(bound, int64_t(m) * n);
}

cudaError_t launch_gemm_tn(const double* A, int64_t lda, const double* B, int64_t ldb, double* C,
                           int64_t ldc, int m, int n, int64_t K, double alpha, double beta,
                           double* scratch, int64_t scratch_doubles, cudaStream_t s) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    const int splits = tn_splits(m, n, K);
    if (int64_t(splits) * m * n > scratch_doubles) return cudaErrorInvalidValue;
    KL_RANGE(A, block_extent(K, m, lda), double, "gemm_tn A");
    KL_RANGE(B, block_extent(K, n, ldb), double, "gemm_tn B");
    KL_RANGE(C, block_extent(m, n, ldc), double, "gemm_tn C");
    KL_RANGE(scratch, int64_t(splits) * m * n, double, "gemm_tn scratch");
    const int64_t kchunk = ((K + splits - 1) / splits + TN_T - 1) / TN_T * TN_T;
    if (n <= TN_NARROW) {
        dim3 grid((m + TN_T - 1) / TN_T, 1, splits);
        gemm_tn_narrow_kernel<<<grid, 256, 0, s>>>(A, lda, B, ldb, m, n, K, kchunk, scratch);
    } else {
        dim3 grid((m + TN_T - 1) / TN_T, (n + TN_T - 1) / TN_T, splits);
        gemm_tn_kernel<<<grid, 256, 0, s>>>(A, lda, B, ldb, m, n, K, kchunk, scratch);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int g = std::max(1, std::min(device_sm_count() * 8, (m * n + 31) / 32));
    gemm_tn_reduce<<<g, 256, 0, s>>>(scratch, splits, m, n, alpha, beta, C, ldc);
    return cudaGetLastError();
}

cudaError_t launch_gemm_nn(const double* A, int64_t lda, const double* B, int64_t ldb, double* C,
                           int64_t ldc, int64_t K, int m, int n, double alpha, double beta,
                           cudaStream_t s) {
    if (K <= 0 || n <= 0) return cudaSuccess;
    KL_RANGE(A, block_extent(K, m, lda), double, "gemm_nn A");
    KL_RANGE(B, block_extent(m, n, ldb), double, "gemm_nn B");
    KL_RANGE(C, block_extent(K, n, ldc), double, "gemm_nn C");
    dim3 grid(unsigned((K + NN_R - 1) / NN_R), unsigned((n + NN_C - 1) / NN_C));
    gemm_nn_kernel<<<grid, 256, 0, s>>>(A, lda, B, ldb, C, ldc, K, m, n, alpha, beta);
    return cudaGetLastError();
}

cudaError_t launch_chol_rinv(double* G, int n, double* Rinv, int* bad, cudaStream_t s) {
    KL_RANGE(G, int64_t(n) * n, double, "chol G");
    KL_RANGE(Rinv, int64_t(n) * n, double, "chol Rinv");
    KL_RANGE(bad, n, int, "chol flags");
    if (n >= 1 && n <= kCholSmemN) {
        static std::once_flag once;
        static cudaError_t attr_error = cudaSuccess;
        std::call_once(once, [] {
            attr_error = cudaFuncSetAttribute(chol_rinv_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              int(chol_smem_bytes(kCholSmemN)));
        });
        if (attr_error != cudaSuccess) return attr_error;
        chol_rinv_smem_kernel<<<1, 256, chol_smem_bytes(n), s>>>(G, n, Rinv, bad);
        return cudaGetLastError();
    }
    chol_rinv_kernel<<<1, 256, n * sizeof(double), s>>>(G, n, Rinv, bad);
    return cudaGetLastError();
}

}  // namespace kl
