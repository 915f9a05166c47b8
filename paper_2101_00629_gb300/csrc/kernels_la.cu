// Dense FP64 linear algebra of the outer eigensolver (Sec. 3: the standard
// form A' v' = lambda v' is solved iteratively; Sec. 3.3: N_iter matvecs).
//
//   gemm_tn    C = alpha A^T B + beta C for tall A, B (projections V^T W,
//              Gram matrices, Rayleigh-Ritz matrices). The long dimension is
//              split over CTAs; partial tiles are summed in a fixed order.
//   gemm_nn    C = alpha A B + beta C for tall A and small B (basis updates).
//   chol_rinv  Cholesky of a small SPD Gram matrix and the inverse of its
//              transpose (CholQR), flagging collapsed pivots.
//   nonsym_eig Householder reduction to Hessenberg form, Francis double-shift
//              QR to real Schur form with accumulated Schur vectors, ordering
//              of the Schur form, and eigenvectors by back substitution (one
//              warp: the bulge chase is a serial chain of small updates, so
//              warp-level synchronisation is what keeps it fast).
//   sym_eig    the same kernel for a symmetric matrix (ordered Schur vectors
//              are its eigenvectors).
#include <cfloat>
#include <cmath>

#include "kl_internal.h"

namespace kl {

namespace {

// ------------------------------- gemm_tn ----------------------------------
constexpr int TN_T = 32;

inline int tn_splits(int m, int n, int64_t K) {
    // the long dimension is cut into chunks of >= 256 rows until about eight
    // CTAs per SM exist (FP64 work is the limit: ~2 DFMA/clock/SM on GB300)
    const int tiles = ((m + TN_T - 1) / TN_T) * ((n + TN_T - 1) / TN_T);
    int64_t s = (K + 255) / 256;
    int64_t cap = (8 * 152) / tiles;
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

__global__ void gemm_tn_reduce(const double* __restrict__ part, int splits, int m, int n,
                               double alpha, double beta, double* C, int64_t ldc) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * n; e += gridDim.x * blockDim.x) {
        const int i = e % m, j = e / m;
        double s = 0.0;
        for (int sp = 0; sp < splits; ++sp) s += part[(int64_t(sp) * n + j) * m + i];
        double v = alpha * s;
        if (beta != 0.0) v += beta * C[i + j * ldc];
        C[i + j * ldc] = v;
    }
}

// ------------------------------- gemm_nn ----------------------------------
constexpr int NN_C = 8;     // columns per thread
constexpr int NN_M = 512;   // rows of B staged per pass

__global__ void __launch_bounds__(256) gemm_nn_kernel(const double* __restrict__ A, int64_t lda,
                                                      const double* __restrict__ B, int64_t ldb,
                                                      double* C, int64_t ldc, int64_t K, int m,
                                                      int n, double alpha, double beta) {
    __shared__ double Bs[NN_M][NN_C];
    const int64_t i = int64_t(blockIdx.x) * 256 + threadIdx.x;
    const int c0 = blockIdx.y * NN_C;
    const int nc = min(NN_C, n - c0);
    double acc[NN_C];
#pragma unroll
    for (int c = 0; c < NN_C; ++c) acc[c] = 0.0;
    for (int m0 = 0; m0 < m; m0 += NN_M) {
        const int mm = min(NN_M, m - m0);
        __syncthreads();
        for (int e = threadIdx.x; e < NN_M * NN_C; e += 256) {
            const int j = e / NN_C, c = e % NN_C;
            Bs[j][c] = (j < mm && c < nc) ? B[(m0 + j) + int64_t(c0 + c) * ldb] : 0.0;
        }
        __syncthreads();
        if (i < K) {
            for (int j = 0; j < mm; ++j) {
                const double a = A[i + int64_t(m0 + j) * lda];
#pragma unroll
                for (int c = 0; c < NN_C; ++c) acc[c] = fma(a, Bs[j][c], acc[c]);
            }
        }
    }
    if (i < K) {
        for (int c = 0; c < nc; ++c) {
            double* p = C + i + int64_t(c0 + c) * ldc;
            double v = alpha * acc[c];
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

// ------------------------------ nonsym_eig --------------------------------
struct cplx {
    double re, im;
};
__device__ inline cplx cmul(cplx a, cplx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ inline cplx cdiv(cplx a, cplx b) {
    // Smith's algorithm
    if (fabs(b.re) >= fabs(b.im)) {
        const double r = b.im / b.re, d = b.re + b.im * r;
        return {(a.re + a.im * r) / d, (a.im - a.re * r) / d};
    }
    const double r = b.re / b.im, d = b.re * r + b.im;
    return {(a.re * r + a.im) / d, (a.im * r - a.re) / d};
}

// Apply the reflector (I - beta v v^T) (v of length len, len <= 3) to rows
// r0..r0+len-1 of M, columns c0..c1-1 (left) -- work split over threads.
__device__ inline void refl_rows(double* M, int n, int r0, int len, int c0, int c1, const double* v,
                                 double beta) {
    for (int j = c0 + threadIdx.x; j < c1; j += blockDim.x) {
        double s = 0.0;
        for (int t = 0; t < len; ++t) s += v[t] * M[(r0 + t) + int64_t(j) * n];
        s *= beta;
        for (int t = 0; t < len; ++t) M[(r0 + t) + int64_t(j) * n] -= s * v[t];
    }
}
// Right application to columns c0..c0+len-1, rows r0..r1-1.
__device__ inline void refl_cols(double* M, int n, int c0, int len, int r0, int r1, const double* v,
                                 double beta) {
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        double s = 0.0;
        for (int t = 0; t < len; ++t) s += M[i + int64_t(c0 + t) * n] * v[t];
        s *= beta;
        for (int t = 0; t < len; ++t) M[i + int64_t(c0 + t) * n] -= s * v[t];
    }
}

// Householder vector for x (length len <= 3): (I - beta v v^T) x = alpha e1.
__device__ inline void house(const double* x, int len, double* v, double& beta) {
    double nrm = 0.0;
    for (int t = 0; t < len; ++t) nrm += x[t] * x[t];
    nrm = sqrt(nrm);
    for (int t = 0; t < len; ++t) v[t] = x[t];
    if (nrm == 0.0) {
        beta = 0.0;
        return;
    }
    v[0] += (x[0] >= 0.0 ? nrm : -nrm);
    double vv = 0.0;
    for (int t = 0; t < len; ++t) vv += v[t] * v[t];
    beta = vv > 0.0 ? 2.0 / vv : 0.0;
}

__global__ void __launch_bounds__(32) nonsym_eig_kernel(const double* __restrict__ H, int n,
                                                        double* wr_out, double* wi_out,
                                                        double* Vout, double* Qout, double* work,
                                                        int* status, int use_smem, int sym) {
    extern __shared__ double smem_a[];
    // the Schur form lives in shared memory when it fits: thread 0's serial
    // scans (deflation, block search) then cost shared- not global-memory
    // latency
    double* A = use_smem ? smem_a : work;    // n x n (Schur form)
    double* Z = work + int64_t(n) * n;       // n x n (Schur vectors), always global
    double* X = Z + int64_t(n) * n;          // n x n (eigenvectors of T, real/imag)
    double* wr = X + int64_t(n) * n;         // n
    double* wi = wr + n;                     // n
    double* hv = wi + n;                     // n (Householder vector for Hessenberg)
    __shared__ double s_v[3];
    __shared__ double s_beta;
    __shared__ int s_l, s_u, s_its, s_fail, s_action;
    __shared__ double s_sh, s_th;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < n * n; e += nt) {
        A[e] = sym ? 0.5 * (H[e] + H[(e % n) * n + e / n]) : H[e];
        Z[e] = (e % n == e / n) ? 1.0 : 0.0;
    }
    __syncwarp();
    // ---- Hessenberg reduction ----
    for (int k = 0; k + 2 < n; ++k) {
        const int len = n - k - 1;
        if (tid == 0) {
            double nrm = 0.0;
            for (int t = 0; t < len; ++t) nrm += A[(k + 1 + t) + int64_t(k) * n] * A[(k + 1 + t) + int64_t(k) * n];
            nrm = sqrt(nrm);
            for (int t = 0; t < len; ++t) hv[t] = A[(k + 1 + t) + int64_t(k) * n];
            double beta = 0.0;
            if (nrm > 0.0) {
                hv[0] += (hv[0] >= 0.0 ? nrm : -nrm);
                double vv = 0.0;
                for (int t = 0; t < len; ++t) vv += hv[t] * hv[t];
                beta = 2.0 / vv;
            }
            s_beta = beta;
        }
        __syncwarp();
        const double beta = s_beta;
        if (beta != 0.0) {
            // left: rows k+1..n-1, columns k..n-1
            for (int j = k + tid; j < n; j += nt) {
                double s = 0.0;
                for (int t = 0; t < len; ++t) s += hv[t] * A[(k + 1 + t) + int64_t(j) * n];
                s *= beta;
                for (int t = 0; t < len; ++t) A[(k + 1 + t) + int64_t(j) * n] -= s * hv[t];
            }
            __syncwarp();
            // right: all rows, columns k+1..n-1 ; and Z
            for (int i = tid; i < n; i += nt) {
                double s = 0.0, sz = 0.0;
                for (int t = 0; t < len; ++t) {
                    s += A[i + int64_t(k + 1 + t) * n] * hv[t];
                    sz += Z[i + int64_t(k + 1 + t) * n] * hv[t];
                }
                s *= beta;
                sz *= beta;
                for (int t = 0; t < len; ++t) {
                    A[i + int64_t(k + 1 + t) * n] -= s * hv[t];
                    Z[i + int64_t(k + 1 + t) * n] -= sz * hv[t];
                }
            }
        }
        __syncwarp();
        for (int i = k + 2 + tid; i < n; i += nt) A[i + int64_t(k) * n] = 0.0;
        __syncwarp();
    }
    // ---- Francis double-shift QR to real Schur form ----
    double anorm = 0.0;
    for (int e = 0; e < n * n; ++e) anorm = fmax(anorm, fabs(A[e]));
    if (tid == 0) {
        s_u = n - 1;
        s_its = 0;
        s_fail = 0;
    }
    __syncwarp();
    int total_its = 0;
    while (true) {
        __syncwarp();
        if (tid == 0) {
            const int u = s_u;
            int l = 0;
            int action = 0;  // 1: one root, 2: two roots, 3: Francis step, 4: done, 5: split
            if (u < 0) {
                action = 4;
            } else {
                for (l = u; l >= 1; --l) {
                    double s = fabs(A[(l - 1) + int64_t(l - 1) * n]) + fabs(A[l + int64_t(l) * n]);
                    if (s == 0.0) s = anorm;
                    const double sub = fabs(A[l + int64_t(l - 1) * n]);
                    // absolute test at roundoff of the whole matrix: next to
                    // eigenvalues that are themselves at roundoff level a
                    // relative test can never be met
                    if (sub <= double(n) * DBL_EPSILON * anorm) {
                        A[l + int64_t(l - 1) * n] = 0.0;
                        break;
                    }
                    // relative test, confirmed by the more conservative
                    // Ahues-Kressner criterion (off-diagonal product against
                    // the gap of the diagonal pair)
                    if (sub <= DBL_EPSILON * s) {
                        const double up = fabs(A[(l - 1) + int64_t(l) * n]);
                        const double ab = fmax(sub, up), ba = fmin(sub, up);
                        const double dd = fabs(A[(l - 1) + int64_t(l - 1) * n] - A[l + int64_t(l) * n]);
                        const double aa = fmax(fabs(A[l + int64_t(l) * n]), dd);
                        const double bb = fmin(fabs(A[l + int64_t(l) * n]), dd);
                        const double ss = aa + ab;
                        if (ba * (ab / ss) <= fmax(DBL_MIN, DBL_EPSILON * (bb * (aa / ss)))) {
                            A[l + int64_t(l - 1) * n] = 0.0;
                            break;
                        }
                    }
                }
                if (l < 0) l = 0;
                if (l == u) action = 1;
                else if (l == u - 1) action = 2;
                else action = 3;
            }
            if (action == 3 && s_its >= 30 && s_its % 10 == 5) {
                // A window that resists the shifts for 30 iterations is a
                // cluster of (numerically) equal eigenvalues perturbed into a
                // near-Jordan block. The window is already decoupled from its
                // neighbours, so zeroing its smallest subdiagonal leaves every
                // other eigenvalue and the window's invariant subspace as
                // they are; it only splits the cluster (by about
                // sqrt(|sub * super|)).
                // Only a subdiagonal far below any tolerance of the outer
                // solver is dropped (backward error 1e-10 * ||H||).
                int m = l + 1;
                for (int i = l + 2; i <= u; ++i)
                    if (fabs(A[i + int64_t(i - 1) * n]) < fabs(A[m + int64_t(m - 1) * n])) m = i;
                if (fabs(A[m + int64_t(m - 1) * n]) <= 1e-10 * anorm) {
                    A[m + int64_t(m - 1) * n] = 0.0;
                    action = 5;
                }
            }
            s_l = l;
            s_action = action;
            if (action == 3) {
                if (s_its >= 300 || total_its > 120 * max(10, n)) {
                    s_fail = 1;
                    s_action = 4;
                } else {
                    double sh, th;
                    if (s_its > 0 && s_its % 10 == 0) {  // exceptional shift
                        const double ex = fabs(A[u + int64_t(u - 1) * n]) + fabs(A[(u - 1) + int64_t(u - 2) * n]);
                        const double c = A[u + int64_t(u) * n] + 0.75 * ex;
                        sh = 2.0 * c;
                        th = c * c + 0.4375 * ex * ex;
                    } else {
                        const double a = A[(u - 1) + int64_t(u - 1) * n], b = A[(u - 1) + int64_t(u) * n];
                        const double c = A[u + int64_t(u - 1) * n], d = A[u + int64_t(u) * n];
                        sh = a + d;
                        th = a * d - b * c;
                    }
                    s_sh = sh;
                    s_th = th;
                    s_its = s_its + 1;
                }
            }
        }
        __syncwarp();
        const int action = s_action;
        const int u = s_u, l = s_l;
        if (action == 4) break;
        if (action == 5) {
            // a stalled window was split; look for deflations again
            if (tid == 0) s_its = s_its + 1;
            continue;
        }
        if (action == 1) {
            if (tid == 0) {
                wr[u] = A[u + int64_t(u) * n];
                wi[u] = 0.0;
                s_u = u - 1;
                s_its = 0;
            }
            continue;
        }
        if (action == 2) {
            // 2x2 block at (u-1, u): triangularise if its eigenvalues are real
            __shared__ double s_cs, s_sn;
            __shared__ int s_rot;
            if (tid == 0) {
                const double a = A[(u - 1) + int64_t(u - 1) * n], b = A[(u - 1) + int64_t(u) * n];
                const double c = A[u + int64_t(u - 1) * n], d = A[u + int64_t(u) * n];
                const double p = 0.5 * (a - d);
                // a symmetric matrix has real eigenvalues: rounding may leave
                // b c slightly negative, which must not create a complex pair
                const double q = sym ? fmax(p * p + b * c, 0.0) : p * p + b * c;
                s_rot = 0;
                if (q >= 0.0) {
                    const double zz = p + (p >= 0.0 ? sqrt(q) : -sqrt(q));
                    const double r = hypot(zz, c);
                    if (r > 0.0) {
                        s_cs = zz / r;
                        s_sn = c / r;
                        s_rot = 1;
                    }
                    wr[u - 1] = d + zz;
                    wr[u] = (zz != 0.0) ? d - b * c / zz : d + zz;
                    wi[u - 1] = wi[u] = 0.0;
                } else {
                    wr[u - 1] = wr[u] = d + p;
                    wi[u - 1] = sqrt(-q);
                    wi[u] = -sqrt(-q);
                }
            }
            __syncwarp();
            if (s_rot) {
                const double cs = s_cs, sn = s_sn;
                for (int j = u - 1 + tid; j < n; j += nt) {
                    const double x1 = A[(u - 1) + int64_t(j) * n], x2 = A[u + int64_t(j) * n];
                    A[(u - 1) + int64_t(j) * n] = cs * x1 + sn * x2;
                    A[u + int64_t(j) * n] = -sn * x1 + cs * x2;
                }
                __syncwarp();
                for (int i = tid; i < n; i += nt) {
                    if (i <= u) {
                        const double x1 = A[i + int64_t(u - 1) * n], x2 = A[i + int64_t(u) * n];
                        A[i + int64_t(u - 1) * n] = cs * x1 + sn * x2;
                        A[i + int64_t(u) * n] = -sn * x1 + cs * x2;
                    }
                    const double z1 = Z[i + int64_t(u - 1) * n], z2 = Z[i + int64_t(u) * n];
                    Z[i + int64_t(u - 1) * n] = cs * z1 + sn * z2;
                    Z[i + int64_t(u) * n] = -sn * z1 + cs * z2;
                }
                __syncwarp();
                if (tid == 0) {
                    A[u + int64_t(u - 1) * n] = 0.0;
                    // diagonal entries now hold the two real eigenvalues
                    wr[u - 1] = A[(u - 1) + int64_t(u - 1) * n];
                    wr[u] = A[u + int64_t(u) * n];
                }
            }
            __syncwarp();
            if (tid == 0) {
                s_u = u - 2;
                s_its = 0;
            }
            continue;
        }
        // Francis double-shift step on the window [l, u] (size ns >= 3)
        ++total_its;
        const int ns = u - l + 1;
        __shared__ double s_x[3];
        if (tid == 0) {
            const double h11 = A[l + int64_t(l) * n], h12 = A[l + int64_t(l + 1) * n];
            const double h21 = A[(l + 1) + int64_t(l) * n], h22 = A[(l + 1) + int64_t(l + 1) * n];
            const double h32 = A[(l + 2) + int64_t(l + 1) * n];
            s_x[0] = h11 * h11 + h12 * h21 - s_sh * h11 + s_th;
            s_x[1] = h21 * (h11 + h22 - s_sh);
            s_x[2] = h21 * h32;
        }
        __syncwarp();
        for (int kk = 0; kk <= ns - 3; ++kk) {
            if (tid == 0) {
                double v[3], beta;
                house(s_x, 3, v, beta);
                s_v[0] = v[0];
                s_v[1] = v[1];
                s_v[2] = v[2];
                s_beta = beta;
            }
            __syncwarp();
            const int r0 = l + kk;
            const int c0 = l + (kk > 0 ? kk - 1 : 0);
            refl_rows(A, n, r0, 3, c0, n, s_v, s_beta);
            __syncwarp();
            const int rmax = min(l + kk + 3, u);  // last row touched (inclusive)
            refl_cols(A, n, r0, 3, 0, rmax + 1, s_v, s_beta);
            refl_cols(Z, n, r0, 3, 0, n, s_v, s_beta);
            __syncwarp();
            if (tid == 0) {
                s_x[0] = A[(r0 + 1) + int64_t(r0) * n];
                s_x[1] = A[(r0 + 2) + int64_t(r0) * n];
                s_x[2] = (kk < ns - 3) ? A[(r0 + 3) + int64_t(r0) * n] : 0.0;
            }
            __syncwarp();
        }
        if (tid == 0) {
            double v[3], beta;
            house(s_x, 2, v, beta);
            s_v[0] = v[0];
            s_v[1] = v[1];
            s_beta = beta;
        }
        __syncwarp();
        refl_rows(A, n, u - 1, 2, u - 2, n, s_v, s_beta);
        __syncwarp();
        refl_cols(A, n, u - 1, 2, 0, u + 1, s_v, s_beta);
        refl_cols(Z, n, u - 1, 2, 0, n, s_v, s_beta);
        __syncwarp();
        // clean the bulge remnants below the subdiagonal of the window
        for (int e = tid; e < ns * ns; e += nt) {
            const int i = l + e % ns, j = l + e / ns;
            if (i > j + 1) A[i + int64_t(j) * n] = 0.0;
        }
    }
    __syncwarp();
    // ---- reorder the real Schur form: eigenvalues by decreasing real part ----
    // Selection sort over the diagonal blocks (1x1 real eigenvalues, 2x2
    // complex pairs). Adjacent blocks A (n1 x n1) and B (n2 x n2) with
    // coupling C are exchanged by the direct swap: solve A X - X B = C, the
    // columns of [X; -I] span the B-invariant subspace, and the orthogonal
    // factor Q of their QR factorisation gives Q^T [A C; 0 B] Q = [B' *; 0 A'].
    // The leading Schur vectors then span the invariant subspace of the
    // largest eigenvalues, which is what a Krylov-Schur restart keeps.
    __shared__ double s_q[16];
    __shared__ int s_k, s_m, s_n2, s_act, s_pos;
    if (tid == 0) s_pos = 0;
    while (!s_fail) {
        // every lane has read the previous decision before lane 0 rewrites it
        __syncwarp();
        if (tid == 0) {
            const int pos = s_pos;
            s_act = 0;
            if (pos < n) {
                // best block at or after pos (max real part, earliest on ties)
                int best = -1, bsz = 1, prev = -1, psz = 1, before_best = -1, before_sz = 1;
                double bkey = -DBL_MAX;
                for (int i = pos; i < n;) {
                    const int sz = (i + 1 < n && A[(i + 1) + int64_t(i) * n] != 0.0) ? 2 : 1;
                    const double key = sz == 1 ? A[i + int64_t(i) * n]
                                               : 0.5 * (A[i + int64_t(i) * n] + A[(i + 1) + int64_t(i + 1) * n]);
                    if (key > bkey) {
                        bkey = key;
                        best = i;
                        bsz = sz;
                        before_best = prev;
                        before_sz = psz;
                    }
                    prev = i;
                    psz = sz;
                    i += sz;
                }
                if (best == pos) {
                    s_pos = pos + bsz;
                    s_act = 2;
                } else {
                    // swap the block before `best` (k, n1) with best (n2)
                    const int k = before_best, n1 = before_sz, n2 = bsz, m = n1 + n2;
                    double K[16], x[4], W[8], Qm[16];
                    const int pdim = n1 * n2;
                    for (int r = 0; r < pdim * pdim; ++r) K[r] = 0.0;
                    // K = I_{n2} (x) A - B^T (x) I_{n1}, x = vec(X) column-major
                    for (int j = 0; j < n2; ++j)
                        for (int i = 0; i < n1; ++i) {
                            const int row = i + n1 * j;
                            for (int i2 = 0; i2 < n1; ++i2)
                                K[row + pdim * (i2 + n1 * j)] += A[(k + i) + int64_t(k + i2) * n];
                            for (int j2 = 0; j2 < n2; ++j2)
                                K[row + pdim * (i + n1 * j2)] -= A[(k + n1 + j2) + int64_t(k + n1 + j) * n];
                            x[row] = A[(k + i) + int64_t(k + n1 + j) * n];
                        }
                    // Gaussian elimination with partial pivoting (pdim <= 4)
                    double kn = 0.0;
                    for (int r = 0; r < pdim * pdim; ++r) kn = fmax(kn, fabs(K[r]));
                    const double tiny = DBL_EPSILON * fmax(kn, anorm);
                    for (int c = 0; c < pdim; ++c) {
                        int pr = c;
                        for (int r = c + 1; r < pdim; ++r)
                            if (fabs(K[r + pdim * c]) > fabs(K[pr + pdim * c])) pr = r;
                        if (pr != c) {
                            for (int cc = 0; cc < pdim; ++cc) {
                                const double t = K[c + pdim * cc]; K[c + pdim * cc] = K[pr + pdim * cc]; K[pr + pdim * cc] = t;
                            }
                            const double t = x[c]; x[c] = x[pr]; x[pr] = t;
                        }
                        if (fabs(K[c + pdim * c]) < tiny) K[c + pdim * c] = K[c + pdim * c] >= 0.0 ? tiny : -tiny;
                        for (int r = c + 1; r < pdim; ++r) {
                            const double f = K[r + pdim * c] / K[c + pdim * c];
                            for (int cc = c; cc < pdim; ++cc) K[r + pdim * cc] -= f * K[c + pdim * cc];
                            x[r] -= f * x[c];
                        }
                    }
                    for (int r = pdim - 1; r >= 0; --r) {
                        double t = x[r];
                        for (int cc = r + 1; cc < pdim; ++cc) t -= K[r + pdim * cc] * x[cc];
                        x[r] = t / K[r + pdim * r];
                    }
                    // W = [X; -I] (m x n2), Householder QR, Q accumulated
                    for (int j = 0; j < n2; ++j)
                        for (int i = 0; i < m; ++i) W[i + m * j] = (i < n1) ? x[i + n1 * j] : (i - n1 == j ? -1.0 : 0.0);
                    for (int r = 0; r < m * m; ++r) Qm[r] = (r % m == r / m) ? 1.0 : 0.0;
                    for (int j = 0; j < n2; ++j) {
                        double v[4], beta, xx[4];
                        const int len = m - j;
                        for (int t = 0; t < len; ++t) xx[t] = W[(j + t) + m * j];
                        house(xx, len, v, beta);
                        for (int c = j; c < n2; ++c) {
                            double sdot = 0.0;
                            for (int t = 0; t < len; ++t) sdot += v[t] * W[(j + t) + m * c];
                            for (int t = 0; t < len; ++t) W[(j + t) + m * c] -= beta * sdot * v[t];
                        }
                        for (int r = 0; r < m; ++r) {
                            double sdot = 0.0;
                            for (int t = 0; t < len; ++t) sdot += Qm[r + m * (j + t)] * v[t];
                            for (int t = 0; t < len; ++t) Qm[r + m * (j + t)] -= beta * sdot * v[t];
                        }
                    }
                    for (int r = 0; r < m * m; ++r) s_q[r] = Qm[r];
                    s_k = k;
                    s_m = m;
                    s_n2 = n2;
                    s_act = 1;
                }
            }
        }
        __syncwarp();
        const int act = s_act;
        if (act == 0) break;
        if (act == 1) {
            const int k = s_k, m = s_m;
            // rows k..k+m-1 <- Q^T rows (columns k..n-1)
            for (int j = k + tid; j < n; j += nt) {
                double old[4];
                for (int t = 0; t < m; ++t) old[t] = A[(k + t) + int64_t(j) * n];
                for (int t = 0; t < m; ++t) {
                    double acc = 0.0;
                    for (int u2 = 0; u2 < m; ++u2) acc += s_q[u2 + m * t] * old[u2];
                    A[(k + t) + int64_t(j) * n] = acc;
                }
            }
            __syncwarp();
            // columns k..k+m-1 <- columns Q (rows 0..k+m-1), and Z (all rows)
            for (int r = tid; r < n; r += nt) {
                double old[4], oz[4];
                for (int t = 0; t < m; ++t) {
                    old[t] = A[r + int64_t(k + t) * n];
                    oz[t] = Z[r + int64_t(k + t) * n];
                }
                for (int t = 0; t < m; ++t) {
                    double acc = 0.0, accz = 0.0;
                    for (int u2 = 0; u2 < m; ++u2) {
                        acc += old[u2] * s_q[u2 + m * t];
                        accz += oz[u2] * s_q[u2 + m * t];
                    }
                    if (r < k + m) A[r + int64_t(k + t) * n] = acc;
                    Z[r + int64_t(k + t) * n] = accz;
                }
            }
            __syncwarp();
            if (tid == 0) {
                // the exchanged blocks: zero the new (2,1) block
                const int n2 = s_n2;
                for (int i = k + n2; i < k + m; ++i)
                    for (int j = k; j < k + n2; ++j) A[i + int64_t(j) * n] = 0.0;
            }
            __syncwarp();
        }
    }
    // eigenvalues from the (re)ordered blocks
    if (tid == 0 && !s_fail) {
        for (int i = 0; i < n;) {
            if (i + 1 < n && A[(i + 1) + int64_t(i) * n] != 0.0) {
                const double a = A[i + int64_t(i) * n], b = A[i + int64_t(i + 1) * n];
                const double c = A[(i + 1) + int64_t(i) * n], d = A[(i + 1) + int64_t(i + 1) * n];
                const double pp = 0.5 * (a - d), q = pp * pp + b * c;
                wr[i] = wr[i + 1] = d + pp;
                const double im = q < 0.0 ? sqrt(-q) : 0.0;
                wi[i] = im;
                wi[i + 1] = -im;
                i += 2;
            } else {
                wr[i] = A[i + int64_t(i) * n];
                wi[i] = 0.0;
                i += 1;
            }
        }
    }
    __syncwarp();
    // ---- eigenvectors of the quasi-triangular T by back substitution ----
    // Diagonal entries within 1e-10 ||T|| of the eigenvalue belong to its
    // cluster; their components are set to zero instead of dividing by a
    // vanishing pivot, so the vectors of a (numerically) multiple eigenvalue
    // stay independent (its invariant subspace is spanned by Schur vectors).
    const double small = DBL_EPSILON * fmax(anorm, DBL_MIN);
    const double clus = 1e-10 * anorm;
    for (int col = tid; col < n && !sym; col += nt) {
        double* xr = X + int64_t(col) * n;
        if (wi[col] == 0.0) {
            const double lam = wr[col];
            for (int i = 0; i < n; ++i) xr[i] = 0.0;
            xr[col] = 1.0;
            for (int j = col - 1; j >= 0; --j) {
                const bool two = (j > 0) && A[j + int64_t(j - 1) * n] != 0.0;
                if (!two) {
                    double s = 0.0;
                    for (int l2 = j + 1; l2 <= col; ++l2) s += A[j + int64_t(l2) * n] * xr[l2];
                    double den = A[j + int64_t(j) * n] - lam;
                    if (fabs(den) <= clus) {
                        xr[j] = 0.0;
                        continue;
                    }
                    if (fabs(den) < small) den = small;
                    xr[j] = -s / den;
                } else {
                    // 2x2 system for rows j-1, j
                    double s1 = 0.0, s2 = 0.0;
                    for (int l2 = j + 1; l2 <= col; ++l2) {
                        s1 += A[(j - 1) + int64_t(l2) * n] * xr[l2];
                        s2 += A[j + int64_t(l2) * n] * xr[l2];
                    }
                    const double a11 = A[(j - 1) + int64_t(j - 1) * n] - lam, a12 = A[(j - 1) + int64_t(j) * n];
                    const double a21 = A[j + int64_t(j - 1) * n], a22 = A[j + int64_t(j) * n] - lam;
                    double det = a11 * a22 - a12 * a21;
                    if (fabs(det) < small * small) det = small * small;
                    xr[j - 1] = (-s1 * a22 + s2 * a12) / det;
                    xr[j] = (-s2 * a11 + s1 * a21) / det;
                    --j;
                }
            }
        } else if (wi[col] > 0.0) {
            // complex pair (col, col+1): vector for lambda = wr + i wi, stored
            // as real part in column col and imaginary part in column col+1
            double* xi = X + int64_t(col + 1) * n;
            const cplx lam = {wr[col], wi[col]};
            for (int i = 0; i < n; ++i) xr[i] = xi[i] = 0.0;
            // eigenvector of the 2x2 block rows/cols (col, col+1)
            // (b12, lambda - b11) solves the first row of (B - lambda I) x = 0
            // and is non-zero because lambda is not real
            const int q = col;
            xr[q] = A[q + int64_t(q + 1) * n];
            xi[q] = 0.0;
            xr[q + 1] = lam.re - A[q + int64_t(q) * n];
            xi[q + 1] = lam.im;
            for (int j = q - 1; j >= 0; --j) {
                const bool two = (j > 0) && A[j + int64_t(j - 1) * n] != 0.0;
                if (!two) {
                    cplx s = {0.0, 0.0};
                    for (int l2 = j + 1; l2 <= q + 1; ++l2) {
                        s.re += A[j + int64_t(l2) * n] * xr[l2];
                        s.im += A[j + int64_t(l2) * n] * xi[l2];
                    }
                    cplx den = {A[j + int64_t(j) * n] - lam.re, -lam.im};
                    if (fabs(den.re) + fabs(den.im) < small) den.re = small;
                    const cplx r = cdiv({-s.re, -s.im}, den);
                    xr[j] = r.re;
                    xi[j] = r.im;
                } else {
                    cplx s1 = {0.0, 0.0}, s2 = {0.0, 0.0};
                    for (int l2 = j + 1; l2 <= q + 1; ++l2) {
                        s1.re += A[(j - 1) + int64_t(l2) * n] * xr[l2];
                        s1.im += A[(j - 1) + int64_t(l2) * n] * xi[l2];
                        s2.re += A[j + int64_t(l2) * n] * xr[l2];
                        s2.im += A[j + int64_t(l2) * n] * xi[l2];
                    }
                    const cplx a11 = {A[(j - 1) + int64_t(j - 1) * n] - lam.re, -lam.im};
                    const cplx a12 = {A[(j - 1) + int64_t(j) * n], 0.0};
                    const cplx a21 = {A[j + int64_t(j - 1) * n], 0.0};
                    const cplx a22 = {A[j + int64_t(j) * n] - lam.re, -lam.im};
                    cplx det = {cmul(a11, a22).re - cmul(a12, a21).re, cmul(a11, a22).im - cmul(a12, a21).im};
                    if (fabs(det.re) + fabs(det.im) < small * small) det.re = small * small;
                    const cplx n1 = {-(cmul(s1, a22).re) + cmul(s2, a12).re, -(cmul(s1, a22).im) + cmul(s2, a12).im};
                    const cplx n2 = {-(cmul(s2, a11).re) + cmul(s1, a21).re, -(cmul(s2, a11).im) + cmul(s1, a21).im};
                    const cplx r1 = cdiv(n1, det), r2 = cdiv(n2, det);
                    xr[j - 1] = r1.re;
                    xi[j - 1] = r1.im;
                    xr[j] = r2.re;
                    xi[j] = r2.im;
                    --j;
                }
            }
        }
        // wi < 0: second member of a pair, written by its partner
    }
    __syncwarp();
    // V = Z X (each thread one row), then normalise columns (pairs jointly);
    // the symmetric mode returns the ordered Schur vectors instead
    double* Vt = A;  // reuse (Schur form no longer needed)
    for (int i = tid; i < n && !sym; i += nt) {
        for (int c = 0; c < n; ++c) {
            double s = 0.0;
            for (int l2 = 0; l2 < n; ++l2) s += Z[i + int64_t(l2) * n] * X[l2 + int64_t(c) * n];
            Vt[i + int64_t(c) * n] = s;
        }
    }
    __syncwarp();
    for (int c = tid; c < n && !sym; c += nt) {
        if (wi[c] < 0.0) continue;
        double s = 0.0;
        const int w2 = (wi[c] > 0.0) ? 2 : 1;
        for (int t = 0; t < w2; ++t)
            for (int i = 0; i < n; ++i) s += Vt[i + int64_t(c + t) * n] * Vt[i + int64_t(c + t) * n];
        s = s > 0.0 ? 1.0 / sqrt(s) : 1.0;
        for (int t = 0; t < w2; ++t)
            for (int i = 0; i < n; ++i) Vt[i + int64_t(c + t) * n] *= s;
    }
    __syncwarp();
    // sort by real part descending; a complex pair keeps its (+, -) order
    for (int i = tid; i < n; i += nt) {
        int rank = 0;
        for (int j = 0; j < n; ++j)
            if (wr[j] > wr[i] || (wr[j] == wr[i] && j < i)) ++rank;
        wr_out[rank] = wr[i];
        if (wi_out) wi_out[rank] = wi[i];
        if (Vout && !sym)
            for (int r = 0; r < n; ++r) Vout[r + int64_t(rank) * n] = Vt[r + int64_t(i) * n];
    }
    if (Qout) {
        for (int e = tid; e < n * n; e += nt) Qout[e] = Z[e];
    }
    if (tid == 0) {
        status[0] = s_fail ? 1 : 0;
        // diagnostics after the status word: QR iterations, last window end,
        // iterations spent on it
        status[1] = total_its;
        status[2] = s_u;
        status[3] = s_its;
    }
}

}  // namespace

int64_t gemm_tn_scratch_doubles(int m, int n, int64_t K) {
    return int64_t(tn_splits(m, n, K)) * m * n;
}

cudaError_t launch_gemm_tn(const double* A, int64_t lda, const double* B, int64_t ldb, double* C,
                           int64_t ldc, int m, int n, int64_t K, double alpha, double beta,
                           double* scratch, int64_t scratch_doubles, cudaStream_t s) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    const int splits = tn_splits(m, n, K);
    if (int64_t(splits) * m * n > scratch_doubles) return cudaErrorInvalidValue;
    const int64_t kchunk = ((K + splits - 1) / splits + TN_T - 1) / TN_T * TN_T;
    dim3 grid((m + TN_T - 1) / TN_T, (n + TN_T - 1) / TN_T, splits);
    gemm_tn_kernel<<<grid, 256, 0, s>>>(A, lda, B, ldb, m, n, K, kchunk, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int g = std::max(1, std::min(152 * 8, (m * n + 255) / 256));
    gemm_tn_reduce<<<g, 256, 0, s>>>(scratch, splits, m, n, alpha, beta, C, ldc);
    return cudaGetLastError();
}

cudaError_t launch_gemm_nn(const double* A, int64_t lda, const double* B, int64_t ldb, double* C,
                           int64_t ldc, int64_t K, int m, int n, double alpha, double beta,
                           cudaStream_t s) {
    if (K <= 0 || n <= 0) return cudaSuccess;
    dim3 grid(unsigned((K + 255) / 256), unsigned((n + NN_C - 1) / NN_C));
    gemm_nn_kernel<<<grid, 256, 0, s>>>(A, lda, B, ldb, C, ldc, K, m, n, alpha, beta);
    return cudaGetLastError();
}

cudaError_t launch_chol_rinv(double* G, int n, double* Rinv, int* bad, cudaStream_t s) {
    chol_rinv_kernel<<<1, 256, n * sizeof(double), s>>>(G, n, Rinv, bad);
    return cudaGetLastError();
}

int64_t sym_eig_work_doubles(int n) { return nonsym_eig_work_doubles(n); }

// Symmetric eigenproblem: the same Hessenberg (here tridiagonal) reduction and
// Francis QR; the ordered real Schur form of a symmetric matrix is diagonal,
// so the ordered Schur vectors are orthonormal eigenvectors.
cudaError_t launch_sym_eig(const double* H, int n, double* w, double* V, double* work, int* status,
                           cudaStream_t s) {
    const size_t smem = size_t(n) * n * sizeof(double);
    const int use_smem = smem <= 200 * 1024;
    if (use_smem) {
        cudaError_t e = cudaFuncSetAttribute(nonsym_eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
    }
    nonsym_eig_kernel<<<1, 32, use_smem ? smem : 0, s>>>(H, n, w, nullptr, nullptr, V, work, status, use_smem, 1);
    return cudaGetLastError();
}

int64_t nonsym_eig_work_doubles(int n) { return 3 * int64_t(n) * n + 3 * int64_t(n); }

cudaError_t launch_nonsym_eig(const double* H, int n, double* wr, double* wi, double* V, double* Q,
                              double* work, int* status, cudaStream_t s) {
    const size_t smem = size_t(n) * n * sizeof(double);
    const int use_smem = smem <= 200 * 1024;
    if (use_smem) {
        cudaError_t e = cudaFuncSetAttribute(nonsym_eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
    }
    nonsym_eig_kernel<<<1, 32, use_smem ? smem : 0, s>>>(H, n, wr, wi, V, Q, work, status, use_smem, 0);
    return cudaGetLastError();
}

}  // namespace kl
