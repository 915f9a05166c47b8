// Symmetric Rayleigh-Ritz eigenproblems by parallel cyclic Jacobi.
//
// The Galerkin operator in standard form, A' = L^-1 A L^-T (Sec. 3.1), is
// symmetric, so its Rayleigh-Ritz matrix H = V^T A' V is too; its ordered
// eigenpairs give the Ritz pairs (Sec. 3.3 leaves the eigensolver open).
//
// One CTA holds H and its eigenvector matrix in shared memory. A sweep is
// m - 1 rounds of the circle schedule on m = n rounded up to even indices;
// the n/2 rotations of a round act on disjoint index pairs, so each round is
// one parallel computation of the rotations, one parallel row update and one
// parallel column update (of H and of the vectors). A rotation is skipped when
// its off-diagonal entry is below n eps sqrt(|h_pp h_qq|) (or eps ||H||_F),
// and the sweeps stop when a sweep skips all of them.
//
// GB300's FP64 arithmetic is slow (one dependent FMA: 63 cycles; a square
// root or division ~650), so an FP64 problem is solved in FP32 first and
// refined: the FP32 vectors Q0 are made orthonormal in FP64 by a Cholesky QR,
// B = Q^T H Q (nearly diagonal) is diagonalised by FP64 Jacobi in two or three
// sweeps, and the vectors are Q W. The products are the multi-SM FP64 GEMMs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cstdint>
#include <mutex>

#include "kl_internal.h"

namespace kl {

namespace {

constexpr int kJacThreads = 256;
constexpr int kJacMaxN = 90;  // H and the vectors in shared memory, FP64

template <class R>
struct JacEps;
template <>
struct JacEps<float> {
    static constexpr float eps = FLT_EPSILON;
    static constexpr float big = 1e9f;  // |theta| beyond which t = 1 / (2 theta)
};
template <>
struct JacEps<double> {
    static constexpr double eps = DBL_EPSILON;
    static constexpr double big = 1e18;
};

// Pair k of round r of the circle schedule on m (even) indices: index m - 1
// meets r, and r + k meets r - k (mod m - 1). Every pair occurs once in the
// m - 1 rounds. Returned with p < q.
__device__ __forceinline__ void circle_pair(int m, int r, int k, int& p, int& q) {
    if (k == 0) {
        p = r;
        q = m - 1;
    } else {
        p = (r + k) % (m - 1);
        q = (r - k + (m - 1)) % (m - 1);
    }
    if (p > q) {
        const int t = p;
        p = q;
        q = t;
    }
}

size_t jacobi_smem_bytes(int n, size_t esize) {
    return 2 * size_t(n) * (n + 1) * esize + 4 * size_t(kJacMaxN) * 8;
}

// Eigenpairs of the symmetric part of the n x n column-major H: w (n,
// descending) and V (n x n column-major, column j for w[j]). status: 0, or 1
// if the off-diagonal part is still above sqrt(eps) ||H||_F after max_sweeps.
template <class R>
__global__ void __launch_bounds__(kJacThreads) jacobi_kernel(const double* __restrict__ H, int n, int max_sweeps,
                                                            double* __restrict__ w, double* __restrict__ V,
                                                            int* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char jac_smem[];
    const int ld = n + 1;
    R* A = reinterpret_cast<R*>(jac_smem);  // A[i * ld + j] = H(i, j)
    R* U = A + size_t(n) * ld;              // U[i * ld + j] = vector j, entry i
    R* rc = U + size_t(n) * ld;             // the round's rotations (and, at the end, the ranks)
    R* rs = rc + kJacMaxN;
    int* rp = reinterpret_cast<int*>(rs + kJacMaxN);
    int* rq = rp + kJacMaxN;
    __shared__ double red[kJacThreads / 32];
    __shared__ int any_rot;
    const int tid = threadIdx.x;
    const int m = n + (n & 1);
    const int npairs = m / 2;
    constexpr R eps = JacEps<R>::eps;

    double ss = 0.0;
    for (int idx = tid; idx < n * n; idx += blockDim.x) {
        const int i = idx % n, j = idx / n;
        const double h = 0.5 * (H[idx] + H[j + int64_t(i) * n]);
        A[i * ld + j] = R(h);
        U[i * ld + j] = R(i == j ? 1 : 0);
        ss += h * h;
    }
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if ((tid & 31) == 0) red[tid >> 5] = ss;
    __syncthreads();
    double fro2 = 0.0;
    for (int i = 0; i < kJacThreads / 32; ++i) fro2 += red[i];
    const R floor = R(double(eps) * sqrt(fro2));
    const R rel = R(n) * eps;

    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        if (tid == 0) any_rot = 0;
        __syncthreads();
        for (int r = 0; r < m - 1; ++r) {
            if (tid < npairs) {
                int p, q;
                circle_pair(m, r, tid, p, q);
                R c = R(1), s = R(0);
                if (q < n) {
                    const R apq = A[p * ld + q], app = A[p * ld + p], aqq = A[q * ld + q];
                    if (fabs(apq) > fmax(rel * sqrt(fabs(app) * fabs(aqq)), floor)) {
                        const R theta = (aqq - app) / (R(2) * apq);
                        const R t = fabs(theta) > JacEps<R>::big
                                        ? R(0.5) / theta
                                        : copysign(R(1), theta) / (fabs(theta) + sqrt(R(1) + theta * theta));
                        c = R(1) / sqrt(R(1) + t * t);
                        s = t * c;
                        any_rot = 1;
                    }
                }
                rp[tid] = p;
                rq[tid] = (q < n && s != R(0)) ? q : -1;
                rc[tid] = c;
                rs[tid] = s;
            }
            __syncthreads();
            // rows p, q <- J^T rows
            for (int idx = tid; idx < npairs * n; idx += blockDim.x) {
                const int k = idx / n, j = idx - k * n;
                const int q = rq[k];
                if (q < 0) continue;
                const int p = rp[k];
                const R c = rc[k], s = rs[k];
                const R ap = A[p * ld + j], aq = A[q * ld + j];
                A[p * ld + j] = c * ap - s * aq;
                A[q * ld + j] = s * ap + c * aq;
            }
            __syncthreads();
            // columns p, q of A and of the vectors <- (.) J
            for (int idx = tid; idx < npairs * n; idx += blockDim.x) {
                const int k = idx / n, i = idx - k * n;
                const int q = rq[k];
                if (q < 0) continue;
                const int p = rp[k];
                const R c = rc[k], s = rs[k];
                const R ap = A[i * ld + p], aq = A[i * ld + q];
                A[i * ld + p] = c * ap - s * aq;
                A[i * ld + q] = s * ap + c * aq;
                const R up = U[i * ld + p], uq = U[i * ld + q];
                U[i * ld + p] = c * up - s * uq;
                U[i * ld + q] = s * up + c * uq;
            }
            __syncthreads();
        }
        if (!any_rot) break;
    }

    // off-diagonal size for the status
    double off = 0.0;
    for (int idx = tid; idx < n * n; idx += blockDim.x) {
        const int i = idx % n, j = idx / n;
        if (i != j) off += double(A[i * ld + j]) * double(A[i * ld + j]);
    }
    for (int o = 16; o > 0; o >>= 1) off += __shfl_xor_sync(0xffffffffu, off, o);
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = off;
    __syncthreads();
    // descending order: rank of each eigenvalue (ties by index)
    int* rank = rp;
    for (int i = tid; i < n; i += blockDim.x) {
        const R di = A[i * ld + i];
        int rk = 0;
        for (int j = 0; j < n; ++j) {
            const R dj = A[j * ld + j];
            rk += (dj > di || (dj == di && j < i)) ? 1 : 0;
        }
        rank[i] = rk;
    }
    __syncthreads();
    for (int i = tid; i < n; i += blockDim.x) w[rank[i]] = double(A[i * ld + i]);
    for (int idx = tid; idx < n * n; idx += blockDim.x) {
        const int i = idx % n, j = idx / n;
        V[i + int64_t(rank[j]) * n] = double(U[i * ld + j]);
    }
    if (tid == 0) {
        double o = 0.0;
        for (int i = 0; i < kJacThreads / 32; ++i) o += red[i];
        *status = o > double(eps) * fro2 ? 1 : 0;  // ||off||_F > sqrt(eps) ||H||_F
    }
}

template <class R>
cudaError_t launch_jacobi(const double* H, int n, int max_sweeps, double* w, double* V, int* status,
                          cudaStream_t s) {
    static std::once_flag once;
    static cudaError_t attr_error = cudaSuccess;
    std::call_once(once, [] {
        attr_error = cudaFuncSetAttribute(jacobi_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          int(jacobi_smem_bytes(kJacMaxN, sizeof(R))));
    });
    if (attr_error != cudaSuccess) return attr_error;
    jacobi_kernel<R><<<1, kJacThreads, jacobi_smem_bytes(n, sizeof(R)), s>>>(H, n, max_sweeps, w, V, status);
    return cudaGetLastError();
}

}  // namespace

int jacobi_max_n() { return kJacMaxN; }

int64_t jacobi_work_doubles(int n) {
    const int64_t nn = int64_t(n) * n;
    return 6 * nn + 2 * int64_t(n) + gemm_tn_scratch_doubles(n, n, n) + 64;
}

cudaError_t launch_sym_eig_jacobi(const double* H, int n, double* w, double* V, double* work, int* status,
                                  cudaStream_t s, bool fp32) {
    if (n <= 0 || n > kJacMaxN) return cudaErrorInvalidValue;
    KL_RANGE(H, int64_t(n) * n, double, "jacobi H");
    KL_RANGE(w, n, double, "jacobi w");
    KL_RANGE(V, int64_t(n) * n, double, "jacobi V");
    KL_RANGE(status, 1, int, "jacobi status");
    if (fp32) return launch_jacobi<float>(H, n, 30, w, V, status, s);
    KL_RANGE(work, jacobi_work_doubles(n), double, "jacobi work");
    const int64_t nn = int64_t(n) * n;
    double* Q0 = work;       // FP32 eigenvectors
    double* G = Q0 + nn;     // Q0^T Q0, then H Q
    double* Rinv = G + nn;   // L^-T of the Cholesky factor of Q0^T Q0
    double* Q = Rinv + nn;   // orthonormal in FP64
    double* B = Q + nn;      // Q^T H Q
    double* W = B + nn;      // eigenvectors of B
    double* w32 = W + nn;
    int* bad = reinterpret_cast<int*>(w32 + n);
    double* scratch = w32 + 2 * int64_t(n);
    const int64_t scratch_len = gemm_tn_scratch_doubles(n, n, n);
    cudaError_t e;
    if ((e = launch_jacobi<float>(H, n, 30, w32, Q0, status, s)) != cudaSuccess) return e;
    if ((e = launch_gemm_tn(Q0, n, Q0, n, G, n, n, n, n, 1.0, 0.0, scratch, scratch_len, s)) != cudaSuccess) return e;
    if ((e = launch_chol_rinv(G, n, Rinv, bad, s)) != cudaSuccess) return e;
    if ((e = launch_gemm_nn(Q0, n, Rinv, n, Q, n, n, n, n, 1.0, 0.0, s)) != cudaSuccess) return e;
    if ((e = launch_gemm_nn(H, n, Q, n, G, n, n, n, n, 1.0, 0.0, s)) != cudaSuccess) return e;
    if ((e = launch_gemm_tn(Q, n, G, n, B, n, n, n, n, 1.0, 0.0, scratch, scratch_len, s)) != cudaSuccess) return e;
    if ((e = launch_jacobi<double>(B, n, 10, w, W, status, s)) != cudaSuccess) return e;
    return launch_gemm_nn(Q, n, W, n, V, n, n, n, n, 1.0, 0.0, s);
}

}  // namespace kl
