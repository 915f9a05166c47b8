// Point tables (geometry map F and det DF) and the sum-factorisation mode
// products: the Kronecker-structured factors of Sec. 3.1, applied one
// direction at a time in (nearly) linear time, and the interpolation of the
// trial field at the quadrature points in Algorithm 1, plus small block
// utilities.
//
// Layout: a block of k vectors over a tensor grid (n1, n2, n3) is
// column-major, point index i1 + n1 * (i2 + n2 * i3), column stride ld.
#include <algorithm>
#include <cmath>

#include "kl_internal.h"

namespace kl {

namespace {

constexpr int kThreads = 256;

// Grid of a mode product: the k columns along y, the rows of a column along x
// (both grid-stride beyond their caps: 65535 columns, and the row blocks of
// grid_for's cap shared among the columns).
inline dim3 grid_cols(int64_t per_col, int k) {
    int64_t gx = (per_col + kThreads - 1) / kThreads;
    const int64_t cap = std::max<int64_t>(1, int64_t(device_sm_count()) * 64 / std::max(1, k));
    if (gx > cap) gx = cap;
    return dim3(unsigned(gx < 1 ? 1 : gx), unsigned(std::min(k, 65535)));
}

inline int grid_for(int64_t n, int per_block = kThreads) {
    int64_t g = (n + per_block - 1) / per_block;
    const int64_t cap = int64_t(device_sm_count()) * 64;
    if (g > cap) g = cap;  // grid-stride beyond this
    return int(g < 1 ? 1 : g);
}

// Quadratic NURBS quarter arc (control points (1,0), (1,1), (0,1), weights
// 1, sqrt(2)/2, 1): unit-circle point and d(theta)/du.
__device__ inline void arc_point(double u, double& cx, double& cy, double& dtheta) {
    const double w = 0.70710678118654752440;
    const double a = 1.0 - u;
    const double nx = a * a + 2.0 * w * u * a;
    const double ny = 2.0 * w * u * a + u * u;
    const double W = a * a + 2.0 * w * u * a + u * u;
    const double dnx = -2.0 * a + 2.0 * w * (1.0 - 2.0 * u);
    const double dny = 2.0 * w * (1.0 - 2.0 * u) + 2.0 * u;
    const double dW = -2.0 * a + 2.0 * w * (1.0 - 2.0 * u) + 2.0 * u;
    cx = nx / W;
    cy = ny / W;
    const double dcx = (dnx * W - nx * dW) / (W * W);
    const double dcy = (dny * W - ny * dW) / (W * W);
    dtheta = cx * dcy - cy * dcx;
}

// geo: annulus r_in, r_out, height; projective cube c_1, c_2, c_3.
__global__ void tensor_points_kernel(int geometry, double g0, double g1, double g2,
                                     const double* __restrict__ t1, const double* __restrict__ t2,
                                     const double* __restrict__ t3, int n1, int n2, int n3,
                                     const double* __restrict__ w1, const double* __restrict__ w2,
                                     const double* __restrict__ w3, double jac_power, double* out_x,
                                     double* out_y, double* out_z, double* out_w) {
    const int64_t n = int64_t(n1) * n2 * n3;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int i1 = int(i % n1);
        const int i2 = int((i / n1) % n2);
        const int i3 = int(i / (int64_t(n1) * n2));
        const double u1 = t1[i1], u2 = t2[i2], u3 = t3[i3];
        double x, y, z, det;
        if (geometry == KL_GEOM_QUARTER_ANNULUS || geometry == KL_GEOM_HALF_ANNULUS) {
            double cx, cy, dth;
            if (geometry == KL_GEOM_QUARTER_ANNULUS) {
                arc_point(u1, cx, cy, dth);
            } else {
                // two quarter arcs, the second turned by 90 degrees (C^0 at 1/2)
                const bool second = u1 >= 0.5;
                double ax, ay;
                arc_point(second ? 2.0 * u1 - 1.0 : 2.0 * u1, ax, ay, dth);
                cx = second ? -ay : ax;
                cy = second ? ax : ay;
                dth *= 2.0;
            }
            const double r_in = g0, r_out = g1, h = g2;
            const double r = r_in + (r_out - r_in) * u2;
            x = r * cx;
            y = r * cy;
            z = h * u3;
            det = r * dth * (r_out - r_in) * h;
        } else if (geometry == KL_GEOM_PROJECTIVE_CUBE) {
            // x = u / D, D = 1 + c . u: DF = (I - x c^T) / D, det DF = 1 / D^4
            const double D = 1.0 + g0 * u1 + g1 * u2 + g2 * u3;
            const double iD = 1.0 / D;
            x = u1 * iD;
            y = u2 * iD;
            z = u3 * iD;
            const double iD2 = iD * iD;
            det = iD2 * iD2;
        } else {
            x = u1;
            y = u2;
            z = u3;
            det = 1.0;
        }
        double w = 1.0;
        if (w1) w *= w1[i1] * w2[i2] * w3[i3];
        if (jac_power == 0.5) w *= sqrt(det);
        else if (jac_power == 1.0) w *= det;
        else if (jac_power == -0.5) w /= sqrt(det);  // Galerkin trial functions B / sqrt(det DF)
        if (out_x) out_x[i] = x;
        if (out_y) out_y[i] = y;
        if (out_z) out_z[i] = z;
        if (out_w) out_w[i] = w;
    }
}

// out[(ia, i, ib), c] = sum_l A[i + m l] pre[(ia, l, ib)] X[(ia, l, ib), c],
// optional pre (input rows) and post (output rows) scales. Column c is
// blockIdx.y; the row r = ia + a (i + m ib) of that column is decomposed with
// index type I (32-bit whenever a m b fits: a 64-bit division costs several
// times the 18 FMAs of a typical output).
template <class I>
__global__ void modeprod_kernel(const double* __restrict__ A, int m, int n,
                                const double* __restrict__ X, int64_t ldx, double* __restrict__ Y,
                                int64_t ldy, I a, I b, int k, const double* __restrict__ post,
                                const double* __restrict__ pre) {
    const I per_col = a * I(m) * b;
    for (int64_t c = blockIdx.y; c < k; c += gridDim.y) {
    for (I r = I(blockIdx.x) * blockDim.x + threadIdx.x; r < per_col; r += I(gridDim.x) * blockDim.x) {
        const I rest = r / a;
        const I ia = r - rest * a;
        const I ib = rest / I(m);
        const int i = int(rest - ib * I(m));
        const int64_t base = int64_t(ia) + int64_t(a) * n * int64_t(ib);
        const double* x = X + c * ldx + base;
        // four partial sums: the n-term FP64 FMA chain of one output would
        // otherwise wait on the FMA latency (~63 cycles on GB300) n times
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        int l = 0;
        const int64_t as = int64_t(a);
        if (pre) {
            const double* s = pre + base;
            for (; l + 4 <= n; l += 4) {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    acc[q] = fma(A[i + int64_t(m) * (l + q)], x[as * (l + q)] * s[as * (l + q)], acc[q]);
            }
            for (; l < n; ++l) acc[0] = fma(A[i + int64_t(m) * l], x[as * l] * s[as * l], acc[0]);
        } else {
            for (; l + 4 <= n; l += 4) {
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[q] = fma(A[i + int64_t(m) * (l + q)], x[as * (l + q)], acc[q]);
            }
            for (; l < n; ++l) acc[0] = fma(A[i + int64_t(m) * l], x[as * l], acc[0]);
        }
        double sum = (acc[0] + acc[1]) + (acc[2] + acc[3]);
        if (post) sum *= post[r];
        Y[c * ldy + int64_t(r)] = sum;
    }
    }
}

// Banded form: out[(ia, i, ib), c] = sum_j V[i w + j] pre[(ia, s_i + j, ib)]
// X[(ia, s_i + j, ib), c] with s_i = start[i]; the same thread mapping.
template <class I>
__global__ void modeprod_band_kernel(const double* __restrict__ V, const int* __restrict__ start, int w, int m,
                                     int n, const double* __restrict__ X, int64_t ldx, double* __restrict__ Y,
                                     int64_t ldy, I a, I b, int k, const double* __restrict__ post,
                                     const double* __restrict__ pre) {
    const I per_col = a * I(m) * b;
    for (int64_t c = blockIdx.y; c < k; c += gridDim.y) {
    for (I r = I(blockIdx.x) * blockDim.x + threadIdx.x; r < per_col; r += I(gridDim.x) * blockDim.x) {
        const I rest = r / a;
        const I ia = r - rest * a;
        const I ib = rest / I(m);
        const int i = int(rest - ib * I(m));
        const int64_t off = int64_t(ia) + int64_t(a) * (int64_t(start[i]) + int64_t(n) * int64_t(ib));
        const double* x = X + c * ldx + off;
        const double* v = V + int64_t(i) * w;
        const int64_t as = int64_t(a);
        double acc = 0.0;
        if (pre) {
            const double* s = pre + off;
            for (int j = 0; j < w; ++j) acc = fma(v[j], x[as * j] * s[as * j], acc);
        } else {
            for (int j = 0; j < w; ++j) acc = fma(v[j], x[as * j], acc);
        }
        if (post) acc *= post[r];
        Y[c * ldy + int64_t(r)] = acc;
    }
    }
}

__device__ inline unsigned long long splitmix64(unsigned long long x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// Standard normal numbers: SplitMix64 of (seed, counter) -> two uniforms ->
// Box-Muller (one output per counter).
__global__ void randn_kernel(double* X, int64_t ldx, int64_t K, int n, unsigned long long seed,
                             unsigned long long offset) {
    const int64_t total = K * n;
    for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
         t += int64_t(gridDim.x) * blockDim.x) {
        const int64_t c = t / K, i = t - c * K;
        const unsigned long long ctr = offset + (unsigned long long)t;
        const unsigned long long h1 = splitmix64(seed ^ splitmix64(2 * ctr));
        const unsigned long long h2 = splitmix64(seed ^ splitmix64(2 * ctr + 1));
        const double u1 = ((h1 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        const double u2 = ((h2 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        X[c * ldx + i] = sqrt(-2.0 * log(u1)) * cos(6.283185307179586477 * u2);
    }
}

__global__ void scale_cols_kernel(double* X, int64_t ldx, int64_t K, int n,
                                  const double* __restrict__ s, int invert) {
    const int64_t total = K * n;
    for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
         t += int64_t(gridDim.x) * blockDim.x) {
        const int64_t c = t / K, i = t - c * K;
        const double f = invert ? 1.0 / s[c] : s[c];
        X[c * ldx + i] *= f;
    }
}

// X(i, j) *= scale[i] (K x n block, column-major).
__global__ void scale_rows_kernel(double* X, int64_t ldx, int64_t K, int n, const double* __restrict__ scale) {
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < K * n; e += int64_t(gridDim.x) * blockDim.x) {
        const int64_t i = e % K, j = e / K;
        X[i + j * ldx] *= scale[i];
    }
}

// From W at the Gauss points (in place in w_inv): w_inv = 1 / W and
// scale_out = scale / W.
__global__ void rational_scales_kernel(double* w_inv, const double* __restrict__ scale,
                                       double* __restrict__ scale_out, int64_t n) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const double inv = 1.0 / w_inv[i];
        w_inv[i] = inv;
        scale_out[i] = scale[i] * inv;
    }
}

__global__ void copy_block_kernel(const double* __restrict__ X, int64_t ldx, double* Y,
                                  int64_t ldy, int64_t K, int n) {
    const int64_t total = K * n;
    for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
         t += int64_t(gridDim.x) * blockDim.x) {
        const int64_t c = t / K, i = t - c * K;
        Y[c * ldy + i] = X[c * ldx + i];
    }
}

template <int BS>
__device__ inline double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x < 32) {
        r = (threadIdx.x < BS / 32) ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    }
    return r;  // valid in thread 0
}

// One block per column: out[c] = sqrt(sum_i w_i X_ic^2) (w may be NULL).
__global__ void weighted_norms_kernel(const double* __restrict__ X, int64_t ldx, int64_t K,
                                      const double* __restrict__ w, double* out) {
    // four independent loads and partial sums per step: one dependent chain
    // of DRAM round trips per thread would be K / blockDim long
    __shared__ double sh[32];
    const int c = blockIdx.x;
    const double* x = X + c * ldx;
    const int64_t bd = blockDim.x;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int64_t i = threadIdx.x;
    for (; i + 3 * bd < K; i += 4 * bd) {
        const double v0 = x[i], v1 = x[i + bd], v2 = x[i + 2 * bd], v3 = x[i + 3 * bd];
        const double w0 = w ? w[i] : 1.0, w1 = w ? w[i + bd] : 1.0;
        const double w2 = w ? w[i + 2 * bd] : 1.0, w3 = w ? w[i + 3 * bd] : 1.0;
        s0 = fma(w0 * v0, v0, s0);
        s1 = fma(w1 * v1, v1, s1);
        s2 = fma(w2 * v2, v2, s2);
        s3 = fma(w3 * v3, v3, s3);
    }
    for (; i < K; i += bd) {
        const double v = x[i];
        s0 = fma((w ? w[i] : 1.0) * v, v, s0);
    }
    double s = (s0 + s1) + (s2 + s3);
    s = block_sum<kThreads>(s, sh);
    if (threadIdx.x == 0) out[c] = sqrt(s);
}

// One block per column: flip the sign so that the largest-magnitude entry is
// positive (first index wins ties).
__global__ void sign_fix_kernel(double* X, int64_t ldx, int64_t K) {
    __shared__ double sv[kThreads];
    __shared__ int64_t si[kThreads];
    const int c = blockIdx.x;
    double* x = X + c * ldx;
    double best = -1.0, val = 0.0;
    int64_t bi = 0;
    for (int64_t i = threadIdx.x; i < K; i += blockDim.x) {
        const double a = fabs(x[i]);
        if (a > best) best = a, bi = i, val = x[i];
    }
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __shared__ double sval[kThreads];
    sval[threadIdx.x] = val;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const int o = threadIdx.x + s;
            if (sv[o] > sv[threadIdx.x] || (sv[o] == sv[threadIdx.x] && si[o] < si[threadIdx.x])) {
                sv[threadIdx.x] = sv[o];
                si[threadIdx.x] = si[o];
                sval[threadIdx.x] = sval[o];
            }
        }
        __syncthreads();
    }
    const double sign = sval[0] < 0.0 ? -1.0 : 1.0;
    if (sign < 0.0)
        for (int64_t i = threadIdx.x; i < K; i += blockDim.x) x[i] = -x[i];
}

// One block per column: ||AY_c - theta_c Y_c||.
__global__ void resid_norms_kernel(const double* __restrict__ Y, int64_t ldy,
                                   const double* __restrict__ AY, int64_t lday,
                                   const double* __restrict__ theta, int64_t K, double* out) {
    // four independent loads and partial sums per step (see weighted_norms_kernel)
    __shared__ double sh[32];
    const int c = blockIdx.x;
    const double th = theta[c];
    const double* y = Y + c * ldy;
    const double* ay = AY + c * lday;
    const int64_t bd = blockDim.x;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int64_t i = threadIdx.x;
    for (; i + 3 * bd < K; i += 4 * bd) {
        const double r0 = ay[i] - th * y[i], r1 = ay[i + bd] - th * y[i + bd];
        const double r2 = ay[i + 2 * bd] - th * y[i + 2 * bd], r3 = ay[i + 3 * bd] - th * y[i + 3 * bd];
        s0 = fma(r0, r0, s0);
        s1 = fma(r1, r1, s1);
        s2 = fma(r2, r2, s2);
        s3 = fma(r3, r3, s3);
    }
    for (; i < K; i += bd) {
        const double r = ay[i] - th * y[i];
        s0 = fma(r, r, s0);
    }
    double s = (s0 + s1) + (s2 + s3);
    s = block_sum<kThreads>(s, sh);
    if (threadIdx.x == 0) out[c] = sqrt(s);
}

}  // namespace

cudaError_t launch_tensor_points(int geometry, const double* geo, const double* t1, const double* t2,
                                 const double* t3, int n1, int n2, int n3, const double* w1,
                                 const double* w2, const double* w3, double jac_power, double* out_x,
                                 double* out_y, double* out_z, double* out_w, cudaStream_t s) {
    const int64_t n = int64_t(n1) * n2 * n3;
    KL_RANGE(t1, n1, double, "tensor_points t1");
    KL_RANGE(t2, n2, double, "tensor_points t2");
    KL_RANGE(t3, n3, double, "tensor_points t3");
    if (w1) {
        KL_RANGE(w1, n1, double, "tensor_points w1");
        KL_RANGE(w2, n2, double, "tensor_points w2");
        KL_RANGE(w3, n3, double, "tensor_points w3");
    }
    KL_RANGE(out_x, n, double, "tensor_points x");
    KL_RANGE(out_y, n, double, "tensor_points y");
    KL_RANGE(out_z, n, double, "tensor_points z");
    KL_RANGE(out_w, n, double, "tensor_points w");
    tensor_points_kernel<<<grid_for(n), kThreads, 0, s>>>(geometry, geo[0], geo[1], geo[2], t1, t2,
                                                          t3, n1, n2, n3, w1, w2, w3, jac_power,
                                                          out_x, out_y, out_z, out_w);
    return cudaGetLastError();
}

cudaError_t launch_modeprod(const double* A, int m, int n, const double* X, int64_t ldx, double* Y,
                            int64_t ldy, int64_t a, int64_t b, int k, const double* post,
                            const double* pre, cudaStream_t s) {
    const int64_t total = a * m * b * k;
    if (total == 0) return cudaSuccess;
    KL_RANGE(A, int64_t(m) * n, double, "modeprod table");
    KL_RANGE(X, block_extent(a * n * b, k, ldx), double, "modeprod X");
    KL_RANGE(Y, block_extent(a * m * b, k, ldy), double, "modeprod Y");
    KL_RANGE(post, a * m * b, double, "modeprod post");
    KL_RANGE(pre, a * n * b, double, "modeprod pre");
    const int64_t per_col = a * m * b;
    if (per_col < (int64_t(1) << 31))
        modeprod_kernel<uint32_t><<<grid_cols(per_col, k), kThreads, 0, s>>>(A, m, n, X, ldx, Y, ldy, uint32_t(a),
                                                                             uint32_t(b), k, post, pre);
    else
        modeprod_kernel<uint64_t><<<grid_cols(per_col, k), kThreads, 0, s>>>(A, m, n, X, ldx, Y, ldy, uint64_t(a),
                                                                             uint64_t(b), k, post, pre);
    return cudaGetLastError();
}

cudaError_t launch_modeprod_band(const Band& A, int m, int n, const double* X, int64_t ldx, double* Y,
                                 int64_t ldy, int64_t a, int64_t b, int k, const double* post,
                                 const double* pre, cudaStream_t s) {
    const int64_t total = a * m * b * k;
    if (total == 0) return cudaSuccess;
    KL_RANGE(A.vals, int64_t(m) * A.w, double, "band table");
    KL_RANGE(A.start, m, int, "band starts");
    KL_RANGE(X, block_extent(a * n * b, k, ldx), double, "band modeprod X");
    KL_RANGE(Y, block_extent(a * m * b, k, ldy), double, "band modeprod Y");
    KL_RANGE(post, a * m * b, double, "band modeprod post");
    KL_RANGE(pre, a * n * b, double, "band modeprod pre");
    const int64_t per_col = a * m * b;
    if (per_col < (int64_t(1) << 31))
        modeprod_band_kernel<uint32_t><<<grid_cols(per_col, k), kThreads, 0, s>>>(
            A.vals, A.start, A.w, m, n, X, ldx, Y, ldy, uint32_t(a), uint32_t(b), k, post, pre);
    else
        modeprod_band_kernel<uint64_t><<<grid_cols(per_col, k), kThreads, 0, s>>>(
            A.vals, A.start, A.w, m, n, X, ldx, Y, ldy, uint64_t(a), uint64_t(b), k, post, pre);
    return cudaGetLastError();
}

cudaError_t launch_rational_scales(double* w_inv, const double* scale, double* scale_out, int64_t n,
                                   cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    KL_RANGE(w_inv, n, double, "rational w_inv");
    KL_RANGE(scale, n, double, "rational scale");
    KL_RANGE(scale_out, n, double, "rational scale_out");
    rational_scales_kernel<<<grid_for(n), kThreads, 0, s>>>(w_inv, scale, scale_out, n);
    return cudaGetLastError();
}

cudaError_t launch_randn(double* X, int64_t ldx, int64_t K, int n, unsigned long long seed,
                         unsigned long long offset, cudaStream_t s) {
    KL_RANGE(X, block_extent(K, n, ldx), double, "randn X");
    randn_kernel<<<grid_for(K * n), kThreads, 0, s>>>(X, ldx, K, n, seed, offset);
    return cudaGetLastError();
}

cudaError_t launch_scale_cols(double* X, int64_t ldx, int64_t K, int n, const double* scale,
                              int invert, cudaStream_t s) {
    KL_RANGE(X, block_extent(K, n, ldx), double, "scale_cols X");
    KL_RANGE(scale, n, double, "scale_cols scale");
    scale_cols_kernel<<<grid_for(K * n), kThreads, 0, s>>>(X, ldx, K, n, scale, invert);
    return cudaGetLastError();
}

cudaError_t launch_scale_rows(double* X, int64_t ldx, int64_t K, int n, const double* scale, cudaStream_t s) {
    if (K * n == 0) return cudaSuccess;
    KL_RANGE(X, block_extent(K, n, ldx), double, "scale_rows X");
    KL_RANGE(scale, K, double, "scale_rows scale");
    scale_rows_kernel<<<grid_for(K * n), kThreads, 0, s>>>(X, ldx, K, n, scale);
    return cudaGetLastError();
}

cudaError_t launch_copy_block(const double* X, int64_t ldx, double* Y, int64_t ldy, int64_t K,
                              int n, cudaStream_t s) {
    if (K * n == 0) return cudaSuccess;
    KL_RANGE(X, block_extent(K, n, ldx), double, "copy_block X");
    KL_RANGE(Y, block_extent(K, n, ldy), double, "copy_block Y");
    copy_block_kernel<<<grid_for(K * n), kThreads, 0, s>>>(X, ldx, Y, ldy, K, n);
    return cudaGetLastError();
}

cudaError_t launch_col_norms(const double* X, int64_t ldx, int64_t K, int n, double* out,
                             cudaStream_t s) {
    KL_RANGE(X, block_extent(K, n, ldx), double, "col_norms X");
    KL_RANGE(out, n, double, "col_norms out");
    weighted_norms_kernel<<<n, kThreads, 0, s>>>(X, ldx, K, nullptr, out);
    return cudaGetLastError();
}

cudaError_t launch_weighted_norms(const double* X, int64_t ldx, int64_t K, int n, const double* w,
                                  double* out, cudaStream_t s) {
    KL_RANGE(X, block_extent(K, n, ldx), double, "weighted_norms X");
    KL_RANGE(w, K, double, "weighted_norms w");
    KL_RANGE(out, n, double, "weighted_norms out");
    weighted_norms_kernel<<<n, kThreads, 0, s>>>(X, ldx, K, w, out);
    return cudaGetLastError();
}

cudaError_t launch_sign_fix(double* X, int64_t ldx, int64_t K, int n, cudaStream_t s) {
    KL_RANGE(X, block_extent(K, n, ldx), double, "sign_fix X");
    sign_fix_kernel<<<n, kThreads, 0, s>>>(X, ldx, K);
    return cudaGetLastError();
}

cudaError_t launch_resid_norms(const double* Y, int64_t ldy, const double* AY, int64_t lday,
                               const double* theta, int64_t K, int n, double* out,
                               cudaStream_t s) {
    KL_RANGE(Y, block_extent(K, n, ldy), double, "resid_norms Y");
    KL_RANGE(AY, block_extent(K, n, lday), double, "resid_norms AY");
    KL_RANGE(theta, n, double, "resid_norms theta");
    KL_RANGE(out, n, double, "resid_norms out");
    resid_norms_kernel<<<n, kThreads, 0, s>>>(Y, ldy, AY, lday, theta, K, out);
    return cudaGetLastError();
}

}  // namespace kl
