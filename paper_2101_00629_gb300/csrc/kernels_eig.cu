// Small dense FP64 eigenproblems of the Rayleigh-Ritz step (Sec. 3: the
// standard form A' v' = lambda v' is solved by an iterative projection
// method, whose projected matrix H = V^T A' V is decomposed here).
//
// One CTA of four warps per matrix: Householder reduction to Hessenberg form,
// then, for a general matrix, Francis double-shift QR to real Schur form with
// accumulated Schur vectors, ordering of the Schur form by decreasing real
// part, and eigenvectors of the leading columns by back substitution; for a
// symmetric matrix (whose Hessenberg form is tridiagonal) implicit QR steps
// with Wilkinson shifts on the tridiagonal form, the rotations accumulated
// into the eigenvectors.
//
// GB300 has a small FP64 unit: one warp-wide FP64 instruction issues every
// 64 cycles per SM sub-partition, and a dependent FP64 FMA waits 63 cycles
// (square root and division take about 650). The kernel is therefore laid
// out so that every operation that can run in parallel does (four warps on
// the four sub-partitions, reductions by shuffles, deflation and ordering
// decisions evaluated by all threads at once); the one-thread chains are the
// core of each bulge step with its next Householder vector (general case)
// and the scalar sweep of the tridiagonal QR (symmetric case), which the
// other warps' updates of the Schur vectors run beside.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <mutex>
#include <type_traits>

#include "kl_internal.h"

namespace kl {

// Double-float arithmetic for the small eigenproblems: a value is hi + lo, two
// FP32 numbers with |lo| at most about half an ulp of hi (about 46-48
// significant bits, the FP32 exponent range). Error-free transformations
// (Knuth's two-sum, the FMA two-product) on the FP32 pipe: on GB300 a
// dependent FP64 operation waits about 63 cycles and the FP64 unit issues one
// warp instruction per 64 cycles per sub-partition, while a double-float
// operation is a handful of 4-cycle FP32 steps on a pipe 64 times as wide.
// The bulge chase of a Francis step is one long chain of dependent operations,
// so the whole decomposition gets several times faster at ~1e-14 relative
// accuracy. Used for the Rayleigh-Ritz problems of the reduced-precision solves
// (whose residuals are resolved to ~1e-6); FP64 solves keep FP64. Operations
// use the _rn intrinsics so that the compiler neither contracts nor
// reassociates them.
namespace dfa {
struct dfl {
    float hi, lo;
    dfl() = default;
    __device__ dfl(float h, float l) : hi(h), lo(l) {}
    __device__ dfl(double x) {
        hi = __double2float_rn(x);
        lo = __double2float_rn(x - double(hi));
    }
    __device__ dfl(int x) : hi(float(x)), lo(0.f) {}
};
__device__ inline dfl fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return dfl(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ inline dfl operator+(dfl a, dfl b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    return fast_two_sum(s, e);
}
__device__ inline dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
__device__ inline dfl operator-(dfl a, dfl b) { return a + (-b); }
__device__ inline dfl operator*(dfl a, dfl b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}
__device__ inline dfl operator/(dfl a, dfl b) {
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const dfl r = a - b * dfl(q1, 0.f);
    return fast_two_sum(q1, __fdiv_rn(r.hi, b.hi));
}
// 1 / b: an FP32 reciprocal refined by one Newton step in double-float
// (r + r (1 - b r)), about 2^-46 relative
__device__ inline dfl recip(dfl b) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(b.hi));  // ~1 ulp; the Newton step squares the error
    const dfl e = dfl(1.f, 0.f) - b * dfl(r, 0.f);
    return fast_two_sum(r, __fmul_rn(r, e.hi));
}
// sqrt(a) for a > 0 from an approximate FP32 reciprocal square root y: s = a y,
// corrected by one Newton step s + (a - s^2) y / 2 in double-float
__device__ inline dfl sqrt_fast(dfl a) {
    if (!(a.hi > 0.f)) return dfl(0.f, 0.f);
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a.hi));
    const float s = __fmul_rn(a.hi, y);
    const float p = __fmul_rn(s, s);
    const dfl r = a - dfl(p, __fmaf_rn(s, s, -p));  // a - s^2, s^2 exactly
    return fast_two_sum(s, __fmul_rn(__fmul_rn(r.hi, y), 0.5f));
}
__device__ inline dfl& operator+=(dfl& a, dfl b) { return a = a + b; }
__device__ inline dfl& operator-=(dfl& a, dfl b) { return a = a - b; }
__device__ inline dfl& operator*=(dfl& a, dfl b) { return a = a * b; }
__device__ inline bool operator<(dfl a, dfl b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ inline bool operator>(dfl a, dfl b) { return b < a; }
__device__ inline bool operator<=(dfl a, dfl b) { return !(b < a); }
__device__ inline bool operator>=(dfl a, dfl b) { return !(a < b); }
__device__ inline bool operator==(dfl a, dfl b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ inline bool operator!=(dfl a, dfl b) { return !(a == b); }
__device__ inline dfl fabs(dfl a) { return a.hi < 0.f ? -a : a; }
__device__ inline dfl fmax(dfl a, dfl b) { return a < b ? b : a; }
__device__ inline dfl fmin(dfl a, dfl b) { return b < a ? b : a; }
__device__ inline dfl fma(dfl a, dfl b, dfl c) { return a * b + c; }
__device__ inline dfl sqrt(dfl a) {
    if (!(a.hi > 0.f)) return dfl(0.f, 0.f);
    const float s = __fsqrt_rn(a.hi);
    const float p = __fmul_rn(s, s);
    const dfl r = a - dfl(p, __fmaf_rn(s, s, -p));  // a - s^2, s^2 exactly
    return fast_two_sum(s, __fdiv_rn(r.hi, __fmul_rn(2.f, s)));
}
// sqrt(a^2 + b^2) with a and b first scaled by a power of two (exact), so
// that tiny entries neither underflow nor lose their low part
__device__ inline dfl hypot(dfl a, dfl b) {
    const float m = fmaxf(fabsf(a.hi), fabsf(b.hi));
    if (!(m > 0.f)) return dfl(0.f, 0.f);
    int e;
    frexpf(m, &e);
    const float sc = ldexpf(1.f, -e), inv = ldexpf(1.f, e);
    const dfl as(a.hi * sc, a.lo * sc), bs(b.hi * sc, b.lo * sc);
    const dfl r = sqrt(as * as + bs * bs);
    return dfl(r.hi * inv, r.lo * inv);
}
__device__ inline double to_d(dfl a) { return double(a.hi) + double(a.lo); }
}  // namespace dfa
using dfa::dfl;

namespace {

__device__ inline double to_d(double a) { return a; }
__device__ inline double to_d(float a) { return double(a); }
template <class R>
__device__ inline R shfl_xor(R v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
template <>
__device__ inline dfl shfl_xor<dfl>(dfl v, int o) {
    return dfl(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
}
template <class R>
__device__ inline R shfl_idx(R v, int src) { return __shfl_sync(0xffffffffu, v, src); }
template <>
__device__ inline dfl shfl_idx<dfl>(dfl v, int src) {
    return dfl(__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src));
}

constexpr int kEigThreads = 128;
constexpr size_t kEigSmemLimit = 220 * 1024;  // dynamic shared memory of the largest level
constexpr int kEigWarps = kEigThreads / 32;
constexpr unsigned kFull = 0xffffffffu;

// Arithmetic of the kernel: FP64 for the Rayleigh-Ritz problems of FP64
// solves, double-float for the final ones of reduced-precision solves, FP32
// for their restarts (shorter dependency chains). split:
// relative size (to ||H||) below which a stalled window's subdiagonal may be
// dropped and diagonal entries count as one eigenvalue cluster.
template <class R>
struct EigNum;
template <>
struct EigNum<double> {
    static constexpr double eps = DBL_EPSILON;
    static constexpr double tiny = DBL_MIN;
    static constexpr double split = 1e-10;
    static constexpr double abs_defl = 1.0;  // absolute deflation at n eps ||H||
    static constexpr double hess_min = 0.0;  // smallest column norm^2 the reduction reflects
};
template <>
struct EigNum<dfl> {
    // the deflation tolerance: about 10 units of the double-float's last place
    // (a tighter one only buys QR iterations spent at the rounding level:
    // 1e-14 took 107 iterations where FP64 took 90)
    static constexpr double eps = 1e-13;
    static constexpr double tiny = 1e-30;  // FP32 range, with room for the low part
    static constexpr double split = 1e-10;
    static constexpr double abs_defl = 1.0;
    // below this a column's entries (< 1e-15) are dropped, not reflected:
    // beta ~ 1 / |x|^2 would leave the FP32 exponent range
    static constexpr double hess_min = 1e-30;
};
template <>
struct EigNum<float> {
    static constexpr float eps = FLT_EPSILON;
    static constexpr float tiny = FLT_MIN;
    static constexpr float split = 1e-5f;
    static constexpr float abs_defl = 1.0f / 64;  // about eps ||H|| for the sizes used
    static constexpr float hess_min = 0.f;
};

// Givens rotation (c, s) with c x - s z = r and s x + c z = 0 (r = |(x, z)|;
// r = x when z = 0). FP32 and double-float: from one approximate reciprocal
// square root of x^2 + z^2 refined by a Newton step (c^2 + s^2 = 1 to the
// working precision), the pair first scaled by a power of two (exact) where
// the squares could leave FP32's exponent range; FP64: hypot and a division.
__device__ inline void givens_r(double x, double z, double& c, double& s, double& r) {
    if (z == 0.0) {
        c = 1.0;
        s = 0.0;
        r = x;
        return;
    }
    r = hypot(x, z);
    const double ir = 1.0 / r;
    c = x * ir;
    s = -(z * ir);
}
__device__ inline void givens_r(float x, float z, float& c, float& s, float& r) {
    if (z == 0.f) {
        c = 1.f;
        s = 0.f;
        r = x;
        return;
    }
    const float m = fmaxf(fabsf(x), fabsf(z));
    float sc = 1.f, isc = 1.f;
    if (m < 1e-18f || m > 1e18f) {
        // 2^-e with 2^(e-1) <= m < 2^e, from the exponent bits
        const int e = ((__float_as_int(m) >> 23) & 0xff) - 126;
        sc = __int_as_float((127 - e) << 23);
        isc = __int_as_float((127 + e) << 23);
    }
    const float xs = x * sc, zs = z * sc;
    const float q = fmaf(xs, xs, zs * zs);
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(q));
    y = y * fmaf(-0.5f * q * y, y, 1.5f);
    c = xs * y;
    s = -(zs * y);
    r = q * y * isc;
}
__device__ inline void givens_r(dfl x, dfl z, dfl& c, dfl& s, dfl& r) {
    if (z.hi == 0.f && z.lo == 0.f) {
        c = dfl(1.f, 0.f);
        s = dfl(0.f, 0.f);
        r = x;
        return;
    }
    const float m = fmaxf(fabsf(x.hi), fabsf(z.hi));
    // scale to [0.5, 1) by a power of two (exact): both parts keep their bits
    const int e = ((__float_as_int(m) >> 23) & 0xff) - 126;
    const float sc = __int_as_float((127 - e) << 23), isc = __int_as_float((127 + e) << 23);
    const dfl xs(x.hi * sc, x.lo * sc), zs(z.hi * sc, z.lo * sc);
    const dfl q = xs * xs + zs * zs;  // in [0.25, 2)
    float y0;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(q.hi));
    // y = y0 + y0 (1 - q y0^2) / 2, the residual in double-float
    const dfl t = q * (dfl(y0, 0.f) * dfl(y0, 0.f));
    const dfl e1 = dfl(1.f, 0.f) - t;
    const dfl y = dfl(y0, 0.f) + dfl(0.5f * y0, 0.f) * e1;
    c = xs * y;
    s = -(zs * y);
    const dfl rq = q * y;
    r = dfl(rq.hi * isc, rq.lo * isc);
}

// complex numbers over the working arithmetic R
template <class R>
struct cpx {
    R re, im;
};
template <class R>
__device__ inline cpx<R> cmul_r(cpx<R> a, cpx<R> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// a / b by Smith's algorithm (ratio of the smaller to the larger part of b)
template <class R>
__device__ inline cpx<R> cdiv_r(cpx<R> a, cpx<R> b) {
    if (fabs(b.re) >= fabs(b.im)) {
        const R r = b.im / b.re, d = R(1.0) / (b.re + b.im * r);
        return {(a.re + a.im * r) * d, (a.im - a.re * r) * d};
    }
    const R r = b.re / b.im, d = R(1.0) / (b.re * r + b.im);
    return {(a.re * r + a.im) * d, (a.im * r - a.re) * d};
}

template <class R>
__device__ inline R blk_sum(R v, R* red) {
    for (int o = 16; o > 0; o >>= 1) v += shfl_xor(v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    R s = R(0.0);
    for (int w = 0; w < kEigWarps; ++w) s += red[w];
    __syncthreads();
    return s;
}
template <class R>
__device__ inline R blk_max(R v, R* red) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, shfl_xor(v, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    R s = red[0];
    for (int w = 1; w < kEigWarps; ++w) s = fmax(s, red[w]);
    __syncthreads();
    return s;
}
__device__ inline int blk_max_int(int v, int* red) {
    v = __reduce_max_sync(kFull, v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    int s = red[0];
    for (int w = 1; w < kEigWarps; ++w) s = max(s, red[w]);
    __syncthreads();
    return s;
}

// Householder vector for x (len 2 or 3): (I - beta v v^T) x = -sign(x0)|x| e1.
// v^T v = 2 |x| (|x| + |x0|), so beta needs one division and no second sum.
template <class R>
__device__ inline void house(const R* x, int len, R* v, R& beta) {
    R ss = x[0] * x[0];
    for (int t = 1; t < len; ++t) ss = fma(x[t], x[t], ss);
    for (int t = 0; t < len; ++t) v[t] = x[t];
    if (ss == R(0.0)) {
        beta = R(0.0);
        return;
    }
    const R nrm = sqrt(ss);
    v[0] += (x[0] >= R(0.0) ? nrm : -nrm);
    beta = R(1.0) / (nrm * (nrm + fabs(x[0])));
}
// Double-float: FP32's exponent range cannot hold |x|^2 or beta ~ |x|^-2 for the
// tiny entries a converging bulge carries (|x| ~ 1e-20 gives beta ~ 1e40), so x
// is first scaled by a power of two (exact) to |x_i| < 1, and the vector is
// normalised to v0 = 1 with beta = 2 / (v^T v) of that vector (bounded, and
// orthogonal to rounding whatever the rounding of |x|).
template <>
__device__ inline void house<dfl>(const dfl* x, int len, dfl* v, dfl& beta) {
    float m = 0.f;
    for (int t = 0; t < len; ++t) m = fmaxf(m, fabsf(x[t].hi));
    for (int t = 0; t < len; ++t) v[t] = x[t];
    if (!(m > 0.f)) {
        beta = dfl(0.f, 0.f);
        return;
    }
    if (m < 1e-30f) {
        // entries this small (below 1e-30) are dropped with the bulge remnants
        beta = dfl(0.f, 0.f);
        return;
    }
    // scale by 2^-e with 2^(e-1) <= m < 2^e (exact): exponent bits of m
    const int e = ((__float_as_int(m) >> 23) & 0xff) - 126;
    const float sc = __int_as_float((127 - e) << 23);
    dfl xs[3];
    for (int t = 0; t < len; ++t) xs[t] = dfl(x[t].hi * sc, x[t].lo * sc);
    dfl ss = xs[0] * xs[0];
    for (int t = 1; t < len; ++t) ss = fma(xs[t], xs[t], ss);
    const dfl nrm = sqrt_fast(ss);  // ss in [0.25, 3)
    const dfl alpha = xs[0] + (xs[0].hi >= 0.f ? nrm : -nrm);
    // one reciprocal (|alpha| >= |x|, in [0.5, 2)), then products
    const dfl ra = recip(alpha);
    dfl vtv = dfl(1.f, 0.f);
    v[0] = dfl(1.f, 0.f);
    for (int t = 1; t < len; ++t) {
        v[t] = xs[t] * ra;
        vtv = fma(v[t], v[t], vtv);
    }
    const dfl rv = recip(vtv);  // v^T v in [1, 3)
    beta = dfl(2.f * rv.hi, 2.f * rv.lo);
}

// Deflation test for the subdiagonal entry (l, l-1).
template <class R>
__device__ inline bool deflatable(const R* A, int n, int ld, int l, R anorm) {
    R s = fabs(A[(l - 1) + int64_t(l - 1) * ld]) + fabs(A[l + int64_t(l) * ld]);
    if (s == R(0.0)) s = anorm;
    const R sub = fabs(A[l + int64_t(l - 1) * ld]);
    // absolute test at roundoff of the whole matrix: next to eigenvalues that
    // are themselves at roundoff level a relative test can never be met
    if (sub <= EigNum<R>::abs_defl * R(n) * EigNum<R>::eps * anorm) return true;
    // relative test, confirmed by the more conservative Ahues-Kressner
    // criterion (off-diagonal product against the gap of the diagonal pair)
    if (sub <= EigNum<R>::eps * s) {
        const R up = fabs(A[(l - 1) + int64_t(l) * ld]);
        const R ab = fmax(sub, up), ba = fmin(sub, up);
        const R dd = fabs(A[(l - 1) + int64_t(l - 1) * ld] - A[l + int64_t(l) * ld]);
        const R aa = fmax(fabs(A[l + int64_t(l) * ld]), dd);
        const R bb = fmin(fabs(A[l + int64_t(l) * ld]), dd);
        const R ss = aa + ab;
        return ba * (ab / ss) <= fmax(EigNum<R>::tiny, EigNum<R>::eps * (bb * (aa / ss)));
    }
    return false;
}

// Largest power of two g <= 32 with items * g <= kEigThreads (at least 1):
// g threads share one dot product and combine it by shuffles.
__device__ inline int group_size(int items) {
    int g = 1;
    while (g < 32 && items * (g * 2) <= kEigThreads) g *= 2;
    return g;
}

// Orthogonal Q (m x m, m = n1 + n2 <= 4, column-major) exchanging the adjacent
// diagonal blocks T11 (n1 x n1, at row/column k) and T22 (n2 x n2) of the
// quasi-triangular T: Q^T [T11 T12; 0 T22] Q = [T22' *; 0 T11'].
// 1x1 with 1x1: the Givens rotation whose first column is the eigenvector
// (t12, t22 - t11) of t22. Otherwise the direct swap: solve the Sylvester
// equation T11 X - X T22 = T12; the columns of [X; -I] span the
// T22-invariant subspace and Q is the orthogonal factor of their QR
// factorisation (Householder).
// The direct swap for blocks of fixed sizes N1, N2 (not both 1): every loop
// bound is a constant, so the small arrays stay in registers.
template <class R, int N1, int N2>
__device__ void swap_transform_nn(const R* A, int ld, int k, R anorm, R* Qm) {
    constexpr int n1 = N1, n2 = N2, m = N1 + N2;
    constexpr int pdim = n1 * n2;
    R K[pdim * pdim], x[pdim], W[m * n2];
#pragma unroll
    for (int r = 0; r < pdim * pdim; ++r) K[r] = R(0.0);
    // K = I_{n2} (x) T11 - T22^T (x) I_{n1}, x = vec(X) column-major
    #pragma unroll
    for (int j = 0; j < n2; ++j)
        #pragma unroll
        for (int i = 0; i < n1; ++i) {
            const int row = i + n1 * j;
            #pragma unroll
            for (int i2 = 0; i2 < n1; ++i2) K[row + pdim * (i2 + n1 * j)] += A[(k + i) + int64_t(k + i2) * ld];
            #pragma unroll
            for (int j2 = 0; j2 < n2; ++j2) K[row + pdim * (i + n1 * j2)] -= A[(k + n1 + j2) + int64_t(k + n1 + j) * ld];
            x[row] = A[(k + i) + int64_t(k + n1 + j) * ld];
        }
    // Gaussian elimination with partial pivoting; a pivot below eps ||T|| is
    // replaced by that bound (the blocks have close eigenvalues)
    R kn = R(0.0);
    #pragma unroll
    for (int r = 0; r < pdim * pdim; ++r) kn = fmax(kn, fabs(K[r]));
    const R tiny = EigNum<R>::eps * fmax(kn, anorm);
    #pragma unroll
    for (int c = 0; c < pdim; ++c) {
        int pr = c;
        #pragma unroll
        for (int r = c + 1; r < pdim; ++r)
            if (fabs(K[r + pdim * c]) > fabs(K[pr + pdim * c])) pr = r;
        // row exchange by constant indices (the arrays stay in registers)
#pragma unroll
        for (int r = c + 1; r < pdim; ++r)
            if (r == pr) {
#pragma unroll
                for (int cc = 0; cc < pdim; ++cc) {
                    const R t = K[c + pdim * cc];
                    K[c + pdim * cc] = K[r + pdim * cc];
                    K[r + pdim * cc] = t;
                }
                const R t = x[c];
                x[c] = x[r];
                x[r] = t;
            }
        if (fabs(K[c + pdim * c]) < tiny) K[c + pdim * c] = K[c + pdim * c] >= R(0.0) ? tiny : -tiny;
        #pragma unroll
        for (int r = c + 1; r < pdim; ++r) {
            const R f = K[r + pdim * c] / K[c + pdim * c];
            #pragma unroll
            for (int cc = c; cc < pdim; ++cc) K[r + pdim * cc] -= f * K[c + pdim * cc];
            x[r] -= f * x[c];
        }
    }
    #pragma unroll
    for (int r = pdim - 1; r >= 0; --r) {
        R t = x[r];
        #pragma unroll
        for (int cc = r + 1; cc < pdim; ++cc) t -= K[r + pdim * cc] * x[cc];
        x[r] = t / K[r + pdim * r];
    }
    // W = [X; -I] (m x n2), Householder QR with Q accumulated
    #pragma unroll
    for (int j = 0; j < n2; ++j)
        #pragma unroll
        for (int i = 0; i < m; ++i) W[i + m * j] = (i < n1) ? x[i + n1 * j] : (i - n1 == j ? -R(1.0) : R(0.0));
    #pragma unroll
    for (int r = 0; r < m * m; ++r) Qm[r] = (r % m == r / m) ? R(1.0) : R(0.0);
    #pragma unroll
    for (int j = 0; j < n2; ++j) {
        R v[4];
        const int len = m - j;
        R ss = R(0.0);
        #pragma unroll
        for (int t = 0; t < len; ++t) {
            v[t] = W[(j + t) + m * j];
            ss += v[t] * v[t];
        }
        if (ss == R(0.0)) continue;
        const R x0 = v[0], nrm = sqrt(ss);
        v[0] += (x0 >= R(0.0) ? nrm : -nrm);
        const R beta = R(1.0) / (nrm * (nrm + fabs(x0)));
        #pragma unroll
        for (int c = j; c < n2; ++c) {
            R sdot = R(0.0);
            #pragma unroll
            for (int t = 0; t < len; ++t) sdot += v[t] * W[(j + t) + m * c];
            #pragma unroll
            for (int t = 0; t < len; ++t) W[(j + t) + m * c] -= beta * sdot * v[t];
        }
        #pragma unroll
        for (int r = 0; r < m; ++r) {
            R sdot = R(0.0);
            #pragma unroll
            for (int t = 0; t < len; ++t) sdot += Qm[r + m * (j + t)] * v[t];
            #pragma unroll
            for (int t = 0; t < len; ++t) Qm[r + m * (j + t)] -= beta * sdot * v[t];
        }
    }
}

template <class R>
__device__ void swap_transform(const R* A, int ld, int k, int n1, int n2, R anorm, R* Qm) {
    if (n1 == 1 && n2 == 1) {
        const R a = A[k + int64_t(k) * ld], d = A[(k + 1) + int64_t(k + 1) * ld];
        const R b = A[k + int64_t(k + 1) * ld];
        const R r = hypot(b, d - a);
        const R c = r > R(0.0) ? b / r : R(1.0), sn = r > R(0.0) ? (d - a) / r : R(0.0);
        Qm[0] = c;
        Qm[1] = sn;
        Qm[2] = -sn;
        Qm[3] = c;
        return;
    }
    if (n1 == 1) swap_transform_nn<R, 1, 2>(A, ld, k, anorm, Qm);
    else if (n2 == 1) swap_transform_nn<R, 2, 1>(A, ld, k, anorm, Qm);
    else swap_transform_nn<R, 2, 2>(A, ld, k, anorm, Qm);
}

// Orders the diagonal blocks (1x1 real eigenvalues, 2x2 complex pairs) of the
// quasi-triangular A so that the blocks holding the nwant eigenvalues of
// largest real part come first, by decreasing real part, updating the Schur
// vectors Z: odd-even transposition over the blocks, exchanging blocks 2p + par
// and 2p + par + 1 where the second is wanted (real part at least the
// smallest wanted one, less the cluster tolerance) and has the larger real part (the
// other blocks keep their relative order: nothing downstream reads it). The
// exchanges of a round act on disjoint row/column ranges and commute, so a
// round is applied as one two-sided update (all rows, then all columns and Z)
// over the exchanged pairs only. Each exchange is computed by its own thread.
// ints: 2n ints of scratch (block starts; per exchanged pair its block start
// and its size/pair index word); ord: 8n values (a 4 x 4 transform per pair;
// before the first round the block keys).
template <class R>
__device__ void order_schur(R* A, R* Z, int n, int ld, int nwant, R anorm, R* ints_d, R* ord, int* oob) {
    constexpr int NT = kEigThreads;
    __shared__ int s_wsum[kEigWarps];
    __shared__ int s_nb;
    __shared__ R s_tau;
    int* bstart = reinterpret_cast<int*>(ints_d);  // n
    int* pk = bstart + n;                           // n / 2 (pairs <= blocks / 2)
    int* pinfo = pk + n / 2;                        // n / 2
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ipt = (n + NT - 1) / NT;
    // exclusive block-wide prefix sum of a per-thread count; total in *tot
    auto scan = [&](int cnt, int* tot) {
        int incl = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_wsum[warp] = incl;
        __syncthreads();
        int pos = incl - cnt, t = 0;
        for (int w = 0; w < kEigWarps; ++w) {
            if (w < warp) pos += s_wsum[w];
            t += s_wsum[w];
        }
        __syncthreads();
        *tot = t;
        return pos;
    };
    // block starts: i = 0 or a zero subdiagonal entry (i, i-1)
    auto find_blocks = [&]() -> int {
        int cnt = 0;
        for (int i = tid * ipt; i < min(n, (tid + 1) * ipt); ++i)
            cnt += (i == 0 || A[i + int64_t(i - 1) * ld] == R(0.0));
        int nb;
        int pos = scan(cnt, &nb);
        for (int i = tid * ipt; i < min(n, (tid + 1) * ipt); ++i)
            if (i == 0 || A[i + int64_t(i - 1) * ld] == R(0.0)) bstart[pos++] = i;
        __syncthreads();
        return nb;
    };
    auto key_of = [&](int k, int sz) {
        return sz == 1 ? A[k + int64_t(k) * ld] : R(0.5) * (A[k + int64_t(k) * ld] + A[(k + 1) + int64_t(k + 1) * ld]);
    };
    // the wanted blocks: those with fewer than nwant eigenvalues in blocks of
    // larger key (ties: lower position first); tau = the smallest wanted key
    {
        const int nb = find_blocks();
        for (int b = tid; b < nb; b += NT) {
            const int k = bstart[b], k2 = b + 1 < nb ? bstart[b + 1] : n;
            ord[b] = key_of(k, k2 - k);
        }
        __syncthreads();
        R tmin = R(0.0);
        bool have = false;
        for (int b = tid; b < nb; b += NT) {
            const R kb = ord[b];
            int above = 0;
            for (int j = 0; j < nb; ++j) {
                const R kj = ord[j];
                if (kj > kb || (kj == kb && j < b)) above += (j + 1 < nb ? bstart[j + 1] : n) - bstart[j];
            }
            if (above < nwant && (!have || kb < tmin)) {
                tmin = kb;
                have = true;
            }
        }
        // block minimum over the threads that have a wanted block
        if (tid == 0) s_nb = 0;
        __syncthreads();
        for (int w = 0; w < NT; w += 32) {
            // one warp at a time keeps this simple: it runs once per call
            if (warp == w / 32) {
                for (int l2 = 0; l2 < 32; ++l2) {
                    if (lane == l2 && have) {
                        if (s_nb == 0 || tmin < s_tau) s_tau = tmin;
                        s_nb = 1;
                    }
                    __syncwarp();
                }
            }
            __syncthreads();
        }
    }
    // a 2x2 block's key (half its trace) moves by rounding as it is exchanged:
    // blocks within the cluster tolerance of the threshold count as wanted, so
    // that the last wanted block never drops out of the set on the way
    const R tau = s_tau - R(EigNum<R>::split) * anorm;
    int quiet = 0;
    for (int round = 0; round < 2 * n + 4 && quiet < 2; ++round) {
        const int nb = find_blocks();
        const int par = round & 1;
        const int npairs = max(0, (nb - par) / 2);
        // each thread decides a contiguous range of at most 4 pairs and
        // computes the exchanges among them
        const int ppt = (npairs + NT - 1) / NT;
        const int pa = min(npairs, tid * ppt), pb = min(npairs, pa + ppt);
        int mykey[4], myk[4];
        int cnt = 0;
        for (int p = pa; p < pb; ++p) {
            const int b0 = par + 2 * p;
            const int k = bstart[b0], k2 = bstart[b0 + 1];
            const int k3 = (b0 + 2 < nb) ? bstart[b0 + 2] : n;
            const int n1 = k2 - k, n2 = k3 - k2;
            const R key1 = key_of(k, n1), key2 = key_of(k2, n2);
            int f = key2 > key1 && key2 >= tau;
#ifdef KL_CHECK_BOUNDS
            // pair and block indices stay inside the scratch (n / 2 pairs), the
            // blocks are 1x1 or 2x2 and a thread has at most 4 pairs;
            // otherwise record it, skip the exchange
            if (b0 + 1 >= nb || p >= n / 2 || n1 < 1 || n1 > 2 || n2 < 1 || n2 > 2 || k3 > n || ppt > 4) {
                atomicExch(oob, 1);
                f = 0;
            }
#endif
            if (f) {
                swap_transform(A, ld, k, n1, n2, anorm, ord + 16 * int64_t(p));
                if (n1 == 1 && n2 == 1) {
                    // exact exchange of the diagonal pair
                    ord[16 * int64_t(p) + 4] = A[k + int64_t(k) * ld];
                    ord[16 * int64_t(p) + 5] = A[k2 + int64_t(k2) * ld];
                }
                mykey[cnt] = (p << 8) | 1 | (n1 << 1) | (n2 << 3);
                myk[cnt] = k;
                ++cnt;
            }
        }
        int nswap;
        int pos = scan(cnt, &nswap);
        for (int c = 0; c < cnt; ++c) {
            pk[pos + c] = myk[c];
            pinfo[pos + c] = mykey[c];
        }
        __syncthreads();
        if (nswap == 0) {
            ++quiet;
            continue;
        }
        quiet = 0;
        // x (m values, stride st) <- Q^T x (rows) or x Q (columns); m fixed
        // at compile time so that the values stay in registers
        auto rot = [&](auto mtag, R* x0, int64_t st, const R* Qm, bool transpose) {
            constexpr int MM = decltype(mtag)::value;
            R old[MM];
#pragma unroll
            for (int t = 0; t < MM; ++t) old[t] = x0[t * st];
#pragma unroll
            for (int t = 0; t < MM; ++t) {
                R acc = R(0.0);
#pragma unroll
                for (int u2 = 0; u2 < MM; ++u2) acc = fma(Qm[u2 + MM * t], old[u2], acc);
                x0[t * st] = acc;
            }
            (void)transpose;
        };
        auto rot_m = [&](int m, R* x0, int64_t st, const R* Qm) {
            if (m == 2) rot(std::integral_constant<int, 2>{}, x0, st, Qm, false);
            else if (m == 3) rot(std::integral_constant<int, 3>{}, x0, st, Qm, false);
            else rot(std::integral_constant<int, 4>{}, x0, st, Qm, false);
        };
        // rows of each exchanged span <- Q^T rows (columns k..n-1)
        for (int e = tid; e < nswap * n; e += NT) {
            const int q = int(unsigned(e) / unsigned(n)), j = e - q * n;
            const int info = pinfo[q];
            const int k = pk[q], m = ((info >> 1) & 3) + ((info >> 3) & 3);
            if (j < k) continue;
            rot_m(m, A + k + int64_t(j) * ld, 1, ord + 16 * int64_t(info >> 8));
        }
        __syncthreads();
        // columns of each exchanged span <- columns Q (rows of A above the
        // span's end, all rows of Z)
        for (int e = tid; e < nswap * 2 * n; e += NT) {
            const int q = int(unsigned(e) / unsigned(2 * n)), i2 = e - q * 2 * n;
            const int info = pinfo[q];
            const int k = pk[q], m = ((info >> 1) & 3) + ((info >> 3) & 3);
            R* M = i2 < n ? A : Z;
            const int r = i2 < n ? i2 : i2 - n;
            if (i2 < n && r >= k + m) continue;
            // (x Q)_t = sum_u x_u Q(u, t): the same sums as Q^T x
            rot_m(m, M + r + int64_t(k) * ld, ld, ord + 16 * int64_t(info >> 8));
        }
        __syncthreads();
        // the exchanged blocks: zero the new (2,1) block; 1x1 pairs take
        // their exchanged diagonal exactly
        for (int q = tid; q < nswap; q += NT) {
            const int info = pinfo[q];
            const int k = pk[q], n1 = (info >> 1) & 3, n2 = (info >> 3) & 3, m = n1 + n2;
            const int p = info >> 8;
            for (int i = k + n2; i < k + m; ++i)
                for (int j = k; j < k + n2; ++j) A[i + int64_t(j) * ld] = R(0.0);
            if (n1 == 1 && n2 == 1) {
                A[k + int64_t(k) * ld] = ord[16 * int64_t(p) + 5];
                A[(k + 1) + int64_t(k + 1) * ld] = ord[16 * int64_t(p) + 4];
            }
        }
        __syncthreads();
    }
}

// smem_level: 2 = A, Z, X, the Householder vector and the ordering scratch in
// shared memory, 1 = A and the Householder vector, 0 = everything in the
// global work array.
// nvec: eigenvectors wanted for the leading nvec ordered eigenvalues
// (non-symmetric mode); the symmetric mode returns all ordered Schur vectors.
template <class R>
__global__ void __launch_bounds__(kEigThreads) nonsym_eig_kernel(const double* __restrict__ H, int n,
                                                                 double* wr_out, double* wi_out,
                                                                 double* Vout, double* Qout, double* work_d,
                                                                 int* status, int smem_level, int sym,
                                                                 int nvec) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* smem_a = reinterpret_cast<R*>(smem_raw);
    R* work = reinterpret_cast<R*>(work_d);
    const int64_t nn = int64_t(n) * n;
    // A, Z and X are stored with leading dimension n + 1: a row of a matrix
    // (consecutive columns, one per thread) then spreads over the shared-
    // memory banks instead of hitting one bank n apart
    const int ld = n + 1;
    const int64_t nl = int64_t(ld) * n;
    R* A = smem_level >= 1 ? smem_a : work;
    R* Z = smem_level == 2 ? smem_a + nl : work + nl;
    R* X = smem_level == 2 ? smem_a + 2 * nl : work + 2 * nl;
    // Householder vector / integer scratch (2n), ordering scratch (8n)
    R* hv = smem_level == 2 ? smem_a + 3 * nl : (smem_level == 1 ? smem_a + nl : work + 3 * nl + 2 * n);
    R* wr = work + 3 * nl;
    R* wi = wr + n;
    R* ord = smem_level == 2 ? smem_a + 3 * nl + 2 * n : work + 3 * nl + 4 * n;
    __shared__ R s_red[kEigWarps];
    __shared__ int s_redi[kEigWarps];
    __shared__ R s_x[3], s_vb[2][3], s_bb[2];
    __shared__ R s_beta, s_sh, s_th;
    __shared__ int s_l, s_u, s_its, s_fail, s_action, s_oob;
    const int tid = threadIdx.x;
    constexpr int NT = kEigThreads;

    R amax = R(0.0);
    for (int e = tid; e < int(nn); e += NT) {
        const int j = int(unsigned(e) / unsigned(n)), i = e - j * n;
        const R a = sym ? R(0.5) * (H[e] + H[j + int64_t(i) * n]) : H[e];
        A[i + int64_t(j) * ld] = a;
        Z[i + int64_t(j) * ld] = (i == j) ? R(1.0) : R(0.0);
        amax = fmax(amax, fabs(a));
    }
    const R anorm = blk_max(amax, s_red);  // also orders the stores above

    // ---- Householder reduction to Hessenberg form ----
    for (int k = 0; k + 2 < n; ++k) {
        const int len = n - k - 1;
        R ss = R(0.0);
        for (int t = tid; t < len; t += NT) {
            const R x = A[(k + 1 + t) + int64_t(k) * ld];
            hv[t] = x;
            ss = fma(x, x, ss);
        }
        ss = blk_sum(ss, s_red);
        if (tid == 0) {
            R beta = R(0.0);
            if (ss > R(EigNum<R>::hess_min)) {
                const R x0 = hv[0], nrm = sqrt(ss);
                hv[0] = x0 + (x0 >= R(0.0) ? nrm : -nrm);
                beta = R(1.0) / (nrm * (nrm + fabs(x0)));
            }
            s_beta = beta;
        }
        __syncthreads();
        const R beta = s_beta;
        if (beta != R(0.0)) {
            // left: rows k+1..n-1 of columns k..n-1
            const int ncols = n - k;
            const int g = group_size(ncols), per = NT / g;
            for (int base = 0; base < ncols; base += per) {
                const int c = base + tid / g, p = tid % g;
                R s = R(0.0);
                if (c < ncols) {
                    // four partial sums: the dependent chain is a quarter as long
                    R s4[4] = {R(0.0), R(0.0), R(0.0), R(0.0)};
                    const R* col = A + (k + 1) + int64_t(k + c) * ld;
                    int t = p;
                    for (; t + 3 * g < len; t += 4 * g)
                        for (int q = 0; q < 4; ++q) s4[q] = fma(hv[t + q * g], col[t + q * g], s4[q]);
                    for (; t < len; t += g) s4[0] = fma(hv[t], col[t], s4[0]);
                    s = (s4[0] + s4[1]) + (s4[2] + s4[3]);
                }
                for (int o = g / 2; o > 0; o >>= 1) s += shfl_xor(s, o);
                s *= beta;
                if (c < ncols) {
                    // four elements per step: loads of a step issue together
                    // (hv and A are both shared memory, so a store orders
                    // every later load)
                    R* col = A + (k + 1) + int64_t(k + c) * ld;
                    int t = p;
                    for (; t + 3 * g < len; t += 4 * g) {
                        R a4[4], h4[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            a4[q] = col[t + q * g];
                            h4[q] = hv[t + q * g];
                        }
#pragma unroll
                        for (int q = 0; q < 4; ++q) col[t + q * g] = a4[q] - s * h4[q];
                    }
                    for (; t < len; t += g) col[t] -= s * hv[t];
                }
            }
            __syncthreads();
            // right: all rows of A and of Z, columns k+1..n-1
            const int items = 2 * n;
            const int g2 = group_size(items), per2 = NT / g2;
            for (int base = 0; base < items; base += per2) {
                const int it = base + tid / g2, p = tid % g2;
                R* M = it < n ? A : Z;
                const int i = it < n ? it : it - n;
                R s = R(0.0);
                if (it < items) {
                    R s4[4] = {R(0.0), R(0.0), R(0.0), R(0.0)};
                    const R* row = M + i + int64_t(k + 1) * ld;
                    int t = p;
                    for (; t + 3 * g2 < len; t += 4 * g2)
                        for (int q = 0; q < 4; ++q) s4[q] = fma(row[int64_t(t + q * g2) * ld], hv[t + q * g2], s4[q]);
                    for (; t < len; t += g2) s4[0] = fma(row[int64_t(t) * ld], hv[t], s4[0]);
                    s = (s4[0] + s4[1]) + (s4[2] + s4[3]);
                }
                for (int o = g2 / 2; o > 0; o >>= 1) s += shfl_xor(s, o);
                s *= beta;
                if (it < items) {
                    R* row = M + i + int64_t(k + 1) * ld;
                    int t = p;
                    for (; t + 3 * g2 < len; t += 4 * g2) {
                        R a4[4], h4[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            a4[q] = row[int64_t(t + q * g2) * ld];
                            h4[q] = hv[t + q * g2];
                        }
#pragma unroll
                        for (int q = 0; q < 4; ++q) row[int64_t(t + q * g2) * ld] = a4[q] - s * h4[q];
                    }
                    for (; t < len; t += g2) row[int64_t(t) * ld] -= s * hv[t];
                }
            }
        }
        __syncthreads();
        for (int i = k + 2 + tid; i < n; i += NT) A[i + int64_t(k) * ld] = R(0.0);
        __syncthreads();
    }

    // ---- Francis R-shift QR to real Schur form ----
    if (tid == 0) {
        s_u = n - 1;
        s_its = 0;
        s_fail = 0;
        s_oob = 0;
    }
    __syncthreads();
    int total_its = 0;
    if (sym) {
        // ---- symmetric: implicit QR steps with Wilkinson shifts on the
        // tridiagonal form (the Hessenberg form of a symmetric matrix):
        // diagonal d, subdiagonal e. A sweep's rotations follow from (d, e)
        // alone, so one thread (warp 3, lane 0) runs the sweeps and writes
        // each one's rotations to one of two buffers, while warps 0..2 apply
        // the previous sweep's rotations to their rows of Z: one block
        // barrier per sweep, no barrier per rotation. ----
        R* dv = X;
        R* ev = X + n;
        R* rot = ord;  // two buffers of (c, s) for up to n - 1 rotations
        __shared__ int s_wl[2], s_wu[2], s_next[2];
        for (int i = tid; i < n; i += NT) {
            dv[i] = A[i + int64_t(i) * ld];
            ev[i] = i + 1 < n ? R(0.5) * (A[(i + 1) + int64_t(i) * ld] + A[i + int64_t(i + 1) * ld]) : R(0.0);
        }
        __syncthreads();
        constexpr int kScalar = NT - 32;
        int l = 0, u = n - 1, sweeps = 0;
        bool failed = false;
        const R eps = R(EigNum<R>::eps);
        // e_i against its two diagonal neighbours (||H|| where both vanish)
        auto negligible = [&](int i) {
            const R sc = fabs(dv[i]) + fabs(dv[i + 1]);
            return fabs(ev[i]) <= eps * (sc > R(0.0) ? sc : anorm);
        };
        // one sweep on the bottom unreduced block [l, u] into buffer b;
        // false when every block has converged (or the sweep limit is hit)
        auto sweep = [&](int b) -> bool {
            while (true) {
                while (u > l && negligible(u - 1)) {
                    ev[u - 1] = R(0.0);
                    --u;
                }
                if (u > l) break;
                // the block is down to one entry: the next block above
                u = l - 1;
                while (u > 0 && negligible(u - 1)) {
                    ev[u - 1] = R(0.0);
                    --u;
                }
                if (u <= 0) return false;
                l = u - 1;
                while (l > 0 && !negligible(l - 1)) --l;
                if (l > 0) ev[l - 1] = R(0.0);
            }
            if (++sweeps > 30 * n) {
                failed = true;
                return false;
            }
            // Wilkinson shift: the eigenvalue of the trailing 2x2 block nearer d_u
            const R du = dv[u], eu = ev[u - 1];
            const R del = R(0.5) * (dv[u - 1] - du);
            const R hyp = hypot(del, eu);
            const R den = del + (del >= R(0.0) ? hyp : -hyp);
            const R mu = den != R(0.0) ? du - eu * (eu / den) : du;
            // chase: rotation k acts on rows and columns k, k+1; (x, z) is the
            // shifted first column (k = l), then the entry (k, k-1) and the
            // bulge (k+1, k-1)
            // register-carried chain: a, bk the current d_k, e_k; d2, en the
            // untouched d_{k+1}, e_{k+1} (loaded one step ahead); each d_k and
            // e_{k-1} is final once written
            R* cs = rot + b * 2 * n;
            R a = dv[l], bk = ev[l], d2 = dv[l + 1];
            R en = l + 1 < u ? ev[l + 1] : R(0.0);
            R x = a - mu, z = bk, dprev = R(0.0);
            int lz = l;
            for (int k = l; k < u; ++k) {
                const R d2n = k + 2 <= u ? dv[k + 2] : R(0.0);
                const R enn = k + 2 < u ? ev[k + 2] : R(0.0);
                R c, sn, r;
                givens_r(x, z, c, sn, r);
                if (k > l) {
                    ev[k - 1] = r;
                    const R sc = fabs(dprev) + fabs(a);
                    if (fabs(r) <= eps * (sc > R(0.0) ? sc : anorm)) lz = k;
                }
                const R cc = c * c, ss = sn * sn, csn = c * sn;
                const R t2 = R(2.0) * bk * csn;
                const R dk = a * cc - t2 + d2 * ss;
                dv[k] = dk;
                dprev = dk;
                const R dk1 = a * ss + t2 + d2 * cc;
                x = (a - d2) * csn + bk * (cc - ss);
                if (k + 1 < u) {
                    z = -(sn * en);
                    bk = c * en;
                }
                cs[2 * k] = c;
                cs[2 * k + 1] = sn;
                a = dk1;
                d2 = d2n;
                en = enn;
            }
            dv[u] = a;
            ev[u - 1] = x;
            s_wl[b] = l;
            s_wu[b] = u;
            if (lz > l) {
                // a negligible entry inside the block: continue below it
                ev[lz - 1] = R(0.0);
                l = lz;
            }
            return true;
        };
        if (tid == kScalar) s_next[0] = sweep(0) ? 1 : 0;
        __syncthreads();
        for (int j = 0; s_next[j & 1]; ++j) {
            const int b = j & 1;
            if (tid == kScalar) {
                s_next[b ^ 1] = sweep(b ^ 1) ? 1 : 0;
            } else if (tid < kScalar) {
                // Z <- Z G_l ... G_{u-1}, one row per thread, the column
                // entry carried from one rotation to the next in a register
                const int wl = s_wl[b], wu = s_wu[b];
                const R* cs = rot + b * 2 * n;
                for (int i = tid; i < n; i += kScalar) {
                    R* zr = Z + i;
                    R a0 = zr[int64_t(wl) * ld];
                    for (int k = wl; k < wu; ++k) {
                        const R b0 = zr[int64_t(k + 1) * ld];
                        const R c = cs[2 * k], sn = cs[2 * k + 1];
                        zr[int64_t(k) * ld] = c * a0 - sn * b0;
                        a0 = sn * a0 + c * b0;
                    }
                    zr[int64_t(wu) * ld] = a0;
                }
            }
            __syncthreads();
        }
        if (tid == kScalar) {
            s_fail = failed ? 1 : 0;
            s_its = sweeps;
            s_u = u;
        }
        for (int i = tid; i < n; i += NT) A[i + int64_t(i) * ld] = dv[i];
        __syncthreads();
        total_its = s_its;
    }
    while (!sym) {
        const int u0 = s_u;
        if (u0 < 0) break;
        // largest l <= u with a negligible subdiagonal (l, l-1); 0 if none
        int cand = 0;
        for (int l = u0 - tid; l >= 1; l -= NT)
            if (deflatable(A, n, ld, l, anorm)) {
                cand = l;
                break;
            }
        cand = blk_max_int(cand, s_redi);
        if (tid == 0) {
            const int u = u0;
            int l = cand;
            if (l >= 1) A[l + int64_t(l - 1) * ld] = R(0.0);
            int action = (l == u) ? 1 : (l == u - 1) ? 2 : 3;  // 1: one root, 2: 2x2 block, 3: Francis step
            if (action == 3 && s_its >= 30 && s_its % 10 == 5) {
                // A window that resists the shifts for 30 iterations is a
                // cluster of (numerically) equal eigenvalues perturbed into a
                // near-Jordan block. The window is already decoupled from its
                // neighbours, so zeroing its smallest subdiagonal leaves every
                // other eigenvalue and the window's invariant subspace as
                // they are; it only splits the cluster (by about
                // sqrt(|sub * super|)). Only a subdiagonal far below any
                // tolerance of the outer solver is dropped (backward error
                // 1e-10 * ||H||).
                int m = l + 1;
                for (int i = l + 2; i <= u; ++i)
                    if (fabs(A[i + int64_t(i - 1) * ld]) < fabs(A[m + int64_t(m - 1) * ld])) m = i;
                if (fabs(A[m + int64_t(m - 1) * ld]) <= EigNum<R>::split * anorm) {
                    A[m + int64_t(m - 1) * ld] = R(0.0);
                    action = 5;  // split: look for deflations again
                    s_its = s_its + 1;
                }
            }
            if (action == 3) {
                if (s_its >= 300 || total_its > 120 * max(10, n)) {
                    s_fail = 1;
                    action = 4;
                } else {
                    R sh, th;
                    if (s_its > 0 && s_its % 10 == 0) {  // exceptional shift
                        const R ex = fabs(A[u + int64_t(u - 1) * ld]) + fabs(A[(u - 1) + int64_t(u - 2) * ld]);
                        const R c = A[u + int64_t(u) * ld] + R(0.75) * ex;
                        sh = R(2.0) * c;
                        th = c * c + R(0.4375) * ex * ex;
                    } else {
                        const R a = A[(u - 1) + int64_t(u - 1) * ld], b = A[(u - 1) + int64_t(u) * ld];
                        const R c = A[u + int64_t(u - 1) * ld], d = A[u + int64_t(u) * ld];
                        sh = a + d;
                        th = a * d - b * c;
                    }
                    s_its = s_its + 1;
                    // first column of (H - s1)(H - s2) restricted to the window
                    const R h11 = A[l + int64_t(l) * ld], h12 = A[l + int64_t(l + 1) * ld];
                    const R h21 = A[(l + 1) + int64_t(l) * ld], h22 = A[(l + 1) + int64_t(l + 1) * ld];
                    const R h32 = A[(l + 2) + int64_t(l + 1) * ld];
                    s_x[0] = h11 * h11 + h12 * h21 - sh * h11 + th;
                    s_x[1] = h21 * (h11 + h22 - sh);
                    s_x[2] = h21 * h32;
                }
            }
            if (action == 1) {
                wr[u] = A[u + int64_t(u) * ld];
                wi[u] = R(0.0);
            }
            s_l = l;
            s_action = action;
        }
        __syncthreads();
        const int action = s_action;
        const int u = u0, l = s_l;
        if (action == 4) break;
        if (action == 5) continue;
        if (action == 1) {
            if (tid == 0) {
                s_u = u - 1;
                s_its = 0;
            }
            __syncthreads();
            continue;
        }
        if (action == 2) {
            // 2x2 block at (u-1, u): triangularise if its eigenvalues are real
            __shared__ R s_cs, s_sn;
            __shared__ int s_rot;
            if (tid == 0) {
                const R a = A[(u - 1) + int64_t(u - 1) * ld], b = A[(u - 1) + int64_t(u) * ld];
                const R c = A[u + int64_t(u - 1) * ld], d = A[u + int64_t(u) * ld];
                const R p = R(0.5) * (a - d);
                const R q = p * p + b * c;
                s_rot = 0;
                if (q >= R(0.0)) {
                    const R zz = p + (p >= R(0.0) ? sqrt(q) : -sqrt(q));
                    const R r = hypot(zz, c);
                    if (r > R(0.0)) {
                        s_cs = zz / r;
                        s_sn = c / r;
                        s_rot = 1;
                    }
                    wr[u - 1] = d + zz;
                    wr[u] = (zz != R(0.0)) ? d - b * c / zz : d + zz;
                    wi[u - 1] = wi[u] = R(0.0);
                } else {
                    wr[u - 1] = wr[u] = d + p;
                    wi[u - 1] = sqrt(-q);
                    wi[u] = -sqrt(-q);
                }
            }
            __syncthreads();
            if (s_rot) {
                const R cs = s_cs, sn = s_sn;
                for (int j = u - 1 + tid; j < n; j += NT) {
                    const R x1 = A[(u - 1) + int64_t(j) * ld], x2 = A[u + int64_t(j) * ld];
                    A[(u - 1) + int64_t(j) * ld] = cs * x1 + sn * x2;
                    A[u + int64_t(j) * ld] = -sn * x1 + cs * x2;
                }
                __syncthreads();
                for (int e = tid; e < u + 1 + n; e += NT) {
                    R* M = e <= u ? A : Z;
                    const int i = e <= u ? e : e - (u + 1);
                    const R x1 = M[i + int64_t(u - 1) * ld], x2 = M[i + int64_t(u) * ld];
                    M[i + int64_t(u - 1) * ld] = cs * x1 + sn * x2;
                    M[i + int64_t(u) * ld] = -sn * x1 + cs * x2;
                }
                __syncthreads();
                if (tid == 0) {
                    A[u + int64_t(u - 1) * ld] = R(0.0);
                    // diagonal entries now hold the two real eigenvalues
                    wr[u - 1] = A[(u - 1) + int64_t(u - 1) * ld];
                    wr[u] = A[u + int64_t(u) * ld];
                }
            }
            if (tid == 0) {
                s_u = u - 2;
                s_its = 0;
            }
            __syncthreads();
            continue;
        }
        // Francis R-shift step on the window [l, u] (size ns >= 3). Bulge
        // step kk applies the reflector P (rows and columns r0..r0+2) as
        // H <- P H P and Z <- Z P. Only the core block, rows r0..rmax
        // (rmax = min(r0 + 3, u)) of columns r0..r0+2, takes both the left
        // and the right product; the next reflector is formed from its
        // column r0 (rows r0+1..r0+3). Warp 0 applies P to the core (left
        // product on its three columns, lanes 0..2, then right product on
        // its rows, lanes 0..nq) and lane 0 forms the next reflector, while
        // the other warps apply the left product to the other columns
        // (c0 = r0 - 1 and r0+3..), the right product to the rows above the
        // core, and Z. These sets are disjoint and the left and right
        // products commute, so one block barrier per bulge step suffices:
        // after it, the next core's columns carry every earlier update.
        // Reflectors alternate between two shared slots (the next one is
        // written while the current one is still being read).
        ++total_its;
        const int ns = u - l + 1;
        if (tid == 0) {
            R v[3], beta;
            house(s_x, 3, v, beta);
            for (int t = 0; t < 3; ++t) s_vb[0][t] = v[t];
            s_bb[0] = beta;
        }
        __syncthreads();
        for (int kk = 0; kk <= ns - 3; ++kk) {
            const int b = kk & 1;
            const R v0 = s_vb[b][0], v1 = s_vb[b][1], v2 = s_vb[b][2], beta = s_bb[b];
            const int r0 = l + kk;
            const int c0 = l + (kk > 0 ? kk - 1 : 0);
            const int rmax = min(r0 + 3, u);
            const int nq = rmax - r0;
            if (tid < 32) {
                // core, left product: columns r0 + lane, rows r0..r0+2
                if (tid < 3) {
                    R* col = A + int64_t(r0 + tid) * ld + r0;
                    const R a0 = col[0], a1 = col[1], a2 = col[2];
                    const R sc = beta * fma(v2, a2, fma(v1, a1, v0 * a0));
                    col[0] = a0 - sc * v0;
                    col[1] = a1 - sc * v1;
                    col[2] = a2 - sc * v2;
                }
                __syncwarp();
                // core, right product: rows r0 + lane, columns r0..r0+2
                R xnew = R(0.0);
                if (tid <= nq) {
                    R* row = A + (r0 + tid) + int64_t(r0) * ld;
                    const R a0 = row[0], a1 = row[ld], a2 = row[2 * int64_t(ld)];
                    const R sc = beta * fma(a2, v2, fma(a1, v1, a0 * v0));
                    xnew = a0 - sc * v0;
                    row[0] = xnew;
                    row[ld] = a1 - sc * v1;
                    row[2 * int64_t(ld)] = a2 - sc * v2;
                }
                R xx[3];
                xx[0] = shfl_idx(xnew, 1);
                xx[1] = shfl_idx(xnew, 2);
                xx[2] = shfl_idx(xnew, 3);
                if (tid == 0) {
                    // the 2-element reflector of the window's end after the
                    // last 3-element one
                    R v[3], bt;
                    house(xx, kk < ns - 3 ? 3 : 2, v, bt);
                    for (int t = 0; t < 3; ++t) s_vb[b ^ 1][t] = v[t];
                    s_bb[b ^ 1] = bt;
                }
            } else {
                // left product on column c0 (kk > 0) and columns r0+3..n-1,
                // right product on rows 0..r0-1 of A and on every row of Z
                const int lc = c0 < r0 ? 1 : 0;
                const int nl = lc + max(0, n - (r0 + 3));
                const int nr = r0;
                for (int e = tid - 32; e < nl + nr + n; e += NT - 32) {
                    if (e < nl) {
                        const int j = (e < lc) ? c0 : r0 + 3 + (e - lc);
                        R* col = A + int64_t(j) * ld + r0;
                        const R a0 = col[0], a1 = col[1], a2 = col[2];
                        const R sc = beta * fma(v2, a2, fma(v1, a1, v0 * a0));
                        col[0] = a0 - sc * v0;
                        col[1] = a1 - sc * v1;
                        col[2] = a2 - sc * v2;
                    } else {
                        R* M = e < nl + nr ? A : Z;
                        const int i = e < nl + nr ? e - nl : e - nl - nr;
                        R* row = M + i + int64_t(r0) * ld;
                        const R a0 = row[0], a1 = row[ld], a2 = row[2 * int64_t(ld)];
                        const R sc = beta * fma(a2, v2, fma(a1, v1, a0 * v0));
                        row[0] = a0 - sc * v0;
                        row[ld] = a1 - sc * v1;
                        row[2 * int64_t(ld)] = a2 - sc * v2;
                    }
                }
            }
            __syncthreads();
        }
        {
            // the last reflector (2 elements, rows u - 1 and u)
            const int b = (ns - 2) & 1;
            const R v0 = s_vb[b][0], v1 = s_vb[b][1], beta = s_bb[b];
            for (int j = u - 2 + tid; j < n; j += NT) {
                R* col = A + int64_t(j) * ld + (u - 1);
                const R a0 = col[0], a1 = col[1];
                const R s = beta * fma(v1, a1, v0 * a0);
                col[0] = a0 - s * v0;
                col[1] = a1 - s * v1;
            }
            __syncthreads();
            for (int e = tid; e < u + 1 + n; e += NT) {
                R* M = e <= u ? A : Z;
                const int i = e <= u ? e : e - (u + 1);
                R* row = M + i + int64_t(u - 1) * ld;
                const R a0 = row[0], a1 = row[ld];
                const R s = beta * fma(a1, v1, a0 * v0);
                row[0] = a0 - s * v0;
                row[ld] = a1 - s * v1;
            }
            __syncthreads();
        }
        // clean the bulge remnants of the window: the chase leaves rounding
        // remnants only on its second and third subdiagonals (each step's
        // left product annihilates rows r0+1, r0+2 of column r0-1)
        for (int e = tid; e < 2 * ns; e += NT) {
            const int j = l + (e >> 1), i = j + 2 + (e & 1);
            if (i <= u) A[i + int64_t(j) * ld] = R(0.0);
        }
        __syncthreads();
    }

    const int fail = s_fail;
    const int nv = min(max(nvec, 1), n);
    if (!fail && sym) {
        // ---- symmetric: the real Schur form is diagonal, so ordering is a
        // permutation of the Schur vectors (stable for ties) ----
        int* rk = reinterpret_cast<int*>(hv);
        for (int i = tid; i < n; i += NT) {
            const R di = A[i + int64_t(i) * ld];
            int rank = 0;
            for (int j = 0; j < n; ++j) {
                const R dj = A[j + int64_t(j) * ld];
                if (dj > di || (dj == di && j < i)) ++rank;
            }
#ifdef KL_CHECK_BOUNDS
            if (rank < 0 || rank >= n) {
                atomicExch(&s_oob, 1);
                rank = 0;
            }
#endif
            wr_out[rank] = to_d(di);
            if (wi_out) wi_out[rank] = 0.0;
            rk[i] = rank;
        }
        __syncthreads();
        for (int e = tid; e < int(nn); e += NT) {
            const int c = int(unsigned(e) / unsigned(n)), i = e - c * n;
            const R z = Z[i + int64_t(c) * ld];
            if (Vout) Vout[i + int64_t(rk[c]) * n] = to_d(z);
            if (Qout) Qout[i + int64_t(rk[c]) * n] = to_d(z);
        }
    } else if (!fail) {
        // ---- ordering of the real Schur form by decreasing real part ----
        order_schur(A, Z, n, ld, nv, anorm, hv, ord, &s_oob);
        __syncthreads();

        // ---- eigenvalues of the ordered blocks ----
        for (int i = tid; i < n; i += NT) {
            const bool first = (i + 1 < n) && A[(i + 1) + int64_t(i) * ld] != R(0.0);
            const bool second = (i > 0) && A[i + int64_t(i - 1) * ld] != R(0.0);
            if (first || second) {
                const int b0 = first ? i : i - 1;
                const R a = A[b0 + int64_t(b0) * ld], b = A[b0 + int64_t(b0 + 1) * ld];
                const R c = A[(b0 + 1) + int64_t(b0) * ld], d = A[(b0 + 1) + int64_t(b0 + 1) * ld];
                const R pp = R(0.5) * (a - d), q = pp * pp + b * c;
                const R im = q < R(0.0) ? sqrt(-q) : R(0.0);
                wr[i] = d + pp;
                wi[i] = first ? im : -im;
            } else {
                wr[i] = A[i + int64_t(i) * ld];
                wi[i] = R(0.0);
            }
        }
        __syncthreads();

        // ---- eigenvectors of the leading nv columns of T by back substitution ----
        // Diagonal entries within 1e-10 ||T|| of the eigenvalue belong to its
        // cluster; their components are set to zero instead of dividing by a
        // vanishing pivot, so the vectors of a (numerically) multiple
        // eigenvalue stay independent (its invariant subspace is spanned by
        // Schur vectors).
        // All columns are solved together, one block row of T (1x1 or 2x2)
        // per step from the bottom up: X(i, c) holds the partial sum
        // sum_{l > i} T(i, l) x_c(l) until row i is reached, then x_c(i). A
        // step solves its rows for every active column (one thread each),
        // then adds their contributions to the rows above (one thread per
        // entry). The real and imaginary columns of a complex pair take the
        // same real update.
        const int nve = (nv < n && wi[nv - 1] > R(0.0)) ? nv + 1 : nv;
        const R small = EigNum<R>::eps * fmax(anorm, EigNum<R>::tiny);
        const R clus = EigNum<R>::split * anorm;
        for (int e = tid; e < n * nve; e += NT) {
            const int c = int(unsigned(e) / unsigned(n)), i = e - c * n;
            R v = R(0.0);
            if (wi[c] == R(0.0)) {
                // real eigenvalue: x_c(c) = 1, zero below
                v = i < c ? A[i + int64_t(c) * ld] : i == c ? R(1.0) : R(0.0);
            } else if (wi[c] > R(0.0)) {
                // complex pair (c, c+1), lambda = wr + i wi: the vector is
                // real part in column c, imaginary part in column c+1. Its
                // rows c, c+1 are (b12, lambda - b11), which solves the first
                // row of (B - lambda I) x = 0 for the 2x2 block B and is non-
                // zero because lambda is not real.
                const R b12 = A[c + int64_t(c + 1) * ld], d = wr[c] - A[c + int64_t(c) * ld];
                if (i < c) v = A[i + int64_t(c) * ld] * b12 + A[i + int64_t(c + 1) * ld] * d;
                else if (i == c) v = b12;
                else if (i == c + 1) v = d;
            } else {
                // imaginary part of the pair (c-1, c)
                const int q = c - 1;
                if (i < q) v = A[i + int64_t(c) * ld] * wi[q];
                else if (i == c) v = wi[q];
            }
            X[i + int64_t(c) * ld] = v;
        }
        __syncthreads();
        {
            // rows below the block of the last column's eigenvalue are known
            const int cl = nve - 1;
            int j = (wi[cl] < R(0.0) ? cl - 1 : cl) - 1;
            while (j >= 0) {
                // j is the bottom row of a diagonal block of T, so columns
                // c > j are exactly those whose eigenvalue block lies below
                const bool two = (j > 0) && A[j + int64_t(j - 1) * ld] != R(0.0);
                const int jl = two ? j - 1 : j;
                for (int c = j + 1 + tid; c < nve; c += NT) {
                    if (wi[c] < R(0.0)) continue;  // solved with its partner
                    R* xr = X + int64_t(c) * ld;
                    if (wi[c] == R(0.0)) {
                        const R lam = wr[c];
                        if (!two) {
                            R den = A[j + int64_t(j) * ld] - lam;
                            if (fabs(den) <= clus) {
                                xr[j] = R(0.0);
                            } else {
                                if (fabs(den) < small) den = small;
                                xr[j] = -xr[j] / den;
                            }
                        } else {
                            // 2x2 system for rows j-1, j
                            const R s1 = xr[j - 1], s2 = xr[j];
                            const R a11 = A[(j - 1) + int64_t(j - 1) * ld] - lam, a12 = A[(j - 1) + int64_t(j) * ld];
                            const R a21 = A[j + int64_t(j - 1) * ld], a22 = A[j + int64_t(j) * ld] - lam;
                            R det = a11 * a22 - a12 * a21;
                            if (fabs(det) < small * small) det = small * small;
                            const R rdet = R(1.0) / det;
                            xr[j - 1] = (s2 * a12 - s1 * a22) * rdet;
                            xr[j] = (s1 * a21 - s2 * a11) * rdet;
                        }
                    } else {
                        R* xi = X + int64_t(c + 1) * ld;
                        const cpx<R> lam = {wr[c], wi[c]};
                        if (!two) {
                            cpx<R> den = {A[j + int64_t(j) * ld] - lam.re, -lam.im};
                            if (fabs(den.re) + fabs(den.im) < small) den.re = small;
                            const cpx<R> r = cdiv_r(cpx<R>{-xr[j], -xi[j]}, den);
                            xr[j] = r.re;
                            xi[j] = r.im;
                        } else {
                            const cpx<R> s1 = {xr[j - 1], xi[j - 1]}, s2 = {xr[j], xi[j]};
                            const cpx<R> a11 = {A[(j - 1) + int64_t(j - 1) * ld] - lam.re, -lam.im};
                            const R a12 = A[(j - 1) + int64_t(j) * ld], a21 = A[j + int64_t(j - 1) * ld];
                            const cpx<R> a22 = {A[j + int64_t(j) * ld] - lam.re, -lam.im};
                            const cpx<R> p = cmul_r(a11, a22);
                            cpx<R> det = {p.re - a12 * a21, p.im};
                            if (fabs(det.re) + fabs(det.im) < small * small) det.re = small * small;
                            const cpx<R> q1 = cmul_r(s1, a22), q2 = cmul_r(s2, a11);
                            const cpx<R> r1 = cdiv_r(cpx<R>{s2.re * a12 - q1.re, s2.im * a12 - q1.im}, det);
                            const cpx<R> r2 = cdiv_r(cpx<R>{s1.re * a21 - q2.re, s1.im * a21 - q2.im}, det);
                            xr[j - 1] = r1.re;
                            xi[j - 1] = r1.im;
                            xr[j] = r2.re;
                            xi[j] = r2.im;
                        }
                    }
                }
                __syncthreads();
                // contributions of rows jl..j to the rows above
                const int nact = nve - (j + 1);
                for (int e = tid; e < jl * nact; e += NT) {
                    const int i = e % jl;
                    R* x = X + int64_t(j + 1 + e / jl) * ld;
                    R sum = fma(A[i + int64_t(j) * ld], x[j], x[i]);
                    if (two) sum = fma(A[i + int64_t(j - 1) * ld], x[j - 1], sum);
                    x[i] = sum;
                }
                __syncthreads();
                j = jl - 1;
            }
        }
        // V = Z X for the leading columns (X(:, c) vanishes below row c + 1),
        // four columns per thread, then unit columns (complex pairs jointly)
        R* Vt = A;  // the Schur form is no longer needed
        const int ng = (nve + 3) / 4;
        for (int e = tid; e < n * ng; e += NT) {
            const int cg = int(unsigned(e) / unsigned(n)), i = e - cg * n, c0 = 4 * cg;
            const int top = min(n - 1, c0 + 4);
            // columns past the last one repeat it (computed, not stored)
            const R* x0 = X + int64_t(c0) * ld;
            const R* x1 = X + int64_t(min(c0 + 1, nve - 1)) * ld;
            const R* x2 = X + int64_t(min(c0 + 2, nve - 1)) * ld;
            const R* x3 = X + int64_t(min(c0 + 3, nve - 1)) * ld;
            R s0 = R(0.0), s1 = R(0.0), s2 = R(0.0), s3 = R(0.0);
            for (int l2 = 0; l2 <= top; ++l2) {
                const R z = Z[i + int64_t(l2) * ld];
                s0 = fma(z, x0[l2], s0);
                s1 = fma(z, x1[l2], s1);
                s2 = fma(z, x2[l2], s2);
                s3 = fma(z, x3[l2], s3);
            }
            Vt[i + int64_t(c0) * n] = s0;
            if (c0 + 1 < nve) Vt[i + int64_t(c0 + 1) * n] = s1;
            if (c0 + 2 < nve) Vt[i + int64_t(c0 + 2) * n] = s2;
            if (c0 + 3 < nve) Vt[i + int64_t(c0 + 3) * n] = s3;
        }
        __syncthreads();
        {
            const int lane = tid & 31, warp = tid >> 5;
            for (int c = warp; c < nve; c += kEigWarps) {
                if (wi[c] < R(0.0)) continue;
                const int w2 = (wi[c] > R(0.0)) ? 2 : 1;
                R s = R(0.0);
                for (int t = 0; t < w2; ++t)
                    for (int i = lane; i < n; i += 32) s = fma(Vt[i + int64_t(c + t) * n], Vt[i + int64_t(c + t) * n], s);
                for (int o = 16; o > 0; o >>= 1) s += shfl_xor(s, o);
                s = s > R(0.0) ? R(1.0) / sqrt(s) : R(1.0);
                for (int t = 0; t < w2; ++t)
                    for (int i = lane; i < n; i += 32) Vt[i + int64_t(c + t) * n] *= s;
            }
        }
        __syncthreads();
        for (int i = tid; i < n; i += NT) {
            wr_out[i] = to_d(wr[i]);
            if (wi_out) wi_out[i] = to_d(wi[i]);
        }
        if (Vout)
            for (int64_t e = tid; e < int64_t(n) * nve; e += NT) Vout[e] = to_d(Vt[e]);
        if (Qout)
            for (int e = tid; e < int(nn); e += NT) {
                const int c = int(unsigned(e) / unsigned(n));
                Qout[e] = to_d(Z[(e - c * n) + int64_t(c) * ld]);
            }
    }
    if (tid == 0) {
        // 3: the bounds-checking build found an index out of range
        status[0] = s_oob ? 3 : fail ? 1 : 0;
        // diagnostics after the status word: QR iterations, last window end,
        // iterations spent on it
        status[1] = total_its;
        status[2] = s_u;
        status[3] = s_its;
    }
}

// Shared-memory level for an n x n problem (see the kernel).
int eig_smem_level(int n, size_t esize, size_t* bytes) {
    const size_t nn = size_t(n + 1) * n;  // matrices with leading dimension n + 1
    if ((3 * nn + 10 * size_t(n)) * esize <= kEigSmemLimit) {
        *bytes = (3 * nn + 10 * size_t(n)) * esize;
        return 2;
    }
    if ((nn + 2 * size_t(n)) * esize <= kEigSmemLimit) {
        *bytes = (nn + 2 * size_t(n)) * esize;
        return 1;
    }
    *bytes = 0;
    return 0;
}

template <class R>
cudaError_t launch_eig_t(const double* H, int n, double* wr, double* wi, double* V, double* Q, double* work,
                         int* status, int sym, int nvec, cudaStream_t s) {
    size_t bytes = 0;
    const int level = eig_smem_level(n, sizeof(R), &bytes);
    // the attribute is set once to the largest size any call uses: host
    // threads launching concurrently must not lower it under each other
    static std::once_flag once;
    static cudaError_t attr_error = cudaSuccess;
    std::call_once(once, [] {
        attr_error = cudaFuncSetAttribute(nonsym_eig_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          int(kEigSmemLimit));
    });
    if (attr_error != cudaSuccess) return attr_error;
    nonsym_eig_kernel<R><<<1, kEigThreads, bytes, s>>>(H, n, wr, wi, V, Q, work, status, level, sym, nvec);
    return cudaGetLastError();
}

cudaError_t launch_eig(const double* H, int n, double* wr, double* wi, double* V, double* Q, double* work,
                       int* status, int sym, int nvec, int arith, cudaStream_t s) {
    // the ordering gives each thread at most 4 block pairs: n <= 1024
    if (n <= 0 || n > 1024) return cudaErrorInvalidValue;
    const int64_t nn = int64_t(n) * n;
    KL_RANGE(H, nn, double, "eig H");
    KL_RANGE(wr, n, double, "eig wr");
    KL_RANGE(wi, n, double, "eig wi");
    // eigenvectors: all n (symmetric) or the leading nvec (one more to keep
    // a complex pair whole), n rows each
    KL_RANGE(V, sym ? nn : int64_t(n) * std::min(n, std::max(nvec, 1) + 1), double, "eig V");
    KL_RANGE(Q, nn, double, "eig Q");
    KL_RANGE(work, nonsym_eig_work_doubles(n), double, "eig work");
    KL_RANGE(status, 4, int, "eig status");
    if (arith == kEigFP32) return launch_eig_t<float>(H, n, wr, wi, V, Q, work, status, sym, nvec, s);
    if (arith == kEigDF) return launch_eig_t<dfl>(H, n, wr, wi, V, Q, work, status, sym, nvec, s);
    return launch_eig_t<double>(H, n, wr, wi, V, Q, work, status, sym, nvec, s);
}

}  // namespace

int64_t nonsym_eig_work_doubles(int n) { return 3 * int64_t(n + 1) * n + 12 * int64_t(n); }
int64_t sym_eig_work_doubles(int n) { return std::max(nonsym_eig_work_doubles(n), jacobi_work_doubles(n)); }

// Symmetric eigenproblem. FP64: parallel Jacobi in FP32 refined in FP64 up to
// jacobi_max_n(). FP32, double-float, and FP64 beyond that order: the same
// Householder reduction as the non-symmetric one (here to tridiagonal form),
// then implicit QR steps with Wilkinson shifts on the tridiagonal form, the
// rotations accumulated into the orthonormal eigenvectors. (FP32 Jacobi alone accumulates the
// rounding of thousands of rotations in its vectors: invariant subspaces of
// clustered K-L eigenvalues came out 1e-4 off, against 1e-6 for the QR path,
// and restarts from them slowed convergence.)
cudaError_t launch_sym_eig(const double* H, int n, double* w, double* V, double* work, int* status,
                           cudaStream_t s, bool fp32, bool dfloat) {
    if (!fp32 && dfloat) return launch_eig(H, n, w, nullptr, V, nullptr, work, status, 1, n, kEigDF, s);
    if (!fp32 && n <= jacobi_max_n()) return launch_sym_eig_jacobi(H, n, w, V, work, status, s, false);
    return launch_eig(H, n, w, nullptr, V, nullptr, work, status, 1, n, fp32 ? kEigFP32 : kEigFP64, s);
}

cudaError_t launch_nonsym_eig(const double* H, int n, double* wr, double* wi, double* V, double* Q,
                              double* work, int* status, cudaStream_t s, int nvec, int arith) {
    return launch_eig(H, n, wr, wi, V, Q, work, status, 0, nvec > 0 ? nvec : n, arith, s);
}

}  // namespace kl
