// Pairwise kernel products on CUDA cores: W = Gamma(targets, sources) X.
//
// This is the O(N~^2) step of the IBQ-Galerkin matvec (Sec. 3.1: the rows of
// Gamma are evaluated when needed, never stored) and the kernel product of
// Algorithm 1 in the collocation matvec (Sec. 3.2). Gamma is never stored: every CTA owns 128
// target points (one per thread, coordinates in registers), streams tiles of
// source points and their k vector values through shared memory, evaluates
// the kernel for each (target, source) pair in registers and accumulates
// Gamma_ts * X_s into k per-thread accumulators.
//
// The source range is split across blockIdx.y so that small target counts
// still fill the GPU; each split writes its partial sums to scratch and a
// second kernel adds the splits in a fixed order (deterministic results) and
// applies sigma^2 and the optional per-target scale (J of Sec. 3.1).
#include <cmath>

#include "kernel_eval.cuh"
#include "kernels_tc.h"
#include "kl_internal.h"

namespace kl {

namespace {

constexpr int kTgt = 128;  // targets per CTA (= threads)
constexpr int kSrc = 128;  // sources per shared-memory tile

template <int KIND, int KB>
__global__ void __launch_bounds__(kTgt) pair_f64_kernel(
    const double* __restrict__ tx, const double* __restrict__ ty, const double* __restrict__ tz,
    int64_t T, const double* __restrict__ sx, const double* __restrict__ sy,
    const double* __restrict__ sz, int64_t S, const double* __restrict__ X, int64_t ldx, int k,
    int c0, double a, double* __restrict__ part, int64_t per_split) {
    __shared__ double s_x[kSrc], s_y[kSrc], s_z[kSrc];
    __shared__ double s_v[kSrc][KB];
    const int64_t t = int64_t(blockIdx.x) * kTgt + threadIdx.x;
    const int split = blockIdx.y;
    const int64_t s0 = int64_t(split) * per_split;
    const int64_t s1 = min(S, s0 + per_split);
    const double px = t < T ? tx[t] : 0.0, py = t < T ? ty[t] : 0.0, pz = t < T ? tz[t] : 0.0;
    const int kc = min(KB, k - c0);
    double acc[KB];
#pragma unroll
    for (int c = 0; c < KB; ++c) acc[c] = 0.0;
    for (int64_t base = s0; base < s1; base += kSrc) {
        const int n = int(s1 - base < kSrc ? s1 - base : int64_t(kSrc));
        __syncthreads();
        for (int i = threadIdx.x; i < kSrc; i += kTgt) {
            const bool v = i < n;
            s_x[i] = v ? sx[base + i] : 0.0;
            s_y[i] = v ? sy[base + i] : 0.0;
            s_z[i] = v ? sz[base + i] : 0.0;
        }
        for (int i = threadIdx.x; i < kSrc * KB; i += kTgt) {
            const int c = i / kSrc, j = i - c * kSrc;
            s_v[j][c] = (j < n && c < kc) ? X[base + j + int64_t(c0 + c) * ldx] : 0.0;
        }
        __syncthreads();
        for (int j = 0; j < n; ++j) {
            const double g = gamma64<KIND>(px - s_x[j], py - s_y[j], pz - s_z[j], a);
#pragma unroll
            for (int c = 0; c < KB; ++c) acc[c] = fma(g, s_v[j][c], acc[c]);
        }
    }
    if (t < T) {
        for (int c = 0; c < kc; ++c) part[(int64_t(split) * k + c0 + c) * T + t] = acc[c];
    }
}

template <int KIND, int KB>
__global__ void __launch_bounds__(kTgt) pair_f32_kernel(
    const float* __restrict__ tx, const float* __restrict__ ty, const float* __restrict__ tz,
    int64_t T, const float* __restrict__ sx, const float* __restrict__ sy,
    const float* __restrict__ sz, int64_t S, const double* __restrict__ X, int64_t ldx, int k,
    int c0, float a, float a2, double* __restrict__ part, int64_t per_split) {
    __shared__ float s_x[kSrc], s_y[kSrc], s_z[kSrc];
    __shared__ float s_v[kSrc][KB];
    const int64_t t = int64_t(blockIdx.x) * kTgt + threadIdx.x;
    const int split = blockIdx.y;
    const int64_t s0 = int64_t(split) * per_split;
    const int64_t s1 = min(S, s0 + per_split);
    const float px = t < T ? tx[t] : 0.f, py = t < T ? ty[t] : 0.f, pz = t < T ? tz[t] : 0.f;
    const int kc = min(KB, k - c0);
    float acc[KB];
    double accd[KB];
#pragma unroll
    for (int c = 0; c < KB; ++c) acc[c] = 0.f, accd[c] = 0.0;
    for (int64_t base = s0; base < s1; base += kSrc) {
        const int n = int(s1 - base < kSrc ? s1 - base : int64_t(kSrc));
        __syncthreads();
        for (int i = threadIdx.x; i < kSrc; i += kTgt) {
            const bool v = i < n;
            s_x[i] = v ? sx[base + i] : 0.f;
            s_y[i] = v ? sy[base + i] : 0.f;
            s_z[i] = v ? sz[base + i] : 0.f;
        }
        for (int i = threadIdx.x; i < kSrc * KB; i += kTgt) {
            const int c = i / kSrc, j = i - c * kSrc;
            s_v[j][c] = (j < n && c < kc) ? float(X[base + j + int64_t(c0 + c) * ldx]) : 0.f;
        }
        __syncthreads();
        for (int j = 0; j < n; ++j) {
            const float g = gamma32<KIND>(px - s_x[j], py - s_y[j], pz - s_z[j], a, a2);
#pragma unroll
            for (int c = 0; c < KB; ++c) acc[c] = fmaf(g, s_v[j][c], acc[c]);
        }
        // flush the FP32 tile sums into FP64 once per tile
#pragma unroll
        for (int c = 0; c < KB; ++c) accd[c] += double(acc[c]), acc[c] = 0.f;
    }
    if (t < T) {
        for (int c = 0; c < kc; ++c) part[(int64_t(split) * k + c0 + c) * T + t] = accd[c];
    }
}

__global__ void pair_reduce_kernel(const double* __restrict__ part, int splits, int64_t T, int k,
                                   double sigma2, const double* __restrict__ post, double* Y,
                                   int64_t ldy) {
    const int64_t total = T * k;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t c = i / T, t = i - c * T;
        double s = 0.0;
        for (int sp = 0; sp < splits; ++sp) s += part[(int64_t(sp) * k + c) * T + t];
        s *= sigma2;
        if (post) s *= post[t];
        Y[c * ldy + t] = s;
    }
}

template <int KIND>
cudaError_t launch_kind(const PairArgs& a, bool fp32, cudaStream_t s) {
    const int64_t per_split = (a.S + a.splits - 1) / a.splits;
    if (fp32) {
        KL_RANGE(a.tx32, a.T, float, "pair targets x");
        KL_RANGE(a.ty32, a.T, float, "pair targets y");
        KL_RANGE(a.tz32, a.T, float, "pair targets z");
        KL_RANGE(a.sx32, a.S, float, "pair sources x");
        KL_RANGE(a.sy32, a.S, float, "pair sources y");
        KL_RANGE(a.sz32, a.S, float, "pair sources z");
    } else {
        KL_RANGE(a.tx, a.T, double, "pair targets x");
        KL_RANGE(a.ty, a.T, double, "pair targets y");
        KL_RANGE(a.tz, a.T, double, "pair targets z");
        KL_RANGE(a.sx, a.S, double, "pair sources x");
        KL_RANGE(a.sy, a.S, double, "pair sources y");
        KL_RANGE(a.sz, a.S, double, "pair sources z");
    }
    KL_RANGE(a.X, block_extent(a.S, a.k, a.ldx), double, "pair X");
    KL_RANGE(a.scratch, pair_scratch_doubles(a.T, a.k, a.splits), double, "pair partial sums");
    KL_RANGE(a.Y, block_extent(a.T, a.k, a.ldy), double, "pair Y");
    KL_RANGE(a.post, a.T, double, "pair post");
    dim3 grid(unsigned((a.T + kTgt - 1) / kTgt), unsigned(a.splits));
    const double l2e = 1.4426950408889634074;
    for (int c0 = 0; c0 < a.k; c0 += 32) {
        const int kc = a.k - c0;
        if (fp32) {
            const float fa = float(a.ks.a), fa2 = float(a.ks.a * l2e);
            if (kc <= 8)
                pair_f32_kernel<KIND, 8><<<grid, kTgt, 0, s>>>(a.tx32, a.ty32, a.tz32, a.T, a.sx32, a.sy32, a.sz32, a.S, a.X, a.ldx, a.k, c0, fa, fa2, a.scratch, per_split);
            else if (kc <= 16)
                pair_f32_kernel<KIND, 16><<<grid, kTgt, 0, s>>>(a.tx32, a.ty32, a.tz32, a.T, a.sx32, a.sy32, a.sz32, a.S, a.X, a.ldx, a.k, c0, fa, fa2, a.scratch, per_split);
            else
                pair_f32_kernel<KIND, 32><<<grid, kTgt, 0, s>>>(a.tx32, a.ty32, a.tz32, a.T, a.sx32, a.sy32, a.sz32, a.S, a.X, a.ldx, a.k, c0, fa, fa2, a.scratch, per_split);
        } else {
            if (kc <= 8)
                pair_f64_kernel<KIND, 8><<<grid, kTgt, 0, s>>>(a.tx, a.ty, a.tz, a.T, a.sx, a.sy, a.sz, a.S, a.X, a.ldx, a.k, c0, a.ks.a, a.scratch, per_split);
            else if (kc <= 16)
                pair_f64_kernel<KIND, 16><<<grid, kTgt, 0, s>>>(a.tx, a.ty, a.tz, a.T, a.sx, a.sy, a.sz, a.S, a.X, a.ldx, a.k, c0, a.ks.a, a.scratch, per_split);
            else
                pair_f64_kernel<KIND, 32><<<grid, kTgt, 0, s>>>(a.tx, a.ty, a.tz, a.T, a.sx, a.sy, a.sz, a.S, a.X, a.ldx, a.k, c0, a.ks.a, a.scratch, per_split);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const int64_t total = a.T * a.k;
    int g = int(std::min<int64_t>((total + 255) / 256, int64_t(device_sm_count()) * 32));
    pair_reduce_kernel<<<g < 1 ? 1 : g, 256, 0, s>>>(a.scratch, a.splits, a.T, a.k, a.ks.sigma2, a.post, a.Y, a.ldy);
    return cudaGetLastError();
}

}  // namespace

int64_t pair_scratch_doubles(int64_t T, int k, int splits) { return T * int64_t(k) * splits; }

int pair_choose_splits(int64_t T, int64_t S, int sm_count) {
    const int64_t tb = (T + kTgt - 1) / kTgt;
    int64_t want = (16LL * sm_count + tb - 1) / tb;
    int64_t cap = S / 512;
    if (cap < 1) cap = 1;
    if (want > cap) want = cap;
    if (want < 1) want = 1;
    if (want > 64) want = 64;
    return int(want);
}

cudaError_t launch_pair_reduce(const double* part, int splits, int64_t T, int k, double sigma2,
                               const double* post, double* Y, int64_t ldy, cudaStream_t s) {
    KL_RANGE(part, pair_scratch_doubles(T, k, splits), double, "pair_reduce partial sums");
    KL_RANGE(Y, block_extent(T, k, ldy), double, "pair_reduce Y");
    KL_RANGE(post, T, double, "pair_reduce post");
    const int64_t total = T * k;
    int g = int(std::min<int64_t>((total + 255) / 256, int64_t(device_sm_count()) * 32));
    pair_reduce_kernel<<<g < 1 ? 1 : g, 256, 0, s>>>(part, splits, T, k, sigma2, post, Y, ldy);
    return cudaGetLastError();
}

cudaError_t launch_pair_simt(const PairArgs& a, bool fp32, cudaStream_t s) {
    switch (a.ks.kind) {
        case KL_KERNEL_GAUSS: return launch_kind<KL_KERNEL_GAUSS>(a, fp32, s);
        case KL_KERNEL_EXP_SEP: return launch_kind<KL_KERNEL_EXP_SEP>(a, fp32, s);
        case KL_KERNEL_EXP: return launch_kind<KL_KERNEL_EXP>(a, fp32, s);
        case KL_KERNEL_MATERN32: return launch_kind<KL_KERNEL_MATERN32>(a, fp32, s);
        default: return launch_kind<KL_KERNEL_CONST>(a, fp32, s);
    }
}

}  // namespace kl
