// Covariance kernel evaluation shared by the pairwise-product kernels.
//
// Gamma(x, x') without the factor sigma^2, which is applied once per output
// entry. `a` is 1/L^2 (Gaussian), 1/L (the exponential kernels) or
// sqrt(3)/L (Matern-3/2); the FP32 variants also take a2 = a * log2(e) so
// that the exponential is a single base-2 exponential.
#pragma once

#include "../../include/kl.h"

namespace kl {

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Kernel value without sigma^2. `a` is 1/L^2 (Gauss), 1/L (exponentials) or
// sqrt(3)/L (Matern-3/2); the FP32 variants take a * log2(e) in `a2`.
template <int KIND>
__device__ __forceinline__ double gamma64(double dx, double dy, double dz, double a) {
    if (KIND == KL_KERNEL_GAUSS) return exp(-a * (dx * dx + dy * dy + dz * dz));
    if (KIND == KL_KERNEL_EXP_SEP) return exp(-a * (fabs(dx) + fabs(dy) + fabs(dz)));
    if (KIND == KL_KERNEL_EXP) return exp(-a * sqrt(dx * dx + dy * dy + dz * dz));
    if (KIND == KL_KERNEL_MATERN32) {
        const double s = a * sqrt(dx * dx + dy * dy + dz * dz);
        return (1.0 + s) * exp(-s);
    }
    return 1.0;
}

template <int KIND>
__device__ __forceinline__ float gamma32(float dx, float dy, float dz, float a, float a2) {
    if (KIND == KL_KERNEL_GAUSS) return ex2_approx(-a2 * fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
    if (KIND == KL_KERNEL_EXP_SEP) return ex2_approx(-a2 * (fabsf(dx) + fabsf(dy) + fabsf(dz)));
    if (KIND == KL_KERNEL_EXP) return ex2_approx(-a2 * sqrt_approx(fmaf(dx, dx, fmaf(dy, dy, dz * dz))));
    if (KIND == KL_KERNEL_MATERN32) {
        const float r = sqrt_approx(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
        return fmaf(a, r, 1.0f) * ex2_approx(-a2 * r);
    }
    return 1.0f;
}


}  // namespace kl
