// Microbenchmarks of the arithmetic units that bound the pairwise kernel
// evaluation: FP32 FMA issue, the base-2 exponential of the special function
// unit (MUFU ex2) and FP64 FMA. Each kernel runs independent dependency
// chains in every thread of a full grid; rates are operations per second.
#include <cuda_runtime.h>

#include "kl_internal.h"

namespace kl {
namespace {

constexpr int kIters = 4096;

__global__ void ffma_kernel(float* out, float a, float b) {
    float x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    for (int i = 0; i < kIters; ++i) {
        x0 = fmaf(x0, a, b); x1 = fmaf(x1, a, b); x2 = fmaf(x2, a, b); x3 = fmaf(x3, a, b);
        x4 = fmaf(x4, a, b); x5 = fmaf(x5, a, b); x6 = fmaf(x6, a, b); x7 = fmaf(x7, a, b);
    }
    const float s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
    if (s == 1234.5f) out[0] = s;
}

__global__ void ex2_kernel(float* out, float a) {
    float x0 = threadIdx.x * 1e-3f, x1 = x0 + 0.1f, x2 = x0 + 0.2f, x3 = x0 + 0.3f;
    for (int i = 0; i < kIters; ++i) {
        float y0, y1, y2, y3;
        asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(x0));
        asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y1) : "f"(x1));
        asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y2) : "f"(x2));
        asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y3) : "f"(x3));
        x0 = -y0 * a; x1 = -y1 * a; x2 = -y2 * a; x3 = -y3 * a;
    }
    const float s = x0 + x1 + x2 + x3;
    if (s == 1234.5f) out[0] = s;
}

__global__ void dfma_kernel(double* out, double a, double b) {
    double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
    for (int i = 0; i < kIters / 8; ++i) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    }
    const double s = x0 + x1 + x2 + x3;
    if (s == 1234.5) out[0] = s;
}

template <class F>
double time_ms(F launch) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    launch();  // warm-up
    cudaEventRecord(e0);
    for (int r = 0; r < 3; ++r) launch();
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms / 3.0;
}

}  // namespace
}  // namespace kl

extern "C" int kl_measure_peaks(double* fp32_fma_per_s, double* ex2_per_s, double* fp64_fma_per_s) {
    using namespace kl;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return KL_ERR_CUDA;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return KL_ERR_CUDA;
    const int blocks = prop.multiProcessorCount * 8, threads = 256;
    float* buf = nullptr;
    if (cudaMalloc(&buf, 64) != cudaSuccess) return KL_ERR_OOM;
    const double nthr = double(blocks) * threads;
    const double t1 = time_ms([&] { ffma_kernel<<<blocks, threads>>>(buf, 0.999f, 1e-3f); });
    const double t2 = time_ms([&] { ex2_kernel<<<blocks, threads>>>(buf, 0.5f); });
    const double t3 = time_ms([&] { dfma_kernel<<<blocks, threads>>>(reinterpret_cast<double*>(buf), 0.999, 1e-3); });
    const cudaError_t e = cudaGetLastError();
    cudaFree(buf);
    if (e != cudaSuccess) return KL_ERR_CUDA;
    if (fp32_fma_per_s) *fp32_fma_per_s = nthr * 8.0 * kIters / (t1 * 1e-3);
    if (ex2_per_s) *ex2_per_s = nthr * 4.0 * kIters / (t2 * 1e-3);
    if (fp64_fma_per_s) *fp64_fma_per_s = nthr * 4.0 * (kIters / 8) / (t3 * 1e-3);
    return KL_OK;
}
