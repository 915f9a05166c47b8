// tcgen05 (5th-generation tensor core) pairwise product W = Gamma X.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "kl_internal.h"

namespace kl {

struct TcArgs {
    const float *tx, *ty, *tz;  // targets (T), FP32
    const float *sx, *sy, *sz;  // sources (S), FP32
    int64_t T, S;
    const double* X;  // S x k (ldx), FP64 source values
    int64_t ldx;
    double* Y;  // T x k (ldy)
    int64_t ldy;
    int k;
    const double* post;  // optional per-target scale
    KernelSpec ks;
    bool tf32;  // split TF32 products instead of split BF16
    double* scratch;
    int64_t scratch_len;  // doubles
    int sm_count;
};

// Scratch needed by launch_pair_tc for T targets and k vectors (doubles).
int64_t tc_scratch_doubles(int64_t T, int64_t S, int k, int sm_count);
// Enqueues the conversion, the tcgen05 kernel and the split reduction.
// *launched receives the number of kernels launched. Returns
// cudaErrorLaunchTimeout if a bounded wait inside the kernel gave up.
cudaError_t launch_pair_tc(const TcArgs& a, cudaStream_t s, int* launched);

// Reduction of split partials shared with the CUDA-core kernels.
cudaError_t launch_pair_reduce(const double* part, int splits, int64_t T, int k, double sigma2,
                               const double* post, double* Y, int64_t ldy, cudaStream_t s);

}  // namespace kl
