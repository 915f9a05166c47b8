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
    int* err;  // device word set when a bounded wait inside the kernel gives up
    long long wait_limit;  // clock cycles per pipeline wait (0: default, about a second)
};

// One pairwise product inside a persistent launch: its target points, the
// chunk records of X (split images and pre-scaled source coordinates, written
// by the conversion kernel; srcc is unused), its (hi, lo) partial sums, and
// its range of work units [unit0, unit0 + tiles * splits) in the launch.
struct TcInstance {
    const float *tx, *ty, *tz;
    const float* srcc;
    const uint8_t* img;
    float2* part;
    int64_t T, nchunks, unit0;
    int cps, splits, kind, k_total, c0, kc;
    float cscale;
};
// Instances of one launch (same precision and N rounded to 16); passed by
// value as a kernel parameter.
constexpr int kTcMaxBatch = 32;
struct TcBatch {
    TcInstance inst[kTcMaxBatch];
    int ninst;
    int64_t nunits;
    long long wait_limit;  // clock cycles of each pipeline wait (0: about a second)
};

// Phase 1 of a pairwise product: conversion kernels on stream s and the
// instance descriptors (unit0 = 0) of its column blocks of at most 64
// vectors (*n of them, <= 4). tf32/np of the descriptors in *tf32, *np.
cudaError_t tc_prepare(const TcArgs& a, cudaStream_t s, TcInstance* out, int* n, int* np, int* launched);
// Phase 2: one persistent launch over the instances of b (same tf32 and np),
// units assigned contiguously in order; err: device word set on a timeout.
cudaError_t tc_launch_batch(TcBatch& b, bool tf32, int np, int sm_count, int* err, cudaStream_t s);
// Phase 3: reduction of the partial sums into Y on stream s.
cudaError_t tc_finish(const TcArgs& a, cudaStream_t s, int* launched);
// Scratch needed by launch_pair_tc for T targets and any block of at most k
// vectors (doubles).
int64_t tc_scratch_doubles(int64_t T, int64_t S, int k, int sm_count);
// Enqueues the conversion, the tcgen05 kernel and the split reduction.
// *launched receives the number of kernels launched. A bounded wait that gives
// up inside the kernel sets *a.err (read by the caller after a synchronisation).
cudaError_t launch_pair_tc(const TcArgs& a, cudaStream_t s, int* launched);

// Reduction of split partials shared with the CUDA-core kernels.
cudaError_t launch_pair_reduce(const double* part, int splits, int64_t T, int k, double sigma2,
                               const double* post, double* Y, int64_t ldy, cudaStream_t s);

}  // namespace kl
