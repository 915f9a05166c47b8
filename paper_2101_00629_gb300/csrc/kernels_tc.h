// tcgen05 (5th-generation tensor core) pairwise product W = Gamma X.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "kl_internal.h"

namespace kl {

struct TcSymPlan;

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
    // SMs the persistent pairwise grid spans (2 CTAs each; 0: sm_count):
    // fewer leave SMs free for kernels of other streams
    int grid_sms;
    int* err;  // device word set when a bounded wait inside the kernel gives up
    long long wait_limit;  // clock cycles per pipeline wait (0: default, about a second)
    // symmetric mode (Galerkin: targets = sources, same coordinates): the plan
    // of launch_pair_tc_sym, whose scratch is `scratch`; null for the dense
    // product
    const TcSymPlan* sym;
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
    // symmetric mode only: per tile {first unit, chunks per unit} (one entry
    // more than tiles, global unit numbering), the launch's first unit and
    // tile range [sym_tile0, sym_tile1) and the band's transposed partial
    // sums (chunk-major within the band)
    const int2* sym_tab;
    float* part2;
    int64_t sym_unit_begin;
    int sym_tile0, sym_tile1;
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

// Symmetric pairwise product (Galerkin form: Gamma over one point set is
// symmetric, Sec. 3.1). Tiles of 128 points, chunks of 64: tile I takes the
// source chunks from its own first chunk 2I onwards; each kernel tile of a
// chunk c >= 2I + 2 is evaluated once and applied twice, W_I += Gamma_Ic X_c
// and W_c += Gamma_Ic^T X_I. Split BF16 and at most 16 vectors per product.
// The work units of a tile (chunk ranges of cps chunks each) are numbered
// tile after tile; tiles are grouped into bands whose transposed partial
// sums fit a fixed cap, one launch and one reduction per band.
struct TcSymPlan {
    int64_t T = 0, nchunks = 0;
    int nt = 0, kcap = 0, sm_count = 0;
    std::vector<int2> tab;      // per tile {first unit, cps}; tab[nt] = {units, 0}
    std::vector<int> band;      // band boundaries in tiles (bands + 1 entries)
    int64_t max_band_units = 0;
    int64_t max_band_p2 = 0;    // transposed partial sums of the largest band (floats, kcap columns)
    // scratch layout (doubles from the start of the scratch)
    int64_t off_img = 0, off_tab = 0, off_part1 = 0, off_part2 = 0, off_acc = 0, total = 0;
};
// Whether the symmetric product applies to T points and blocks of k vectors.
bool tc_sym_eligible(int64_t T, int k, bool tf32);
// Plan for blocks of at most kcap vectors (kcap <= 16).
TcSymPlan tc_sym_plan(int64_t T, int kcap, int sm_count);
// Copies the unit table into the scratch (synchronous; before any capture).
cudaError_t tc_sym_upload(const TcSymPlan& p, double* scratch, cudaStream_t s);
// Conversion, one tcgen05 launch and one ordered reduction per band.
cudaError_t launch_pair_tc_sym(const TcArgs& a, cudaStream_t s, int* launched);

// Reduction of split partials shared with the CUDA-core kernels.
cudaError_t launch_pair_reduce(const double* part, int splits, int64_t T, int k, double sigma2,
                               const double* post, double* Y, int64_t ldy, cudaStream_t s);

}  // namespace kl
