// Pairwise product W = Gamma X on the tcgen05 tensor cores (sm_100 family).
//
// The O(N~^2) step of the IBQ-Galerkin matvec (Sec. 3.1) and the kernel
// product of Algorithm 1 in the collocation matvec (Sec. 3.2), with Gamma
// never stored:
//
//   * A CTA owns 128 target points; target t is tensor-memory lane t. Eight
//     producer warps (two warpgroups, warp w serving lanes 32*(w%4)..) share
//     every chunk of 64 (BF16) or 32 (TF32) sources, each warpgroup one half;
//     each thread evaluates Gamma(x_t, y_j) for its sources in FP32
//     registers, splits every value into a high and a low part (BF16 + BF16
//     or TF32 + TF32) and writes both straight into tensor memory with
//     tcgen05.st: the kernel tile becomes the A operand of the MMA without
//     passing through shared memory. Two tiles alternate, so the producers
//     fill one while the tensor core reads the other.
//   * The source values X (FP64 in HBM) are converted once per application
//     into the same hi/lo split, laid out as K-major no-swizzle core matrices
//     (8 rows x 16 bytes) chunk by chunk together with the chunk's source
//     coordinates; a loader warp streams the chunk records into a shared
//     memory ring (up to 16 stages) with bulk copies. They are the B operand.
//   * One thread of a ninth warp issues, per chunk and K step,
//     D += A_hi B_hi + A_hi B_lo + A_lo B_hi  (tcgen05.mma, FP32 accumulator
//     D in tensor memory, M = 128, N = k rounded up to 16; for N = 16 two
//     MMAs with a combined [hi | lo] B operand), and tcgen05.commit releases
//     the stage when the tensor core has read it.
//   * The FP32 accumulator is double-buffered in tensor memory and restarted
//     every kGroup chunks: both warpgroups read the finished buffer with
//     tcgen05.ld (half of the columns each) and fold it into (hi, lo) FP32
//     running sums of their rows by an error-free two-sum while the tensor
//     core fills the other buffer. Long FP32 accumulations on the tensor
//     core drift (the error grows linearly with their length); the fold
//     bounds every FP32 sum to kGroup chunks.
//   * The partial sums of each source split are reduced by a second kernel in
//     a fixed order, which also applies sigma^2 and the per-target scale.
//   * Coordinates are pre-scaled so that the kernel argument needs no
//     multiplication (see gamma_scaled), and the hi/lo splits cost three
//     (BF16) or two (TF32) instructions per value.
//
// Every mbarrier wait is bounded by a clock limit (about a second, or the
// launch's wait_limit); on timeout the kernel records an error flag. Before
// the tensor memory is freed the issuing thread always waits (bounded by the
// default limit) for every MMA it issued, and the loader for every copy it
// issued, so that a short limit ends the kernel early but never frees memory
// still in use.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <mutex>
#include <type_traits>

#include "kernel_eval.cuh"
#include "kernels_tc.h"

namespace kl {

namespace {

constexpr int kStages = 2;                // TMEM A-operand ring (kernel tiles of one chunk)
constexpr int kProducers = 256;           // two warpgroups
constexpr int kThreads = kProducers + 64; // + MMA warp + loader warp
constexpr int kTmemCols = 256;
constexpr int kAColsPerStage = 64;        // hi 32 + lo 32 columns (64 BF16 / 32 TF32 sources)
constexpr int kKSteps = 4;                // MMA K steps per chunk (K = 16 BF16 / 8 TF32 each)
constexpr int kGroup = 8;                 // chunks accumulated in FP32 before a fold
                                          // (512 BF16 / 256 TF32 sources; measured on
                                          // GB300: 4% faster than 4 chunks, relative
                                          // error 1.8e-6 against 1.4e-6, while 16 chunks
                                          // let single columns reach 1.8e-5)
constexpr int kFlushLag = 2;              // chunks between a group's end and its fold
// Tensor memory of a CTA (256 columns): two accumulator buffers (32 columns
// each for N <= 32, else 64); for N <= 32 the running (hi, lo) sums of the
// unit (2N columns); then the 2-slot ring of kernel tiles (64 columns each).
template <int NP>
struct TmemLayout {
    static constexpr bool kSum = NP <= 32;             // running sums in TMEM
    static constexpr int kDStride = NP <= 32 ? 32 : 64;
    static constexpr int kSBase = 2 * kDStride;
    static constexpr int kAColBase = kSum ? kSBase + (2 * NP + 31) / 32 * 32 : 2 * kDStride;
    static_assert(kAColBase + kStages * kAColsPerStage <= kTmemCols, "tensor memory overflow");
};
constexpr long long kWaitLimit = 2000000000LL;  // clock cycles (~1 s): the default pipeline limit
                                                // and always the limit of the final drains

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait on the phase with the given parity. False on timeout. Each
// try_wait lets the thread sleep in hardware until the phase completes (at
// most the 1 ms hint), so waiting warps take no issue slots from producing
// ones (polling cost 5 % of the pairwise kernel's time).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit) {
    const uint32_t a = smem_u32(bar);
    // suspend hint (ns): 1 ms under the default limit, about half the limit
    // under a short one, so that the limit, not the hint, ends the wait
    const uint32_t hint = limit >= 2000000LL ? 1000000u : uint32_t(limit / 4 + 16);
    uint32_t ready;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ready)
        : "r"(a), "r"(parity)
        : "memory");
    if (ready) return true;
    const long long t0 = clock64();
    while (true) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(a), "r"(parity), "r"(hint)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > limit) return false;
    }
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor, K-major, no swizzle: start address,
// leading byte offset (stride between core matrices along K), stride byte
// offset (between 8-row groups along M/N), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= uint64_t((addr >> 4) & 0x3FFFu);
    d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;
    d |= uint64_t((sbo >> 4) & 0x3FFFu) << 32;
    d |= uint64_t(1) << 46;
    return d;
}

// Instruction descriptor: dense, D = F32, A = B = BF16 (1) or TF32 (2),
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t instr_desc(int n, bool tf32) {
    return (1u << 4) | ((tf32 ? 2u : 1u) << 7) | ((tf32 ? 2u : 1u) << 10) |
           (uint32_t(n >> 3) << 17) | (uint32_t(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_tmemA(bool tf32, uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc,
                                          uint32_t idesc, uint32_t accumulate) {
    if (tf32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
            "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
            "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
            : "memory");
    }
}

// Instruction descriptor of the transposed product of the symmetric mode:
// dense, D = F32, A = B = BF16, A MN-major (transposed, bit 15), B K-major,
// N >> 3 at bit 17, M = 64 (M >> 4 at bit 24).
__host__ __device__ constexpr uint32_t instr_desc_t64(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (uint32_t(n >> 3) << 17) | (uint32_t(64 >> 4) << 24);
}

// D (tensor memory) += A B with both operands in shared memory (BF16).
__device__ __forceinline__ void mma_smemA(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void st_global_v4(float* p, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.global.v4.b32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

__device__ __forceinline__ void st_shared_v4(void* p, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(smem_u32(p)), "r"(a), "r"(b), "r"(c), "r"(d)
                 : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]),
        "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t* v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                 "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* v) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ uint32_t tf32_rna(float x) {
    uint32_t y;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(y) : "f"(x));
    return y;
}

// Two K-adjacent values -> packed BF16 pair (even K in the low half).
__device__ __forceinline__ uint32_t cvt_bf16x2(float even_k, float odd_k) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(odd_k), "f"(even_k));
    return r;
}

// Packed FP32 pairs (sm_100 f32x2 arithmetic: one instruction, two values;
// the first value in the low half).
__device__ __forceinline__ uint64_t pk2(float a, float b) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void up2(uint64_t v, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ uint64_t f2sub(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t f2mul(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t f2fma(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// Split (g0, g1) into packed hi and lo BF16 pairs with g ~ hi + lo.
__device__ __forceinline__ void split_bf16(float g0, float g1, uint32_t& hi, uint32_t& lo) {
    hi = cvt_bf16x2(g0, g1);
    const uint64_t h = pk2(__uint_as_float(hi << 16), __uint_as_float(hi & 0xffff0000u));
    float l0, l1;
    up2(f2sub(pk2(g0, g1), h), l0, l1);
    lo = cvt_bf16x2(l0, l1);
}

// Split (g0, g1) into hi (mantissa truncated to the 10 bits a TF32 operand
// keeps) and lo = g - hi (exact in FP32; the tensor core uses its leading 10
// bits).
__device__ __forceinline__ void split_tf32(float g0, float g1, uint32_t& hi0, uint32_t& hi1, uint32_t& lo0,
                                           uint32_t& lo1) {
    hi0 = __float_as_uint(g0) & 0xffffe000u;
    hi1 = __float_as_uint(g1) & 0xffffe000u;
    float l0, l1;
    up2(f2sub(pk2(g0, g1), pk2(__uint_as_float(hi0), __uint_as_float(hi1))), l0, l1);
    lo0 = __float_as_uint(l0);
    lo1 = __float_as_uint(l1);
}

// Kernel value without sigma^2 from pre-scaled coordinate differences: the
// conversion multiplies every coordinate by c (c^2 = a log2(e) for the
// Gaussian, c = a log2(e) otherwise), so the base-2 exponent is a plain sum.
template <int KIND>
__device__ __forceinline__ float gamma_scaled(float dx, float dy, float dz) {
    if (KIND == KL_KERNEL_GAUSS) return ex2_approx(-fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
    if (KIND == KL_KERNEL_EXP_SEP) return ex2_approx(-(fabsf(dx) + fabsf(dy) + fabsf(dz)));
    if (KIND == KL_KERNEL_EXP) return ex2_approx(-sqrt_approx(fmaf(dx, dx, fmaf(dy, dy, dz * dz))));
    if (KIND == KL_KERNEL_MATERN32) {
        // a r = r' ln 2 with r' = a log2(e) r
        const float r = sqrt_approx(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
        return fmaf(0.69314718055994531f, r, 1.0f) * ex2_approx(-r);
    }
    return 1.0f;
}

// Two kernel values from packed pre-scaled differences (dx0, dx1), ...
template <int KIND>
__device__ __forceinline__ void gamma2(uint64_t dx, uint64_t dy, uint64_t dz, float& g0, float& g1) {
    if (KIND == KL_KERNEL_EXP_SEP) {
        float x0, x1, y0, y1, z0, z1;
        up2(dx, x0, x1);
        up2(dy, y0, y1);
        up2(dz, z0, z1);
        g0 = ex2_approx(-(fabsf(x0) + fabsf(y0) + fabsf(z0)));
        g1 = ex2_approx(-(fabsf(x1) + fabsf(y1) + fabsf(z1)));
        return;
    }
    if (KIND == KL_KERNEL_CONST) {
        g0 = g1 = 1.0f;
        return;
    }
    float r0, r1;
    up2(f2fma(dz, dz, f2fma(dy, dy, f2mul(dx, dx))), r0, r1);
    if (KIND == KL_KERNEL_GAUSS) {
        g0 = ex2_approx(-r0);
        g1 = ex2_approx(-r1);
        return;
    }
    r0 = sqrt_approx(r0);
    r1 = sqrt_approx(r1);
    if (KIND == KL_KERNEL_EXP) {
        g0 = ex2_approx(-r0);
        g1 = ex2_approx(-r1);
        return;
    }
    // Matern-3/2: a r = r' ln 2 with r' = a log2(e) r
    g0 = fmaf(0.69314718055994531f, r0, 1.0f) * ex2_approx(-r0);
    g1 = fmaf(0.69314718055994531f, r1, 1.0f) * ex2_approx(-r1);
}

// Kernel kind chosen per work unit at run time (batched launches of several
// problems); other values of KIND fix it at compile time.
constexpr int kKindAny = -1;
template <int KIND>
__device__ __forceinline__ void gamma2_k(int kind, uint64_t dx, uint64_t dy, uint64_t dz, float& g0, float& g1) {
    if (KIND != kKindAny) {
        gamma2<(KIND == kKindAny ? KL_KERNEL_CONST : KIND)>(dx, dy, dz, g0, g1);
        return;
    }
    switch (kind) {
        case KL_KERNEL_GAUSS: gamma2<KL_KERNEL_GAUSS>(dx, dy, dz, g0, g1); break;
        case KL_KERNEL_EXP_SEP: gamma2<KL_KERNEL_EXP_SEP>(dx, dy, dz, g0, g1); break;
        case KL_KERNEL_EXP: gamma2<KL_KERNEL_EXP>(dx, dy, dz, g0, g1); break;
        case KL_KERNEL_MATERN32: gamma2<KL_KERNEL_MATERN32>(dx, dy, dz, g0, g1); break;
        default: gamma2<KL_KERNEL_CONST>(dx, dy, dz, g0, g1); break;
    }
}

// Coordinate scale c of gamma_scaled: the argument a r^2 log2(e) (Gaussian) or
// a r log2(e) (exponentials, Matern) becomes |c x - c y|^2 or |c x - c y|.
float coord_scale(const KernelSpec& ks) {
    const double l2e = 1.4426950408889634074;
    if (ks.kind == KL_KERNEL_GAUSS) return float(std::sqrt(ks.a * l2e));
    if (ks.kind == KL_KERNEL_CONST) return 1.0f;
    return float(ks.a * l2e);
}

// Depth of the shared-memory stage ring: the largest power of two (16 at
// most, 4 at least) whose stages fit in ~100 KB (two CTAs per SM). Powers of
// two keep the ring arithmetic to shifts and masks.
__host__ __device__ constexpr int smem_stages(int stage_bytes) {
    return (99 * 1024) / stage_bytes >= 16 ? 16 : (99 * 1024) / stage_bytes >= 8 ? 8 : 4;
}

// Byte offset of element (n, kk) inside one hi or lo image of a chunk:
// K steps of 32 bytes per row, each made of two 8x16-byte core matrices
// along K; np/8 core matrices along N. esize = 2 (BF16) or 4 (TF32).
__host__ __device__ inline uint32_t img_offset(int n, int kk, int np, int esize) {
    const int per_core = 16 / esize;   // K elements per core-matrix row
    const int per_step = 32 / esize;   // K elements per MMA
    const int ks = kk / per_step, rem = kk % per_step;
    const int kb = rem / per_core, e = rem % per_core;
    const int nb = n / 8, r = n % 8;
    return uint32_t(((ks * 2 + kb) * (np / 8) + nb) * 128 + r * 16 + e * esize);
}

// BF16 products with N = 16 use one combined image per chunk: rows 0..15 the
// hi part and rows 16..31 the lo part of X, so that one MMA of N = 32 forms
// A_hi [X_hi | X_lo] and a second of N = 16 (the first 16 rows) adds A_lo X_hi
// into the first half: four MMAs per chunk instead of six. The issuing
// thread, not the tensor core, limits the pipeline at these shapes (an MMA
// of N <= 128 costs the same issue time whatever N is).
__host__ __device__ constexpr bool tc_concat(bool tf32, int np) { return !tf32 && np == 16; }

// X (FP64) -> split images + FP32 source coordinates, chunk by chunk. A chunk
// is one contiguous record [hi image | lo image | x[kchunk] y[kchunk]
// z[kchunk]] (the stage layout), so that one bulk copy loads it; with the
// combined layout the two images form one image of 2 np rows.
__global__ void tc_convert_kernel(const double* __restrict__ X, int64_t ldx, int64_t S, int c0, int kc,
                                  int np, int kchunk, bool tf32, float cscale, const float* __restrict__ sx,
                                  const float* __restrict__ sy, const float* __restrict__ sz,
                                  uint8_t* __restrict__ img, int64_t nchunks) {
    const int esize = tf32 ? 4 : 2;
    const int64_t img_bytes = int64_t(np) * kchunk * esize;  // one of hi / lo
    const int64_t rec_bytes = 2 * img_bytes + 12 * int64_t(kchunk);
    const int64_t total = nchunks * kchunk * np;
    for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
         t += int64_t(gridDim.x) * blockDim.x) {
        const int n = int(t % np);
        const int64_t s = t / np;
        const int64_t ch = s / kchunk;
        const int kk = int(s % kchunk);
        const float v = (s < S && n < kc) ? float(X[s + int64_t(c0 + n) * ldx]) : 0.f;
        uint8_t* base = img + ch * rec_bytes;
        const uint32_t off = img_offset(n, kk, np, esize);
        if (tc_concat(tf32, np)) {
            const __nv_bfloat16 h = __float2bfloat16_rn(v);
            const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
            *reinterpret_cast<__nv_bfloat16*>(base + img_offset(n, kk, 2 * np, esize)) = h;
            *reinterpret_cast<__nv_bfloat16*>(base + img_offset(np + n, kk, 2 * np, esize)) = l;
        } else if (tf32) {
            const uint32_t hi = tf32_rna(v);
            const uint32_t lo = tf32_rna(v - __uint_as_float(hi));
            *reinterpret_cast<uint32_t*>(base + off) = hi;
            *reinterpret_cast<uint32_t*>(base + img_bytes + off) = lo;
        } else {
            const __nv_bfloat16 h = __float2bfloat16_rn(v);
            const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
            *reinterpret_cast<__nv_bfloat16*>(base + off) = h;
            *reinterpret_cast<__nv_bfloat16*>(base + img_bytes + off) = l;
        }
        if (n == 0) {
            // chunk-wise structure of arrays: x[kchunk], y[kchunk], z[kchunk]
            float* c = reinterpret_cast<float*>(base + 2 * img_bytes) + kk;
            c[0] = s < S ? cscale * sx[s] : 0.f;
            c[kchunk] = s < S ? cscale * sy[s] : 0.f;
            c[2 * kchunk] = s < S ? cscale * sz[s] : 0.f;
        }
    }
}

// Bulk asynchronous copy global -> shared memory, completion counted in bytes
// on an mbarrier (both addresses 16-byte aligned, size a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// Bounded wait by every lane of a warp, then a warp-uniform verdict.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, long long limit) {
    const bool ok = mbar_wait(bar, parity, limit);
    return __all_sync(0xffffffffu, ok);
}

// Work unit u of the persistent schedule: target tile u / splits, source
// chunk range [c0, c1) of split u % splits.
struct Unit {
    int64_t tile;
    int split;
    int64_t c0;
    int nloc;
};
__device__ __forceinline__ Unit unit_of(int64_t u, int splits, int64_t nchunks, int cps) {
    Unit r;
    r.tile = u / splits;
    r.split = int(u % splits);
    r.c0 = int64_t(r.split) * cps;
    const int64_t left = nchunks - r.c0;
    r.nloc = int(left < cps ? left : int64_t(cps));
    return r;
}

// Instance of global work unit u (units are assigned contiguously).
__device__ __forceinline__ int inst_of(const TcBatch& b, int64_t u) {
    int p = 0;
    while (p + 1 < b.ninst && b.inst[p + 1].unit0 <= u) ++p;
    return p;
}

// Symmetric mode: unit u of the launch (global unit sym_unit_begin + u) ->
// tile (binary search of the per-tile first units) and chunk range.
__device__ __forceinline__ Unit sym_unit_of(const TcInstance& I, int64_t u) {
    const int64_t g = I.sym_unit_begin + u;
    int lo = I.sym_tile0, hi = I.sym_tile1 - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (int64_t(I.sym_tab[mid].x) <= g) lo = mid;
        else hi = mid - 1;
    }
    Unit r;
    r.tile = lo;
    r.split = int(g - I.sym_tab[lo].x);
    const int cps = I.sym_tab[lo].y;
    r.c0 = 2 * int64_t(lo) + int64_t(r.split) * cps;
    const int64_t left = I.nchunks - r.c0;
    r.nloc = int(left < cps ? left : int64_t(cps));
    return r;
}

// Index of the transposed partial sum of tile I and chunk c >= 2I + 2 within
// the band of tiles [b0, b1), chunk by chunk and, within a chunk, tile by
// tile: the sums a chunk's reduction reads are contiguous. Chunk c' holds
// g(c' / 2) of them, g(m) = clamp(m, b0, b1) - b0 (the band's tiles I < c' / 2),
// and the sum of g(m) over m < M is G(M) = x (x - 1) / 2 + max(0, M - b1) (b1 - b0)
// with x = max(0, min(M, b1) - b0).
// Every term is below the band's block count (its transposed sums fit the
// band cap, or the band is one tile), so 32-bit arithmetic holds; the kernel
// evaluates this once per drained product.
__host__ __device__ __forceinline__ int sym_p2_index(int c, int I, int b0, int b1) {
    const int M = c >> 1;
    const int x = (M < b1 ? M : b1) - b0;
    const int G = x > 0 ? x * (x - 1) / 2 + (M > b1 ? (M - b1) * (b1 - b0) : 0) : 0;
    const int gM = (M < b0 ? b0 : M > b1 ? b1 : M) - b0;
    return 2 * G + ((c & 1) ? gM : 0) + (I - b0);
}

// Symmetric mode layout (split BF16, N = 16): shared memory holds the ring of
// kernel tiles of the transposed product (hi and lo image of 128 targets x
// 64 sources each, 16 KB), then the split images of X on the unit's own tile
// (two chunks, double-buffered across units), then the chunk-record ring.
constexpr int kSymGBytes = 32768;               // one kernel tile: hi + lo image
constexpr int kSymXBytes = 8192;                // X of one 128-point tile (two 4 KB images)
constexpr int kSymRecBase = 2 * kSymGBytes + 2 * kSymXBytes;
constexpr int kSymRecStages = 4;
constexpr int kSymDJ = 224;                     // TMEM columns of the transposed product's two
                                                // accumulators (16 columns each)
// Kernel tile image of the transposed product (MN-major: sources contiguous):
// 8 x 8 core matrices of 128 bytes, element (target t, source j) at
// (j / 8) * 2048 + (t / 8) * 128 + (t % 8) * 16 + (j % 8) * 2.
constexpr uint32_t kSymSrcGroupStride = 2048;   // along M (sources) of the transposed product
constexpr uint32_t kSymTgtGroupStride = 128;    // along K (targets)

template <int KIND, bool TF32, int NP, bool SYM>
__global__ void __launch_bounds__(kThreads, 2)
pair_tc_kernel(const __grid_constant__ TcBatch batch, int* __restrict__ err) {
    static_assert(!SYM || (!TF32 && NP == 16), "symmetric mode: split BF16, N = 16");
    const int64_t nunits = batch.nunits;
    const long long wlim = batch.wait_limit > 0 ? batch.wait_limit : kWaitLimit;
    constexpr int ESIZE = TF32 ? 4 : 2;
    constexpr int KC = TF32 ? 32 : 64;                  // sources per chunk (32 TMEM columns)
    constexpr int SW = KC / 2;                          // sources of each warpgroup
    constexpr int IMG = NP * KC * ESIZE;                // bytes of one of hi / lo
    constexpr int STAGE_BYTES = 2 * IMG + KC * 12;      // hi, lo, coordinates x[KC] y[KC] z[KC]
    constexpr int SSTAGES = SYM ? kSymRecStages : smem_stages(STAGE_BYTES);  // shared-memory ring (>= kStages)
    constexpr int REC_BASE = SYM ? kSymRecBase : 0;
    constexpr uint32_t IDESC = instr_desc(NP, TF32);
    constexpr bool kConcat = tc_concat(TF32, NP);
    constexpr uint32_t IDESC2 = instr_desc(2 * NP, TF32);  // combined [hi | lo] operand
    // transposed product: M = 64 sources, A (kernel tile) MN-major
    constexpr uint32_t IDESC_T = instr_desc_t64(NP);
    static_assert(!kConcat || 2 * NP <= TmemLayout<NP>::kDStride, "combined accumulator wider than its buffer");
    constexpr bool kSum = TmemLayout<NP>::kSum;
    constexpr int kDStride = TmemLayout<NP>::kDStride;
    constexpr int kSBase = TmemLayout<NP>::kSBase;
    constexpr int kAColBase = TmemLayout<NP>::kAColBase;
    static_assert(!SYM || (kAColBase + kStages * kAColsPerStage <= kSymDJ && kSymDJ + 2 * NP <= kTmemCols),
                  "symmetric mode: tensor memory overflow");

    extern __shared__ __align__(1024) uint8_t smem[];
    // loaded/sempty: shared-memory ring (bulk copies ahead of use);
    // full/tfree: TMEM ring of kernel tiles; dfull/dfree: accumulators;
    // symmetric mode: gfree (shared-memory kernel tiles read), d2full/d2free
    // (transposed accumulator), xload/xfree (X of the unit's tile)
    __shared__ uint64_t loaded_bar[SSTAGES], sempty_bar[SSTAGES], full_bar[kStages], tfree_bar[kStages];
    __shared__ uint64_t dfull_bar[2], dfree_bar[2], drain_bar;
    __shared__ uint64_t gfree_bar[2], d2full_bar[2], d2free_bar[2], xload_bar[2], xfree_bar[2];
    __shared__ uint32_t tmem_slot;

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int s = 0; s < SSTAGES; ++s) {
            mbar_init(&loaded_bar[s], 1);
            mbar_init(&sempty_bar[s], 1);
        }
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full_bar[s], 256);  // both warpgroups write half of every tile
            mbar_init(&tfree_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&dfull_bar[b], 1);
            mbar_init(&dfree_bar[b], 256);  // both warpgroups fold half of the columns
            mbar_init(&gfree_bar[b], 1);
            mbar_init(&xload_bar[b], 1);
            mbar_init(&xfree_bar[b], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&d2full_bar[b], 1);
            mbar_init(&d2free_bar[b], 256);
        }
        mbar_init(&drain_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 8) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp < 8) {
        // ---------------- producers (two warpgroups, half of each chunk) ----------------
        const int wg = warp >> 2;
        const int ptid = tid & 127;
        const uint32_t lane_base = uint32_t((warp & 3) * 32) << 16;
        bool ok = true;
        uint32_t jbase = 0;  // chunks of earlier units (stage ring position)
        uint32_t gbase = 0;  // accumulator groups of earlier units
        uint32_t og = 0;     // symmetric mode: transposed products so far
        uint32_t drained = 0;  // symmetric mode: transposed products drained so far
        for (int64_t u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
            const TcInstance& I = batch.inst[SYM ? 0 : inst_of(batch, u)];
            const Unit un = SYM ? sym_unit_of(I, u) : unit_of(u - I.unit0, I.splits, I.nchunks, I.cps);
            const int64_t T = I.T;
            const float cscale = I.cscale;
            const int kc = I.kc;
            const float *tx = I.tx, *ty = I.ty, *tz = I.tz;
            const int64_t t = un.tile * 128 + ptid;
            const float px = t < T ? cscale * tx[t] : 0.f;
            const float py = t < T ? cscale * ty[t] : 0.f;
            const float pz = t < T ? cscale * tz[t] : 0.f;
            const uint64_t ppx = pk2(px, px), ppy = pk2(py, py), ppz = pk2(pz, pz);
            // partial sums of this unit: by source split (dense) or by unit
            // of the band (symmetric, 128 rows per unit and column)
            float2* prow = SYM ? I.part + (u * I.k_total + I.c0) * 128 + ptid
                               : I.part + (int64_t(un.split) * I.k_total + I.c0) * T + t;
            const int64_t pstride = SYM ? 128 : T;
            const int kind = I.kind;
            const int ngroups = (un.nloc + kGroup - 1) / kGroup;
            int flushed = 0;
            // Both warpgroups fold the finished accumulator of local group g
            // (warpgroup w the columns [w NP/2, (w+1) NP/2)) into the unit's
            // running sums of the rows owned by the thread, as FP32 (hi, lo)
            // pairs: an error-free two-sum of hi and the group's sum, its error
            // added into lo (about 48 significant bits at FP32 instruction
            // cost). For N <= 32 the running sums stay in tensor memory and
            // the last group writes them to the partial-sum array; otherwise
            // every group updates that array in global memory. With the
            // combined operand the group's sum is the sum of its two halves.
            auto flush = [&](int g, bool last) {
                const uint32_t gg = gbase + uint32_t(g);
                const bool got = ok && warp_wait(&dfull_bar[gg & 1], uint32_t((gg >> 1) & 1), wlim);
                if (!got) ok = false;
                tc_fence_after();
                const uint32_t dcol = uint32_t((gg & 1) * kDStride);
#pragma unroll 1
                for (int cb = wg * (NP / 2); cb < (wg + 1) * (NP / 2); cb += 8) {
                    uint32_t v[8], h[8], l[8];
                    __syncwarp();
                    tmem_ld8(tmem + lane_base + dcol + uint32_t(cb), v);
                    if (kConcat) {
                        uint32_t v2[8];
                        tmem_ld8(tmem + lane_base + dcol + uint32_t(NP + cb), v2);
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            v[q] = __float_as_uint(__fadd_rn(__uint_as_float(v[q]), __uint_as_float(v2[q])));
                    }
                    if (kSum && g > 0) {
                        tmem_ld8(tmem + lane_base + uint32_t(kSBase + cb), h);
                        tmem_ld8(tmem + lane_base + uint32_t(kSBase + NP + cb), l);
                    }
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const float x = __uint_as_float(v[q]);
                        float hs = x, ls = 0.f;
                        if (kSum) {
                            if (g > 0) {
                                const float o = __uint_as_float(h[q]);
                                hs = __fadd_rn(o, x);
                                const float bb = __fsub_rn(hs, o);
                                const float er = __fadd_rn(__fsub_rn(o, __fsub_rn(hs, bb)), __fsub_rn(x, bb));
                                ls = __fadd_rn(__uint_as_float(l[q]), er);
                            }
                        } else if (g > 0 && got && t < T && cb + q < kc) {
                            const float2 o = prow[int64_t(cb + q) * pstride];
                            hs = __fadd_rn(o.x, x);
                            const float bb = __fsub_rn(hs, o.x);
                            const float er = __fadd_rn(__fsub_rn(o.x, __fsub_rn(hs, bb)), __fsub_rn(x, bb));
                            ls = __fadd_rn(o.y, er);
                        }
                        h[q] = __float_as_uint(hs);
                        l[q] = __float_as_uint(ls);
                    }
                    if (kSum && !last) {
                        tmem_st8(tmem + lane_base + uint32_t(kSBase + cb), h);
                        tmem_st8(tmem + lane_base + uint32_t(kSBase + NP + cb), l);
                    } else if (got && t < T) {
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            if (cb + q < kc)
                                prow[int64_t(cb + q) * pstride] =
                                    make_float2(__uint_as_float(h[q]), __uint_as_float(l[q]));
                    }
                }
                if (kSum && !last) asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                tc_fence_before();
                mbar_arrive(&dfree_bar[gg & 1]);
            };
            // Symmetric mode: both warpgroups read the finished transposed
            // accumulator of product m (buffer m & 1; M = 64 rows: row 16 q + l
            // in lane l < 16 of the lane quarter q; warpgroup w the columns
            // [8 w, 8 w + 8)) and store it as the FP32 partial sum of the 64
            // sources of its chunk ch.
            auto drain = [&](int64_t ch, uint32_t m) {
                const int64_t p2 = sym_p2_index(int(ch), int(un.tile), I.sym_tile0, I.sym_tile1);
                const bool got = ok && warp_wait(&d2full_bar[m & 1], (m >> 1) & 1u, wlim);
                if (!got) ok = false;
                tc_fence_after();
                const int cb = wg * (NP / 2);
                uint32_t v[8];
                __syncwarp();
                tmem_ld8(tmem + lane_base + uint32_t(kSymDJ + NP * int(m & 1) + cb), v);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                // rows of kstride (k rounded up to 8) floats: two 16-byte
                // stores per row and warpgroup
                const int kstride = (I.k_total + 7) & ~7;
                if (got && lane < 16 && cb < kstride) {
                    const int row = (warp & 3) * 16 + lane;
                    float* dst = I.part2 + (p2 * 64 + row) * kstride + cb;
                    st_global_v4(dst, v[0], v[1], v[2], v[3]);
                    st_global_v4(dst + 4, v[4], v[5], v[6], v[7]);
                }
                tc_fence_before();
                mbar_arrive(&d2free_bar[m & 1]);
            };
            const int first_offd = SYM ? int(2 * un.tile + 2 - un.c0) : un.nloc;  // local index
            // One chunk: wait for its record and a free kernel-tile stage,
            // evaluate, split, store into tensor memory (and, for a transposed
            // product, into the shared-memory tile), arrive. OFFD is fixed per
            // loop so that neither path tests it per source.
            auto chunk_step = [&](int jl, auto offd_tag) -> bool {
                constexpr bool OFFD = decltype(offd_tag)::value;
                // group g is folded kFlushLag chunks after it ends, when the
                // tensor core has long finished it (never the last group of
                // the unit here)
                while (ok && jl >= kFlushLag && flushed < (jl - kFlushLag) / kGroup) {
                    flush(flushed, false);
                    ++flushed;
                }
                if (!ok) return false;
                const uint32_t jg = jbase + uint32_t(jl);
                const int ss = int(jg % SSTAGES), s = int(jg % kStages);
                if (!warp_wait(&loaded_bar[ss], uint32_t((jg / SSTAGES) & 1), wlim)) return false;
                if (jg >= kStages && !warp_wait(&tfree_bar[s], uint32_t(((jg / kStages) - 1) & 1), wlim)) return false;
                if (OFFD && og >= 2 && !warp_wait(&gfree_bar[og & 1], ((og >> 1) - 1) & 1u, wlim)) return false;
                const float* cx = reinterpret_cast<const float*>(smem + REC_BASE + ss * STAGE_BYTES + 2 * IMG) + wg * SW;
                const uint32_t acol = uint32_t(kAColBase + s * kAColsPerStage);
                // this thread's 16-byte rows of the shared-memory kernel tile
                // (target ptid; sources wg SW + 16 half + 0..15)
                uint8_t* grow = smem + (og & 1) * kSymGBytes + (wg * SW / 8) * kSymSrcGroupStride +
                                (ptid / 8) * kSymTgtGroupStride + (ptid % 8) * 16;
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    // 16 (BF16) or 8 (TF32) sources: four per 16-byte load of
                    // each coordinate, differences and squares two at a time
                    uint32_t hi[8], lo[8];
#pragma unroll
                    for (int q4 = 0; q4 < (TF32 ? 2 : 4); ++q4) {
                        const int j0 = (SW / 2) * half + 4 * q4;
                        const ulonglong2 xv = *reinterpret_cast<const ulonglong2*>(cx + j0);
                        const ulonglong2 yv = *reinterpret_cast<const ulonglong2*>(cx + KC + j0);
                        const ulonglong2 zv = *reinterpret_cast<const ulonglong2*>(cx + 2 * KC + j0);
                        float g0, g1, g2, g3;
                        gamma2_k<KIND>(kind, f2sub(ppx, xv.x), f2sub(ppy, yv.x), f2sub(ppz, zv.x), g0, g1);
                        gamma2_k<KIND>(kind, f2sub(ppx, xv.y), f2sub(ppy, yv.y), f2sub(ppz, zv.y), g2, g3);
                        if (TF32) {
                            split_tf32(g0, g1, hi[4 * q4], hi[4 * q4 + 1], lo[4 * q4], lo[4 * q4 + 1]);
                            split_tf32(g2, g3, hi[4 * q4 + 2], hi[4 * q4 + 3], lo[4 * q4 + 2], lo[4 * q4 + 3]);
                        } else {
                            split_bf16(g0, g1, hi[2 * q4], lo[2 * q4]);
                            split_bf16(g2, g3, hi[2 * q4 + 1], lo[2 * q4 + 1]);
                        }
                    }
                    __syncwarp();
                    tmem_st8(tmem + lane_base + acol + uint32_t(16 * wg + 8 * half), hi);
                    tmem_st8(tmem + lane_base + acol + 32u + uint32_t(16 * wg + 8 * half), lo);
                    if (OFFD) {
                        uint8_t* gr = grow + half * 2 * kSymSrcGroupStride;
                        st_shared_v4(gr, hi[0], hi[1], hi[2], hi[3]);
                        st_shared_v4(gr + kSymSrcGroupStride, hi[4], hi[5], hi[6], hi[7]);
                        st_shared_v4(gr + kSymGBytes / 2, lo[0], lo[1], lo[2], lo[3]);
                        st_shared_v4(gr + kSymGBytes / 2 + kSymSrcGroupStride, lo[4], lo[5], lo[6], lo[7]);
                    }
                }
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                // generic-proxy stores to shared memory become visible to the
                // tensor core (async proxy) before the arrival
                if (OFFD) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                tc_fence_before();
                mbar_arrive(&full_bar[s]);
                if (OFFD) {
                    // transposed products are drained two behind: product
                    // og - 2 has long finished, and its buffer is the one the
                    // next product needs
                    if (og >= drained + 2) {
                        drain(un.c0 + (jl - 2), drained);
                        ++drained;
                    }
                    ++og;
                }
                return true;
            };
            const int ndiag = first_offd < 0 ? 0 : (first_offd > un.nloc ? un.nloc : first_offd);
            int jl = 0;
            for (; jl < ndiag && ok; ++jl)
                if (!chunk_step(jl, std::false_type{})) ok = false;
            if constexpr (SYM) {
                for (; jl < un.nloc && ok; ++jl)
                    if (!chunk_step(jl, std::true_type{})) ok = false;
                // the unit's last (up to two) transposed products
                while (ok && drained < og) {
                    drain(un.c0 + (un.nloc - int(og - drained)), drained);
                    ++drained;
                }
            }
            while (ok && flushed < ngroups) {
                flush(flushed, flushed == ngroups - 1);
                ++flushed;
            }
            jbase += un.nloc;
            gbase += ngroups;
        }
        if (!ok && lane == 0) atomicExch(err, 1);
    } else if (warp == 8) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            bool ok = true;
            uint32_t jbase = 0, gbase = 0, og = 0, xu = 0;
            // B descriptors: stage ss, K step ks is the stage-0 descriptor plus
            // (ss * STAGE_BYTES + K-step offset) / 16 in its 14-bit start
            // address field (shared memory ends below 256 KB, so the field never
            // carries); the issuing thread, which shares its issue slots with
            // producer warps, then spends one add per MMA on addresses
            constexpr uint32_t kLbo = (kConcat ? 2 * NP : NP) / 8 * 128;
            constexpr uint32_t kStep = 2 * kLbo;  // bytes of one K step of one image
            const uint64_t bdesc0 = smem_desc(smem_u32(smem + REC_BASE), kLbo, 128);
            // symmetric mode: kernel tiles of the transposed product (MN-major:
            // leading byte offset along K = targets, stride byte offset along
            // M = sources) and the split images of X on the unit's tile (the
            // chunk-record layout, K = the tile's 128 points in 8 steps)
            const uint64_t gdesc0 = smem_desc(smem_u32(smem), kSymTgtGroupStride, kSymSrcGroupStride);
            const uint64_t xdesc0 = smem_desc(smem_u32(smem + 2 * kSymGBytes), kLbo, 128);
            for (int64_t u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
                const TcInstance& I = batch.inst[SYM ? 0 : inst_of(batch, u)];
                const Unit un = SYM ? sym_unit_of(I, u) : unit_of(u - I.unit0, I.splits, I.nchunks, I.cps);
                const int64_t first_offd = 2 * un.tile + 2;  // first chunk with a transposed product
                const bool unit_offd = SYM && un.c0 + un.nloc > first_offd;
                const uint32_t xb = xu & 1u;
                bool xwaited = false;
                for (int jl = 0; jl < un.nloc; ++jl) {
                    const uint32_t jg = jbase + uint32_t(jl);
                    const int s = int(jg % kStages), ss = int(jg % SSTAGES);
                    const uint32_t gg = gbase + uint32_t(jl / kGroup);
                    const bool first = (jl % kGroup) == 0;
                    const uint32_t d_tmem = tmem + uint32_t((gg & 1) * kDStride);
                    if (first && gg >= 2 && !mbar_wait(&dfree_bar[gg & 1], uint32_t(((gg >> 1) - 1) & 1), wlim)) { ok = false; break; }
                    if (!mbar_wait(&full_bar[s], uint32_t((jg / kStages) & 1), wlim)) { ok = false; break; }
                    tc_fence_after();
                    const uint64_t bst = bdesc0 + uint64_t(uint32_t(ss * STAGE_BYTES) >> 4);
                    const uint32_t acol = tmem + uint32_t(kAColBase + s * kAColsPerStage);
#pragma unroll
                    for (int ks = 0; ks < kKSteps; ++ks) {
                        const uint32_t ah = acol + uint32_t(ks * 8), al = acol + 32u + uint32_t(ks * 8);
                        if (kConcat) {
                            // rows 0..2NP-1 of the combined image: [X_hi | X_lo];
                            // its first NP rows: X_hi
                            const uint64_t bb = bst + uint64_t((ks * kStep) >> 4);
                            mma_tmemA(TF32, d_tmem, ah, bb, IDESC2, (first && ks == 0) ? 0u : 1u);
                            mma_tmemA(TF32, d_tmem, al, bb, IDESC, 1u);
                        } else {
                            const uint64_t bh = bst + uint64_t((ks * kStep) >> 4);
                            const uint64_t bl = bst + uint64_t((IMG + ks * kStep) >> 4);
                            mma_tmemA(TF32, d_tmem, ah, bh, IDESC, (first && ks == 0) ? 0u : 1u);
                            mma_tmemA(TF32, d_tmem, ah, bl, IDESC, 1u);
                            mma_tmemA(TF32, d_tmem, al, bh, IDESC, 1u);
                        }
                    }
                    mma_commit(&sempty_bar[ss]);
                    mma_commit(&tfree_bar[s]);
                    if ((jl % kGroup) == kGroup - 1 || jl == un.nloc - 1) mma_commit(&dfull_bar[gg & 1]);
                    if (SYM && un.c0 + jl >= first_offd) {
                        // transposed product m into accumulator m & 1:
                        // D_c = Gamma^T X_hi (hi and lo tiles) + Gamma_hi^T X_lo
                        // of the unit's tile, M = 64 sources, K = 128 targets
                        const uint32_t m = og++;
                        if (m >= 2 && !mbar_wait(&d2free_bar[m & 1], ((m >> 1) - 1) & 1u, wlim)) { ok = false; break; }
                        if (!xwaited) {
                            if (!mbar_wait(&xload_bar[xb], (xu >> 1) & 1u, wlim)) { ok = false; break; }
                            xwaited = true;
                        }
                        tc_fence_after();
                        const uint64_t gd = gdesc0 + uint64_t(uint32_t((m & 1) * kSymGBytes) >> 4);
                        const uint64_t xd = xdesc0 + uint64_t(uint32_t(xb * kSymXBytes) >> 4);
                        const uint32_t dj = tmem + uint32_t(kSymDJ + NP * int(m & 1));
#pragma unroll
                        for (int ks = 0; ks < 8; ++ks) {
                            // K step ks: targets 16 ks .. 16 ks + 15 (two core
                            // matrices along K), X rows of the same targets:
                            // rows 0..NP-1 X_hi, rows NP..2NP-1 X_lo
                            const uint64_t ah = gd + uint64_t((ks * 2 * kSymTgtGroupStride) >> 4);
                            const uint64_t al = ah + uint64_t((kSymGBytes / 2) >> 4);
                            const uint64_t bh = xd + uint64_t((ks * kStep) >> 4);
                            const uint64_t bl = bh + uint64_t((NP / 8 * 128) >> 4);
                            mma_smemA(dj, ah, bh, IDESC_T, ks == 0 ? 0u : 1u);
                            mma_smemA(dj, ah, bl, IDESC_T, 1u);
                            mma_smemA(dj, al, bh, IDESC_T, 1u);
                        }
                        mma_commit(&gfree_bar[m & 1]);
                        mma_commit(&d2full_bar[m & 1]);
                    }
                }
                if (!ok) break;
                if (unit_offd) {
                    mma_commit(&xfree_bar[xb]);
                    ++xu;
                }
                jbase += un.nloc;
                gbase += (un.nloc + kGroup - 1) / kGroup;
            }
            if (!ok) atomicExch(err, 1);
            // every MMA issued here completes before the tensor memory is
            // freed, also when the producers gave up first (bounded by the
            // default limit whatever the pipeline limit is)
            mma_commit(&drain_bar);
            mbar_wait(&drain_bar, 0, kWaitLimit);
        }
        __syncwarp();
    } else {
        // ---------------- loader: stage images and coordinates ahead ----------------
        if (lane == 0) {
            bool ok = true;
            int64_t jbase = 0, issued = 0;
            uint32_t xu = 0;
            for (int64_t u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
                const TcInstance& I = batch.inst[SYM ? 0 : inst_of(batch, u)];
                const Unit un = SYM ? sym_unit_of(I, u) : unit_of(u - I.unit0, I.splits, I.nchunks, I.cps);
                const uint8_t* img = I.img;
                if (SYM && un.c0 + un.nloc > 2 * un.tile + 2) {
                    // split images of X on the unit's own tile (its two chunk
                    // records' image parts) for the transposed products
                    const uint32_t xb = xu & 1u;
                    if (xu >= 2 && !mbar_wait(&xfree_bar[xb], ((xu >> 1) - 1) & 1u, wlim)) { ok = false; break; }
                    uint8_t* dst = smem + 2 * kSymGBytes + xb * kSymXBytes;
                    mbar_arrive_expect_tx(&xload_bar[xb], uint32_t(kSymXBytes));
                    bulk_g2s(dst, img + 2 * un.tile * int64_t(STAGE_BYTES), uint32_t(2 * IMG), &xload_bar[xb]);
                    bulk_g2s(dst + 2 * IMG, img + (2 * un.tile + 1) * int64_t(STAGE_BYTES), uint32_t(2 * IMG),
                             &xload_bar[xb]);
                    ++xu;
                }
                for (int jl = 0; jl < un.nloc; ++jl) {
                    const int64_t jg = jbase + jl;
                    const int ss = int(jg % SSTAGES);
                    const int64_t use = jg / SSTAGES;
                    if (use > 0 && !mbar_wait(&sempty_bar[ss], uint32_t((use - 1) & 1), wlim)) { ok = false; break; }
                    issued = jg + 1;
                    uint8_t* st = smem + REC_BASE + ss * STAGE_BYTES;
                    const int64_t ch = un.c0 + jl;
                    mbar_arrive_expect_tx(&loaded_bar[ss], uint32_t(STAGE_BYTES));
                    bulk_g2s(st, img + ch * int64_t(STAGE_BYTES), uint32_t(STAGE_BYTES), &loaded_bar[ss]);
                }
                jbase += un.nloc;
            }
            if (!ok) atomicExch(err, 1);
            // every copy issued here lands before the CTA exits: wait for the
            // last use of each stage (already complete unless an error cut
            // the pipeline short; bounded in any case)
            for (int64_t jg = issued - 1; jg >= 0 && jg >= issued - SSTAGES; --jg)
                mbar_wait(&loaded_bar[jg % SSTAGES], uint32_t((jg / SSTAGES) & 1), kWaitLimit);
            for (int64_t x = int64_t(xu) - 1; SYM && x >= 0 && x >= int64_t(xu) - 2; --x)
                mbar_wait(&xload_bar[x & 1], uint32_t((x >> 1) & 1), kWaitLimit);
        }
        __syncwarp();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 8) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

template <int KIND, bool TF32, int NP, bool SYM>
cudaError_t launch_batch_np(const TcBatch& b, int sm_count, int* err, cudaStream_t s) {
    constexpr int ESIZE = TF32 ? 4 : 2;
    constexpr int KC = TF32 ? 32 : 64;
    constexpr int STAGE_BYTES = 2 * NP * KC * ESIZE + KC * 12;
    constexpr int ring = SYM ? kSymRecBase + kSymRecStages * STAGE_BYTES : smem_stages(STAGE_BYTES) * STAGE_BYTES;
    // at least ~100 KB so that no more than two CTAs share an SM (256 TMEM
    // columns each)
    const int smem = std::max(ring + 1024, 100 * 1024);
    auto kern = pair_tc_kernel<KIND, TF32, NP, SYM>;
    // set once per instantiation (before any stream capture of a launch)
    static std::once_flag once;
    static cudaError_t attr_error = cudaSuccess;
    std::call_once(once, [&] { attr_error = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); });
    if (attr_error != cudaSuccess) return attr_error;
    const int64_t grid = std::min<int64_t>(b.nunits, 2LL * sm_count);
    kern<<<unsigned(grid), kThreads, smem, s>>>(b, err);
    return cudaGetLastError();
}

template <int KIND, bool TF32>
cudaError_t launch_batch_kind(const TcBatch& b, int np, bool sym, int sm_count, int* err, cudaStream_t s) {
    if constexpr (!TF32) {
        if (sym) return launch_batch_np<KIND, false, 16, true>(b, sm_count, err, s);
    }
    switch (np) {
        case 16: return launch_batch_np<KIND, TF32, 16, false>(b, sm_count, err, s);
        case 32: return launch_batch_np<KIND, TF32, 32, false>(b, sm_count, err, s);
        case 48: return launch_batch_np<KIND, TF32, 48, false>(b, sm_count, err, s);
        default: return launch_batch_np<KIND, TF32, 64, false>(b, sm_count, err, s);
    }
}

template <bool TF32>
cudaError_t launch_batch_prec(const TcBatch& b, int np, bool sym, int sm_count, int* err, cudaStream_t s) {
    int kind = b.inst[0].kind;
    for (int i = 1; i < b.ninst; ++i)
        if (b.inst[i].kind != kind) kind = kKindAny;
    switch (kind) {
        case KL_KERNEL_GAUSS: return launch_batch_kind<KL_KERNEL_GAUSS, TF32>(b, np, sym, sm_count, err, s);
        case KL_KERNEL_EXP_SEP: return launch_batch_kind<KL_KERNEL_EXP_SEP, TF32>(b, np, sym, sm_count, err, s);
        case KL_KERNEL_EXP: return launch_batch_kind<KL_KERNEL_EXP, TF32>(b, np, sym, sm_count, err, s);
        case KL_KERNEL_MATERN32: return launch_batch_kind<KL_KERNEL_MATERN32, TF32>(b, np, sym, sm_count, err, s);
        case KL_KERNEL_CONST: return launch_batch_kind<KL_KERNEL_CONST, TF32>(b, np, sym, sm_count, err, s);
        default: return launch_batch_kind<kKindAny, TF32>(b, np, sym, sm_count, err, s);
    }
}

// Adds v (FP32, or an FP32 (hi, lo) pair) into the double-float (hi, lo):
// error-free two-sum into hi, the error and v's low part into lo.
__device__ __forceinline__ void df_add(float& hi, float& lo, float v, float vlo) {
    const float sum = __fadd_rn(hi, v);
    const float bb = __fsub_rn(sum, hi);
    const float er = __fadd_rn(__fsub_rn(hi, __fsub_rn(sum, bb)), __fsub_rn(v, bb));
    hi = sum;
    lo = __fadd_rn(lo, __fadd_rn(er, vlo));
}

// W = sigma^2 * post * sum over source splits of the (hi, lo) partial sums,
// in a fixed order. A block serves 32 consecutive points of one column with
// 8 warps: warp y sums the y-th eighth of the splits as a double-float (eight
// loads in flight per thread), then warp 0 adds the eight sums in the order
// y = 0..7. Many outputs are short of threads otherwise (T k / 256 blocks of
// one load chain each cannot keep enough loads in flight to stream the
// partial sums at HBM rate).
constexpr int kRedSplit = 8;
__global__ void __launch_bounds__(32 * kRedSplit)
tc_reduce_kernel(const float2* __restrict__ part, int splits, int64_t T, int k, double sigma2,
                 const double* __restrict__ post, double* __restrict__ Y, int64_t ldy) {
    __shared__ float2 sh[kRedSplit][32];
    const int64_t tblocks = (T + 31) / 32;
    const int y = threadIdx.y;
    const int sa = splits * y / kRedSplit, sb = splits * (y + 1) / kRedSplit;
    const int64_t st = int64_t(k) * T;  // from one split to the next
    for (int64_t b = blockIdx.x; b < tblocks * k; b += gridDim.x) {
        const int c = int(b / tblocks);
        const int64_t t = (b - int64_t(c) * tblocks) * 32 + threadIdx.x;
        float hi = 0.f, lo = 0.f;
        if (t < T) {
            // groups of 8 splits, the last one predicated: every group's
            // loads are in flight together
            const float2* pp = part + (int64_t(sa) * k + c) * T + t;
            for (int sp = sa; sp < sb; sp += 8) {
                float2 v[8];
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (sp + q < sb) v[q] = pp[q * st];
                pp += 8 * st;
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (sp + q < sb) df_add(hi, lo, v[q].x, v[q].y);
            }
        }
        sh[y][threadIdx.x] = make_float2(hi, lo);
        __syncthreads();
        if (y == 0 && t < T) {
            float h = 0.f, l = 0.f;
            for (int q = 0; q < kRedSplit; ++q) df_add(h, l, sh[q][threadIdx.x].x, sh[q][threadIdx.x].y);
            double v = (double(h) + double(l)) * sigma2;
            if (post) v *= post[t];
            Y[c * ldy + t] = v;
        }
        __syncthreads();
    }
}


// Symmetric mode, one band of tiles [tile0, tile1). A block serves one chunk
// of 64 points (chunks from the last, the largest sums, to the first 2 tile0):
// a thread takes one row (point) and four columns of it (16 bytes of a
// transposed-sum row; kstride = k rounded up to 8), and the block's S =
// 512 / (16 kstride) slices (threadIdx.x / (16 kstride)) split the work by
// range: slice y sums, as double-floats, the y-th part of the direct partial
// sums of the point's tile (when the tile is in the band) and the y-th part of
// the transposed partial sums of the band's tiles I below it (I ascending).
// The transposed sums of one chunk are consecutive 64 x kstride blocks (chunk-
// major layout), so a slice's loads stream one contiguous range, six 16-byte
// loads in flight per thread (the last group predicated). The S sums
// are then added in slice order after the running sum of the earlier bands
// (acc; none for the first band): a fixed order. Columns k..kstride-1 of a
// transposed row are padding (products with zero columns of X): read, never
// written out. 32-bit offsets: a band's partial sums stay under 2^31 floats
// and points under 2^26 (tc_sym_eligible).
constexpr int kSymRedThreads = 512;
constexpr int kSymRedLoads = 6;  // 16-byte loads in flight per thread
__global__ void __launch_bounds__(kSymRedThreads, 2)
tc_sym_reduce_kernel(const float2* __restrict__ part1, const float* __restrict__ part2,
                     const int2* __restrict__ tab, int64_t nchunks, int64_t T, int k, int tile0, int tile1,
                     int64_t unit_begin, int first, float2* __restrict__ acc, double sigma2,
                     const double* __restrict__ post, double* __restrict__ Y, int64_t ldy) {
    __shared__ float4 sh[kSymRedThreads][2];
    const int kstride = (k + 7) & ~7;
    const int ng = kstride / 4;   // 16-byte column groups per row
    const int per = 64 * ng;      // threads per 64 x kstride block
    const int S = kSymRedThreads / per;
    const int tid = threadIdx.x;
    const int y = tid / per, lane = tid % per;
    const int r = lane / ng, c0 = 4 * (lane % ng);
    const int nch = int(nchunks) - 2 * tile0;  // chunks of the band's points and the later ones
    const int step = 16 * kstride;             // one block of transposed sums, in 16-byte vectors
    const float4* p2base = reinterpret_cast<const float4*>(part2);
    for (int b = blockIdx.x; b < nch; b += gridDim.x) {
        const int ch = int(nchunks) - 1 - b;
        const int t = ch * 64 + r;
        const int J = ch >> 1;
        const bool valid = t < int(T);
        float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
        if (valid) {
            if (J < tile1) {
                const int u0 = tab[J].x, n1 = tab[J + 1].x - u0;
                const int ua = u0 + n1 * y / S, ub = u0 + n1 * (y + 1) / S;
                for (int u = ua; u < ub; ++u) {
                    const float2* pu = part1 + ((int(u - unit_begin) * k + c0) * 128 + (t & 127));
                    float2 v[4];
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc)
                        if (c0 + cc < k) v[cc] = pu[cc * 128];
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc)
                        if (c0 + cc < k) df_add(hi[cc], lo[cc], v[cc].x, v[cc].y);
                }
            }
            const int n2 = (J < tile1 ? J : tile1) - tile0;
            const int ia = tile0 + n2 * y / S, ib = tile0 + n2 * (y + 1) / S;
            const float4* p2 = p2base + (r * kstride + c0) / 4;
            int off = sym_p2_index(ch, ia, tile0, tile1) * step;
            for (int I = ia; I < ib; I += kSymRedLoads) {
                float4 v[kSymRedLoads];
#pragma unroll
                for (int q = 0; q < kSymRedLoads; ++q) {
                    if (I + q < ib) v[q] = p2[off];
                    off += step;
                }
#pragma unroll
                for (int q = 0; q < kSymRedLoads; ++q)
                    if (I + q < ib) {
                        df_add(hi[0], lo[0], v[q].x, 0.f);
                        df_add(hi[1], lo[1], v[q].y, 0.f);
                        df_add(hi[2], lo[2], v[q].z, 0.f);
                        df_add(hi[3], lo[3], v[q].w, 0.f);
                    }
            }
        }
        sh[tid][0] = make_float4(hi[0], hi[1], hi[2], hi[3]);
        sh[tid][1] = make_float4(lo[0], lo[1], lo[2], lo[3]);
        __syncthreads();
        if (y == 0 && valid) {
            float h[4] = {0.f, 0.f, 0.f, 0.f}, l[4] = {0.f, 0.f, 0.f, 0.f};
            if (!first) {
#pragma unroll
                for (int cc = 0; cc < 4; ++cc)
                    if (c0 + cc < k) {
                        const float2 a2 = acc[int64_t(c0 + cc) * T + t];
                        h[cc] = a2.x;
                        l[cc] = a2.y;
                    }
            }
            for (int q = 0; q < S; ++q) {
                const float4 w = sh[q * per + lane][0], wl = sh[q * per + lane][1];
                df_add(h[0], l[0], w.x, wl.x);
                df_add(h[1], l[1], w.y, wl.y);
                df_add(h[2], l[2], w.z, wl.z);
                df_add(h[3], l[3], w.w, wl.w);
            }
            const bool done = J < tile1;
            const double m = post ? sigma2 * post[t] : sigma2;
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                if (c0 + cc >= k) break;
                if (done) Y[(c0 + cc) * ldy + t] = (double(h[cc]) + double(l[cc])) * m;
                else acc[int64_t(c0 + cc) * T + t] = make_float2(h[cc], l[cc]);
            }
        }
        __syncthreads();
    }
}

struct TcPlan {
    int kchunk;
    int64_t nchunks;
    int np_max;
    int splits, cps;
    int nblk;  // column blocks of at most 64 vectors (one instance each)
    int64_t img_blk_doubles, img_doubles, src_doubles, part_doubles;
};

// Persistent schedule: 2 CTAs per SM walk the units (tile, source range)
// round-robin. Splitting every tile's sources into `splits` ranges of equal
// length gives about 16 units per CTA (load imbalance <= 1/16) while keeping
// ranges >= 768 sources long and the partial sums <= 64 MiB.
TcPlan plan(int64_t T, int64_t S, int k, int sm_count, bool tf32) {
    TcPlan p;
    p.kchunk = tf32 ? 32 : 64;
    p.nchunks = std::max<int64_t>(1, (S + p.kchunk - 1) / p.kchunk);
    const int kmax = std::min(k, 64);
    p.np_max = std::max(16, (kmax + 15) / 16 * 16);
    const int64_t tiles = (T + 127) / 128;
    const int64_t grid = 2LL * sm_count;
    int64_t want = (16 * grid + tiles - 1) / tiles;
    want = std::min(want, std::max<int64_t>(1, p.nchunks * p.kchunk / 768));
    want = std::min(want, std::max<int64_t>(1, (int64_t(8) << 20) / (int64_t(k) * T)));
    want = std::max<int64_t>(1, want);
    p.cps = int((p.nchunks + want - 1) / want);
    p.splits = int((p.nchunks + p.cps - 1) / p.cps);
    const int esize = tf32 ? 4 : 2;
    p.nblk = (k + 63) / 64;
    // one record per chunk: hi and lo images and the coordinates (16-byte multiple)
    p.img_blk_doubles = (p.nchunks * (2 * p.np_max * p.kchunk * esize + 12 * p.kchunk) + 7) / 8;
    p.img_doubles = p.nblk * p.img_blk_doubles;
    p.src_doubles = 0;  // coordinates are part of the chunk records
    p.part_doubles = int64_t(p.splits) * k * T;
    return p;
}

}  // namespace

int64_t tc_scratch_doubles(int64_t T, int64_t S, int k, int sm_count) {
    // every block width up to k: a narrower block may take more source
    // splits (the partial sums are capped at 8M doubles per split count, not
    // per width), so the largest need is not always at k itself
    int64_t need = 0;
    for (int kk = 1; kk <= k; ++kk) {
        const TcPlan pb = plan(T, S, kk, sm_count, false), pt = plan(T, S, kk, sm_count, true);
        need = std::max({need, pb.img_doubles + pb.src_doubles + pb.part_doubles,
                         pt.img_doubles + pt.src_doubles + pt.part_doubles});
    }
    return need;
}

cudaError_t tc_prepare(const TcArgs& a, cudaStream_t s, TcInstance* out, int* n, int* np, int* launched) {
    *n = 0;
    const TcPlan p = plan(a.T, a.S, a.k, a.sm_count, a.tf32);
    if (p.img_doubles + p.src_doubles + p.part_doubles > a.scratch_len) return cudaErrorInvalidValue;
    if (p.nblk > 4) return cudaErrorInvalidValue;
    float2* part = reinterpret_cast<float2*>(a.scratch + p.img_doubles + p.src_doubles);
    const float cscale = coord_scale(a.ks);
    KL_RANGE(a.X, block_extent(a.S, a.k, a.ldx), double, "tc convert X");
    KL_RANGE(a.sx, a.S, float, "tc convert sources x");
    KL_RANGE(a.sy, a.S, float, "tc convert sources y");
    KL_RANGE(a.sz, a.S, float, "tc convert sources z");
    KL_RANGE(a.scratch, p.img_doubles + p.src_doubles + p.part_doubles, double, "tc scratch");
    // every column block uses the image layout of the widest one (the last
    // block's missing columns are zero), so that they share one launch
    *np = p.np_max;
    for (int blk = 0; blk < p.nblk; ++blk) {
        const int c0 = 64 * blk, kc = std::min(64, a.k - c0);
        uint8_t* img = reinterpret_cast<uint8_t*>(a.scratch + blk * p.img_blk_doubles);
        const int64_t total = p.nchunks * p.kchunk * p.np_max;
        const int g = int(std::min<int64_t>((total + 255) / 256, int64_t(a.sm_count) * 64));
        tc_convert_kernel<<<g, 256, 0, s>>>(a.X, a.ldx, a.S, c0, kc, p.np_max, p.kchunk, a.tf32, cscale, a.sx,
                                            a.sy, a.sz, img, p.nchunks);
        ++*launched;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        TcInstance& I = out[blk];
        I.tx = a.tx;
        I.ty = a.ty;
        I.tz = a.tz;
        I.srcc = nullptr;
        I.img = img;
        I.part = part;
        I.T = a.T;
        I.nchunks = p.nchunks;
        I.unit0 = 0;
        I.cps = p.cps;
        I.splits = p.splits;
        I.kind = a.ks.kind;
        I.k_total = a.k;
        I.c0 = c0;
        I.kc = kc;
        I.cscale = cscale;
        ++*n;
    }
    return cudaSuccess;
}

cudaError_t tc_launch_batch(TcBatch& b, bool tf32, int np, int sm_count, int* err, cudaStream_t s) {
    if (b.ninst < 1 || b.ninst > kTcMaxBatch) return cudaErrorInvalidValue;
    int64_t u = 0;
    for (int i = 0; i < b.ninst; ++i) {
        b.inst[i].unit0 = u;
        u += (b.inst[i].T + 127) / 128 * b.inst[i].splits;
    }
    b.nunits = u;
    if (u == 0) return cudaSuccess;
#ifdef KL_CHECK_BOUNDS
    {
        const int esize = tf32 ? 4 : 2, kchunk = tf32 ? 32 : 64;
        const int64_t stage_bytes = 2 * int64_t(np) * kchunk * esize + 12 * int64_t(kchunk);
        for (int i = 0; i < b.ninst; ++i) {
            const TcInstance& I = b.inst[i];
            KL_RANGE(I.tx, I.T, float, "tc targets x");
            KL_RANGE(I.ty, I.T, float, "tc targets y");
            KL_RANGE(I.tz, I.T, float, "tc targets z");
            KL_RANGE(I.img, I.nchunks * stage_bytes, uint8_t, "tc chunk records");
            // partial sums of the instance's columns c0 .. c0 + kc - 1 of every split
            KL_RANGE(I.part, (int64_t(I.splits - 1) * I.k_total + I.c0 + I.kc) * I.T, float2, "tc partial sums");
            if (int64_t(I.splits - 1) * I.cps >= I.nchunks || int64_t(I.splits) * I.cps < I.nchunks ||
                I.c0 + I.kc > I.k_total || I.kc > np) {
                std::fprintf(stderr, "kl bounds check: tc instance %d: splits %d x %d chunks against %lld, "
                             "columns %d + %d of %d, N %d\n", i, I.splits, I.cps, (long long)I.nchunks, I.c0, I.kc,
                             I.k_total, np);
                return cudaErrorInvalidValue;
            }
        }
        KL_RANGE(err, 1, int, "tc error word");
    }
#endif
    return tf32 ? launch_batch_prec<true>(b, np, false, sm_count, err, s)
                : launch_batch_prec<false>(b, np, false, sm_count, err, s);
}

cudaError_t tc_finish(const TcArgs& a, cudaStream_t s, int* launched) {
    const TcPlan p = plan(a.T, a.S, a.k, a.sm_count, a.tf32);
    const float2* part = reinterpret_cast<const float2*>(a.scratch + p.img_doubles + p.src_doubles);
    KL_RANGE(part, p.part_doubles, float2, "tc_reduce partial sums");
    KL_RANGE(a.Y, block_extent(a.T, a.k, a.ldy), double, "tc_reduce Y");
    KL_RANGE(a.post, a.T, double, "tc_reduce post");
    const int64_t nblk = (a.T + 31) / 32 * a.k;
    const int g = int(std::max<int64_t>(1, std::min<int64_t>(nblk, int64_t(a.sm_count) * 16)));
    tc_reduce_kernel<<<g, dim3(32, kRedSplit), 0, s>>>(part, p.splits, a.T, a.k, a.ks.sigma2, a.post, a.Y, a.ldy);
    ++*launched;
    return cudaGetLastError();
}

// Transposed partial sums of one band: at most this many floats (512 MB);
// more tiles make more bands.
constexpr int64_t kSymP2Cap = int64_t(128) << 20;

// T <= 2^26 keeps the symmetric reduction's 32-bit offsets in range (one
// tile's transposed sums: at most 2^30 floats)
bool tc_sym_eligible(int64_t T, int k, bool tf32) {
    return !tf32 && k >= 1 && k <= 16 && T >= 1 && T <= (int64_t(1) << 26);
}

TcSymPlan tc_sym_plan(int64_t T, int kcap, int sm_count) {
    TcSymPlan p;
    p.T = T;
    p.kcap = kcap;
    p.sm_count = sm_count;
    p.nchunks = (T + 63) / 64;
    p.nt = int((T + 127) / 128);
    // bands: consecutive tiles while their transposed partial sums fit the cap
    p.band.push_back(0);
    int64_t inband = 0;
    for (int I = 0; I < p.nt; ++I) {
        const int64_t w = int64_t(64) * kcap * std::max<int64_t>(0, p.nchunks - 2 - 2 * int64_t(I));
        if (inband > 0 && inband + w > kSymP2Cap) {
            p.band.push_back(I);
            inband = 0;
        }
        inband += w;
    }
    p.band.push_back(p.nt);
    // units: per band, chunk ranges of cps chunks with cps from the band's
    // chunk work (about 16 units per CTA of the persistent grid, at least 4
    // chunks each)
    p.tab.assign(size_t(p.nt) + 1, make_int2(0, 0));
    const int64_t grid = 2LL * sm_count;
    int64_t unit = 0;
    for (size_t b = 0; b + 1 < p.band.size(); ++b) {
        int64_t work = 0, p2 = 0;
        for (int I = p.band[b]; I < p.band[b + 1]; ++I) {
            work += p.nchunks - 2 * int64_t(I);
            p2 += std::max<int64_t>(0, p.nchunks - 2 - 2 * int64_t(I));
        }
        const int cps = int(std::max<int64_t>(4, (work + 16 * grid - 1) / (16 * grid)));
        const int64_t u0 = unit;
        for (int I = p.band[b]; I < p.band[b + 1]; ++I) {
            p.tab[I] = make_int2(int(unit), cps);
            unit += (p.nchunks - 2 * int64_t(I) + cps - 1) / cps;
        }
        p.max_band_units = std::max(p.max_band_units, unit - u0);
        p.max_band_p2 = std::max(p.max_band_p2, p2 * 64 * kcap);
    }
    p.tab[p.nt] = make_int2(int(unit), 0);
    // scratch: chunk records | unit table | direct partials (float2 per unit,
    // column and row) | transposed partials (float) | running sums (float2,
    // with more than one band)
    const int stage_bytes = 2 * 16 * 64 * 2 + 64 * 12;
    p.off_img = 0;
    p.off_tab = (p.nchunks * stage_bytes + 15) / 16 * 2;
    p.off_part1 = p.off_tab + (int64_t(p.nt) + 2) / 2 * 2;
    p.off_part2 = p.off_part1 + p.max_band_units * kcap * 128;
    p.off_acc = p.off_part2 + (p.max_band_p2 + 1) / 2;
    p.total = p.off_acc + (p.band.size() > 2 ? T * kcap : 0);
    return p;
}

cudaError_t tc_sym_upload(const TcSymPlan& p, double* scratch, cudaStream_t s) {
    cudaError_t e = cudaMemcpyAsync(scratch + p.off_tab, p.tab.data(), p.tab.size() * sizeof(int2),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
}

cudaError_t launch_pair_tc_sym(const TcArgs& a, cudaStream_t s, int* launched) {
    *launched = 0;
    const TcSymPlan& p = *a.sym;
    if (a.tf32 || a.k < 1 || a.k > p.kcap || a.T != p.T || a.S != p.T || a.scratch_len < p.total)
        return cudaErrorInvalidValue;
    const float cscale = coord_scale(a.ks);
    uint8_t* img = reinterpret_cast<uint8_t*>(a.scratch + p.off_img);
    const int2* tab = reinterpret_cast<const int2*>(a.scratch + p.off_tab);
    float2* part1 = reinterpret_cast<float2*>(a.scratch + p.off_part1);
    float* part2 = reinterpret_cast<float*>(a.scratch + p.off_part2);
    float2* acc = reinterpret_cast<float2*>(a.scratch + p.off_acc);
    KL_RANGE(a.X, block_extent(a.S, a.k, a.ldx), double, "tc sym convert X");
    KL_RANGE(a.sx, a.S, float, "tc sym sources x");
    KL_RANGE(a.sy, a.S, float, "tc sym sources y");
    KL_RANGE(a.sz, a.S, float, "tc sym sources z");
    KL_RANGE(a.scratch, p.total, double, "tc sym scratch");
    KL_RANGE(a.Y, block_extent(a.T, a.k, a.ldy), double, "tc sym Y");
    KL_RANGE(a.post, a.T, double, "tc sym post");
    {
        const int64_t total = p.nchunks * 64 * 16;
        const int g = int(std::min<int64_t>((total + 255) / 256, int64_t(a.sm_count) * 64));
        tc_convert_kernel<<<g, 256, 0, s>>>(a.X, a.ldx, a.S, 0, a.k, 16, 64, false, cscale, a.sx, a.sy, a.sz, img,
                                            p.nchunks);
        ++*launched;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const int nbands = int(p.band.size()) - 1;
    for (int b = 0; b < nbands; ++b) {
        const int tile0 = p.band[b], tile1 = p.band[b + 1];
        TcBatch batch;
        batch.ninst = 1;
        batch.wait_limit = a.wait_limit;
        TcInstance& I = batch.inst[0];
        I.tx = a.tx;
        I.ty = a.ty;
        I.tz = a.tz;
        I.srcc = nullptr;
        I.img = img;
        I.part = part1;
        I.T = a.T;
        I.nchunks = p.nchunks;
        I.unit0 = 0;
        I.cps = 0;
        I.splits = 0;
        I.kind = a.ks.kind;
        I.k_total = a.k;
        I.c0 = 0;
        I.kc = a.k;
        I.cscale = cscale;
        I.sym_tab = tab;
        I.part2 = part2;
        I.sym_unit_begin = p.tab[tile0].x;
        I.sym_tile0 = tile0;
        I.sym_tile1 = tile1;
        batch.nunits = int64_t(p.tab[tile1].x) - p.tab[tile0].x;
#ifdef KL_CHECK_BOUNDS
        {
            // direct partials of the band's units, transposed partials of its
            // tiles (those index the band's own ranges of the scratch)
            int64_t p2 = 0;
            for (int t = tile0; t < tile1; ++t) p2 += std::max<int64_t>(0, p.nchunks - 2 - 2 * int64_t(t));
            if (batch.nunits > p.max_band_units || p2 * 64 * ((a.k + 7) / 8 * 8) > p.max_band_p2) {
                std::fprintf(stderr, "kl bounds check: tc sym band %d: %lld units (max %lld), %lld transposed sums\n",
                             b, (long long)batch.nunits, (long long)p.max_band_units,
                             (long long)(p2 * 64 * ((a.k + 7) / 8 * 8)));
                return cudaErrorInvalidValue;
            }
            KL_RANGE(a.tx, a.T, float, "tc sym targets x");
            KL_RANGE(a.err, 1, int, "tc error word");
        }
#endif
        cudaError_t e = launch_batch_prec<false>(batch, 16, true, a.grid_sms > 0 ? a.grid_sms : a.sm_count, a.err, s);
        ++*launched;
        if (e != cudaSuccess) return e;
        // one block per chunk of the band's points and the later ones
        const int g = int(std::max<int64_t>(1, p.nchunks - 2 * int64_t(tile0)));
        tc_sym_reduce_kernel<<<g, kSymRedThreads, 0, s>>>(part1, part2, tab, p.nchunks, a.T, a.k, tile0, tile1,
                                               I.sym_unit_begin, b == 0, acc, a.ks.sigma2, a.post,
                                               a.Y, a.ldy);
        ++*launched;
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_pair_tc(const TcArgs& a, cudaStream_t s, int* launched) {
    *launched = 0;
    TcBatch b;
    b.wait_limit = a.wait_limit;
    int np = 16;
    cudaError_t e = tc_prepare(a, s, b.inst, &b.ninst, &np, launched);
    if (e != cudaSuccess) return e;
    e = tc_launch_batch(b, a.tf32, np, a.grid_sms > 0 ? a.grid_sms : a.sm_count, a.err, s);
    ++*launched;
    if (e != cudaSuccess) return e;
    return tc_finish(a, s, launched);
}

}  // namespace kl
