// Pairwise product with no device allocation.
//
// Some callers cannot allocate device memory: code running inside a CUDA
// graph that is being captured or replayed, applications whose memory pools
// are fixed up front, or hosts that hand out one pre-sized arena and forbid
// cudaMalloc/cudaFree afterwards. kl_pairwise_noalloc serves them: it is the
// FP64 CUDA-core pairwise kernel of the library, but its split partial sums
// live in a file-scope device array instead of a handle's workspace.
//
// The array (kNoallocScratch doubles, 16 MiB) exists once per device that
// loads the library and stays allocated until the process exits. Every call
// on a device shares it and leaves the previous call's partial sums in it;
// each call overwrites every partial sum it reads, so nothing has to be
// cleared between calls. Calls that overlap on the GPU (different streams,
// or concurrent host threads) race on the array and must be serialised by
// the caller.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "handle.h"

namespace kl {
namespace {

constexpr int64_t kNoallocScratch = int64_t(1) << 21;  // doubles (16 MiB)
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kNoallocScratch];

// Host-side set-up, once per device with that device current: the symbol
// above is only a host stand-in, the kernel needs its device address.
std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {};
int g_sm_count[kMaxDevices] = {};

int device_scratch(double** ptr, int* sm_count) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(nullptr, KL_ERR_UNSUPPORTED, "device index beyond 63");
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetSymbolAddress");
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaDeviceGetAttribute");
        g_sm_count[dev] = sms;
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *ptr = g_scratch_ptr[dev];
    *sm_count = g_sm_count[dev];
    return KL_OK;
}

}  // namespace
}  // namespace kl

using namespace kl;

extern "C" int kl_pairwise_noalloc(int kernel, double sigma, double L, const double* tgt, int64_t T,
                                   const double* src, int64_t S, const double* X, int64_t ldx,
                                   double* Y, int64_t ldy, int k, void* stream) {
    if (kernel < KL_KERNEL_GAUSS || kernel > KL_KERNEL_CONST) return fail(nullptr, KL_ERR_ARG, "unknown kernel");
    if (!(sigma > 0) || !(L > 0) || !std::isfinite(sigma) || !std::isfinite(L))
        return fail(nullptr, KL_ERR_ARG, "sigma and L must be > 0");
    if (!tgt || !src || !X || !Y) return fail(nullptr, KL_ERR_ARG, "pointers must not be NULL");
    if (T < 1 || S < 1 || k < 1 || k > 256) return fail(nullptr, KL_ERR_ARG, "need T, S >= 1 and 1 <= k <= 256");
    if (ldx < S || ldy < T) return fail(nullptr, KL_ERR_ARG, "leading dimensions too small");
    // T is compared against the quotient so that k * T is never formed for
    // a T that would overflow it
    if (T > kNoallocScratch / k)
        return fail(nullptr, KL_ERR_ARG, "k * T exceeds the static scratch of 2^21 doubles (16 MiB)");
    double* scratch = nullptr;
    int sms = 0;
    int rc = device_scratch(&scratch, &sms);
    if (rc != KL_OK) return rc;
    int splits = pair_choose_splits(T, S, sms);
    const int64_t cap = kNoallocScratch / (int64_t(k) * T);
    if (splits > cap) splits = int(cap);
    PairArgs a{};
    a.tx = tgt; a.ty = tgt + T; a.tz = tgt + 2 * T;
    a.sx = src; a.sy = src + S; a.sz = src + 2 * S;
    a.T = T; a.S = S;
    a.X = X; a.ldx = ldx; a.Y = Y; a.ldy = ldy; a.k = k;
    a.post = nullptr;
    a.ks.kind = kernel;
    a.ks.sigma2 = sigma * sigma;
    a.ks.a = kernel == KL_KERNEL_GAUSS ? 1.0 / (L * L) : (kernel == KL_KERNEL_MATERN32 ? std::sqrt(3.0) / L : 1.0 / L);
    a.scratch = scratch;
    a.splits = splits;
    cudaError_t e = launch_pair_simt(a, false, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "pairwise launch");
    return KL_OK;
}
