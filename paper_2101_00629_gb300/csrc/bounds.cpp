// Bounds-checking build (KL_CHECK_BOUNDS): before every kernel launch the
// launchers check, on the host, that each device range the kernel will read
// or write -- [p, p + bytes), computed from the kernel's own index formulas
// and the launch's sizes and leading dimensions -- lies inside one live
// device allocation. The driver reports the allocation that contains p
// (cuMemGetAddressRange), so a range that runs past its buffer, or a buffer
// that was already freed, is caught before the launch instead of faulting the
// GPU. A failed check prints the launch, the argument and both extents to
// stderr and the launch returns cudaErrorInvalidValue (the call then fails
// with KL_ERR_CUDA). The regular build compiles none of this.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cinttypes>
#include <cstdio>
#include <mutex>

#include "kl_internal.h"

#ifdef KL_CHECK_BOUNDS
namespace kl {

namespace {
using AddressRangeFn = CUresult (*)(CUdeviceptr*, size_t*, CUdeviceptr);
AddressRangeFn g_range = nullptr;
std::once_flag g_once;
}  // namespace

cudaError_t check_range(const void* p, int64_t bytes, const char* what) {
    if (bytes <= 0) return cudaSuccess;
    std::call_once(g_once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_range = reinterpret_cast<AddressRangeFn>(fn);
    });
    if (!g_range) {
        std::fprintf(stderr, "kl bounds check: cuMemGetAddressRange unavailable\n");
        return cudaErrorInvalidValue;
    }
    CUdeviceptr base = 0;
    size_t size = 0;
    const CUresult r = g_range(&base, &size, reinterpret_cast<CUdeviceptr>(p));
    const uint64_t a = reinterpret_cast<uint64_t>(p);
    if (r != CUDA_SUCCESS) {
        std::fprintf(stderr, "kl bounds check: %s: %p (%" PRId64 " bytes) is not inside a live device allocation\n",
                     what, p, bytes);
        return cudaErrorInvalidValue;
    }
    if (a + uint64_t(bytes) > uint64_t(base) + size) {
        std::fprintf(stderr,
                     "kl bounds check: %s: range %p + %" PRId64 " bytes ends %" PRIu64
                     " bytes past its allocation (base %p, %zu bytes)\n",
                     what, p, bytes, a + uint64_t(bytes) - (uint64_t(base) + size),
                     reinterpret_cast<void*>(base), size);
        return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}

}  // namespace kl
#endif

extern "C" int kl_bounds_checked(void) {
#ifdef KL_CHECK_BOUNDS
    return 1;
#else
    return 0;
#endif
}
