// C ABI entry points: handle creation (Sec. 3.1 / 3.2 set-up), the
// matrix-free operator applications and profiling counters.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "handle.h"
#include "kernels_tc.h"
#include "serve.h"

namespace {
thread_local std::string g_create_error;  // per host thread (servers create handles concurrently)
}

namespace kl {

int device_sm_count() {
    constexpr int kMax = 64;
    static std::atomic<int> cache[kMax];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMax) {
        cudaGetLastError();
        return 152;
    }
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
        cudaGetLastError();
        return 152;
    }
    cache[dev].store(v, std::memory_order_relaxed);
    return v;
}

namespace {
// allocations left before the injected failure (kl_debug_set with
// KL_DEBUG_FAIL_ALLOC; 0: none pending)
std::atomic<long long> g_fail_alloc_in{0};
}  // namespace

cudaError_t device_alloc(void** p, size_t bytes) {
    *p = nullptr;
    long long left = g_fail_alloc_in.load();
    while (left > 0 && !g_fail_alloc_in.compare_exchange_weak(left, left - 1)) {
    }
    if (left == 1) return cudaErrorMemoryAllocation;  // this is the allocation that fails
    return cudaMalloc(p, bytes);
}

int fail(kl_solver* h, int code, const std::string& msg) {
    if (h) h->err = msg; else g_create_error = msg;
    return code;
}

int cuda_fail(kl_solver* h, cudaError_t e, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(h, e == cudaErrorMemoryAllocation ? KL_ERR_OOM : KL_ERR_CUDA, m);
}

ProfScope::ProfScope(kl_solver* h_, const char* n, double u) : h(h_), name(n), units(u) {
    if (!h->profiling) return;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, h->stream);
}

ProfScope::~ProfScope() {
    if (!e0) return;
    cudaEventRecord(e1, h->stream);
    auto& p = h->prof[name];
    p.pending.emplace_back(e0, e1);
    p.pending_units.push_back(units);
}

namespace {

// y = x - origin rounded to FP32. The kernels depend on coordinate
// differences only, so the origin (the centre of the domain's bounding box)
// changes nothing but the rounding: FP32 coordinates of half the magnitude
// carry half the absolute error into every difference.
__global__ void to_float_kernel(const double* __restrict__ x, float* __restrict__ y, int64_t n, double origin) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x)
        y[i] = float(x[i] - origin);
}

// Centre of the bounding box of the physical domain (per coordinate).
void domain_centre(const kl_params& p, double c[3]) {
    c[0] = c[1] = c[2] = 0.0;
    if (p.geometry == KL_GEOM_QUARTER_ANNULUS) {
        c[0] = c[1] = 0.5 * p.geo[1];
        c[2] = 0.5 * p.geo[2];
    } else if (p.geometry == KL_GEOM_HALF_ANNULUS) {
        c[1] = 0.5 * p.geo[1];
        c[2] = 0.5 * p.geo[2];
    } else if (p.geometry == KL_GEOM_PROJECTIVE_CUBE) {
        // a hexahedron with planar faces: the box of its eight corners
        double lo[3] = {HUGE_VAL, HUGE_VAL, HUGE_VAL}, hi[3] = {-HUGE_VAL, -HUGE_VAL, -HUGE_VAL};
        for (int v = 0; v < 8; ++v) {
            const double u[3] = {double(v & 1), double((v >> 1) & 1), double((v >> 2) & 1)};
            const double D = 1.0 + p.geo[0] * u[0] + p.geo[1] * u[1] + p.geo[2] * u[2];
            for (int d = 0; d < 3; ++d) {
                lo[d] = std::min(lo[d], u[d] / D);
                hi[d] = std::max(hi[d], u[d] / D);
            }
        }
        for (int d = 0; d < 3; ++d) c[d] = 0.5 * (lo[d] + hi[d]);
    } else {
        for (int d = 0; d < p.dim; ++d) c[d] = 0.5;
    }
}

template <class T>
cudaError_t dalloc(kl_solver* h, T** p, int64_t count) {
    *p = nullptr;
    if (count <= 0) count = 1;
    cudaError_t e = device_alloc((void**)p, size_t(count) * sizeof(T));
    if (e == cudaSuccess) h->dev_bytes += count * int64_t(sizeof(T));
    return e;
}

void dfree(void* p) {
    if (p) cudaFree(p);
}

int64_t prod3(const int* a) { return int64_t(a[0]) * a[1] * a[2]; }

}  // namespace

int ensure_workspace(kl_solver* h, int k) {
    if (k <= h->k_cap) return KL_OK;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "workspace sync");
    clear_graphs(h);
    for (int i = 0; i < 3; ++i) {
        dfree(h->ws[i]);
        h->ws[i] = nullptr;
    }
    dfree(h->pair_scratch);
    h->pair_scratch = nullptr;
    const int64_t big = std::max(h->S, h->T) * int64_t(k);
    for (int i = 0; i < 3; ++i)
        if ((e = dalloc(h, &h->ws[i], big)) != cudaSuccess) return cuda_fail(h, e, "workspace alloc");
    h->pair_splits = pair_choose_splits(h->T, h->S, h->sm_count);
    h->pair_scratch_len = std::max<int64_t>(pair_scratch_doubles(h->T, k, h->pair_splits),
                                            tc_scratch_doubles(h->T, h->S, k, h->sm_count));
    if ((e = dalloc(h, &h->pair_scratch, h->pair_scratch_len)) != cudaSuccess)
        return cuda_fail(h, e, "pair scratch alloc");
    h->k_cap = k;
    return KL_OK;
}

// Symmetric split-BF16 Galerkin product: plan and scratch for blocks of k
// vectors (k rounded up to 8, at most 16), created on the first application
// that uses it (stand-alone handles only: served handles share batched
// launches of the dense form). Before any graph capture of the application.
static bool sym_applies(const kl_solver* h, int precision, int k) {
    return galerkin_form(h->prm.method) && precision == KL_MIXED_BF16 && !h->batcher && !h->pair_dense &&
           h->cc_major == 10 && h->T == h->S && tc_sym_eligible(h->T, k, false);
}

static int ensure_sym(kl_solver* h, int k) {
    if (h->sym_plan && k <= h->sym_plan->kcap) return KL_OK;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "workspace sync");
    clear_graphs(h);
    dfree(h->sym_scratch);
    h->dev_bytes -= h->sym_scratch_len * int64_t(sizeof(double));
    h->sym_scratch = nullptr;
    h->sym_scratch_len = 0;
    delete h->sym_plan;
    h->sym_plan = nullptr;
    TcSymPlan* p = new TcSymPlan(tc_sym_plan(h->T, std::min(16, (k + 7) / 8 * 8), h->sm_count));
    if ((e = dalloc(h, &h->sym_scratch, p->total)) != cudaSuccess) {
        delete p;
        return cuda_fail(h, e, "symmetric pair scratch alloc");
    }
    if ((e = tc_sym_upload(*p, h->sym_scratch, h->stream)) != cudaSuccess) {
        delete p;
        return cuda_fail(h, e, "symmetric pair unit table");
    }
    h->sym_scratch_len = p->total;
    h->sym_plan = p;
    return KL_OK;
}

// Y <- (x)_d F_d applied mode by mode: X has dims (n_in[0], n_in[1], n_in[2]),
// F_d is (n_out[d] x n_in[d]). The first product scales the input rows by
// `pre` and the last one writes Y (ldy) with per-point scaling `post` (either
// may be NULL); intermediates use ws[wa], ws[wb].
static int kron3_s(kl_solver* h, const double* const* Fd, const int* n_in, const int* n_out,
                   const double* X, int64_t ldx, double* Y, int64_t ldy, int k, const double* post,
                   double* sa, double* sb, const double* pre = nullptr, const Band* bands = nullptr);

// bands: banded forms of the F_d (per direction; vals NULL: dense product)
static int kron3(kl_solver* h, const double* const* Fd, const int* n_in, const int* n_out,
                 const double* X, int64_t ldx, double* Y, int64_t ldy, int k, const double* post,
                 int wa, int wb, const double* pre = nullptr, const Band* bands = nullptr) {
    return kron3_s(h, Fd, n_in, n_out, X, ldx, Y, ldy, k, post, h->ws[wa], h->ws[wb], pre, bands);
}

// Same with explicit scratch for the two intermediate products.
static int kron3_s(kl_solver* h, const double* const* Fd, const int* n_in, const int* n_out,
                   const double* X, int64_t ldx, double* Y, int64_t ldy, int k, const double* post,
                   double* sa, double* sb, const double* pre, const Band* bands) {
    int dims[3] = {n_in[0], n_in[1], n_in[2]};
    const double* cur = X;
    int64_t ldc = ldx;
    for (int d = 0; d < 3; ++d) {
        int64_t a = 1, b = 1;
        for (int j = 0; j < d; ++j) a *= dims[j];
        for (int j = d + 1; j < 3; ++j) b *= dims[j];
        dims[d] = n_out[d];
        const int64_t out_len = prod3(dims);
        double* out;
        int64_t ldo;
        if (d == 2) {
            out = Y;
            ldo = ldy;
        } else {
            out = d == 0 ? sa : sb;
            ldo = out_len;
        }
        cudaError_t e =
            (bands && bands[d].vals)
                ? launch_modeprod_band(bands[d], n_out[d], n_in[d], cur, ldc, out, ldo, a, b, k,
                                       d == 2 ? post : nullptr, d == 0 ? pre : nullptr, h->stream)
                : launch_modeprod(Fd[d], n_out[d], n_in[d], cur, ldc, out, ldo, a, b, k, d == 2 ? post : nullptr,
                                  d == 0 ? pre : nullptr, h->stream);
        ++h->launches;
        if (e != cudaSuccess) return cuda_fail(h, e, "modeprod");
        cur = out;
        ldc = ldo;
    }
    return KL_OK;
}

static int pairwise(kl_solver* h, int precision, const double* U, double* W, int k,
                    const double* post) {
    const double S2 = h->prm.sigma * h->prm.sigma;
    KernelSpec ks;
    ks.kind = h->prm.kernel;
    ks.sigma2 = S2;
    const double L = h->prm.L;
    switch (h->prm.kernel) {
        case KL_KERNEL_GAUSS: ks.a = 1.0 / (L * L); break;
        case KL_KERNEL_MATERN32: ks.a = std::sqrt(3.0) / L; break;
        default: ks.a = 1.0 / L; break;
    }
    const double pairs = double(h->T) * double(h->S);
    if (precision == KL_FP64 || precision == KL_FP32) {
        PairArgs a{};
        a.tx = h->tx; a.ty = h->ty; a.tz = h->tz;
        a.sx = h->sx; a.sy = h->sy; a.sz = h->sz;
        a.tx32 = h->tx32; a.ty32 = h->ty32; a.tz32 = h->tz32;
        a.sx32 = h->sx32; a.sy32 = h->sy32; a.sz32 = h->sz32;
        a.T = h->T; a.S = h->S;
        a.X = U; a.ldx = h->S; a.Y = W; a.ldy = h->T; a.k = k;
        a.post = post; a.ks = ks;
        a.scratch = h->pair_scratch; a.splits = h->pair_splits;
        ProfScope ps(h, precision == KL_FP64 ? "pair_f64" : "pair_f32", pairs);
        cudaError_t e = launch_pair_simt(a, precision == KL_FP32, h->stream);
        h->launches += (k + 31) / 32 + 1;
        if (e != cudaSuccess) return cuda_fail(h, e, "pairwise (CUDA cores)");
        return KL_OK;
    }
    if (precision == KL_MIXED_BF16 || precision == KL_MIXED_TF32) {
        if (h->cc_major != 10) return fail(h, KL_ERR_UNSUPPORTED, "tcgen05 precisions need an sm_100-class GPU");
        TcArgs a{};
        a.tx = h->tx32; a.ty = h->ty32; a.tz = h->tz32;
        a.sx = h->sx32; a.sy = h->sy32; a.sz = h->sz32;
        a.T = h->T; a.S = h->S;
        a.X = U; a.ldx = h->S; a.Y = W; a.ldy = h->T; a.k = k;
        a.post = post; a.ks = ks; a.tf32 = precision == KL_MIXED_TF32;
        a.scratch = h->pair_scratch; a.scratch_len = h->pair_scratch_len;
        a.sm_count = h->sm_count;
        a.grid_sms = h->sm_count - h->shared_sms;
        a.err = h->d_err;
        a.wait_limit = h->wait_limit;
        int launched = 0;
        if (sym_applies(h, precision, k) && h->sym_plan && k <= h->sym_plan->kcap) {
            // each symmetric pair once (units of the method's work: N~(N~+1)/2)
            a.sym = h->sym_plan;
            a.scratch = h->sym_scratch;
            a.scratch_len = h->sym_scratch_len;
            ProfScope ps(h, "pair_tc_bf16_sym", 0.5 * double(h->T) * double(h->T + 1));
            cudaError_t e = launch_pair_tc_sym(a, h->stream, &launched);
            h->launches += launched;
            if (e != cudaSuccess) return cuda_fail(h, e, "pairwise (tcgen05, symmetric)");
            return KL_OK;
        }
        ProfScope ps(h, precision == KL_MIXED_TF32 ? "pair_tc_tf32" : "pair_tc_bf16", pairs);
        if (!h->batcher) {
            cudaError_t e = launch_pair_tc(a, h->stream, &launched);
            h->launches += launched;
            if (e != cudaSuccess) return cuda_fail(h, e, "pairwise (tcgen05)");
            return KL_OK;
        }
        // serving: conversion here, the tcgen05 launch shared with the other
        // running solves, the reduction back on this stream
        BatchJob job;
        job.tf32 = a.tf32;
        job.err = h->d_err;
        cudaError_t e = tc_prepare(a, h->stream, job.inst, &job.n, &job.np, &launched);
        if (e == cudaSuccess && !h->ev_ready) e = cudaEventCreateWithFlags(&h->ev_ready, cudaEventDisableTiming);
        if (e == cudaSuccess && !h->ev_done) e = cudaEventCreateWithFlags(&h->ev_done, cudaEventDisableTiming);
        job.ready = h->ev_ready;
        job.done = h->ev_done;
        if (e == cudaSuccess) e = cudaEventRecord(job.ready, h->stream);
        if (e == cudaSuccess) {
            h->announced = false;  // run() takes the announcement over
            e = h->batcher->run(job);
        }
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, job.done, 0);
        if (e == cudaSuccess) e = tc_finish(a, h->stream, &launched);
        h->launches += launched + 1;
        if (e != cudaSuccess) return cuda_fail(h, e, "pairwise (tcgen05, batched)");
        return KL_OK;
    }
    return fail(h, KL_ERR_ARG, "unknown precision");
}

int check_device_error(kl_solver* h) {
    int v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "device error word");
    if (v != 0) {
        cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream);
        return fail(h, KL_ERR_TIMEOUT, "a bounded wait inside a tensor-core kernel gave up");
    }
    return KL_OK;
}

void clear_graphs(kl_solver* h) {
    for (auto& kv : h->graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    h->graphs.clear();
}

// 1) sum factorisation to the source points, scaled by J (Galerkin) or
//    w det DF (collocation: the field at the quadrature points and its
//    weights, Algorithm 1): X -> ws[0]. With
//    non-tensor NURBS weights R X = (B (w X)) / W, the 1 / W folded into the
//    point scale.
static int apply_pre(kl_solver* h, int which, const double* X, int64_t ldx, int k) {
    const bool gal = galerkin_form(h->prm.method);
    const bool proj = gal && which == 1;
    const double* const* F = proj ? h->P : h->F;
    const double* post = h->rat_w ? h->rat_src_scale : h->src_scale;
    return kron3(h, F, h->N1, h->Ns1, X, ldx, h->ws[0], h->S, k, post, 1, 2, h->rat_w, proj ? nullptr : h->bF);
}

// 3) back to the trial space: Galerkin J, B~^-1, M^T (and L^-1); collocation
//    Z^-1 for A': ws[1] -> Y
static int apply_post(kl_solver* h, int which, double* Y, int64_t ldy, int k) {
    const bool gal = galerkin_form(h->prm.method);
    const bool proj = gal && which == 1;
    const double* const* FT = proj ? h->PT : h->FT;
    double* W = h->ws[1];
    if (gal) return kron3(h, FT, h->Ns1, h->N1, W, h->T, Y, ldy, k, nullptr, 0, 2, nullptr, proj ? nullptr : h->bFT);
    if (which == 1) return kron3(h, h->Zinv, h->N1, h->N1, W, h->T, Y, ldy, k, h->rat_invw, 0, 2, h->rat_Wc);
    cudaError_t e = launch_copy_block(W, h->T, Y, ldy, h->T, k, h->stream);
    ++h->launches;
    if (e != cudaSuccess) return cuda_fail(h, e, "copy");
    return KL_OK;
}

// 2) pairwise product over all (target, source) pairs (the kernel product of
//    Algorithm 1):
//    ws[0] -> ws[1]
static int apply_pair(kl_solver* h, int precision, int k) {
    const bool gal = galerkin_form(h->prm.method);
    return pairwise(h, precision, h->ws[0], h->ws[1], k, gal ? h->src_scale : nullptr);
}

// Runs `enqueue` (kernel launches on the handle's stream only) through the
// graph cache: the first call of a key runs eagerly, the second is captured
// into a CUDA graph (thread-local capture) and later ones replay it.
template <class F>
static int with_graph(kl_solver* h, const kl_solver::GraphKey& key, F&& enqueue) {
    kl_solver::GraphEntry& g = h->graphs[key];
    if (g.exec) {
        cudaError_t e = cudaGraphLaunch(g.exec, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "graph launch");
        h->launches += g.launches;
        return KL_OK;
    }
    if (g.failed || g.uses == 0) {
        const long long l0 = h->launches;
        const int rc = enqueue();
        g.launches = h->launches - l0;
        ++g.uses;
        return rc;
    }
    cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaGetLastError();
        g.failed = true;
        return enqueue();
    }
    const long long l0 = h->launches;
    const int rc = enqueue();
    h->launches = l0;
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(h->stream, &graph);
    if (rc == KL_OK && e == cudaSuccess && graph) e = cudaGraphInstantiate(&g.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (rc != KL_OK || e != cudaSuccess || !g.exec) {
        // capture not possible here: run this and later calls eagerly
        cudaGetLastError();
        g.exec = nullptr;
        g.failed = true;
        if (rc != KL_OK) return rc;
        return enqueue();
    }
    e = cudaGraphLaunch(g.exec, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "graph launch");
    h->launches += g.launches;
    return KL_OK;
}

// An operator application is a fixed sequence of about ten kernels for given
// buffers and block width; with graphs on (default) the solver's repeated
// applications replay captured graphs: the whole application in one graph,
// or, while profiling, the sum-factorisation parts as two graphs around the
// pairwise product, which is launched eagerly between its timing events.
// Served handles run eagerly (the batcher works on the host in the middle
// of the sequence).
int apply_operator(kl_solver* h, int which, int precision, const double* X, int64_t ldx, double* Y,
                   int64_t ldy, int k) {
    if (sym_applies(h, precision, k)) {
        if (int rc = ensure_sym(h, k); rc != KL_OK) return rc;
    }
    auto whole = [&]() -> int {
        int rc = apply_pre(h, which, X, ldx, k);
        if (rc == KL_OK) rc = apply_pair(h, precision, k);
        if (rc == KL_OK) rc = apply_post(h, which, Y, ldy, k);
        return rc;
    };
    if (h->batcher) {
        // served handle: the batcher waits for this product from now on
        if (precision == KL_MIXED_BF16 || precision == KL_MIXED_TF32) {
            h->batcher->announce();
            h->announced = true;
        }
        const int rc = whole();
        if (h->announced) {  // failed before its product reached the batcher
            h->batcher->withdraw();
            h->announced = false;
        }
        return rc;
    }
    if (!h->use_graphs) return whole();
    if (!h->profiling) return with_graph(h, {which, precision, k, X, ldx, Y, ldy, 0}, whole);
    int rc = with_graph(h, {which, precision, k, X, ldx, nullptr, 0, 1}, [&] { return apply_pre(h, which, X, ldx, k); });
    if (rc == KL_OK) rc = apply_pair(h, precision, k);
    if (rc == KL_OK)
        rc = with_graph(h, {which, precision, k, nullptr, 0, Y, ldy, 2}, [&] { return apply_post(h, which, Y, ldy, k); });
    return rc;
}

// Z^-1 (Kronecker LU solves, Sec. 3.2); with non-tensor NURBS weights
// Z = diag(1 / W(x_i)) B diag(w), so Z^-1 = diag(1 / w) B^-1 diag(W(x_i)).
int apply_zinv(kl_solver* h, const double* X, int64_t ldx, double* Y, int64_t ldy, int k) {
    return kron3(h, h->Zinv, h->N1, h->N1, X, ldx, Y, ldy, k, h->rat_invw, 0, 1, h->rat_Wc);
}

int back_transform(kl_solver* h, const double* Yv, int64_t ldy, double* V, int64_t ldv, int k) {
    if (galerkin_form(h->prm.method))
        return kron3(h, h->LinvT, h->N1, h->N1, Yv, ldy, V, ldv, k, nullptr, 0, 1);
    cudaError_t e = launch_copy_block(Yv, ldy, V, ldv, h->N, k, h->stream);
    ++h->launches;
    return e == cudaSuccess ? KL_OK : cuda_fail(h, e, "copy");
}

int field_at_quadrature(kl_solver* h, const double* V, int64_t ldv, double* out, int k) {
    return kron3(h, h->F, h->N1, h->Nq1, V, ldv, out, h->S, k, h->rat_invWq, 1, 2, h->rat_w, h->bF);
}

}  // namespace kl

using namespace kl;

extern "C" {

void kl_default_params(kl_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->dim = 3;
    p->geometry = KL_GEOM_CUBE;
    p->geo[0] = 1.0;
    p->geo[1] = 2.0;
    p->geo[2] = 1.0;
    p->degree = 2;
    p->elems[0] = p->elems[1] = p->elems[2] = 4;
    p->kernel = KL_KERNEL_GAUSS;
    p->sigma = 1.0;
    p->L = 0.5;
    p->method = KL_GALERKIN_IBQ;
    p->interp_continuity = -2;
    p->precision = KL_FP64;
    p->block_k = 8;
    p->refine = -1;
    p->max_restarts = 0;
    p->seed = 2101;
}

const char* kl_status_string(int s) {
    switch (s) {
        case KL_OK: return "ok";
        case KL_ERR_ARG: return "invalid argument";
        case KL_ERR_CUDA: return "CUDA error";
        case KL_ERR_OOM: return "out of device memory";
        case KL_ERR_NOCONV: return "eigensolver did not converge";
        case KL_ERR_NUMERIC: return "numerical breakdown";
        case KL_ERR_TIMEOUT: return "device wait timed out";
        case KL_ERR_UNSUPPORTED: return "unsupported";
        case KL_WARN_COMPLEX: return "complex eigenvalues met";
        default: return "unknown status";
    }
}

const char* kl_last_error(const kl_solver* h) {
    return h ? h->err.c_str() : g_create_error.c_str();
}

// y = ((x)_d A_d) x on the host for square 1D factors A_d (n[d] x n[d]),
// direction 1 fastest.
static void kron3_host(const Mat* const* A, const int* n, const double* x, double* y) {
    const int64_t len = int64_t(n[0]) * n[1] * n[2];
    std::vector<double> cur(x, x + len), nxt(len);
    for (int d = 0; d < 3; ++d) {
        int64_t a = 1, b = 1;
        for (int j = 0; j < d; ++j) a *= n[j];
        for (int j = d + 1; j < 3; ++j) b *= n[j];
        const Mat& M = *A[d];
        for (int64_t ib = 0; ib < b; ++ib)
            for (int i = 0; i < n[d]; ++i)
                for (int64_t ia = 0; ia < a; ++ia) {
                    double s = 0.0;
                    for (int l = 0; l < n[d]; ++l) s += M(i, l) * cur[ia + a * (l + int64_t(n[d]) * ib)];
                    nxt[ia + a * (i + int64_t(n[d]) * ib)] = s;
                }
        cur.swap(nxt);
    }
    std::copy(cur.begin(), cur.end(), y);
}

static std::string check_params(const kl_params& p) {
    if (p.dim < 1 || p.dim > 3) return "dim must be 1, 2 or 3";
    if (p.geometry != KL_GEOM_CUBE && p.geometry != KL_GEOM_QUARTER_ANNULUS && p.geometry != KL_GEOM_HALF_ANNULUS &&
        p.geometry != KL_GEOM_PROJECTIVE_CUBE)
        return "unknown geometry";
    if (p.geometry == KL_GEOM_PROJECTIVE_CUBE) {
        if (p.dim != 3) return "the projective cube needs dim = 3";
        double dmin = 1.0;
        for (int d = 0; d < 3; ++d) {
            if (!std::isfinite(p.geo[d])) return "projective cube: c must be finite";
            dmin += std::min(p.geo[d], 0.0);
        }
        if (!(dmin > 0.0)) return "projective cube: 1 + c . x must stay positive on the unit cube";
    }
    if (p.geometry == KL_GEOM_HALF_ANNULUS && (p.elems[0] < 2 || p.elems[0] % 2))
        return "the half annulus needs an even number of angle elements (both halves together)";
    if (p.geometry == KL_GEOM_QUARTER_ANNULUS || p.geometry == KL_GEOM_HALF_ANNULUS) {
        if (p.dim != 3) return "the annulus needs dim = 3";
        if (!(p.geo[0] > 0 && p.geo[1] > p.geo[0] && p.geo[2] > 0)) return "annulus needs 0 < r_in < r_out, height > 0";
    }
    if (p.degree < 1 || p.degree > 8) return "degree must be in 1..8";
    for (int d = 0; d < p.dim; ++d)
        if (p.elems[d] < 1 || p.elems[d] > 4096) return "elements per direction must be in 1..4096";
    if (p.kernel < KL_KERNEL_GAUSS || p.kernel > KL_KERNEL_CONST) return "unknown kernel";
    if (!(p.sigma > 0) || !std::isfinite(p.sigma)) return "sigma must be > 0";
    if (!(p.L > 0) || !std::isfinite(p.L)) return "L must be > 0";
    if (p.method != KL_GALERKIN_IBQ && p.method != KL_COLLOCATION && p.method != KL_GALERKIN_STD)
        return "unknown method";
    if (p.interp_continuity != -2 && (p.interp_continuity < 0 || p.interp_continuity > p.degree - 1))
        return "interp_continuity must be -2 or in 0..p-1";
    if (p.precision < KL_FP64 || p.precision > KL_MIXED_TF32) return "unknown precision";
    if (p.block_k < 0 || p.block_k > 64) return "block_k must be in 0..64";
    if (p.refine < -1 || p.refine > 2) return "refine must be -1, 0, 1 or 2";
    if (p.max_restarts < 0) return "max_restarts must be >= 0";
    return "";
}

int kl_create(const kl_params* params, void* stream, kl_solver** out) {
    g_create_error.clear();
    if (!params || !out) return fail(nullptr, KL_ERR_ARG, "params and out must not be NULL");
    *out = nullptr;
    std::string msg = check_params(*params);
    if (!msg.empty()) return fail(nullptr, KL_ERR_ARG, msg);

    kl_solver* h = new kl_solver();
    h->prm = *params;
    if (h->prm.block_k == 0) {
        h->prm.block_k = 8;
        h->autotune = true;
    }
    if (h->prm.refine < 0) h->prm.refine = 1;
    if (h->prm.max_restarts == 0) h->prm.max_restarts = 200;
    h->stream = static_cast<cudaStream_t>(stream);
    auto bail = [&](int code) {
        g_create_error = h->err;
        kl_destroy(h);
        return code;
    };
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) return bail(cuda_fail(h, e, "cudaGetDevice"));
    cudaDeviceProp prop;
    if ((e = cudaGetDeviceProperties(&prop, h->device)) != cudaSuccess)
        return bail(cuda_fail(h, e, "cudaGetDeviceProperties"));
    h->sm_count = prop.multiProcessorCount;
    h->cc_major = prop.major;
    h->cc_minor = prop.minor;
    if ((h->prm.precision == KL_MIXED_BF16 || h->prm.precision == KL_MIXED_TF32) && h->cc_major != 10)
        return bail(fail(h, KL_ERR_UNSUPPORTED, "tcgen05 precisions need an sm_100-class GPU"));

    const kl_params& p = h->prm;
    const bool ibq = p.method == KL_GALERKIN_IBQ;
    const bool stdg = p.method == KL_GALERKIN_STD;  // Gauss points as sources and targets
    const bool gal = ibq || stdg;
    const bool exp_kernel = p.kernel == KL_KERNEL_EXP || p.kernel == KL_KERNEL_EXP_SEP;
    const int icont = p.interp_continuity == -2 ? (exp_kernel ? 0 : p.degree - 1) : p.interp_continuity;

    // ---- host set-up per direction ----
    Dir1D dir[3];
    for (int d = 0; d < 3; ++d) {
        const bool present = d < p.dim;
        const int arc = d != 0 ? 0 : p.geometry == KL_GEOM_QUARTER_ANNULUS ? 1 : p.geometry == KL_GEOM_HALF_ANNULUS ? 2 : 0;
        std::string m = setup_direction(dir[d], present, present ? p.elems[d] : 1, p.degree, icont,
                                        arc, gal, !gal);
        if (!m.empty()) return bail(fail(h, KL_ERR_NUMERIC, "set-up: " + m));
        h->N1[d] = dir[d].N;
        h->Nt1[d] = dir[d].Nt;
        h->Nq1[d] = dir[d].nq;
        h->Ns1[d] = ibq ? dir[d].Nt : stdg ? dir[d].ne : dir[d].nq;
    }
    h->N = prod3(h->N1);
    h->S = prod3(h->Ns1);
    h->T = gal ? h->S : h->N;

    // ---- tables: pack every 1D array into one host buffer, upload once ----
    std::vector<double> buf;
    std::vector<size_t> off;
    auto push = [&](const std::vector<double>& v) {
        off.push_back(buf.size());
        buf.insert(buf.end(), v.begin(), v.end());
        while (buf.size() % 4) buf.push_back(0.0);  // 32-byte alignment
    };
    for (int d = 0; d < 3; ++d) {
        const Dir1D& q = dir[d];
        if (ibq) {
            push(q.Q.a);
            push(transpose(q.Q).a);
            push(q.P.a);
            push(transpose(q.P).a);
            push(q.Zinv_gal.a);
            push(q.LinvT.a);
        } else if (stdg) {
            // trial functions at the Gauss points (times sqrt(det DF) on the
            // device), and with L^-T folded in for A'
            const Mat EL = matmul(q.E, q.LinvT);
            push(q.E.a);
            push(transpose(q.E).a);
            push(EL.a);
            push(transpose(EL).a);
            push(q.Zinv_gal.a);
            push(q.LinvT.a);
        } else {
            push(q.R.a);
            push(transpose(q.R).a);
            push(q.R.a);  // unused P slot
            push(transpose(q.R).a);
            push(q.Zinv_col.a);
            push(identity(q.N).a);
        }
    }
    for (int d = 0; d < 3; ++d) push(ibq ? dir[d].xg : stdg ? dir[d].xe : dir[d].xc);  // target params
    for (int d = 0; d < 3; ++d) push(ibq ? dir[d].xg : stdg ? dir[d].xe : dir[d].xq);  // source params
    for (int d = 0; d < 3; ++d) push(ibq ? std::vector<double>(dir[d].Nt, 1.0) : stdg ? dir[d].we : dir[d].wq);
    for (int d = 0; d < 3; ++d) push(dir[d].E.a);   // trial basis at the Gauss points
    for (int d = 0; d < 3; ++d) push(dir[d].xe);    // those points
    if ((e = dalloc(h, &h->d_tables, int64_t(buf.size()))) != cudaSuccess)
        return bail(cuda_fail(h, e, "table alloc"));
    if ((e = cudaMemcpyAsync(h->d_tables, buf.data(), buf.size() * sizeof(double),
                             cudaMemcpyHostToDevice, h->stream)) != cudaSuccess)
        return bail(cuda_fail(h, e, "table upload"));
    h->h2d_bytes += int64_t(buf.size() * sizeof(double));
    for (int d = 0; d < 3; ++d) {
        h->F[d] = h->d_tables + off[6 * d + 0];
        h->FT[d] = h->d_tables + off[6 * d + 1];
        h->P[d] = h->d_tables + off[6 * d + 2];
        h->PT[d] = h->d_tables + off[6 * d + 3];
        h->Zinv[d] = h->d_tables + off[6 * d + 4];
        h->LinvT[d] = h->d_tables + off[6 * d + 5];
    }
    for (int j = 0; j < 9; ++j) h->pts1d[j] = h->d_tables + off[18 + j];
    {
        // banded forms of F, F^T and E (B-spline supports: p + 1 entries per
        // row of F and E; a trial function spans p + 1 elements of Gauss
        // points in F^T); dense projections are left dense
        std::vector<double> bv;
        std::vector<int> bs;
        struct Pending {
            Band* dst;
            size_t v0, s0;
            int w;
        };
        std::vector<Pending> pend;
        for (int d = 0; d < 3; ++d) {
            const Dir1D& q = dir[d];
            const Mat* Fm = ibq ? &q.Q : stdg ? &q.E : &q.R;
            const Mat FTm = transpose(*Fm);
            const Mat* tabs[3] = {Fm, &FTm, &q.E};
            Band* dst[3] = {&h->bF[d], &h->bFT[d], &h->bE[d]};
            for (int t = 0; t < 3; ++t) {
                const Mat& T = *tabs[t];
                std::vector<int> lo(T.rows, 0);
                int w = 1;
                for (int i = 0; i < T.rows; ++i) {
                    int a = -1, b = -1;
                    for (int j = 0; j < T.cols; ++j)
                        if (T(i, j) != 0.0) {
                            if (a < 0) a = j;
                            b = j;
                        }
                    lo[i] = a < 0 ? 0 : a;
                    if (a >= 0) w = std::max(w, b - a + 1);
                }
                if (2 * w > T.cols) continue;  // not worth a band
                Pending p{dst[t], bv.size(), bs.size(), w};
                for (int i = 0; i < T.rows; ++i) {
                    const int s0 = std::min(lo[i], T.cols - w);
                    bs.push_back(s0);
                    for (int j = 0; j < w; ++j) bv.push_back(T(i, s0 + j));
                }
                while (bv.size() % 4) bv.push_back(0.0);
                while (bs.size() % 4) bs.push_back(0);
                pend.push_back(p);
            }
        }
        if (!pend.empty()) {
            if ((e = dalloc(h, &h->d_band_vals, int64_t(bv.size()))) != cudaSuccess)
                return bail(cuda_fail(h, e, "band alloc"));
            if ((e = device_alloc((void**)&h->d_band_start, bs.size() * sizeof(int))) != cudaSuccess)
                return bail(cuda_fail(h, e, "band alloc"));
            h->dev_bytes += int64_t(bs.size() * sizeof(int));
            e = cudaMemcpyAsync(h->d_band_vals, bv.data(), bv.size() * sizeof(double), cudaMemcpyHostToDevice,
                                h->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(h->d_band_start, bs.data(), bs.size() * sizeof(int), cudaMemcpyHostToDevice,
                                    h->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);  // host vectors are temporaries
            if (e != cudaSuccess) return bail(cuda_fail(h, e, "band upload"));
            h->h2d_bytes += int64_t(bv.size() * sizeof(double) + bs.size() * sizeof(int));
            for (const Pending& p : pend) {
                p.dst->vals = h->d_band_vals + p.v0;
                p.dst->start = h->d_band_start + p.s0;
                p.dst->w = p.w;
            }
        }
    }
    for (int d = 0; d < 3; ++d) {
        h->E[d] = h->d_tables + off[27 + d];
        h->xe[d] = h->d_tables + off[30 + d];
        h->Ne1[d] = dir[d].ne;
    }

    // ---- point sets and geometry factors on the device ----
    const int64_t T = h->T, S = h->S;
    const int64_t npts = gal ? 4 * S : 3 * T + 4 * S;
    if ((e = dalloc(h, &h->d_points, npts)) != cudaSuccess) return bail(cuda_fail(h, e, "points alloc"));
    if ((e = dalloc(h, &h->d_points32, 3 * T + 3 * S)) != cudaSuccess)
        return bail(cuda_fail(h, e, "points alloc"));
    if ((e = dalloc(h, &h->d_err, 1)) != cudaSuccess) return bail(cuda_fail(h, e, "error word alloc"));
    if ((e = cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream)) != cudaSuccess)
        return bail(cuda_fail(h, e, "error word"));
    double geo[3] = {p.geo[0], p.geo[1], p.geo[2]};
    const int* nsrc = h->Ns1;
    h->sx = h->d_points;
    h->sy = h->sx + S;
    h->sz = h->sy + S;
    h->src_scale = h->sz + S;
    e = launch_tensor_points(p.geometry, geo, h->pts1d[3], h->pts1d[4], h->pts1d[5], nsrc[0], nsrc[1],
                             nsrc[2], ibq ? nullptr : h->pts1d[6], ibq ? nullptr : h->pts1d[7],
                             ibq ? nullptr : h->pts1d[8], gal ? 0.5 : 1.0, h->sx, h->sy, h->sz,
                             h->src_scale, h->stream);
    ++h->launches;
    if (e != cudaSuccess) return bail(cuda_fail(h, e, "source points"));
    if (gal) {
        h->tx = h->sx;
        h->ty = h->sy;
        h->tz = h->sz;
    } else {
        h->tx = h->src_scale + S;
        h->ty = h->tx + T;
        h->tz = h->ty + T;
        e = launch_tensor_points(p.geometry, geo, h->pts1d[0], h->pts1d[1], h->pts1d[2], h->N1[0],
                                 h->N1[1], h->N1[2], nullptr, nullptr, nullptr, 0.0, h->tx, h->ty,
                                 h->tz, nullptr, h->stream);
        ++h->launches;
        if (e != cudaSuccess) return bail(cuda_fail(h, e, "target points"));
    }
    h->tx32 = h->d_points32;
    h->ty32 = h->tx32 + T;
    h->tz32 = h->ty32 + T;
    h->sx32 = h->tz32 + T;
    h->sy32 = h->sx32 + S;
    h->sz32 = h->sy32 + S;
    const double* src64[6] = {h->tx, h->ty, h->tz, h->sx, h->sy, h->sz};
    float* dst32[6] = {h->tx32, h->ty32, h->tz32, h->sx32, h->sy32, h->sz32};
    double centre[3];
    domain_centre(p, centre);
    for (int j = 0; j < 6; ++j) {
        const int64_t n = j < 3 ? T : S;
        to_float_kernel<<<int(std::min<int64_t>((n + 255) / 256, 4096)), 256, 0, h->stream>>>(src64[j], dst32[j], n,
                                                                                                centre[j % 3]);
        ++h->launches;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return bail(cuda_fail(h, e, "points fp32"));
    int rc = ensure_workspace(h, h->prm.block_k);
    if (rc != KL_OK) return bail(rc);
    if (p.geometry == KL_GEOM_PROJECTIVE_CUBE && !gal) {
        // NURBS weights of the collocation trial space: the coefficients of
        // the weight function W = 1 + c . x^ in the B-spline basis, found by
        // interpolation at the Greville points (Kronecker solves, exact:
        // W lies in the space); W itself at the Gauss points is B w.
        const int64_t N = h->N;
        std::vector<double> host(3 * N);
        double* w = host.data();
        double* iw = w + N;
        double* Wc = iw + N;
        for (int i3 = 0; i3 < h->N1[2]; ++i3)
            for (int i2 = 0; i2 < h->N1[1]; ++i2)
                for (int i1 = 0; i1 < h->N1[0]; ++i1)
                    Wc[i1 + int64_t(h->N1[0]) * (i2 + int64_t(h->N1[1]) * i3)] =
                        1.0 + p.geo[0] * dir[0].xc[i1] + p.geo[1] * dir[1].xc[i2] + p.geo[2] * dir[2].xc[i3];
        const Mat* Zi[3] = {&dir[0].Zinv_col, &dir[1].Zinv_col, &dir[2].Zinv_col};
        kron3_host(Zi, h->N1, Wc, w);
        for (int64_t i = 0; i < N; ++i) {
            if (!(w[i] > 0.0)) return bail(fail(h, KL_ERR_NUMERIC, "set-up: NURBS weight not positive"));
            iw[i] = 1.0 / w[i];
        }
        if ((e = dalloc(h, &h->d_rat, 3 * N + 2 * S)) != cudaSuccess) return bail(cuda_fail(h, e, "weights alloc"));
        h->rat_w = h->d_rat;
        h->rat_invw = h->rat_w + N;
        h->rat_Wc = h->rat_invw + N;
        h->rat_invWq = h->rat_Wc + N;
        h->rat_src_scale = h->rat_invWq + S;
        if ((e = cudaMemcpyAsync(h->d_rat, host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice,
                                 h->stream)) != cudaSuccess)
            return bail(cuda_fail(h, e, "weights upload"));
        h->h2d_bytes += int64_t(host.size() * sizeof(double));
        if ((rc = kron3_s(h, h->F, h->N1, h->Ns1, h->rat_w, N, h->rat_invWq, S, 1, nullptr, h->ws[1], h->ws[2])) !=
            KL_OK)
            return bail(rc);
        e = launch_rational_scales(h->rat_invWq, h->src_scale, h->rat_src_scale, S, h->stream);
        ++h->launches;
        if (e != cudaSuccess) return bail(cuda_fail(h, e, "weight scales"));
        // the host buffer is a temporary
        if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return bail(cuda_fail(h, e, "weights sync"));
    }
    if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return bail(cuda_fail(h, e, "create sync"));
    *out = h;
    return KL_OK;
}

int64_t kl_sample_size(const kl_solver* h) {
    return h ? int64_t(h->Ne1[0]) * h->Ne1[1] * h->Ne1[2] : 0;
}

int kl_sample_points(kl_solver* h, double* xyz) {
    if (!h) return KL_ERR_ARG;
    if (!xyz) return fail(h, KL_ERR_ARG, "xyz must not be NULL");
    const int64_t Q = kl_sample_size(h);
    double geo[3] = {h->prm.geo[0], h->prm.geo[1], h->prm.geo[2]};
    cudaError_t e = launch_tensor_points(h->prm.geometry, geo, h->xe[0], h->xe[1], h->xe[2], h->Ne1[0], h->Ne1[1],
                                         h->Ne1[2], nullptr, nullptr, nullptr, 0.0, xyz, xyz + Q, xyz + 2 * Q,
                                         nullptr, h->stream);
    ++h->launches;
    if (e != cudaSuccess) return cuda_fail(h, e, "sample points");
    return KL_OK;
}

int kl_sample(kl_solver* h, int M, const double* lambda, const double* V, int64_t ldv, const double* xi,
              int64_t ldxi, int ns, double* out, int64_t ldo) {
    if (!h) return KL_ERR_ARG;
    const int64_t Q = kl_sample_size(h), N = h->N;
    if (!lambda || !V || !xi || !out) return fail(h, KL_ERR_ARG, "lambda, V, xi and out must not be NULL");
    if (M < 1 || M > N) return fail(h, KL_ERR_ARG, "M must be in 1..N");
    if (ns < 1) return fail(h, KL_ERR_ARG, "ns must be >= 1");
    if (ldv < N || ldxi < M || ldo < Q) return fail(h, KL_ERR_ARG, "leading dimensions too small");
    // scratch: sqrt(lambda) (M), diag(sqrt lambda) xi (M x ns), C = V diag xi (N x ns),
    // two intermediate products of the evaluation (<= Q x ns each)
    const bool gal = galerkin_form(h->prm.method);
    const int64_t need = (M + 3) / 4 * 4 + int64_t(M) * ns + N * ns + 2 * Q * ns + (gal ? 4 * Q : 0);
    if (need > h->smp_cap) {
        cudaError_t e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "sample sync");
        if (h->smp_ws) {
            cudaFree(h->smp_ws);
            h->dev_bytes -= h->smp_cap * int64_t(sizeof(double));
            h->smp_ws = nullptr;
            h->smp_cap = 0;
        }
        e = device_alloc((void**)&h->smp_ws, size_t(need) * sizeof(double));
        if (e != cudaSuccess) return cuda_fail(h, e, "sample workspace");
        h->smp_cap = need;
        h->dev_bytes += need * int64_t(sizeof(double));
    }
    std::vector<double> sq(M);
    for (int m = 0; m < M; ++m) sq[m] = std::sqrt(std::max(lambda[m], 0.0));
    double* d_sq = h->smp_ws;
    double* Xs = d_sq + (M + 3) / 4 * 4;
    double* C = Xs + int64_t(M) * ns;
    double* sa = C + N * ns;
    double* sb = sa + Q * ns;
    // Galerkin trial functions are B_j(x^) / sqrt(det DF(x^)) (Sec. 3.1):
    // per-point factor |det DF|^(-1/2) at the grid (x, y, z scratch before it)
    double* jscale = gal ? sb + Q * ns + 3 * Q : nullptr;
    cudaError_t e = cudaSuccess;
    if (gal) {
        double geo[3] = {h->prm.geo[0], h->prm.geo[1], h->prm.geo[2]};
        double* xyz = sb + Q * ns;
        e = launch_tensor_points(h->prm.geometry, geo, h->xe[0], h->xe[1], h->xe[2], h->Ne1[0], h->Ne1[1],
                                 h->Ne1[2], nullptr, nullptr, nullptr, -0.5, xyz, xyz + Q, xyz + 2 * Q, jscale,
                                 h->stream);
        ++h->launches;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_sq, sq.data(), M * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);  // sq is a host temporary
    // diag(sqrt lambda) xi: the transpose view (ns x M) scaled by columns
    if (e == cudaSuccess) e = launch_copy_block(xi, ldxi, Xs, M, M, ns, h->stream);
    if (e == cudaSuccess) e = launch_scale_rows(Xs, M, M, ns, d_sq, h->stream);
    if (e == cudaSuccess) e = launch_gemm_nn(V, ldv, Xs, M, C, N, N, M, ns, 1.0, 0.0, h->stream);
    h->launches += 3;
    if (e != cudaSuccess) return cuda_fail(h, e, "sample");
    // collocation with non-tensor NURBS weights: (B (w C)) / W at the Gauss grid
    return kron3_s(h, h->E, h->N1, h->Ne1, C, N, out, ldo, ns, gal ? jscale : h->rat_invWq, sa, sb, h->rat_w, h->bE);
}

int kl_set_graphs(kl_solver* h, int on) {
    if (!h) return KL_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "kl_set_graphs");
    h->use_graphs = on != 0;
    if (!h->use_graphs) clear_graphs(h);
    return KL_OK;
}

int kl_set_shared_sms(kl_solver* h, int n) {
    if (!h) return KL_ERR_ARG;
    if (n < 0 || n >= h->sm_count) return fail(h, KL_ERR_ARG, "shared SMs must lie in [0, SM count)");
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "kl_set_shared_sms");
    if (n != h->shared_sms) {
        h->shared_sms = n;
        clear_graphs(h);  // captured launches hold the old grid
    }
    return KL_OK;
}

int kl_block_size(const kl_solver* h) { return h ? h->prm.block_k : 0; }

int kl_estimate_bytes(const kl_params* params, int M, int64_t* bytes) {
    g_create_error.clear();
    if (!params || !bytes) return fail(nullptr, KL_ERR_ARG, "params and bytes must not be NULL");
    if (M < 1) return fail(nullptr, KL_ERR_ARG, "M must be >= 1");
    std::string msg = check_params(*params);
    if (!msg.empty()) return fail(nullptr, KL_ERR_ARG, msg);
    kl_params p = *params;
    if (p.block_k == 0) p.block_k = 8;
    const bool ibq = p.method == KL_GALERKIN_IBQ;
    const bool stdg = p.method == KL_GALERKIN_STD;
    const bool gal = ibq || stdg;
    const bool exp_kernel = p.kernel == KL_KERNEL_EXP || p.kernel == KL_KERNEL_EXP_SEP;
    const int icont = p.interp_continuity == -2 ? (exp_kernel ? 0 : p.degree - 1) : p.interp_continuity;
    int64_t N = 1, Ns = 1, tab = 0;
    auto add = [&](int64_t n) { tab += (n + 3) / 4 * 4; };
    for (int d = 0; d < 3; ++d) {
        Dir1D q;
        const bool present = d < p.dim;
        const int arc = d != 0 ? 0 : p.geometry == KL_GEOM_QUARTER_ANNULUS ? 1 : p.geometry == KL_GEOM_HALF_ANNULUS ? 2 : 0;
        std::string m = setup_direction(q, present, present ? p.elems[d] : 1, p.degree, icont, arc, gal, !gal);
        if (!m.empty()) return fail(nullptr, KL_ERR_NUMERIC, "set-up: " + m);
        const int64_t ns = ibq ? q.Nt : stdg ? q.ne : q.nq;
        N *= q.N;
        Ns *= ns;
        for (int i = 0; i < 4; ++i) add(ns * q.N);
        add(int64_t(q.N) * q.N);
        add(int64_t(q.N) * q.N);
        add(gal ? ns : q.N);
        add(ns);
        add(ns);
        add(int64_t(q.ne) * q.N);
        add(q.ne);
    }
    const int64_t S = Ns, T = gal ? S : N;
    int sm = 152;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) == cudaSuccess && ndev > 0) sm = device_sm_count();
    else cudaGetLastError();
    const int b = int(std::min<int64_t>(p.block_k, N));
    const int mcap = eig_basis_cap(N, std::min<int64_t>(M, N), b);
    // widest operator application: the final refinement of nkeep + 1 vectors
    const int kmax = std::max(b, (M + 2 * b - 1) / b * b + 1);
    const int64_t points = (gal ? 4 * S : 3 * T + 4 * S) + (3 * T + 3 * S + 1) / 2 + 1 +
                           (p.geometry == KL_GEOM_PROJECTIVE_CUBE && !gal ? 3 * N + 2 * S : 0);
    const int64_t ws = 3 * std::max(S, T) * int64_t(kmax);
    const int64_t pair = std::max<int64_t>(pair_scratch_doubles(T, kmax, pair_choose_splits(T, S, sm)),
                                           tc_scratch_doubles(T, S, kmax, sm));
    const int64_t eig = eig_workspace_doubles(N, mcap);
    const int64_t total = 8 * (tab + points + ws + pair + eig);
    // allocation granularity and runtime bookkeeping
    *bytes = total + total / 32 + (int64_t(8) << 20);
    return KL_OK;
}

int kl_destroy(kl_solver* h) {
    if (!h) return KL_OK;
    if (h->stream || true) cudaStreamSynchronize(h->stream);
    for (auto& kv : h->prof)
        for (auto& pe : kv.second.pending) {
            cudaEventDestroy(pe.first);
            cudaEventDestroy(pe.second);
        }
    dfree(h->d_tables);
    dfree(h->d_points);
    dfree(h->d_points32);
    dfree(h->d_rat);
    dfree(h->d_band_vals);
    dfree(h->d_band_start);
    for (int i = 0; i < 3; ++i) dfree(h->ws[i]);
    dfree(h->pair_scratch);
    dfree(h->sym_scratch);
    delete h->sym_plan;
    dfree(h->eig_ws);
    dfree(h->d_err);
    dfree(h->smp_ws);
    clear_graphs(h);
    if (h->ev_ready) cudaEventDestroy(h->ev_ready);
    if (h->ev_done) cudaEventDestroy(h->ev_done);
    delete h;
    return KL_OK;
}

int kl_dims(const kl_solver* h, int64_t* N, int64_t* n_src, int64_t* n_tgt) {
    if (!h) return KL_ERR_ARG;
    if (N) *N = h->N;
    if (n_src) *n_src = h->S;
    if (n_tgt) *n_tgt = h->T;
    return KL_OK;
}

static int check_block(kl_solver* h, const double* X, int64_t ldx, const double* Y, int64_t ldy, int k) {
    if (!X || !Y) return fail(h, KL_ERR_ARG, "X and Y must not be NULL");
    if (k < 1 || k > 256) return fail(h, KL_ERR_ARG, "k must be in 1..256");
    if (ldx < h->N || ldy < h->N) return fail(h, KL_ERR_ARG, "leading dimensions must be >= N");
    return KL_OK;
}

int kl_apply_A(kl_solver* h, const double* X, int64_t ldx, double* Y, int64_t ldy, int k) {
    if (!h) return KL_ERR_ARG;
    int rc = check_block(h, X, ldx, Y, ldy, k);
    if (rc != KL_OK) return rc;
    if ((rc = ensure_workspace(h, k)) != KL_OK) return rc;
    return apply_operator(h, 0, h->prm.precision, X, ldx, Y, ldy, k);
}

int kl_apply_Aprime(kl_solver* h, const double* X, int64_t ldx, double* Y, int64_t ldy, int k) {
    if (!h) return KL_ERR_ARG;
    int rc = check_block(h, X, ldx, Y, ldy, k);
    if (rc != KL_OK) return rc;
    if ((rc = ensure_workspace(h, k)) != KL_OK) return rc;
    return apply_operator(h, 1, h->prm.precision, X, ldx, Y, ldy, k);
}

int kl_apply_Zinv(kl_solver* h, const double* X, int64_t ldx, double* Y, int64_t ldy, int k) {
    if (!h) return KL_ERR_ARG;
    int rc = check_block(h, X, ldx, Y, ldy, k);
    if (rc != KL_OK) return rc;
    if ((rc = ensure_workspace(h, k)) != KL_OK) return rc;
    return apply_zinv(h, X, ldx, Y, ldy, k);
}

int kl_profile_enable(kl_solver* h, int on) {
    if (!h) return KL_ERR_ARG;
    cudaStreamSynchronize(h->stream);
    for (auto& kv : h->prof)
        for (auto& pe : kv.second.pending) {
            cudaEventDestroy(pe.first);
            cudaEventDestroy(pe.second);
        }
    h->prof.clear();
    h->profiling = on != 0;
    return KL_OK;
}

int kl_profile_read(kl_solver* h, kl_kernel_stats* out, int cap, int* n) {
    if (!h) return KL_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "profile sync");
    int i = 0;
    for (auto& kv : h->prof) {
        kl_prof_entry& p = kv.second;
        for (size_t j = 0; j < p.pending.size(); ++j) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, p.pending[j].first, p.pending[j].second);
            p.ms += ms;
            p.units += p.pending_units[j];
            p.launches += 1;
            cudaEventDestroy(p.pending[j].first);
            cudaEventDestroy(p.pending[j].second);
        }
        p.pending.clear();
        p.pending_units.clear();
        if (out && i < cap) {
            std::memset(&out[i], 0, sizeof(kl_kernel_stats));
            std::snprintf(out[i].name, sizeof(out[i].name), "%s", kv.first.c_str());
            out[i].launches = p.launches;
            out[i].ms = p.ms;
            out[i].units = p.units;
        }
        ++i;
    }
    if (n) *n = i;
    return KL_OK;
}

long long kl_launch_count(const kl_solver* h) { return h ? h->launches : 0; }

int kl_debug_set(kl_solver* h, int what, long long value) {
    switch (what) {
        case KL_DEBUG_WAIT_LIMIT:
            if (!h) return fail(nullptr, KL_ERR_ARG, "KL_DEBUG_WAIT_LIMIT needs a handle");
            if (value < 0) return fail(h, KL_ERR_ARG, "wait limit must be >= 0");
            if (cudaError_t e = cudaStreamSynchronize(h->stream); e != cudaSuccess)
                return cuda_fail(h, e, "kl_debug_set");
            h->wait_limit = value;
            clear_graphs(h);  // captured launches carry the old limit
            return KL_OK;
        case KL_DEBUG_FAIL_ALLOC:
            if (value < 0) return fail(h, KL_ERR_ARG, "allocation count must be >= 0");
            g_fail_alloc_in.store(value);
            return KL_OK;
        case KL_DEBUG_NAN_START:
            if (!h) return fail(nullptr, KL_ERR_ARG, "KL_DEBUG_NAN_START needs a handle");
            h->nan_start = value != 0;
            return KL_OK;
        case KL_DEBUG_PAIR_DENSE:
            if (!h) return fail(nullptr, KL_ERR_ARG, "KL_DEBUG_PAIR_DENSE needs a handle");
            if (cudaError_t e = cudaStreamSynchronize(h->stream); e != cudaSuccess)
                return cuda_fail(h, e, "kl_debug_set");
            h->pair_dense = value != 0;
            clear_graphs(h);  // captured launches use the other form
            return KL_OK;
        default:
            return fail(h, KL_ERR_ARG, "unknown debug setting");
    }
}

int kl_memory(const kl_solver* h, int64_t* h2d_bytes, int64_t* device_bytes) {
    if (!h) return KL_ERR_ARG;
    if (h2d_bytes) *h2d_bytes = h->h2d_bytes;
    if (device_bytes) *device_bytes = h->dev_bytes;
    return KL_OK;
}

}  // extern "C"
