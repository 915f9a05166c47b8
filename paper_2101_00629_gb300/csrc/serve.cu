// Serving: continuous batching of K-L solves on one GPU (no paper passage:
// the paper solves one problem at a time on one CPU core, Sec. 4).
//
//   * kl_server: a FIFO queue of requests, max_slots worker threads and an
//     HBM budget. A worker takes the first queued request (of the first 8)
//     whose memory estimate fits what is left of the budget, creates a
//     handle on its own stream and runs kl_eigs; the handle (tables, Krylov
//     basis, workspaces) stays on the device for the whole solve and is freed
//     at the end, which admits the next requests.
//   * Batcher: the tensor-core pairwise products of all running solves go
//     through one thread. A worker converts its source block on its own
//     stream, records an event and hands the product's instance descriptors
//     to the batcher; the batcher waits (at most batch_window_us) for the
//     other running solves' products, makes its stream wait on their events
//     and issues ONE persistent launch over all of them (instances of
//     different meshes, degrees and kernels; one launch per precision and
//     block width), then records an event per product. Each worker's stream
//     waits on its event and reduces its own partial sums.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "handle.h"
#include "kernels_tc.h"
#include "serve.h"

namespace kl {

namespace {

using Clock = std::chrono::steady_clock;

double ms_since(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct ErrTargets {
    int* dst[kTcMaxBatch];
    int n;
};

// A bounded wait inside a batched launch sets the batcher's word; pass it on
// to every handle whose product was in the launch, then clear it.
__global__ void forward_error_kernel(int* src, const __grid_constant__ ErrTargets t) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const int v = *src;
        if (v) {
            for (int i = 0; i < t.n; ++i) *t.dst[i] = 1;
            *src = 0;
        }
    }
}

}  // namespace

Batcher::Batcher(int device, int window_us, int sm_count)
    : device_(device), window_us_(window_us), sm_count_(sm_count) {
    cudaError_t e = cudaSetDevice(device_);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&stream_, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&d_err_, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(d_err_, 0, sizeof(int));
    init_error_ = e;
    thread_ = std::thread([this] { loop(); });
}

Batcher::~Batcher() {
    {
        std::lock_guard<std::mutex> lk(mu_);
        stop_ = true;
    }
    cv_work_.notify_all();
    if (thread_.joinable()) thread_.join();
    if (stream_) cudaStreamDestroy(stream_);
    if (d_err_) cudaFree(d_err_);
}

void Batcher::set_expected(int n) {
    {
        std::lock_guard<std::mutex> lk(mu_);
        expected_ = n;
    }
    cv_work_.notify_all();
}

void Batcher::announce() {
    std::lock_guard<std::mutex> lk(mu_);
    ++announced_;
}

void Batcher::withdraw() {
    {
        std::lock_guard<std::mutex> lk(mu_);
        if (announced_ > 0) --announced_;
    }
    cv_work_.notify_all();
}

cudaError_t Batcher::run(BatchJob& job) {
    std::unique_lock<std::mutex> lk(mu_);
    if (announced_ > 0) --announced_;
    if (init_error_ != cudaSuccess) return init_error_;
    job.launched = false;
    job.error = cudaSuccess;
    pending_.push_back(&job);
    cv_work_.notify_all();
    cv_done_.wait(lk, [&] { return job.launched; });
    return job.error;
}

BatcherStats Batcher::stats() {
    std::lock_guard<std::mutex> lk(mu_);
    return stats_;
}

void Batcher::loop() {
    cudaSetDevice(device_);
    while (true) {
        std::vector<BatchJob*> take;
        {
            std::unique_lock<std::mutex> lk(mu_);
            cv_work_.wait(lk, [&] { return stop_ || !pending_.empty(); });
            if (pending_.empty()) {
                if (stop_) break;
                continue;
            }
            // gather: wait for the products the running solves have announced
            // (they are in their sum factorisation and submit within
            // microseconds), at most window_us after the first one arrived;
            // solves busy with their orthogonalisation or Rayleigh-Ritz step
            // are not waited for
            const auto until = Clock::now() + std::chrono::microseconds(window_us_);
            while (!stop_ && announced_ > 0 && int(pending_.size()) < expected_) {
                if (cv_work_.wait_until(lk, until) == std::cv_status::timeout) break;
            }
            take.swap(pending_);
        }
        // group by (precision, block width); at most kTcMaxBatch instances
        // per launch
        std::vector<bool> used(take.size(), false);
        for (size_t i = 0; i < take.size(); ++i) {
            if (used[i]) continue;
            std::vector<BatchJob*> grp;
            int ninst = 0;
            for (size_t j = i; j < take.size(); ++j) {
                if (used[j] || take[j]->tf32 != take[i]->tf32 || take[j]->np != take[i]->np) continue;
                if (ninst + take[j]->n > kTcMaxBatch) continue;
                used[j] = true;
                grp.push_back(take[j]);
                ninst += take[j]->n;
            }
            TcBatch b;
            b.ninst = 0;
            b.wait_limit = 0;
            ErrTargets et;
            et.n = 0;
            cudaError_t err = cudaSuccess;
            for (BatchJob* jb : grp) {
                if (err == cudaSuccess) err = cudaStreamWaitEvent(stream_, jb->ready, 0);
                for (int q = 0; q < jb->n; ++q) b.inst[b.ninst++] = jb->inst[q];
                et.dst[et.n++] = jb->err;
            }
            if (err == cudaSuccess) err = tc_launch_batch(b, grp[0]->tf32, grp[0]->np, sm_count_, d_err_, stream_);
#ifdef KL_CHECK_BOUNDS
            for (int q = 0; q < et.n && err == cudaSuccess; ++q)
                err = check_range(et.dst[q], sizeof(int), "batch error target");
#endif
            if (err == cudaSuccess) {
                forward_error_kernel<<<1, 32, 0, stream_>>>(d_err_, et);
                err = cudaGetLastError();
            }
            for (BatchJob* jb : grp)
                if (err == cudaSuccess) err = cudaEventRecord(jb->done, stream_);
            std::lock_guard<std::mutex> lk(mu_);
            stats_.batches += 1;
            stats_.products += int64_t(grp.size());
            stats_.max_batch = std::max(stats_.max_batch, int(grp.size()));
            for (BatchJob* jb : grp) {
                jb->error = err;
                jb->launched = true;
            }
        }
        cv_done_.notify_all();
    }
}

}  // namespace kl

// ---------------------------------------------------------------------------
// Server
// ---------------------------------------------------------------------------
using namespace kl;

namespace {

struct ServeRequest {
    kl_params prm;
    int M;
    double tol;
    int64_t id;
    double* lambda_out;
    double* V_out;
    int64_t ldv;
    int64_t est;
    Clock::time_point t_submit;
};

}  // namespace

struct kl_server {
    kl_serve_config cfg{};
    int device = 0;
    Batcher* batcher = nullptr;
    std::vector<std::thread> workers;
    std::mutex mu;
    std::condition_variable cv_queue, cv_done;
    std::deque<ServeRequest> queue;
    std::deque<kl_serve_result> done;
    int64_t used = 0;
    int active = 0, running_workers = 0;
    bool stop = false;
    kl_serve_stats st{};
};

namespace {

// Index (among the first 8) of the first queued request that fits; -1 if none.
int admissible(const kl_server* s) {
    const int n = int(std::min<size_t>(s->queue.size(), 8));
    for (int i = 0; i < n; ++i)
        if (s->used + s->queue[i].est <= s->cfg.hbm_budget_bytes) return i;
    return -1;
}

void worker(kl_server* s) {
    cudaSetDevice(s->device);
    cudaStream_t stream = nullptr;
    const bool have_stream = cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) == cudaSuccess;
    while (true) {
        ServeRequest r;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            int idx = -1;
            s->cv_queue.wait(lk, [&] { return (s->stop && s->queue.empty()) || (idx = admissible(s)) >= 0; });
            if (idx < 0) break;
            r = s->queue[idx];
            s->queue.erase(s->queue.begin() + idx);
            s->used += r.est;
            s->active += 1;
            s->st.max_concurrent = std::max(s->st.max_concurrent, s->active);
            s->st.peak_est_bytes = std::max(s->st.peak_est_bytes, s->used);
            s->batcher->set_expected(s->active);
        }
        const auto t_start = Clock::now();
        kl_serve_result res{};
        res.request_id = r.id;
        res.M = r.M;
        res.est_bytes = r.est;
        kl_solver* h = nullptr;
        int rc = have_stream ? kl_create(&r.prm, stream, &h) : KL_ERR_CUDA;
        if (rc == KL_OK) {
            h->batcher = s->batcher;
            kl_solve_info info{};
            rc = kl_eigs(h, r.M, r.tol, r.lambda_out, r.V_out, r.ldv, 0, nullptr, &info);
            res.applies = info.applies;
            res.restarts = info.restarts;
            res.max_resid = info.max_resid;
            kl_destroy(h);
        }
        res.status = rc;
        const auto t_end = Clock::now();
        res.queue_ms = ms_since(r.t_submit, t_start);
        res.solve_ms = ms_since(t_start, t_end);
        res.latency_ms = ms_since(r.t_submit, t_end);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->used -= r.est;
            s->active -= 1;
            s->batcher->set_expected(s->active);
            s->done.push_back(res);
            s->st.completed += 1;
        }
        s->cv_queue.notify_all();
        s->cv_done.notify_all();
    }
    if (have_stream) cudaStreamDestroy(stream);
}

}  // namespace

int kl_serve_open(const kl_serve_config* cfg, kl_server** out) {
    if (!out) return fail(nullptr, KL_ERR_ARG, "out must not be NULL");
    *out = nullptr;
    kl_server* s = new kl_server();
    if (cfg) s->cfg = *cfg;
    if (s->cfg.max_slots == 0) s->cfg.max_slots = 8;
    if (s->cfg.batch_window_us == 0) s->cfg.batch_window_us = 300;
    if (s->cfg.max_slots < 1 || s->cfg.max_slots > 64 || s->cfg.batch_window_us < 0 || s->cfg.hbm_budget_bytes < 0) {
        delete s;
        return fail(nullptr, KL_ERR_ARG, "max_slots must be in 1..64, batch_window_us and the budget >= 0");
    }
    cudaError_t e = cudaGetDevice(&s->device);
    cudaDeviceProp prop;
    if (e == cudaSuccess) e = cudaGetDeviceProperties(&prop, s->device);
    size_t free_b = 0, total_b = 0;
    if (e == cudaSuccess) e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) {
        delete s;
        return cuda_fail(nullptr, e, "kl_serve_open");
    }
    if (s->cfg.hbm_budget_bytes == 0) s->cfg.hbm_budget_bytes = int64_t(free_b) / 10 * 8;
    s->st.budget_bytes = s->cfg.hbm_budget_bytes;
    s->batcher = new Batcher(s->device, s->cfg.batch_window_us, prop.multiProcessorCount);
    for (int i = 0; i < s->cfg.max_slots; ++i) s->workers.emplace_back(worker, s);
    *out = s;
    return KL_OK;
}

int kl_serve_submit(kl_server* s, const kl_params* params, int M, double tol, int64_t request_id,
                    double* lambda_out, double* V_out, int64_t ldv) {
    if (!s || !params || !lambda_out) return fail(nullptr, KL_ERR_ARG, "server, params and lambda_out must not be NULL");
    int64_t est = 0;
    int rc = kl_estimate_bytes(params, M, &est);
    if (rc != KL_OK) return rc;
    if (est > s->cfg.hbm_budget_bytes)
        return fail(nullptr, KL_ERR_ARG, "request needs more memory than the whole serving budget");
    ServeRequest r;
    r.prm = *params;
    r.M = M;
    r.tol = tol;
    r.id = request_id;
    r.lambda_out = lambda_out;
    r.V_out = V_out;
    r.ldv = ldv;
    r.est = est;
    r.t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return fail(nullptr, KL_ERR_ARG, "server is closing");
        s->queue.push_back(r);
        s->st.submitted += 1;
    }
    s->cv_queue.notify_all();
    return KL_OK;
}

int kl_serve_poll(kl_server* s, kl_serve_result* out, int cap, int* n, int wait_ms) {
    if (!s || !n || (cap > 0 && !out)) return fail(nullptr, KL_ERR_ARG, "invalid arguments");
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->done.empty() && wait_ms > 0)
        s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !s->done.empty(); });
    int k = 0;
    while (k < cap && !s->done.empty()) {
        out[k++] = s->done.front();
        s->done.pop_front();
    }
    *n = k;
    return KL_OK;
}

int kl_serve_get_stats(kl_server* s, kl_serve_stats* out) {
    if (!s || !out) return fail(nullptr, KL_ERR_ARG, "invalid arguments");
    const BatcherStats b = s->batcher->stats();
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->st;
    out->batches = b.batches;
    out->batched_products = b.products;
    out->max_batch = b.max_batch;
    return KL_OK;
}

int kl_serve_close(kl_server* s) {
    if (!s) return KL_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_queue.notify_all();
    for (auto& t : s->workers)
        if (t.joinable()) t.join();
    delete s->batcher;
    delete s;
    return KL_OK;
}
