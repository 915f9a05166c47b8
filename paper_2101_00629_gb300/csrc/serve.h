// Batching of tensor-core pairwise products across concurrently running
// solves (used by the serving loop in serve.cu).
#pragma once

#include <cuda_runtime.h>

#include <condition_variable>
#include <mutex>
#include <thread>
#include <vector>

#include "kernels_tc.h"

namespace kl {

// One solve's pairwise product handed to the batcher: its instance
// descriptors (conversion already enqueued on the solve's stream, which
// recorded `ready`); the batcher records `done` after the launch.
struct BatchJob {
    TcInstance inst[kTcMaxBatch];
    int n = 0;
    bool tf32 = false;
    int np = 16;
    int* err = nullptr;  // the solve's device error word
    cudaEvent_t ready = nullptr, done = nullptr;
    bool launched = false;
    cudaError_t error = cudaSuccess;
};

struct BatcherStats {
    long long batches = 0;   // launches
    long long products = 0;  // jobs in those launches
    int max_batch = 0;
};

class Batcher {
   public:
    Batcher(int device, int window_us, int sm_count);
    ~Batcher();
    // Blocks until the launch containing the job is enqueued on the
    // batcher's stream; the caller's stream must then wait on job.done.
    cudaError_t run(BatchJob& job);
    // Number of solves that may submit (an upper bound on the products a
    // batch waits for).
    void set_expected(int n);
    // A solve starts an operator application: its product will follow after
    // the application's first sum-factorisation pass. The batcher waits (at
    // most window_us) only for products announced this way and not yet
    // submitted, not for solves busy elsewhere (orthogonalisation, the
    // Rayleigh-Ritz eigenproblem).
    void announce();
    // An announced product will not come (the application failed first).
    void withdraw();
    BatcherStats stats();

   private:
    void loop();
    int device_, window_us_, sm_count_;
    cudaStream_t stream_ = nullptr;
    int* d_err_ = nullptr;
    cudaError_t init_error_ = cudaSuccess;
    std::mutex mu_;
    std::condition_variable cv_work_, cv_done_;
    std::vector<BatchJob*> pending_;
    int expected_ = 1;
    int announced_ = 0;  // announced products not yet submitted
    bool stop_ = false;
    BatcherStats stats_;
    std::thread thread_;
};

}  // namespace kl
