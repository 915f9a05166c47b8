// The solver handle behind the opaque kl_solver of the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <tuple>
#include <string>
#include <vector>

#include "kl_internal.h"

struct kl_prof_entry {
    long long launches = 0;
    double ms = 0.0;
    double units = 0.0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
    std::vector<double> pending_units;
};

namespace kl {
class Batcher;
struct TcSymPlan;
}

struct kl_solver {
    kl_params prm{};
    cudaStream_t stream = nullptr;
    int device = 0;
    int sm_count = 152;
    int shared_sms = 0;  // SMs the pairwise product leaves to other streams (kl_set_shared_sms)
    int cc_major = 0, cc_minor = 0;
    std::string err;

    // sizes
    int N1[3] = {1, 1, 1};   // trial dofs per direction
    int Nt1[3] = {1, 1, 1};  // interpolation dofs per direction (Galerkin)
    int Nq1[3] = {1, 1, 1};  // quadrature points per direction (collocation)
    int Ns1[3] = {1, 1, 1};  // source points per direction (Nt1, the Gauss points, Nq1)
    int64_t N = 0;           // trial dofs
    int64_t S = 0;           // pairwise sources (N~ or NeNq)
    int64_t T = 0;           // pairwise targets (N~ or N)

    // device 1D tables (all inside one allocation)
    double* d_tables = nullptr;
    const double* F[3] = {};      // Galerkin: Q_d (A) ; collocation: R_d     (S_d x N_d)
    const double* FT[3] = {};     // transposes                                (N_d x S_d)
    const double* P[3] = {};      // Galerkin standard form P_d                (Nt_d x N_d)
    const double* PT[3] = {};     // transposes
    const double* Zinv[3] = {};   // Z_d^-1                                     (N_d x N_d)
    const double* LinvT[3] = {};  // Galerkin L_d^-T                            (N_d x N_d)
    const double* pts1d[9] = {};  // target params (3), source params (3), source weights (3)
    const double* E[3] = {};      // trial basis at the Gauss points of direction d (Ne_d x N_d)
    // banded forms of the B-spline / NURBS tables (each row has at most p + 1
    // nonzero entries next to each other): row i holds `w` values starting at
    // column start[i]; vals == NULL where a table is not banded (dense
    // projections and inverses)
    kl::Band bF[3], bFT[3], bE[3];
    double* d_band_vals = nullptr;
    int* d_band_start = nullptr;
    const double* xe[3] = {};     // those Gauss points (parameters)
    int Ne1[3] = {1, 1, 1};       // Gauss points per direction (sampling grid)

    // device point sets
    double* d_points = nullptr;   // tx ty tz (T) sx sy sz (S) scale (S)
    float* d_points32 = nullptr;  // tx ty tz sx sy sz in FP32
    double *tx = nullptr, *ty = nullptr, *tz = nullptr;
    double *sx = nullptr, *sy = nullptr, *sz = nullptr;
    float *tx32 = nullptr, *ty32 = nullptr, *tz32 = nullptr;
    float *sx32 = nullptr, *sy32 = nullptr, *sz32 = nullptr;
    double* src_scale = nullptr;  // Galerkin J (= target scale too); collocation w det DF
    double* d_geo = nullptr;      // geometry parameters on the device (unused by kernels)

    // collocation with NURBS weights that are not a tensor product (projective
    // cube): R_j = w_j B_j / W with W = sum_l w_l B_l, so R v = (B (w v)) / W
    // and Z^-1 = diag(1/w) B^-1 diag(W(x_i)) around the B-spline Kronecker
    // tables; NULL otherwise
    double* d_rat = nullptr;       // one allocation for the five arrays below
    double* rat_w = nullptr;       // w_j (N)
    double* rat_invw = nullptr;    // 1 / w_j (N)
    double* rat_Wc = nullptr;      // W at the collocation points (N)
    double* rat_invWq = nullptr;   // 1 / W at the Gauss points (S)
    double* rat_src_scale = nullptr;  // Gauss weight x det DF / W (S)

    // workspaces for operator applications (k_cap vectors)
    int k_cap = 0;
    double* ws[3] = {nullptr, nullptr, nullptr};
    double* pair_scratch = nullptr;
    int64_t pair_scratch_len = 0;
    int pair_splits = 1;
    // symmetric split-BF16 Galerkin product (stand-alone handles): its plan
    // for blocks of up to sym_plan->kcap vectors and its scratch
    kl::TcSymPlan* sym_plan = nullptr;
    double* sym_scratch = nullptr;
    int64_t sym_scratch_len = 0;
    bool pair_dense = false;  // kl_debug_set(KL_DEBUG_PAIR_DENSE): every pair evaluated

    // device word set by kernels whose bounded waits gave up (read after a
    // synchronisation; see check_device_error)
    int* d_err = nullptr;

    // failure injection (kl_debug_set): clock cycles of each pipeline wait
    // of the tcgen05 kernel (0: the default, about a second) and a NaN
    // planted in the eigensolver's start block
    long long wait_limit = 0;
    bool nan_start = false;

    // kl_sample scratch (grown on demand)
    double* smp_ws = nullptr;
    int64_t smp_cap = 0;  // doubles

    // CUDA graphs of operator applications, keyed by operator, precision,
    // block width and the input/output buffers (see apply_operator)
    struct GraphKey {
        int which, precision, k;
        const double* X;
        int64_t ldx;
        double* Y;
        int64_t ldy;
        int part;  // 0: whole application, 1: before the pairwise product, 2: after
        bool operator<(const GraphKey& o) const {
            return std::tie(which, precision, k, X, ldx, Y, ldy, part) <
                   std::tie(o.which, o.precision, o.k, o.X, o.ldx, o.Y, o.ldy, o.part);
        }
    };
    struct GraphEntry {
        int uses = 0;               // eager runs so far (capture on the second)
        long long launches = 0;     // kernels per application
        cudaGraphExec_t exec = nullptr;
        bool failed = false;        // capture not possible: stay eager
    };
    bool use_graphs = true;
    bool autotune = false;  // created with block_k = 0: kl_eigs looks the block size up
    std::map<GraphKey, GraphEntry> graphs;

    // serving: tensor-core pairwise products go through this batcher (set
    // by the server's worker; null for a stand-alone handle)
    kl::Batcher* batcher = nullptr;
    bool announced = false;  // a product announced to the batcher, not yet submitted
    cudaEvent_t ev_ready = nullptr, ev_done = nullptr;

    // eigensolver workspaces
    int64_t eig_cap_bytes = 0;
    void* eig_ws = nullptr;

    // bookkeeping
    long long launches = 0;
    int64_t h2d_bytes = 0;
    int64_t dev_bytes = 0;
    bool profiling = false;
    std::map<std::string, kl_prof_entry> prof;
};

namespace kl {
int fail(kl_solver* h, int code, const std::string& msg);
int cuda_fail(kl_solver* h, cudaError_t e, const char* where);
int ensure_workspace(kl_solver* h, int k);
// Block size cached by kl_autotune for these parameters and M (0: none).
int tune_lookup(const kl_params& p, int M);
// Drops the captured graphs (their kernels point at the old workspaces).
void clear_graphs(kl_solver* h);
// Eigensolver sizing shared by kl_eigs and kl_estimate_bytes.
int eig_basis_cap(int64_t N, int M, int b);
int64_t eig_workspace_doubles(int64_t N, int mcap);
// KL_ERR_TIMEOUT (and clears the word) if a kernel of this handle recorded a
// bounded wait that gave up; synchronises the handle's stream.
int check_device_error(kl_solver* h);
// Operator applications on device blocks (k <= h->k_cap after ensure_workspace).
// which: 0 = A (generalized), 1 = A' (standard form). precision: KL_* precision.
int apply_operator(kl_solver* h, int which, int precision, const double* X, int64_t ldx,
                   double* Y, int64_t ldy, int k);
int apply_zinv(kl_solver* h, const double* X, int64_t ldx, double* Y, int64_t ldy, int k);
// Galerkin back-transform v = L^-T y; collocation: copy.
int back_transform(kl_solver* h, const double* Yv, int64_t ldy, double* V, int64_t ldv, int k);
// Collocation field values R v at the quadrature points into out (S x k).
int field_at_quadrature(kl_solver* h, const double* V, int64_t ldv, double* out, int k);
// Profiling helpers: record an event pair around a launch sequence.
struct ProfScope {
    kl_solver* h;
    const char* name;
    double units;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ProfScope(kl_solver* h_, const char* n, double u);
    ~ProfScope();
};
}  // namespace kl
