// kl_eigs: the outer iterative eigensolver on the standard form of Eq.
// standard (Sec. 3: A' v' = lambda v', v = C v').
//
// The paper leaves the eigensolver unnamed (Sec. 3.3 counts its iterations
// N_iter); this is a thick-restart block Krylov-Schur method that serves both
// forms:
//   * a basis V (N x m) is grown block by block: the newest block of A'V is
//     orthogonalised against V (two classical Gram-Schmidt passes in FP64)
//     and orthonormalised (CholQR2, collapsed columns replaced by fresh
//     random directions);
//   * the Rayleigh-Ritz matrix H = V^T (A'V) is formed explicitly in FP64 and
//     decomposed on the device: cyclic Jacobi for the symmetric Galerkin form
//     (A' = L^-1 A L^-T), Hessenberg + Francis QR for the non-symmetric
//     collocation form (A' = Z^-1 A);
//   * the restart keeps the nkeep leading Ritz vectors (and A' applied to
//     them, so no operator application is repeated) followed by the
//     orthonormalised residual block, which preserves the Krylov-Schur
//     relation A' V = V H + F E^T;
//   * for the reduced precisions a final Rayleigh-Ritz step in FP64 is taken
//     on the converged Ritz vectors (refine = 2: with an FP64 application of
//     the operator).
// Vectors are then mapped back (Galerkin v = L^-T v'), normalised and given a
// sign (largest-magnitude entry positive).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <initializer_list>
#include <string>
#include <vector>

#include "handle.h"

namespace kl {
namespace {

struct EigWs {
    double *V, *AV, *T1, *T2;   // N x mmax each
    double *H, *S, *G, *Rinv;   // mmax^2 each
    double* Q;                  // ordered Schur vectors (non-symmetric), mmax^2
    double *theta, *thetai, *norms, *norms2;  // mmax each (norms: 2 mmax)
    double* la_work;            // eigensolver work
    double* tn_scratch;         // gemm_tn partials
    int64_t tn_len;
    int* ibuf;                  // eigensolver status, or the two CholQR passes' pivot flags
};

struct Ctx {
    kl_solver* h;
    EigWs w;
    int64_t N;
    int mmax;
    bool sym;
    bool schur_ok = false;      // Q holds ordered Schur vectors of the last H
    int nvec = 0;               // eigenvectors of H needed (leading, ordered)
    bool rr_fp32 = false;       // the last Rayleigh-Ritz problem was solved in FP32
    unsigned long long rng_offset = 0;
    int applies = 0, vectors_applied = 0;
};

#define KL_TRY(expr)                         \
    do {                                     \
        int _rc = (expr);                    \
        if (_rc != KL_OK) return _rc;        \
    } while (0)

int ck(Ctx& c, cudaError_t e, const char* where, int n_launch = 1) {
    c.h->launches += n_launch;
    if (e != cudaSuccess) return cuda_fail(c.h, e, where);
    return KL_OK;
}

// C(m x n) = A^T B with A, B tall (N rows)
int tn(Ctx& c, const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc,
       int m, int n, double alpha = 1.0, double beta = 0.0) {
    return ck(c, launch_gemm_tn(A, lda, B, ldb, C, ldc, m, n, c.N, alpha, beta, c.w.tn_scratch,
                                c.w.tn_len, c.h->stream), "gemm_tn", 2);
}

int nn(Ctx& c, const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc,
       int m, int n, double alpha, double beta) {
    return ck(c, launch_gemm_nn(A, lda, B, ldb, C, ldc, c.N, m, n, alpha, beta, c.h->stream), "gemm_nn");
}

int sync_copy(Ctx& c, void* dst, const void* src, size_t bytes) {
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, c.h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.h->stream);
    if (e != cudaSuccess) return cuda_fail(c.h, e, "device->host copy");
    return KL_OK;
}

// Several device->host copies behind one synchronisation (each host round
// trip leaves the GPU idle between the solve's small kernels).
struct HostCopy {
    void* dst;
    const void* src;
    size_t bytes;
};
int sync_copies(Ctx& c, std::initializer_list<HostCopy> list) {
    cudaError_t e = cudaSuccess;
    for (const HostCopy& hc : list)
        if (e == cudaSuccess && hc.bytes) e = cudaMemcpyAsync(hc.dst, hc.src, hc.bytes, cudaMemcpyDeviceToHost, c.h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.h->stream);
    if (e != cudaSuccess) return cuda_fail(c.h, e, "device->host copy");
    return KL_OK;
}

// Two classical Gram-Schmidt passes of W (N x bw) against V[:, :nv].
int project_out(Ctx& c, const double* V, int nv, double* W, int bw) {
    if (nv <= 0) return KL_OK;
    for (int pass = 0; pass < 2; ++pass) {
        KL_TRY(tn(c, V, c.N, W, c.N, c.w.G, nv, nv, bw));
        KL_TRY(nn(c, V, c.N, c.w.G, nv, W, c.N, nv, bw, -1.0, 1.0));
    }
    return KL_OK;
}

// Makes W (N x bw) orthonormal and orthogonal to V[:, :nv]. Columns that
// collapse (W nearly in span(V) or linearly dependent) are replaced by random
// vectors and the procedure repeats.
int orthonormalize(Ctx& c, const double* V, int nv, double* W, int bw) {
    std::vector<double> norms(2 * bw);
    std::vector<int> flags(2 * bw), bad(bw);
    for (int attempt = 0; attempt < 6; ++attempt) {
        // column norms before and after two Gram-Schmidt passes, then CholQR
        // twice (W R^-1 stays orthogonal to V because it only mixes columns
        // of W); a collapsed Cholesky pivot is flagged and replaced by 1, so
        // W stays finite. Everything is checked after one synchronisation:
        // a column that collapsed in the projection or in either pass is
        // replaced by a random direction and the block is done again (the
        // other columns keep their span: the factors are triangular).
        KL_TRY(ck(c, launch_col_norms(W, c.N, c.N, bw, c.w.norms, c.h->stream), "norms"));
        KL_TRY(project_out(c, V, nv, W, bw));
        KL_TRY(ck(c, launch_col_norms(W, c.N, c.N, bw, c.w.norms + bw, c.h->stream), "norms"));
        for (int pass = 0; pass < 2; ++pass) {
            KL_TRY(tn(c, W, c.N, W, c.N, c.w.G, bw, bw, bw));
            KL_TRY(ck(c, launch_chol_rinv(c.w.G, bw, c.w.Rinv, c.w.ibuf + pass * bw, c.h->stream), "chol"));
            KL_TRY(nn(c, W, c.N, c.w.Rinv, bw, c.w.T2, c.N, bw, bw, 1.0, 0.0));
            KL_TRY(ck(c, launch_copy_block(c.w.T2, c.N, W, c.N, c.N, bw, c.h->stream), "copy"));
        }
        KL_TRY(sync_copies(c, {{norms.data(), c.w.norms, 2 * bw * sizeof(double)},
                               {flags.data(), c.w.ibuf, 2 * bw * sizeof(int)}}));
        bool any = false;
        for (int j = 0; j < bw; ++j) {
            // a NaN or Inf in a new block (the operator produced it, or the
            // start block carried it) is an error, not a collapsed column to
            // replace: replacing it would hide the fault
            if (!std::isfinite(norms[j]))
                return fail(c.h, KL_ERR_NUMERIC, "NaN or Inf in a block of the Krylov basis");
            const double before = norms[j], after = norms[bw + j];
            bad[j] = !(after > 1e-10 * before) || !(after > 1e-290) || !std::isfinite(after) || flags[j] != 0 ||
                     flags[bw + j] != 0;
            any |= bad[j] != 0;
        }
        if (!any) return KL_OK;
        for (int j = 0; j < bw; ++j) {
            if (!bad[j]) continue;
            KL_TRY(ck(c, launch_randn(W + int64_t(j) * c.N, c.N, c.N, 1, c.h->prm.seed ^ 0x5bd1e995ull,
                                      c.rng_offset, c.h->stream), "randn"));
            c.rng_offset += uint64_t(c.N);
        }
    }
    return fail(c.h, KL_ERR_NUMERIC, "orthonormalisation failed repeatedly");
}

int apply(Ctx& c, int precision, const double* X, double* Y, int k) {
    KL_TRY(ensure_workspace(c.h, k));
    c.applies += 1;
    c.vectors_applied += k;
    return apply_operator(c.h, 1, precision, X, c.N, Y, c.N, k);
}

// Rayleigh-Ritz on the first nv columns: theta (desc), S (nv x nv, ld nv).
// fp32: the small eigenproblem in FP32 arithmetic (restarts far from the
// tolerance; its vectors are then re-orthonormalised in FP64 by the caller).
int rayleigh_ritz(Ctx& c, const double* V, const double* AV, int nv, double* max_imag, bool fp32 = false) {
    KL_TRY(tn(c, V, c.N, AV, c.N, c.w.H, nv, nv, nv));
    int status = 0;
    c.rr_fp32 = fp32;
    if (c.sym) {
        // reduced-precision solves: FP64-grade problems in double-float (the
        // QR path), FP64 solves in FP64
        const bool dfloat = !fp32 && c.h->prm.precision != KL_FP64;
        KL_TRY(ck(c, launch_sym_eig(c.w.H, nv, c.w.theta, c.w.S, c.w.la_work, c.w.ibuf, c.h->stream, fp32, dfloat),
                  "sym_eig"));
        KL_TRY(sync_copy(c, &status, c.w.ibuf, sizeof(int)));
        if (dfloat && status == 1) {
            // not converged in double-float: the same matrix in FP64
            KL_TRY(ck(c, launch_sym_eig(c.w.H, nv, c.w.theta, c.w.S, c.w.la_work, c.w.ibuf, c.h->stream, false),
                      "sym_eig"));
            KL_TRY(sync_copy(c, &status, c.w.ibuf, sizeof(int)));
        }
        if (max_imag) *max_imag = 0.0;
    } else {
        // reduced-precision solves take their FP64-grade problems in
        // double-float arithmetic (~1e-14 ||H||, several times faster on
        // GB300 than FP64), FP64 solves in FP64
        const int arith = fp32 ? kEigFP32 : (c.h->prm.precision != KL_FP64 ? kEigDF : kEigFP64);
        KL_TRY(ck(c, launch_nonsym_eig(c.w.H, nv, c.w.theta, c.w.thetai, c.w.S, c.w.Q, c.w.la_work,
                                       c.w.ibuf, c.h->stream, c.nvec, arith), "nonsym_eig"));
        KL_TRY(sync_copy(c, &status, c.w.ibuf, sizeof(int)));
        if (arith == kEigDF && status == 1) {
            // not converged in double-float: the same matrix in FP64
            KL_TRY(ck(c, launch_nonsym_eig(c.w.H, nv, c.w.theta, c.w.thetai, c.w.S, c.w.Q, c.w.la_work,
                                           c.w.ibuf, c.h->stream, c.nvec, kEigFP64), "nonsym_eig"));
            KL_TRY(sync_copy(c, &status, c.w.ibuf, sizeof(int)));
        }
        c.schur_ok = status == 0;
        if (status == 2) status = 0;  // complex pairs: eigenvectors valid, Schur order not
    }
    if (status != 0 && status != 3 && fp32) {
        // the FP32 problem did not converge (its shorter precision can stall
        // on tight clusters): solve the same projected matrix in FP64
        return rayleigh_ritz(c, V, AV, nv, max_imag, false);
    }
    if (status != 0) {
        // diagnostics: with KL_DUMP_DIR set, keep the matrix that failed
        if (const char* dir = std::getenv("KL_DUMP_DIR")) {
            std::vector<double> Hh(size_t(nv) * nv);
            if (cudaMemcpy(Hh.data(), c.w.H, Hh.size() * sizeof(double), cudaMemcpyDeviceToHost) == cudaSuccess) {
                const std::string path = std::string(dir) + "/kl_rr_failed_" + std::to_string(nv) + ".f64";
                if (FILE* f = std::fopen(path.c_str(), "wb")) {
                    std::fwrite(Hh.data(), sizeof(double), Hh.size(), f);
                    std::fclose(f);
                }
            }
        }
        if (status == 3) return fail(c.h, KL_ERR_CUDA, "small eigensolver: index out of range (bounds check)");
        return fail(c.h, KL_ERR_NUMERIC, "small eigensolver did not converge");
    }
    return KL_OK;
}

}  // namespace

// Smallest relative tolerance an FP32 Rayleigh-Ritz problem resolves: its
// Ritz values and vectors are accurate to a few 1e-6 ||H|| (measured on
// GB300 for n = 40..170). Tighter tolerances use FP32 only while the
// residuals are above 1e-3 (and 1e3 tol), i.e. for the early restarts.
constexpr double kFp32RrTol = 1e-4;
// Smallest tolerance an FP32 Rayleigh-Ritz claim of convergence is tried at
// (its residuals bottom out near a few 1e-7 of the largest Ritz value).
constexpr double kFp32ClaimTol = 1e-6;

// Basis width limit of kl_eigs for M wanted pairs and block size b (<= N).
int eig_basis_cap(int64_t N, int M, int b) {
    b = int(std::min<int64_t>(b, N));
    const int nkeep_full = (M + b + b - 1) / b * b;
    const int mmax_full = std::max(2 * nkeep_full, nkeep_full + 2 * b);
    const int mmax = int(std::min<int64_t>(mmax_full, N));
    return int(std::min<int64_t>(int64_t(mmax) + b, N));
}

// Doubles of the eigensolver workspace for N dofs and basis width mcap.
int64_t eig_workspace_doubles(int64_t N, int mcap) {
    const int64_t tn_len = std::max(gemm_tn_scratch_doubles(mcap, mcap, N), int64_t(1));
    const int64_t la = std::max(sym_eig_work_doubles(mcap), nonsym_eig_work_doubles(mcap));
    return 4 * N * mcap + 5 * int64_t(mcap) * mcap + 8 * int64_t(mcap) + la + tn_len + (2 * int64_t(mcap) + 8) / 2 + 64;
}

}  // namespace kl

using namespace kl;

namespace {
int eigs_impl(kl_solver* h, int M, double tol, double* lambda, double* Vout, int64_t ldv, int v_on_device,
              double* resid, kl_solve_info* info);
}  // namespace

// A bounded wait that gave up inside a tensor-core kernel leaves its products
// incomplete; the solve may then fail later for that reason (breakdown, NaN,
// no convergence). The recorded timeout is the cause reported.
extern "C" int kl_eigs(kl_solver* h, int M, double tol, double* lambda, double* Vout, int64_t ldv,
                       int v_on_device, double* resid, kl_solve_info* info) {
    if (!h) return KL_ERR_ARG;
    const int rc = eigs_impl(h, M, tol, lambda, Vout, ldv, v_on_device, resid, info);
    if (rc != KL_OK && rc != KL_WARN_COMPLEX && rc != KL_ERR_CUDA && rc != KL_ERR_TIMEOUT && rc != KL_ERR_ARG) {
        const std::string why = h->err;
        if (check_device_error(h) == KL_ERR_TIMEOUT) return KL_ERR_TIMEOUT;
        h->err = why;
    }
    return rc;
}

namespace {
int eigs_impl(kl_solver* h, int M, double tol, double* lambda, double* Vout, int64_t ldv, int v_on_device,
              double* resid, kl_solve_info* info) {
    const auto t_start = std::chrono::steady_clock::now();
    if (!lambda) return fail(h, KL_ERR_ARG, "lambda must not be NULL");
    if (M < 1 || M > 512 || M > h->N) return fail(h, KL_ERR_ARG, "M must be in 1..min(N, 512)");
    if (Vout && ldv < h->N) return fail(h, KL_ERR_ARG, "ldv must be >= N");
    const int prec = h->prm.precision;
    // Default tolerances: the eigenvalue error of the symmetric Galerkin form
    // is quadratic in the residual, that of the non-symmetric collocation form
    // only linear, hence the tighter FP64 default there.
    if (!(tol > 0))
        tol = (prec == KL_FP64) ? (galerkin_form(h->prm.method) ? 1e-10 : 1e-12) : 1e-6;

    Ctx c;
    c.h = h;
    c.N = h->N;
    c.sym = galerkin_form(h->prm.method);
    const int64_t N = h->N;
    if (h->autotune) {
        // block size from the autotuner's cache for this problem and M
        kl_params key = h->prm;
        key.block_k = 0;
        if (const int kt = tune_lookup(key, M); kt > 0) h->prm.block_k = kt;
    }
    const int b = int(std::min<int64_t>(h->prm.block_k, N));
    // nkeep and mmax are multiples of b so that every expansion step takes the
    // images of a full block (the Krylov-Schur relation needs the whole
    // residual of the last block); a basis of N vectors is complete instead
    const int nkeep_full = (M + b + b - 1) / b * b;
    const int mmax_full = std::max(2 * nkeep_full, nkeep_full + 2 * b);
    if (mmax_full + b > 512 && mmax_full < N) return fail(h, KL_ERR_ARG, "M + 3 block_k too large for the basis limit 512");
    const int nkeep = int(std::min<int64_t>(nkeep_full, N));
    // Ritz vectors are used for the M wanted pairs and at most nkeep + 1
    // restart vectors (nkeep >= M + b)
    c.nvec = nkeep + 1;
    const int mmax = int(std::min<int64_t>(mmax_full, N));
    // a restart keeps one extra vector rather than split a complex pair, so
    // the basis may grow to mmax + b - 1 columns
    const int mcap = int(std::min<int64_t>(int64_t(mmax) + b, N));
    c.mmax = mcap;

    // ---- workspace (one allocation, reused across calls) ----
    const int64_t tn_len = std::max(gemm_tn_scratch_doubles(mcap, mcap, N), int64_t(1));
    const int64_t la = std::max(sym_eig_work_doubles(mcap), nonsym_eig_work_doubles(mcap));
    const int64_t need = eig_workspace_doubles(N, mcap);
    if (need * int64_t(sizeof(double)) > h->eig_cap_bytes) {
        cudaStreamSynchronize(h->stream);
        if (h->eig_ws) cudaFree(h->eig_ws);
        h->eig_ws = nullptr;
        cudaError_t e = device_alloc(&h->eig_ws, size_t(need) * sizeof(double));
        if (e != cudaSuccess) {
            h->eig_cap_bytes = 0;
            return cuda_fail(h, e, "eigensolver workspace");
        }
        h->eig_cap_bytes = need * int64_t(sizeof(double));
        h->dev_bytes += h->eig_cap_bytes;
    }
    double* p = static_cast<double*>(h->eig_ws);
    auto take = [&](int64_t n) {
        double* r = p;
        p += (n + 3) / 4 * 4;
        return r;
    };
    c.w.V = take(N * mcap);
    c.w.AV = take(N * mcap);
    c.w.T1 = take(N * mcap);
    c.w.T2 = take(N * mcap);
    c.w.H = take(int64_t(mcap) * mcap);
    c.w.S = take(int64_t(mcap) * mcap);
    c.w.G = take(int64_t(mcap) * mcap);
    c.w.Rinv = take(int64_t(mcap) * mcap);
    c.w.Q = take(int64_t(mcap) * mcap);
    c.w.theta = take(mcap);
    c.w.thetai = take(mcap);
    c.w.norms = take(2 * int64_t(mcap));
    c.w.norms2 = take(mcap);
    c.w.la_work = take(la);
    c.w.tn_scratch = take(tn_len);
    c.w.tn_len = tn_len;
    c.w.ibuf = reinterpret_cast<int*>(take((2 * int64_t(mcap) + 8) / 2 + 2));  // two flag sets of <= mcap

    double* V = c.w.V;
    double* AV = c.w.AV;
    std::vector<double> th(mcap), thi(mcap, 0.0), rn(mcap);

    // ---- start block ----
    int nv = b, na = 0;
    if (int rc = ck(c, launch_randn(V, N, N, b, h->prm.seed, 0, h->stream), "randn"); rc != KL_OK) return rc;
    c.rng_offset = uint64_t(N) * b;
    if (h->nan_start) {
        // failure injection (kl_debug_set): one NaN in the start block
        const double nan = std::nan("");
        cudaError_t e = cudaMemcpyAsync(V, &nan, sizeof(double), cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "NaN injection");
    }
    if (int rc = orthonormalize(c, V, 0, V, b); rc != KL_OK) return rc;

    int restarts = 0, nconv = 0;
    bool done = false, complete = false;
    bool bad_num = false;
    double last_resid = HUGE_VAL;  // largest wanted relative residual of the last Rayleigh-Ritz
    double last_min_resid = HUGE_VAL;  // smallest one
    // reduced precisions: the split (hi + lo) operands of the pairwise
    // product round every application at about 2^-17 of each term, a noise
    // that bounds how far residuals of the computed operator can fall (seen
    // at 1-2e-6 of |theta_1| for narrow Gaussian kernels, L about 0.1, where
    // few terms average the noise); a solve whose largest wanted residual
    // has not decreased for kStallRestarts restarts while within
    // kStallFactor * tol has reached that floor and stops there
    constexpr int kStallRestarts = 10;
    constexpr double kStallFactor = 10.0;
    double best_resid = HUGE_VAL;
    int best_restart = 0;
    // Rayleigh-Ritz on the basis, Ritz vectors Y = V S(:, :mr) in T1 and
    // A'Y = AV S(:, :mr) in T2, residual norms; sets nconv and last_resid
    auto rr_residuals = [&](bool fp32) -> int {
        if (int rc = rayleigh_ritz(c, V, AV, nv, nullptr, fp32); rc != KL_OK) return rc;
        const int mr = std::min(M, nv);
        if (int rc = nn(c, V, N, c.w.S, nv, c.w.T1, N, nv, mr, 1.0, 0.0); rc != KL_OK) return rc;
        if (int rc = nn(c, AV, N, c.w.S, nv, c.w.T2, N, nv, mr, 1.0, 0.0); rc != KL_OK) return rc;
        if (int rc = ck(c, launch_resid_norms(c.w.T1, N, c.w.T2, N, c.w.theta, N, mr, c.w.norms, h->stream), "resid"); rc != KL_OK) return rc;
        if (int rc = sync_copies(c, {{th.data(), c.w.theta, nv * sizeof(double)},
                                     {thi.data(), c.w.thetai, c.sym ? 0 : nv * sizeof(double)},
                                     {rn.data(), c.w.norms, mr * sizeof(double)}});
            rc != KL_OK)
            return rc;
        const double scale = std::max(std::fabs(th[0]), 1e-300);
        nconv = 0;
        last_resid = 0.0;
        last_min_resid = HUGE_VAL;
        bad_num = false;
        for (int i = 0; i < mr; ++i) {
            if (!std::isfinite(rn[i]) || !std::isfinite(th[i])) bad_num = true;
            if (rn[i] <= tol * scale) ++nconv;
            last_resid = std::max(last_resid, rn[i] / scale);
            last_min_resid = std::min(last_min_resid, rn[i] / scale);
        }
        return KL_OK;
    };
    double max_imag = 0.0;
    int status_out = KL_OK;
    while (!done) {
        // ---- expansion ----
        while (true) {
            if (int rc = apply(c, prec, V + na * N, AV + na * N, nv - na); rc != KL_OK) return rc;
            na = nv;
            if (nv >= mmax || nv >= N) break;
            const int bb = int(std::min<int64_t>(b, N - nv));
            double* Wn = V + int64_t(nv) * N;
            if (int rc = ck(c, launch_copy_block(AV + int64_t(nv - bb) * N, N, Wn, N, N, bb, h->stream), "copy"); rc != KL_OK) return rc;
            if (int rc = orthonormalize(c, V, nv, Wn, bb); rc != KL_OK) return rc;
            nv += bb;
        }
        complete = nv >= N;
        // ---- Rayleigh-Ritz ----
        // Mixed precisions: in FP32 while every wanted residual is far above
        // the tolerance (an FP32 restart perturbs the kept vectors by a few
        // 1e-6 of ||H||, which would undo pairs that have converged: with many
        // wanted pairs the slowest one keeps the largest residual high long
        // after the first ones converged); a convergence claim FP32 cannot
        // resolve is re-checked in FP64. FP64 solves stay in FP64.
        // Solves with the final refinement: the residuals of FP32 Ritz pairs
        // are those of actual vectors of the basis (computed in FP64 from
        // A'V), and a small residual is a small backward error (the pair is
        // exact for A' - r y^T; for symmetric A', within a cluster of nearly
        // equal eigenvalues any vector of its invariant subspace has a small
        // residual), so an FP32 claim that all wanted pairs converged is kept:
        // the refinement then computes the pairs in FP64-grade arithmetic on
        // an FP64-orthonormalised basis of the FP32 Ritz (symmetric) or Schur
        // (non-symmetric) vectors. FP32 is tried first also where the restart
        // needs FP64, and the FP64-grade problem is solved only when that try
        // does not converge: for symmetric problems at every such restart
        // (the FP32 problem costs a fraction of the FP64 one), for non-
        // symmetric ones once the last largest wanted residual is within
        // 1e3 tol (their FP32 problem costs a third of the double-float one,
        // a try that fails is paid in full).
        const bool use32 = prec != KL_FP64 && (tol >= kFp32RrTol || last_min_resid > std::max(1e3 * tol, 1e-3));
        const bool trust32 = (c.sym || last_resid <= 1e3 * tol) && prec != KL_FP64 && h->prm.refine > 0 &&
                             tol < kFp32RrTol && tol >= kFp32ClaimTol;
        bool claimed32 = false;
        if (use32 || trust32) {
            if (int rc = rr_residuals(true); rc != KL_OK) return rc;
            claimed32 = trust32 && !bad_num && nconv >= M;
        }
        if (!claimed32 && !use32) {
            if (int rc = rr_residuals(false); rc != KL_OK) return rc;
        } else if (!claimed32 && tol < kFp32RrTol && (nconv >= M || complete || restarts >= h->prm.max_restarts)) {
            if (int rc = rr_residuals(false); rc != KL_OK) return rc;
        }
        if (bad_num) return fail(h, KL_ERR_NUMERIC, "NaN or Inf in the Ritz values");
        if (nconv >= M || complete) break;
        if (prec != KL_FP64) {
            if (last_resid < 0.97 * best_resid) {
                best_resid = last_resid;
                best_restart = restarts;
            } else if (restarts - best_restart >= kStallRestarts && last_resid <= kStallFactor * tol) {
                break;
            }
        }
        if (restarts >= h->prm.max_restarts) {
            status_out = KL_ERR_NOCONV;
            break;
        }
        // ---- restart ----
        ++restarts;
        int keep = std::min(nkeep, nv - b);
        if (!c.sym && thi[keep - 1] > 0.0) ++keep;  // do not split a complex pair
        // next block: newest block of A'V orthogonalised against the full basis
        double* Wn = c.w.T1;  // reuse; Ritz vectors are recomputed after the loop
        if (int rc = ck(c, launch_copy_block(AV + int64_t(nv - b) * N, N, Wn, N, N, b, h->stream), "copy"); rc != KL_OK) return rc;
        if (int rc = orthonormalize(c, V, nv, Wn, b); rc != KL_OK) return rc;
        // Symmetric: the leading Ritz vectors (orthonormal). Non-symmetric:
        // the leading ordered Schur vectors (orthonormal, spanning the
        // invariant subspace of the wanted Ritz values, also for clusters
        // of equal eigenvalues); Ritz vectors only if complex pairs stopped
        // the ordering. V R(:, :keep) and AV R(:, :keep) go back into V, AV.
        const double* Rk = (c.sym || !c.schur_ok) ? c.w.S : c.w.Q;
        if (int rc = nn(c, V, N, Rk, nv, c.w.T2, N, nv, keep, 1.0, 0.0); rc != KL_OK) return rc;
        if (int rc = ck(c, launch_copy_block(c.w.T2, N, V, N, N, keep, h->stream), "copy"); rc != KL_OK) return rc;
        if (int rc = nn(c, AV, N, Rk, nv, c.w.T2, N, nv, keep, 1.0, 0.0); rc != KL_OK) return rc;
        if (int rc = ck(c, launch_copy_block(c.w.T2, N, AV, N, N, keep, h->stream), "copy"); rc != KL_OK) return rc;
        if ((!c.sym && !c.schur_ok) || c.rr_fp32) {
            // Ritz (or real/imaginary) vectors, or vectors of an FP32
            // Rayleigh-Ritz, are not orthonormal to FP64: CholQR2 on V and
            // the same right factor on AV
            for (int pass = 0; pass < 2; ++pass) {
                if (int rc = tn(c, V, N, V, N, c.w.G, keep, keep, keep); rc != KL_OK) return rc;
                if (int rc = ck(c, launch_chol_rinv(c.w.G, keep, c.w.Rinv, c.w.ibuf, h->stream), "chol"); rc != KL_OK) return rc;
                if (int rc = nn(c, V, N, c.w.Rinv, keep, c.w.T2, N, keep, keep, 1.0, 0.0); rc != KL_OK) return rc;
                if (int rc = ck(c, launch_copy_block(c.w.T2, N, V, N, N, keep, h->stream), "copy"); rc != KL_OK) return rc;
                if (int rc = nn(c, AV, N, c.w.Rinv, keep, c.w.T2, N, keep, keep, 1.0, 0.0); rc != KL_OK) return rc;
                if (int rc = ck(c, launch_copy_block(c.w.T2, N, AV, N, N, keep, h->stream), "copy"); rc != KL_OK) return rc;
            }
        }
        if (int rc = ck(c, launch_copy_block(Wn, N, V + int64_t(keep) * N, N, N, b, h->stream), "copy"); rc != KL_OK) return rc;
        nv = keep + b;
        na = keep;
    }

    // the final pairs come from an FP64 Rayleigh-Ritz problem: the refinement
    // below, or the last one of the loop
    if (c.rr_fp32 && !(prec != KL_FP64 && h->prm.refine > 0)) {
        if (int rc = rr_residuals(false); rc != KL_OK) return rc;
    }

    // ---- final Ritz pairs (optionally refined by an FP64 Rayleigh-Ritz) ----
    int nk = std::min(nv, nkeep);
    if (nk < M) nk = std::min(nv, M);
    if (!c.sym && nk < nv && thi[nk - 1] > 0.0) ++nk;  // keep complex pairs whole
    double* Y = c.w.T1;
    double* AY = c.w.T2;
    const bool use_schur = !c.sym && c.schur_ok && prec != KL_FP64 && h->prm.refine > 0;
    if (int rc = nn(c, V, N, use_schur ? c.w.Q : c.w.S, nv, Y, N, nv, nk, 1.0, 0.0); rc != KL_OK) return rc;
    if (prec != KL_FP64 && h->prm.refine > 0) {
        if ((!c.sym && !use_schur) || c.rr_fp32) {
            // orthonormal basis of the Ritz subspace
            for (int pass = 0; pass < 2; ++pass) {
                if (int rc = tn(c, Y, N, Y, N, c.w.G, nk, nk, nk); rc != KL_OK) return rc;
                if (int rc = ck(c, launch_chol_rinv(c.w.G, nk, c.w.Rinv, c.w.ibuf, h->stream), "chol"); rc != KL_OK) return rc;
                if (int rc = nn(c, Y, N, c.w.Rinv, nk, AY, N, nk, nk, 1.0, 0.0); rc != KL_OK) return rc;
                if (int rc = ck(c, launch_copy_block(AY, N, Y, N, N, nk, h->stream), "copy"); rc != KL_OK) return rc;
            }
        }
        const int rprec = h->prm.refine == 2 ? KL_FP64 : prec;
        if (int rc = apply(c, rprec, Y, AY, nk); rc != KL_OK) return rc;
        // Rayleigh-Ritz on span(Y): reuse V/AV storage for the rotated pair;
        // only the M leading pairs are used (and ordered)
        const int nvec_loop = c.nvec;
        c.nvec = M;
        const int rc_rr = rayleigh_ritz(c, Y, AY, nk, nullptr);
        c.nvec = nvec_loop;
        if (rc_rr != KL_OK) return rc_rr;
        if (int rc = nn(c, Y, N, c.w.S, nk, V, N, nk, M, 1.0, 0.0); rc != KL_OK) return rc;
        if (int rc = nn(c, AY, N, c.w.S, nk, AV, N, nk, M, 1.0, 0.0); rc != KL_OK) return rc;
        if (int rc = ck(c, launch_copy_block(V, N, Y, N, N, M, h->stream), "copy"); rc != KL_OK) return rc;
        if (int rc = ck(c, launch_copy_block(AV, N, AY, N, N, M, h->stream), "copy"); rc != KL_OK) return rc;
    } else {
        if (int rc = nn(c, AV, N, c.w.S, nv, AY, N, nv, M, 1.0, 0.0); rc != KL_OK) return rc;
    }
    if (int rc = ck(c, launch_resid_norms(Y, N, AY, N, c.w.theta, N, M, c.w.norms, h->stream), "resid"); rc != KL_OK) return rc;
    if (int rc = sync_copies(c, {{th.data(), c.w.theta, M * sizeof(double)},
                                 {thi.data(), c.w.thetai, c.sym ? 0 : M * sizeof(double)},
                                 {rn.data(), c.w.norms, M * sizeof(double)}});
        rc != KL_OK)
        return rc;
    const double scale = std::max(std::fabs(th[0]), 1e-300);
    double max_res = 0.0;
    nconv = 0;
    for (int i = 0; i < M; ++i) {
        lambda[i] = th[i];
        const double r = rn[i] / scale;
        if (resid) resid[i] = r;
        max_res = std::max(max_res, r);
        if (r <= tol) ++nconv;
        max_imag = std::max(max_imag, std::fabs(thi[i]) / scale);
    }

    // ---- eigenvectors: back-transform, normalise, sign ----
    if (Vout) {
        double* Vd = AV;  // N x M scratch
        // the back-transform's mode products keep two N x M intermediates in
        // the operator workspaces: size them for M vectors (an FP64 solve has
        // only applied blocks of b < M vectors so far)
        if (int rc = ensure_workspace(h, M); rc != KL_OK) return rc;
        if (int rc = back_transform(h, Y, N, Vd, N, M); rc != KL_OK) return rc;
        if (!c.sym) {
            // unit L2 norm of the field sum_j v_j R_j under the Gauss rule
            if (int rc = field_at_quadrature(h, Vd, N, h->ws[0], M); rc != KL_OK) return rc;
            if (int rc = ck(c, launch_weighted_norms(h->ws[0], h->S, h->S, M, h->src_scale, c.w.norms, h->stream), "wnorm"); rc != KL_OK) return rc;
            if (int rc = ck(c, launch_scale_cols(Vd, N, N, M, c.w.norms, 1, h->stream), "scale"); rc != KL_OK) return rc;
        }
        if (int rc = ck(c, launch_sign_fix(Vd, N, N, M, h->stream), "sign"); rc != KL_OK) return rc;
        cudaError_t e = cudaMemcpy2DAsync(Vout, size_t(ldv) * sizeof(double), Vd, size_t(N) * sizeof(double),
                                          size_t(N) * sizeof(double), size_t(M),
                                          v_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                          h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "copy eigenvectors");
    }
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "kl_eigs sync");
    if (int rc = check_device_error(h); rc != KL_OK) return rc;
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    if (info) {
        info->restarts = restarts;
        info->applies = c.applies;
        info->vectors_applied = c.vectors_applied;
        info->converged = nconv;
        info->max_resid = max_res;
        info->max_imag = max_imag;
        info->seconds = secs;
    }
    if (status_out != KL_OK) return fail(h, status_out, "iteration limit reached before convergence");
    // an imaginary part below the residual tolerance (relative to |lambda_1|)
    // is not resolved by the solve: a numerically multiple real eigenvalue
    // of a non-normal projected matrix splits into such pairs
    if (!c.sym && max_imag > std::max(1e-8, tol)) {
        h->err = "complex eigenvalues among the returned pairs";
        return KL_WARN_COMPLEX;
    }
    return KL_OK;
}
}  // namespace
