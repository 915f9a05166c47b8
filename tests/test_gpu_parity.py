"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Tolerances (derivation in the design notes):
  * Operator applications are compared entry by entry: every entry's error
    is bounded by tol * (|op| |X|)_ij, |op| the absolute values of the
    oracle's factors of the operator (tests/_entrywise.py), i.e. the size of
    that entry's rounding error. FP64: tol = 1e-12 (measured ratios of a
    factored FP64 evaluation to the dense oracle are ~2e-16). FP32 kernel
    values carry a relative error of a few 1e-7 and split (hi + lo) BF16 /
    TF32 products keep about 16 / 21 significant bits per term: 2e-6 (fp32,
    tf32) and 5e-5 (bf16); every column's relative error is held to the same
    bound.
  * Eigenvalues: relative error <= 1e-10 (FP64) and <= 1e-5 (mixed), with
    the denominator floored at 1e-6 * lambda_1 for tiny eigenvalues.
  * Z-orthonormality (Galerkin) and the collocation eigen-residual <= 1e-8.
"""
import functools

import numpy as np
import pytest
import scipy.linalg as sla

from _entrywise import assert_entrywise, bound, collocation_abs, galerkin_abs
from kl_inputs import PARITY_CASES, WORKLOADS, problem_args, random_block
from oracle import closed_form, collocation, galerkin
from oracle.problem import Problem

pytestmark = pytest.mark.gpu

APPLY_TOL = {"fp64": 1e-12, "fp32": 2e-6, "tf32": 2e-6, "bf16": 5e-5}
LAM_TOL = {"fp64": 1e-10, "fp32": 1e-5, "tf32": 1e-5, "bf16": 1e-5}


@pytest.fixture(scope="module")
def kl():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_00629_gb300 import _build
    _build.build()
    import paper_2101_00629_gb300 as mod
    return mod


def _problem(spec):
    return Problem(spec["geometry"], spec["p"], spec["elems"], spec["kernel"], spec["sigma"], spec["L"],
                   geo=spec.get("geo"))


@functools.lru_cache(maxsize=None)
def _oracle(case, method):
    spec = PARITY_CASES[case]
    prob = _problem(spec)
    return _oracle_of(prob, method)


def _oracle_of(prob, method):
    if method == "galerkin":
        A, Z, parts = galerkin.matrices(prob, with_parts=True)
        Ap, _ = galerkin.standard_form(prob)
        scales = galerkin_abs(parts, Z)
    else:
        A, Z = collocation.matrices(prob)
        Ap = np.linalg.solve(Z, A)
        scales = collocation_abs(A, Z)
    return prob, A, Z, Ap, scales


def _check(Y, ref, absop, X, tol, label):
    """Entry-by-entry bound and, for the record, the normwise error."""
    r = assert_entrywise(Y, ref, bound(absop, X), tol, label)
    print(f"{label}: worst entry {r:.2e} of the bound, normwise {_normwise(Y, ref):.2e}")
    return r


def _create(kl, spec, method, precision, **kw):
    import torch
    if "geo" in spec:
        kw = dict(kw, geo=spec["geo"])
    p = kl.params(geometry=spec["geometry"], degree=spec["p"], elems=spec["elems"], kernel=spec["kernel"],
                  sigma=spec["sigma"], L=spec["L"], method=method, precision=precision, **kw)
    return kl.kl_create(p, torch.cuda.current_stream())


def _apply(kl, fn, h, X, ldx=None):
    import torch
    k, n = X.shape
    ldx = n if ldx is None else ldx
    Xd = torch.zeros((k, ldx), dtype=torch.float64, device="cuda")
    Xd[:, :n] = torch.from_numpy(X)
    Yd = torch.full((k, ldx), float("nan"), dtype=torch.float64, device="cuda")
    fn(h, Xd, ldx, Yd, ldx, k)
    torch.cuda.synchronize()
    return Yd[:, :n].cpu().numpy()


def _normwise(Y, ref):
    return np.linalg.norm(Y - ref) / np.linalg.norm(ref)


# --------------------------------------------------------------------------
# operator applications
# --------------------------------------------------------------------------

@pytest.mark.parametrize("case", sorted(PARITY_CASES))
@pytest.mark.parametrize("method", ["galerkin", "collocation"])
def test_apply_fp64(kl, case, method):
    prob, A, Z, Ap, sc = _oracle(case, method)
    h = _create(kl, PARITY_CASES[case], method, "fp64")
    try:
        N, S, T = kl.kl_dims(h)
        assert N == A.shape[0]
        mod = galerkin if method == "galerkin" else collocation
        assert (N, S) == mod.dims(prob)
        X = random_block(N, 5, seed=11)
        Y = _apply(kl, kl.kl_apply_A, h, X)
        _check(Y, (A @ X.T).T, sc["A"], X, APPLY_TOL["fp64"], f"{case} {method} apply_A fp64")
        Yz = _apply(kl, kl.kl_apply_Zinv, h, X)
        _check(Yz, np.linalg.solve(Z, X.T).T, sc["Zinv"], X, 1e-12, f"{case} {method} apply_Zinv")
        Yp = _apply(kl, kl.kl_apply_Aprime, h, X)
        _check(Yp, (Ap @ X.T).T, sc["Aprime"], X, 1e-12, f"{case} {method} apply_Aprime")
    finally:
        kl.kl_destroy(h)


@pytest.mark.parametrize("precision", ["fp32", "bf16", "tf32"])
@pytest.mark.parametrize("case", ["cube_p2_e6x5x7_expsep", "annulus_p2_e4x4x2_gauss", "cube_p3_e4x3x3_matern",
                                  "cube_p2_e5x4x4_exp", "projective_p2_e4x3x3_gauss"])
@pytest.mark.parametrize("method", ["galerkin", "collocation"])
def test_apply_mixed(kl, case, method, precision):
    prob, A, Z, Ap, sc = _oracle(case, method)
    h = _create(kl, PARITY_CASES[case], method, precision)
    try:
        N, _, _ = kl.kl_dims(h)
        X = random_block(N, 8, seed=12)
        Y = _apply(kl, kl.kl_apply_A, h, X)
        ref = (A @ X.T).T
        _check(Y, ref, sc["A"], X, APPLY_TOL[precision], f"{case} {method} apply_A {precision}")
        # every column's relative error, the bound widened only where the
        # column's entries cancel (|op||x| larger than |op x|)
        colerr = np.linalg.norm(Y - ref, axis=1) / np.linalg.norm(ref, axis=1)
        amp = np.maximum(1.0, np.linalg.norm(bound(sc["A"], X), axis=1) / np.linalg.norm(ref, axis=1))
        worst = int(np.argmax(colerr / amp))
        print(f"worst column {worst}: relative error {colerr[worst]:.2e}, cancellation factor {amp[worst]:.2f}")
        assert colerr[worst] < APPLY_TOL[precision] * amp[worst], (worst, colerr[worst], amp[worst])
    finally:
        kl.kl_destroy(h)


@pytest.mark.parametrize("precision", ["fp64", "bf16", "tf32"])
@pytest.mark.parametrize("k", [1, 3, 17, 33, 70])
def test_apply_ragged_block_widths(kl, k, precision):
    case, method = "cube_p2_e3x4x5_gauss", "galerkin"
    prob, A, Z, Ap, sc = _oracle(case, method)
    h = _create(kl, PARITY_CASES[case], method, precision)
    try:
        N, _, _ = kl.kl_dims(h)
        X = random_block(N, k, seed=100 + k)
        Y = _apply(kl, kl.kl_apply_A, h, X, ldx=N + 3)
        _check(Y, (A @ X.T).T, sc["A"], X, APPLY_TOL[precision], f"k={k} {precision}")
    finally:
        kl.kl_destroy(h)


@pytest.mark.parametrize("dim,elems", [(1, (7,)), (2, (4, 5))])
@pytest.mark.parametrize("method", ["galerkin", "collocation"])
def test_apply_lower_dimensions(kl, dim, elems, method):
    spec = dict(geometry="cube", p=2, elems=elems, kernel="gauss", sigma=1.0, L=0.4)
    prob, A, Z, Ap, sc = _oracle_of(_problem(spec), method)
    h = _create(kl, spec, method, "fp64")
    try:
        N, _, _ = kl.kl_dims(h)
        assert N == A.shape[0]
        X = random_block(N, 3, seed=5)
        _check(_apply(kl, kl.kl_apply_A, h, X), (A @ X.T).T, sc["A"], X, 1e-12, f"dim {dim} {method}")
    finally:
        kl.kl_destroy(h)


# --------------------------------------------------------------------------
# eigenpairs
# --------------------------------------------------------------------------

def _lam_err(lam, ref):
    floor = 1e-6 * abs(ref[0])
    return np.max(np.abs(lam - ref) / np.maximum(np.abs(ref), floor))


def _clusters(lam, rtol=1e-6):
    groups, cur = [], [0]
    for i in range(1, len(lam)):
        if abs(lam[i] - lam[cur[-1]]) <= rtol * abs(lam[0]):
            cur.append(i)
        else:
            groups.append(cur)
            cur = [i]
    groups.append(cur)
    return groups


def _subspace_angle(U, W, G=None):
    """Largest principal angle between span(U) and span(W) (columns), inner
    product G (identity if None)."""
    G = np.eye(U.shape[0]) if G is None else G
    L = np.linalg.cholesky(G)
    qu, _ = np.linalg.qr(L.T @ U)
    qw, _ = np.linalg.qr(L.T @ W)
    s = np.linalg.svd(qu.T @ qw, compute_uv=False)
    return float(np.arccos(np.clip(np.min(s), -1.0, 1.0)))


def _run_eigs(kl, h, M, N):
    lam = np.zeros(M)
    V = np.zeros((M, N))
    res = np.zeros(M)
    info = kl.kl_solve_info()
    rc = kl.kl_eigs(h, M, 0.0, lam, V, N, 0, res, info)
    return rc, lam, V.T.copy(), res, info


@pytest.mark.parametrize("precision", ["fp64", "bf16", "tf32", "fp32"])
@pytest.mark.parametrize("case", ["cube_p2_e6x5x7_expsep", "annulus_p2_e4x4x2_gauss", "annulus_p3_e4x3x2_exp",
                                  "cube_p3_e4x3x3_matern", "half_annulus_p2_e4x3x2_gauss",
                                  "half_annulus_p2_e6x2x2_exp", "projective_p2_e4x3x3_gauss",
                                  "projective_p3_e3x3x2_exp"])
@pytest.mark.parametrize("method", ["galerkin", "collocation"])
def test_eigs_vs_oracle(kl, case, method, precision):
    prob, A, Z, Ap, _ = _oracle(case, method)
    mod = galerkin if method == "galerkin" else collocation
    M = 8
    lam_ref, V_ref, info_ref = mod.solve(prob, M + 4)
    h = _create(kl, PARITY_CASES[case], method, precision, block_k=8)
    try:
        N, _, _ = kl.kl_dims(h)
        rc, lam, V, res, info = _run_eigs(kl, h, M, N)
        err = _lam_err(lam, lam_ref[:M])
        print(f"{case} {method} {precision}: lambda err {err:.2e} applies {info.applies} restarts {info.restarts} "
              f"max resid {info.max_resid:.1e}")
        assert rc == 0
        assert err < LAM_TOL[precision]
        if method == "galerkin":
            orth = np.max(np.abs(V.T @ Z @ V - np.eye(M)))
            assert orth < 1e-8
            resid = np.linalg.norm(A @ V - (Z @ V) * lam[None, :]) / (np.max(lam) * np.linalg.norm(Z @ V))
        else:
            resid = np.linalg.norm(A @ V - (Z @ V) * lam[None, :]) / (np.max(np.abs(lam)) * np.linalg.norm(Z @ V))
            assert np.allclose(collocation.l2_norms(prob, V), 1.0, atol=1e-8)
        if precision == "fp64":
            assert resid < 1e-8
            # eigenvectors: compare invariant subspaces cluster by cluster
            G = Z if method == "galerkin" else None
            for grp in _clusters(lam_ref[:M]):
                if grp[-1] + 1 < M or abs(lam_ref[M] - lam_ref[M - 1]) > 1e-6 * lam_ref[0]:
                    ang = _subspace_angle(V[:, grp], V_ref[:, grp], G)
                    assert ang < 1e-7, (grp, ang)
            # sign convention: largest-magnitude entry positive
            idx = np.argmax(np.abs(V), axis=0)
            assert np.all(V[idx, np.arange(M)] > 0)
    finally:
        kl.kl_destroy(h)


@pytest.mark.parametrize("method", ["galerkin", "collocation"])
def test_constant_kernel_rank_one_on_gpu(kl, method):
    spec = dict(geometry="cube", p=2, elems=(2, 3, 2), kernel="const", sigma=1.5, L=1.0)
    h = _create(kl, spec, method, "fp64", block_k=4)
    try:
        N, _, _ = kl.kl_dims(h)
        rc, lam, V, res, info = _run_eigs(kl, h, 3, N)
        assert abs(lam[0] - 2.25) < 1e-11
        assert np.max(np.abs(lam[1:])) < 1e-11
    finally:
        kl.kl_destroy(h)


def test_eigs_complete_basis(kl):
    spec = dict(geometry="cube", p=2, elems=(1, 2, 1), kernel="gauss", sigma=1.0, L=0.7)
    prob = _problem(spec)
    lam_ref, _, _ = galerkin.solve(prob)
    h = _create(kl, spec, "galerkin", "fp64", block_k=5)
    try:
        N, _, _ = kl.kl_dims(h)
        rc, lam, V, res, info = _run_eigs(kl, h, N, N)
        # relative bound with the 1e-6 lambda_1 floor, widened only by the
        # backward-error floor of any FP64 symmetric eigensolver (Weyl: an
        # eigenvalue moves by at most ||E|| ~ N eps ||A'||), which the
        # roundoff-level tail of a complete Gaussian spectrum reaches
        eps = np.finfo(np.float64).eps
        allowed = LAM_TOL["fp64"] * np.maximum(np.abs(lam_ref), 1e-6 * lam_ref[0]) + 16 * N * eps * lam_ref[0]
        worst = int(np.argmax(np.abs(lam - lam_ref) / allowed))
        print(f"complete basis N={N}: worst eigenvalue {worst} err {abs(lam[worst] - lam_ref[worst]):.2e} "
              f"allowed {allowed[worst]:.2e}")
        assert abs(lam[worst] - lam_ref[worst]) <= allowed[worst], (worst, lam[worst], lam_ref[worst])
    finally:
        kl.kl_destroy(h)


def test_workload_cube_p2_e4_gauss(kl):
    """The small benchmark workload: 216 dofs, Gaussian, M = 10, dense oracle."""
    w = WORKLOADS["cube_p2_e4_gauss"]
    prob = Problem(**{k: v for k, v in problem_args(w).items()})
    lam_ref, V_ref, info_ref = galerkin.solve(prob, w["M"])
    for precision in ("fp64", "bf16"):
        h = _create(kl, dict(problem_args(w)), "galerkin", precision, block_k=w["k"])
        try:
            N, _, _ = kl.kl_dims(h)
            rc, lam, V, res, info = _run_eigs(kl, h, w["M"], N)
            err = _lam_err(lam, lam_ref)
            print(f"cube_p2_e4_gauss {precision}: {err:.2e}")
            assert err < LAM_TOL[precision]
            orth = np.max(np.abs(V.T @ info_ref["Z"] @ V - np.eye(w["M"])))
            assert orth < 1e-8
        finally:
            kl.kl_destroy(h)


# --------------------------------------------------------------------------
# full-size separable workload: pinned by products of 1D oracle spectra
# --------------------------------------------------------------------------

def _sep_reference(w, method, M):
    mod = galerkin if method == "galerkin" else collocation
    args = problem_args(w)
    l1 = [mod.solve(Problem(args["geometry"], args["p"], (n,), args["kernel"], 1.0, args["L"]))[0]
          for n in args["elems"]]
    return args["sigma"] ** 2 * closed_form.product_spectrum(l1, M)


@pytest.mark.parametrize("method", ["galerkin", "collocation"])
@pytest.mark.parametrize("precision", ["fp64", "bf16"])
def test_workload_cube_p2_e16_expsep_full_size(kl, method, precision):
    """5832 dofs; the separable kernel makes the 3D discrete spectrum the set
    of products of 1D discrete eigenvalues (oracle pin), at any size."""
    w = WORKLOADS["cube_p2_e16_expsep"]
    M = w["M"]
    ref = _sep_reference(w, method, M)
    h = _create(kl, dict(problem_args(w)), method, precision, block_k=w["k"])
    try:
        N, _, _ = kl.kl_dims(h)
        assert N == 18 ** 3
        rc, lam, V, res, info = _run_eigs(kl, h, M, N)
        err = _lam_err(lam, ref)
        print(f"cube_p2_e16_expsep {method} {precision}: lambda err {err:.2e} applies {info.applies} "
              f"restarts {info.restarts} seconds {info.seconds:.3f}")
        assert rc == 0
        assert err < LAM_TOL[precision]
    finally:
        kl.kl_destroy(h)


@pytest.mark.parametrize("method", ["galerkin", "collocation"])
@pytest.mark.parametrize("precision", ["fp64", "bf16"])
def test_large_basis_separable_cube(kl, method, precision):
    """M = 50 with block size 16 (basis width 176) on 13728 dofs: the basis
    projections then split their long dimension more finely for narrower
    blocks than for the full basis (scratch sized for every shape). Pinned by
    the products of 1D oracle spectra (separable kernel on a box)."""
    w = dict(geometry="cube", p=2, elems=(24, 20, 22), kernel="exp_sep", sigma=1.0, L=0.8)
    M = 50
    ref = _sep_reference(w, method, M)
    h = _create(kl, w, method, precision, block_k=16)
    try:
        N, _, _ = kl.kl_dims(h)
        assert N == 26 * 22 * 24
        rc, lam, V, res, info = _run_eigs(kl, h, M, N)
        err = _lam_err(lam, ref)
        print(f"large basis {method} {precision}: lambda err {err:.2e} applies {info.applies} "
              f"restarts {info.restarts} seconds {info.seconds:.3f}")
        assert rc == 0
        assert err < LAM_TOL[precision]
    finally:
        kl.kl_destroy(h)


def _kron3_apply(F, X):
    """(F[2] x F[1] x F[0]) applied to every row of X (k, n), direction 1
    fastest, by three mode products (reference arithmetic of the test)."""
    k = X.shape[0]
    n = [f.shape[1] for f in F]
    T = X.reshape(k, n[2], n[1], n[0])
    T = np.einsum("ia,cdba->cdbi", F[0], T)
    T = np.einsum("ib,cdba->cdia", F[1], T)
    T = np.einsum("id,cdba->ciba", F[2], T)
    return T.reshape(k, -1)


@pytest.mark.parametrize("method", ["galerkin", "collocation"])
@pytest.mark.parametrize("precision", ["fp64", "bf16", "tf32"])
def test_workload_cube_p2_e16_expsep_apply_full_size(kl, method, precision):
    """kl_apply_A at full size against kron(A_z, A_y, A_x) of 1D oracle
    matrices (exact for the separable kernel on the cube)."""
    w = WORKLOADS["cube_p2_e16_expsep"]
    args = problem_args(w)
    mod = galerkin if method == "galerkin" else collocation
    one_d = [_oracle_of(Problem("cube", 2, (n,), args["kernel"], 1.0, args["L"]), method) for n in args["elems"]]
    A1 = [o[1] for o in one_d]
    S1 = [o[4]["A"] for o in one_d]  # |op| of each direction; |kron| = kron of |.|
    h = _create(kl, dict(args), method, precision, block_k=w["k"])
    try:
        N, _, _ = kl.kl_dims(h)
        X = random_block(N, w["k"], seed=21)
        Y = _apply(kl, kl.kl_apply_A, h, X)
        ref = _kron3_apply(A1, X) * args["sigma"] ** 2
        scale = _kron3_apply(S1, np.abs(X)) * args["sigma"] ** 2
        r = assert_entrywise(Y, ref, scale, APPLY_TOL[precision], f"full-size apply {method} {precision}")
        print(f"full-size apply {method} {precision}: worst entry {r:.2e}, normwise {_normwise(Y, ref):.2e}")
    finally:
        kl.kl_destroy(h)


# --------------------------------------------------------------------------
# argument errors on the device path
# --------------------------------------------------------------------------

def test_bad_call_arguments(kl):
    import torch
    spec = PARITY_CASES["cube_p2_e3x4x5_gauss"]
    h = _create(kl, spec, "galerkin", "fp64")
    try:
        N, _, _ = kl.kl_dims(h)
        X = torch.zeros((2, N), dtype=torch.float64, device="cuda")
        with pytest.raises(kl.KLError):
            kl.kl_apply_A(h, X, N, X, N, 0)
        with pytest.raises(kl.KLError):
            kl.kl_apply_A(h, X, N - 1, X, N, 2)
        with pytest.raises(kl.KLError):
            kl.kl_eigs(h, N + 1, 0.0, np.zeros(N + 1), None, N, 0)
    finally:
        kl.kl_destroy(h)
