"""GPU parity of the standard Gauss-Legendre Galerkin method (KL_GALERKIN_STD,
Sec. 3.1: the trial space B_i / sqrt(det DF) with both integrals by the
Gauss-Legendre rule of (p+1)^3 points per element) against the dense FP64
oracle of the same rule. Tolerances as for the IBQ-Galerkin parity tests,
entry by entry: A = N^T W Gamma W N has no sign changes in its factors (the
trial functions B / sqrt(det DF), the weights and the kernel are
non-negative), so |A| |X| bounds each entry's rounding error."""
import functools

import numpy as np
import pytest

from _entrywise import assert_entrywise, bound, dense_abs
from kl_inputs import PARITY_CASES, random_block
from oracle import standard
from oracle.problem import Problem

pytestmark = pytest.mark.gpu

APPLY_TOL = {"fp64": 1e-12, "fp32": 2e-6, "tf32": 2e-6, "bf16": 5e-5}
LAM_TOL = {"fp64": 1e-10, "bf16": 1e-5, "tf32": 1e-5}
CASES = ["cube_p2_e3x4x5_gauss", "annulus_p2_e4x4x2_gauss", "cube_p3_e4x3x3_matern", "cube_p2_e5x4x4_exp",
         "half_annulus_p2_e4x3x2_gauss"]


@pytest.fixture(scope="module")
def kl():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_00629_gb300 import _build
    _build.build()
    import paper_2101_00629_gb300 as mod
    return mod


@functools.lru_cache(maxsize=None)
def _oracle(case):
    s = PARITY_CASES[case]
    prob = Problem(s["geometry"], s["p"], s["elems"], s["kernel"], s["sigma"], s["L"])
    A, Z = standard.matrices(prob, prob.p + 1)
    Ap, _ = standard.standard_form(prob)
    return prob, A, Z, Ap, dense_abs(A, Z)


def _create(kl, case, precision, **kw):
    import torch
    s = PARITY_CASES[case]
    p = kl.params(geometry=s["geometry"], degree=s["p"], elems=s["elems"], kernel=s["kernel"], sigma=s["sigma"],
                  L=s["L"], method="galerkin_std", precision=precision, **kw)
    return kl.kl_create(p, torch.cuda.current_stream())


def _apply(kl, fn, h, X):
    import torch
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    Yd = torch.full_like(Xd, float("nan"))
    fn(h, Xd, X.shape[1], Yd, X.shape[1], X.shape[0])
    torch.cuda.synchronize()
    return Yd.cpu().numpy()


def _nw(Y, ref):
    return np.linalg.norm(Y - ref) / np.linalg.norm(ref)


def _check(Y, ref, absop, X, tol, label):
    r = assert_entrywise(Y, ref, bound(absop, X), tol, label)
    print(f"{label}: worst entry {r:.2e} of the bound, normwise {_nw(Y, ref):.2e}")


@pytest.mark.parametrize("case", CASES)
def test_std_apply_fp64(kl, case):
    prob, A, Z, Ap, sc = _oracle(case)
    h = _create(kl, case, "fp64")
    try:
        N, S, T = kl.kl_dims(h)
        assert (N, S) == standard.dims(prob)
        assert T == S  # the Gauss points are sources and targets
        X = random_block(N, 5, seed=21)
        _check(_apply(kl, kl.kl_apply_A, h, X), (A @ X.T).T, sc["A"], X, APPLY_TOL["fp64"], f"{case} std A")
        _check(_apply(kl, kl.kl_apply_Zinv, h, X), np.linalg.solve(Z, X.T).T, sc["Zinv"], X, 1e-12,
               f"{case} std Zinv")
        _check(_apply(kl, kl.kl_apply_Aprime, h, X), (Ap @ X.T).T, sc["Aprime"], X, 1e-12, f"{case} std A'")
    finally:
        kl.kl_destroy(h)


@pytest.mark.parametrize("precision", ["fp32", "bf16", "tf32"])
@pytest.mark.parametrize("case", CASES)
def test_std_apply_mixed(kl, case, precision):
    prob, A, Z, Ap, sc = _oracle(case)
    h = _create(kl, case, precision)
    try:
        N = kl.kl_dims(h)[0]
        X = random_block(N, 8, seed=22)
        _check(_apply(kl, kl.kl_apply_A, h, X), (A @ X.T).T, sc["A"], X, APPLY_TOL[precision],
               f"{case} std A {precision}")
    finally:
        kl.kl_destroy(h)


@pytest.mark.parametrize("precision", ["fp64", "bf16"])
@pytest.mark.parametrize("case", CASES)
def test_std_eigenpairs(kl, case, precision):
    import torch
    prob, A, Z, Ap, _ = _oracle(case)
    M = 8
    lam_ref, V_ref, _ = standard.solve(prob, M)
    h = _create(kl, case, precision)
    try:
        N = kl.kl_dims(h)[0]
        lam = np.zeros(M)
        Vd = torch.empty((M, N), dtype=torch.float64, device="cuda")
        rc = kl.kl_eigs(h, M, 0.0, lam, Vd, N, 1)
        assert rc == kl.KL_OK
        V = Vd.cpu().numpy().T
    finally:
        kl.kl_destroy(h)
    rel = np.abs(lam - lam_ref) / np.maximum(np.abs(lam_ref), 1e-6 * abs(lam_ref[0]))
    print(f"{case} std eigs {precision}: max rel err {rel.max():.2e}")
    assert rel.max() < LAM_TOL[precision]
    # Z-orthonormal eigenvectors (unit L2 norm of the eigenfunctions)
    assert np.max(np.abs(V.T @ Z @ V - np.eye(M))) < (1e-8 if precision == "fp64" else 1e-5)
