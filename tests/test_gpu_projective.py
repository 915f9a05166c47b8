"""The projective cube on the GPU: collocation with NURBS weights that are not a
tensor product (Sec. 3.2), applied as Z^-1 = diag(1/w) B^-1 diag(W(x_i))
around the B-spline Kronecker solves, and R v = (B (w v)) / W.

Element-by-element parity with the dense oracle (which builds Z = (R_j(x_i))
from the 3D rational basis and solves it densely) runs in the parametrised
tests of test_gpu_parity.py and test_gpu_sampling.py; here: the closed-form
cases and a larger mesh in mixed precision.
"""
import numpy as np
import pytest

from _entrywise import assert_entrywise
from kl_inputs import random_block
from oracle import collocation
from oracle.problem import Problem

pytestmark = pytest.mark.gpu

C = (0.5, 0.25, -0.2)


@pytest.fixture(scope="module")
def kl():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_00629_gb300 import _build
    _build.build()
    import paper_2101_00629_gb300 as mod
    return mod


def _create(kl, method, precision="fp64", geometry="projective_cube", elems=(4, 3, 3), kernel="gauss",
            sigma=1.0, L=0.6, geo=C, **kw):
    import torch
    p = kl.params(geometry=geometry, degree=2, elems=elems, kernel=kernel, sigma=sigma, L=L, method=method,
                  precision=precision, geo=geo, **kw)
    return kl.kl_create(p, torch.cuda.current_stream())


def _eigs(kl, h, M):
    N = kl.kl_dims(h)[0]
    lam = np.zeros(M)
    V = np.zeros((M, N))
    info = kl.kl_solve_info()
    rc = kl.kl_eigs(h, M, 0.0, lam, V, N, 0, None, info)
    return rc, lam, V


def test_constant_kernel_collocation_eigenvalue_is_the_rule_volume(kl):
    sigma = 1.3
    h = _create(kl, "collocation", kernel="const", sigma=sigma, L=1.0, block_k=4)
    try:
        rc, lam, _ = _eigs(kl, h, 3)
        assert rc == 0
        prob = Problem("projective_cube", 2, (4, 3, 3), "const", sigma, 1.0, geo=C)
        Xq, Wq = prob.quadrature()
        rule_vol = float(np.sum(Wq * (1.0 + Xq @ np.array(C)) ** -4))
        assert abs(lam[0] - sigma ** 2 * rule_vol) < 1e-11 * lam[0]
        assert np.max(np.abs(lam[1:])) < 1e-11 * lam[0]
    finally:
        kl.kl_destroy(h)


@pytest.mark.parametrize("method", ["galerkin", "collocation"])
def test_zero_c_matches_the_cube(kl, method):
    h0 = _create(kl, method, geo=(0.0, 0.0, 0.0))
    h1 = _create(kl, method, geometry="cube")
    try:
        rc0, l0, V0 = _eigs(kl, h0, 6)
        rc1, l1, V1 = _eigs(kl, h1, 6)
        assert rc0 == 0 and rc1 == 0
        assert np.max(np.abs(l0 - l1)) < 1e-11 * l1[0]
    finally:
        kl.kl_destroy(h0)
        kl.kl_destroy(h1)


def test_zinv_inverts_the_rational_collocation_matrix(kl):
    """Z (Z^-1 X) = X with Z assembled densely from the oracle's rational basis."""
    import torch
    prob = Problem("projective_cube", 2, (4, 3, 3), "gauss", 1.0, 0.6, geo=C)
    Xc = collocation.collocation_points(prob)
    Z = collocation.rational_basis(prob, Xc, collocation.nurbs_weights(prob))
    h = _create(kl, "collocation")
    try:
        N = kl.kl_dims(h)[0]
        X = random_block(N, 4, seed=31)
        Xd = torch.from_numpy(X).cuda()
        Yd = torch.empty_like(Xd)
        kl.kl_apply_Zinv(h, Xd, N, Yd, N, 4)
        torch.cuda.synchronize()
        Y = Yd.cpu().numpy()
        # residual entry by entry against |Z| |Y| (the size of its rounding)
        assert_entrywise((Z @ Y.T).T, X, (np.abs(Z) @ np.abs(Y.T)).T, 1e-13, "Z (Z^-1 X) = X")
    finally:
        kl.kl_destroy(h)


@pytest.mark.parametrize("method", ["galerkin", "collocation"])
@pytest.mark.parametrize("precision", ["bf16", "tf32"])
def test_mixed_matches_fp64_on_a_larger_mesh(kl, method, precision):
    """12 x 10 x 8 elements, exponential kernel: mixed eigenvalues within 1e-5
    of the GPU's FP64 ones (the tcgen05 path with the rational scalings)."""
    M = 12
    kw = dict(elems=(12, 10, 8), kernel="exp", L=0.8, block_k=8)
    h64 = _create(kl, method, "fp64", **kw)
    hmx = _create(kl, method, precision, **kw)
    try:
        rc0, l0, _ = _eigs(kl, h64, M)
        rc1, l1, _ = _eigs(kl, hmx, M)
        assert rc0 == 0 and rc1 == 0
        err = np.max(np.abs(l1 - l0) / np.abs(l0))
        print(f"{method} {precision}: max relative eigenvalue difference {err:.2e}")
        assert err < 1e-5
    finally:
        kl.kl_destroy(h64)
        kl.kl_destroy(hmx)
