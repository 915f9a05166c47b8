"""Pins of the standard Gauss-Legendre Galerkin oracle, the reference of the
library's KL_GALERKIN_STD method (Sec. 3.1: both integrals of the Galerkin
matrices by a Gauss-Legendre rule on every element)."""
import numpy as np

from oracle import closed_form, standard
from oracle.problem import Problem


def _gauss_exact(L, n):
    # exp(-|x-y|^2/L^2) on the unit cube is the product of three 1D kernels:
    # its eigenvalues are the products of the 1D ones (converged Nystrom)
    l1 = closed_form.nystrom_1d(lambda x, y: np.exp(-(x - y) ** 2 / L ** 2), 400)
    return closed_form.product_spectrum([l1[:n]] * 3, n)


def test_standard_galerkin_ritz_values_below_exact_spectrum():
    """Min-max: with accurately integrated matrices the Galerkin eigenvalues
    are Ritz values of the covariance operator, below its exact eigenvalues,
    and the finer mesh (a larger trial space) is closer."""
    L = 0.5
    exact = _gauss_exact(L, 10)
    errs = []
    for e in (2, 3):
        prob = Problem("cube", 2, (e, e, e), kernel="gauss", sigma=1.0, L=L)
        lam, V, mats = standard.solve(prob, 10, nq=6)
        assert np.all(lam <= exact * (1 + 1e-10)), (lam, exact)
        errs.append(float(np.max((exact - lam) / exact)))
        # Z-orthonormal eigenvectors
        assert np.allclose(V.T @ mats["Z"] @ V, np.eye(10), atol=1e-10)
    assert errs[1] < errs[0]
    assert errs[1] < 2e-3


def test_library_rule_differs_by_quadrature_error_only():
    """The library's rule (p + 1 points per direction per element) gives the
    same spectrum as an accurate rule up to quadrature error."""
    prob = Problem("cube", 2, (3, 3, 3), kernel="gauss", sigma=1.0, L=0.5)
    lam3, _, _ = standard.solve(prob, 10)
    lam6, _, _ = standard.solve(prob, 10, nq=6)
    assert np.max(np.abs(lam3 - lam6) / lam6) < 1e-3
