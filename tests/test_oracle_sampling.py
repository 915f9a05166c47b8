"""Pins of the oracle's K-L sampling (CPU): identities of the expansion that
do not restate its formula.

* The integral of the pointwise variance sum_m lambda_m phi_m^2 equals
  sum_m lambda_m when the modes are L2-orthonormal: exactly for Galerkin on
  both geometries (N_i N_j |det DF| = B_i B_j, a polynomial the Gauss rule
  integrates exactly), and for collocation with its Gauss-rule normalisation.
  A missing sqrt(lambda), a wrong Jacobian power or transposed coefficients
  break it.
* The empirical covariance of many seeded realisations converges to
  sum_m lambda_m phi_m(x) phi_m(y) (law of large numbers).
* Galerkin modes are orthonormal under the Gauss rule (Z-orthonormality of
  the eigenvectors seen through the evaluated basis).
"""
import numpy as np
import pytest

from kl_inputs import PARITY_CASES
from oracle import collocation, galerkin, sampling
from oracle.problem import Problem


def _prob(case):
    c = PARITY_CASES[case]
    return Problem(c["geometry"], c["p"], c["elems"], c["kernel"], c["sigma"], c["L"])


@pytest.mark.parametrize("case", ["cube_p2_e3x4x5_gauss", "annulus_p2_e4x4x2_gauss", "annulus_p3_e4x3x2_exp"])
def test_variance_integral_galerkin(case):
    prob = _prob(case)
    lam, V, _ = galerkin.solve(prob, 12)
    got = sampling.variance_integral(prob, "galerkin", lam, V)
    assert abs(got - lam.sum()) <= 1e-12 * lam.sum()


@pytest.mark.parametrize("case", ["cube_p2_e6x5x7_expsep", "annulus_p2_e4x4x2_gauss"])
def test_variance_integral_collocation(case):
    prob = _prob(case)
    lam, V, _ = collocation.solve(prob, 10)
    got = sampling.variance_integral(prob, "collocation", lam, V)
    assert abs(got - lam.sum()) <= 1e-10 * lam.sum()


def test_galerkin_modes_orthonormal_under_gauss_rule():
    prob = _prob("annulus_p2_e4x4x2_gauss")
    lam, V, _ = galerkin.solve(prob, 10)
    X, W, _ = sampling.grid(prob)
    Phi = sampling.modes(prob, "galerkin", V)
    G = Phi.T @ ((W * np.abs(prob.geom.detDF(X)))[:, None] * Phi)
    assert np.max(np.abs(G - np.eye(10))) < 1e-12


def test_empirical_covariance_converges():
    prob = _prob("cube_p2_e3x4x5_gauss")
    lam, V, _ = galerkin.solve(prob, 6)
    rng = np.random.Generator(np.random.PCG64(7))
    ns = 40000
    xi = rng.standard_normal((6, ns))
    A = sampling.samples(prob, "galerkin", lam, V, xi)       # Q x ns
    Phi = sampling.modes(prob, "galerkin", V)
    pts = [0, 17, 123, A.shape[0] - 1]
    for a in pts:
        for b in pts:
            emp = float(A[a] @ A[b]) / ns
            exact = float(Phi[a] @ (lam * Phi[b]))
            scale = np.sqrt(float(Phi[a] ** 2 @ lam) * float(Phi[b] ** 2 @ lam))
            assert abs(emp - exact) <= 5 * scale / np.sqrt(ns)
