"""Pins of the oracle's Galerkin and collocation solvers (CPU only).

Each test checks the oracle against something other than itself: exact
spectra of special kernels, the Kronecker identity of separable kernels,
textbook closed forms, an independent Nystrom discretisation, brute-force
double quadrature, and invariants of the discrete problems.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import closed_form, collocation, galerkin, kernels, splines, standard
from oracle.problem import Problem


def _rel(a, b):
    return np.max(np.abs(np.asarray(a) - np.asarray(b)) / np.abs(np.asarray(b)))


# --- exact special cases ----------------------------------------------------

@pytest.mark.parametrize("method", [galerkin, collocation])
@pytest.mark.parametrize("p,elems", [(2, (2, 3, 2)), (3, (2, 2, 1))])
def test_constant_kernel_rank_one(method, p, elems):
    """Gamma = sigma^2 on the unit cube: one eigenvalue sigma^2 |D|, the rest 0.
    IBQ is exact (the constant lies in the interpolation space) and the
    collocation quadrature integrates the partition of unity exactly."""
    sigma = 1.7
    prob = Problem("cube", p, elems, "const", sigma, 1.0)
    lam, V, _ = method.solve(prob)
    assert abs(lam[0] - sigma ** 2) < 1e-12
    assert np.max(np.abs(lam[1:])) < 1e-12


@pytest.mark.parametrize("method", [galerkin, collocation])
def test_degenerate_legendre_kernel_exact(method):
    """Gamma = sum mu_m P_m(x) P_m(x') with tensor Legendre polynomials of
    degree <= p per axis: both methods reproduce the mu_m exactly (the
    eigenfunctions lie in the trial space; IBQ and Gauss are exact)."""
    terms = [(0.9, (0, 0, 0)), (0.5, (1, 0, 2)), (0.31, (2, 1, 0)), (0.2, (0, 2, 1)), (0.07, (2, 2, 2))]
    prob = Problem("cube", 2, (2, 1, 3), closed_form.degenerate_kernel(terms))
    lam, _, _ = method.solve(prob)
    mus = np.array(sorted([t[0] for t in terms], reverse=True))
    assert _rel(lam[:5], mus) < 1e-11
    assert np.max(np.abs(lam[5:])) < 1e-11


def test_ibq_equals_brute_force_for_polynomial_kernel():
    """On the cube with a kernel of degree <= p per coordinate, the IBQ matrix
    equals the standard Galerkin matrix computed by brute-force double Gauss
    quadrature (the interpolation is exact)."""
    k = lambda x, y: (1.0 + np.sum(x * y, axis=-1) * 0.7) ** 2 + 0.3 * x[..., 0] * y[..., 1]
    prob = Problem("cube", 2, (2, 3, 1), k)
    A, Z = galerkin.matrices(prob)
    As, Zs = standard.matrices(prob, nq=4)
    assert np.max(np.abs(A - As)) < 1e-13 * np.max(np.abs(As))
    assert np.max(np.abs(Z - Zs)) < 1e-15


def test_collocation_matches_brute_force_for_polynomial_kernel():
    k = lambda x, y: (1.0 + np.sum(x * y, axis=-1)) ** 2
    prob = Problem("cube", 2, (3, 2, 2), k)
    A, Z, parts = collocation.matrices(prob, with_parts=True)
    # the same integral with a 5-point rule per element direction
    Xq, Wq = prob.quadrature(5)
    Rq = collocation.rational_basis(prob, Xq, parts["w"])
    Ab = k(parts["Pc"][:, None, :], Xq[None, :, :]) @ (Wq[:, None] * Rq)
    assert np.max(np.abs(A - Ab)) < 1e-13 * np.max(np.abs(Ab))


# --- separable kernels: Kronecker identity and closed forms --------------------

@pytest.mark.parametrize("kernel,L", [("gauss", 0.5), ("exp_sep", 1.0)])
@pytest.mark.parametrize("method", [galerkin, collocation])
def test_separable_kernel_is_kronecker_of_1d(kernel, L, method):
    """For a kernel that is a product over axes on the cube, the dense 3D
    matrices are exactly A_3 (x) A_2 (x) A_1 and Z_3 (x) Z_2 (x) Z_1 of the 1D
    problems (direction 1 fastest), hence the 3D spectrum is the set of
    products of 1D eigenvalues."""
    elems = (3, 2, 4)
    A, Z = method.matrices(Problem("cube", 2, elems, kernel, 1.0, L))
    A1 = [method.matrices(Problem("cube", 2, (n,), kernel, 1.0, L)) for n in elems]
    Ak = np.kron(A1[2][0], np.kron(A1[1][0], A1[0][0]))
    Zk = np.kron(A1[2][1], np.kron(A1[1][1], A1[0][1]))
    assert np.max(np.abs(A - Ak)) < 1e-14 * np.max(np.abs(A))
    assert np.max(np.abs(Z - Zk)) < 1e-14 * np.max(np.abs(Z))
    lam3, _, _ = method.solve(Problem("cube", 2, elems, kernel, 1.0, L), 12)
    l1 = [method.solve(Problem("cube", 2, (n,), kernel, 1.0, L))[0] for n in elems]
    assert _rel(lam3, closed_form.product_spectrum(l1, 12)) < 1e-12


@pytest.mark.parametrize("method", [galerkin, collocation])
def test_exp_1d_converges_to_closed_form(method):
    """1D exponential kernel: discrete eigenvalues converge to the textbook
    transcendental-equation eigenvalues at second order (C^0 kernel)."""
    ex = closed_form.exp1d_eigenvalues(1.0, 6)
    errs = []
    for n in (16, 32, 64):
        lam, _, _ = method.solve(Problem("cube", 2, (n,), "exp_sep", 1.0, 1.0), 6)
        errs.append(_rel(lam, ex))
    errs = np.array(errs)
    assert np.all(errs[1:] < errs[:-1] / 3.0)
    assert errs[-1] < 2e-3


def test_exp_closed_form_against_nystrom():
    ex = closed_form.exp1d_eigenvalues(0.5, 5)
    ny = closed_form.nystrom_1d(lambda x, y: np.exp(-np.abs(x - y) / 0.5), 3000)[:5]
    assert _rel(ny, ex) < 1e-4


@pytest.mark.parametrize("method", [galerkin, collocation])
def test_gauss_1d_converges_to_nystrom(method):
    ref = closed_form.nystrom_1d(lambda x, y: np.exp(-(x - y) ** 2 / 0.25), 400)[:6]
    errs = [_rel(method.solve(Problem("cube", 2, (n,), "gauss", 1.0, 0.5), 6)[0], ref) for n in (8, 16, 32)]
    assert errs[0] / errs[1] > 8 and errs[1] / errs[2] > 8
    assert errs[-1] < 1e-4


# --- invariants ---------------------------------------------------------------

@pytest.mark.parametrize("geom,kernel", [("cube", "gauss"), ("annulus", "matern32"), ("annulus", "exp")])
def test_galerkin_invariants(geom, kernel):
    prob = Problem(geom, 2, (3, 2, 2), kernel, 1.2, 0.8)
    lam, V, info = galerkin.solve(prob)
    A, Z = info["A"], info["Z"]
    assert np.max(np.abs(A - A.T)) == 0.0
    assert np.max(np.abs(Z - Z.T)) < 1e-15
    assert np.min(np.linalg.eigvalsh(Z)) > 0
    # Z-orthonormal eigenvectors and non-negative spectrum (A is a congruence of PSD Gamma)
    assert np.max(np.abs(V.T @ Z @ V - np.eye(V.shape[1]))) < 1e-10
    assert lam.min() > -1e-13 * lam[0]
    assert np.max(np.abs(A @ V - (Z @ V) * lam[None, :])) < 1e-12 * lam[0]


def test_galerkin_trace_gap_shrinks():
    """sum of all lambda_h = trace(Z^-1 A) approaches sigma^2 |D| (the trace of
    the continuous operator, integral of Gamma(x, x)) under refinement."""
    gaps = []
    for n in (1, 2, 4):
        prob = Problem("annulus", 2, (n, n, n), "gauss", 1.3, 0.7)
        A, Z = galerkin.matrices(prob)
        tr = np.trace(np.linalg.solve(Z, A))
        gaps.append(abs(tr - 1.3 ** 2 * prob.geom.volume()) / (1.3 ** 2 * prob.geom.volume()))
    assert gaps[1] < 0.6 * gaps[0] and gaps[2] < 0.6 * gaps[1]
    assert gaps[-1] < 0.05


def test_annulus_galerkin_converges_to_standard_galerkin():
    """IBQ (with J = sqrt(det DF) on the annulus) approaches the brute-force
    standard Galerkin matrix under refinement of the shared mesh."""
    diffs = []
    for n in (1, 2, 4):
        prob = Problem("annulus", 2, (n, n, n), "gauss", 1.0, 1.5)
        lam, _, _ = galerkin.solve(prob, 4)
        As, Zs = standard.matrices(prob, nq=4)
        ls = sla.eigh(As, Zs, eigvals_only=True)[::-1][:4]
        diffs.append(_rel(lam, ls))
    assert diffs[1] < diffs[0] / 3 and diffs[2] < diffs[1] / 4 and diffs[2] < 0.02


def test_annulus_constant_kernel():
    """Constant kernel on the annulus: collocation reproduces sigma^2 |D| up to
    the Gauss rule's error on the rational det DF; IBQ-Galerkin converges to it."""
    vol = 0.75 * np.pi
    lc, _, _ = collocation.solve(Problem("annulus", 2, (4, 2, 1), "const", 1.0, 1.0), 2)
    assert abs(lc[0] - vol) / vol < 1e-6 and abs(lc[1]) < 1e-12
    errs = []
    for n in (2, 4, 8):
        lg, _, _ = galerkin.solve(Problem("annulus", 2, (n, n, 1), "const", 1.0, 1.0), 1)
        errs.append(abs(lg[0] - vol) / vol)
    assert errs[1] < errs[0] / 8 and errs[2] < errs[1] / 8 and errs[2] < 1e-5


def test_annulus_nurbs_weights_reproduce_geometry_weight():
    prob = Problem("annulus", 3, (5, 2, 2), "gauss")
    w = collocation.nurbs_weights(prob)
    U = prob.trial_knots()
    n1 = splines.n_basis(U[0], 3)
    t = np.linspace(0, 1, 41)
    Wt = splines.bspline_basis(U[0], 3, t) @ w[:n1]
    assert np.max(np.abs(Wt - prob.geom.weight_function(t))) < 1e-14
    X = np.random.default_rng(7).random((30, 3))
    R = collocation.rational_basis(prob, X, w)
    assert np.allclose(R.sum(axis=1), 1.0, atol=1e-14)


@pytest.mark.parametrize("geom", ["cube", "annulus"])
def test_galerkin_and_collocation_agree_under_refinement(geom):
    """Sec. 4.1: both discretisations approximate the same operator; their
    leading eigenvalues approach each other under refinement."""
    d = []
    for n in (2, 4, 6):
        prob = Problem(geom, 2, (n, n, n), "gauss", 1.0, 0.8)
        lg, _, _ = galerkin.solve(prob, 4)
        lc, _, info = collocation.solve(prob, 4)
        assert not info["complex"]
        d.append(_rel(lc, lg))
    assert d[1] < d[0] / 2 and d[2] < d[1] / 2 and d[2] < 0.01


def test_collocation_eigenpairs_satisfy_generalized_problem():
    prob = Problem("annulus", 2, (3, 2, 2), "exp", 1.0, 1.0)
    lam, V, info = collocation.solve(prob, 8)
    A, Z = info["A"], info["Z"]
    res = A @ V - (Z @ V) * lam[None, :]
    assert np.linalg.norm(res) / (np.max(np.abs(lam)) * np.linalg.norm(Z @ V)) < 1e-12
    assert np.allclose(collocation.l2_norms(prob, V), 1.0, atol=1e-12)


def test_kernel_formulas():
    x = np.array([0.1, 0.2, 0.3])
    y = np.array([0.4, 0.0, 0.7])
    r2 = 0.09 + 0.04 + 0.16
    assert abs(kernels.evaluate("gauss", 2.0, 0.5, x, y) - 4 * np.exp(-r2 / 0.25)) < 1e-15
    assert abs(kernels.evaluate("exp_sep", 1.0, 2.0, x, y) - np.exp(-(0.3 + 0.2 + 0.4) / 2)) < 1e-15
    assert abs(kernels.evaluate("exp", 1.0, 2.0, x, y) - np.exp(-np.sqrt(r2) / 2)) < 1e-15
    a = np.sqrt(3 * r2) / 0.5
    assert abs(kernels.evaluate("matern32", 1.0, 0.5, x, y) - (1 + a) * np.exp(-a)) < 1e-15
    assert kernels.interp_continuity("exp", 3) == 0 and kernels.interp_continuity("gauss", 3) == 2
