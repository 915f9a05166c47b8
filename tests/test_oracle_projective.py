"""Pins of the oracle on the projective cube x = x^ / (1 + c . x^).

Its NURBS weight function 1 + c . x^ is not a product of one-parameter
functions, so the collocation trial space is a NURBS space without tensor
structure and Z = (R_j(x_i)) is not a Kronecker product (Sec. 3.2). What is
fixed independently of the oracle's NURBS evaluator:

* the projective map and its Jacobian determinant, det DF = det H / (c . x^ + 1)^4
  for H = [[I, 0], [c^T, 1]] (det H = 1);
* the hexahedron's volume from its corners (six tetrahedra), and in one
  direction the integral of (1 + a t)^-4 in closed form;
* the trial weights: B-splines reproduce affine functions with the Greville
  abscissae as coefficients (Marsden's identity), so w_j = 1 + c . xi_j;
* the constant kernel's single nonzero eigenvalue, sigma^2 times the rule's
  volume (Sec. 3.2 with a partition of unity);
* c = 0 is the unit cube.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import collocation, galerkin, splines
from oracle.problem import Problem

C = (0.5, 0.25, -0.2)


def _prob(p=2, elems=(3, 2, 2), kernel="gauss", c=C, L=0.6, sigma=1.0):
    return Problem("projective_cube", p, elems, kernel, sigma, L, geo=c)


def test_map_and_jacobian_are_the_projective_ones():
    g = _prob().geom
    X = np.random.default_rng(1).random((200, 3))
    D = 1.0 + X @ np.array(C)
    assert np.max(np.abs(g.F(X) - X / D[:, None])) < 1e-15
    assert np.max(np.abs(g.detDF(X) * D ** 4 - 1.0)) < 1e-14
    # det DF is positive: the parametrisation keeps orientation
    assert np.all(np.linalg.det(g.DF(X)) > 0)


def test_faces_stay_planar():
    P = _prob().geom.corners()
    faces = [P[0], P[1], P[:, 0], P[:, 1], P[:, :, 0], P[:, :, 1]]
    for f in faces:
        a, b, c, d = f[0, 0], f[1, 0], f[0, 1], f[1, 1]
        vol = np.linalg.det(np.array([b - a, c - a, d - a]))
        assert abs(vol) < 1e-15


def test_volume_from_corners_matches_quadrature_of_det():
    prob = _prob(p=4, elems=(4, 4, 4))
    Xq, Wq = prob.quadrature()
    quad = float(np.sum(Wq * (1.0 + Xq @ np.array(C)) ** -4))  # closed-form det DF
    assert abs(quad - prob.geom.volume()) < 1e-11 * quad


def test_volume_in_one_direction_closed_form():
    a = 0.7
    g = _prob(c=(a, 0.0, 0.0)).geom
    assert abs(g.volume() - (1.0 - (1.0 + a) ** -3) / (3.0 * a)) < 1e-15


@pytest.mark.parametrize("p,elems", [(1, (2, 3, 2)), (2, (3, 2, 2)), (3, (2, 2, 3))])
def test_trial_weights_are_the_affine_function_at_greville_points(p, elems):
    prob = _prob(p=p, elems=elems)
    w = collocation.nurbs_weights(prob)
    Xc = collocation.collocation_points(prob)
    assert np.max(np.abs(w - (1.0 + Xc @ np.array(C)))) < 1e-13


def test_trial_weights_are_not_a_tensor_product():
    prob = _prob()
    n = [splines.n_basis(k, prob.p) for k in prob.trial_knots()]
    w = collocation.nurbs_weights(prob).reshape(n[2], n[1], n[0])  # direction 1 fastest
    s = np.linalg.svd(w.reshape(n[2] * n[1], n[0]), compute_uv=False)
    assert s[1] > 1e-2 * s[0]  # rank 2: the rational basis has no tensor-product form


def test_rational_basis_is_a_partition_of_unity():
    prob = _prob()
    w = collocation.nurbs_weights(prob)
    X = np.random.default_rng(2).random((100, 3))
    R = collocation.rational_basis(prob, X, w)
    assert np.max(np.abs(R.sum(axis=1) - 1.0)) < 1e-14
    assert np.min(R) >= -1e-15


def test_constant_kernel_collocation_single_eigenvalue():
    sigma = 1.3
    prob = _prob(kernel="const", sigma=sigma)
    A, Z = collocation.matrices(prob)
    lam = np.sort(sla.eigvals(A, Z).real)[::-1]
    Xq, Wq = prob.quadrature()
    rule_vol = float(np.sum(Wq * (1.0 + Xq @ np.array(C)) ** -4))
    assert abs(lam[0] - sigma ** 2 * rule_vol) < 1e-13 * lam[0]
    assert abs(lam[0] - sigma ** 2 * prob.geom.volume()) < 1e-5 * lam[0]
    assert np.max(np.abs(lam[1:])) < 1e-12 * lam[0]


def test_constant_kernel_galerkin_converges_to_volume():
    sigma = 1.0
    errs = []
    for n in (2, 4):
        prob = _prob(kernel="const", sigma=sigma, elems=(n, n, n))
        A, Z = galerkin.matrices(prob)
        lam = sla.eigh(A, Z, eigvals_only=True)[::-1]
        assert np.max(np.abs(lam[1:])) < 1e-12 * lam[0]
        errs.append(abs(lam[0] - prob.geom.volume()) / prob.geom.volume())
    # IBQ interpolates sqrt(det DF), a rational function here, with degree-2
    # splines: O(h^3) (factor 8 per halving asymptotically, 6 measured at
    # these coarse meshes)
    assert errs[1] < errs[0] / 4 and errs[1] < 1e-4


@pytest.mark.parametrize("method", ["galerkin", "collocation"])
def test_zero_c_is_the_cube(method):
    mod = galerkin if method == "galerkin" else collocation
    a = mod.solve(_prob(c=(0.0, 0.0, 0.0)), M=8)[0]
    b = mod.solve(Problem("cube", 2, (3, 2, 2), "gauss", 1.0, 0.6), M=8)[0]
    assert np.max(np.abs(np.asarray(a) - np.asarray(b))) < 1e-13 * abs(b[0])


def test_galerkin_and_collocation_agree_within_discretisation():
    prob = _prob(elems=(4, 4, 4))
    lg = galerkin.solve(prob, M=4)[0]
    lc = collocation.solve(prob, M=4)[0]
    assert np.max(np.abs(np.asarray(lg) - np.asarray(lc)) / np.asarray(lg)) < 5e-3
