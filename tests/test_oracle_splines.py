"""Pins of the oracle's spline and geometry layer against textbook facts and
library routines (CPU only)."""
import os

import numpy as np
import pytest
from scipy.interpolate import BSpline

from oracle import geometry, splines

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("p,cont,n", [(1, 0, 3), (2, 1, 4), (2, 0, 5), (3, 2, 3), (3, 0, 2), (4, 1, 3)])
def test_partition_of_unity_and_nonnegativity(p, cont, n):
    t = splines.open_uniform_knots(n, p, cont)
    x = np.concatenate([np.linspace(0, 1, 101), np.random.default_rng(0).random(50)])
    B = splines.bspline_basis(t, p, x)
    assert np.allclose(B.sum(axis=1), 1.0, atol=1e-14)
    assert B.min() >= -1e-15
    assert B.shape[1] == splines.n_basis(t, p) == (p + 1) + (n - 1) * (p - cont)


@pytest.mark.parametrize("p,cont,n", [(2, 1, 4), (3, 0, 3), (4, 2, 5), (2, 0, 6)])
def test_cox_de_boor_matches_scipy(p, cont, n):
    t = splines.open_uniform_knots(n, p, cont)
    x = np.random.default_rng(1).random(200) * 0.999
    B = splines.bspline_basis(t, p, x)
    ref = BSpline.design_matrix(x, t, p).toarray()
    assert np.max(np.abs(B - ref)) < 1e-14
    # derivatives against scipy's BSpline.derivative of unit coefficient vectors
    D = splines.bspline_basis_deriv(t, p, x)
    nb = splines.n_basis(t, p)
    for i in range(nb):
        c = np.zeros(nb)
        c[i] = 1.0
        d = BSpline(t, c, p).derivative()(x)
        assert np.max(np.abs(D[:, i] - d)) < 1e-11


@pytest.mark.parametrize("p,cont,n", [(2, 1, 4), (3, 0, 3), (4, 3, 2), (2, 0, 5)])
def test_greville_linear_precision(p, cont, n):
    # sum_i xi*_i B_i(x) = x for every knot vector (Greville abscissae)
    t = splines.open_uniform_knots(n, p, cont)
    g = splines.greville(t, p)
    x = np.linspace(0, 1, 57)
    assert np.allclose(splines.bspline_basis(t, p, x) @ g, x, atol=1e-14)
    assert g[0] == 0.0 and g[-1] == 1.0
    assert np.all(np.diff(g) > 0)


def test_greville_p2_closed_form():
    n = 4
    g = splines.greville(splines.open_uniform_knots(n, 2, 1), 2)
    h = 1.0 / n
    assert np.allclose(g, [0, h / 2, 3 * h / 2, 5 * h / 2, 7 * h / 2, 1.0], atol=1e-15)


def test_p1_mass_matrix_closed_form():
    # linear hat functions: element mass matrix h/6 [[2,1],[1,2]]
    n = 5
    h = 1.0 / n
    t = splines.open_uniform_knots(n, 1, 0)
    x, w = splines.element_gauss(t, 2)
    B = splines.bspline_basis(t, 1, x)
    Z = B.T @ (w[:, None] * B)
    ref = np.zeros((n + 1, n + 1))
    for e in range(n):
        ref[e:e + 2, e:e + 2] += h / 6 * np.array([[2, 1], [1, 2]])
    assert np.max(np.abs(Z - ref)) < 1e-15


@pytest.mark.parametrize("nq", [1, 2, 3, 5])
def test_element_gauss_exactness(nq):
    t = splines.open_uniform_knots(3, 2, 1)
    x, w = splines.element_gauss(t, nq)
    for deg in range(2 * nq):
        assert abs(np.sum(w * x ** deg) - 1.0 / (deg + 1)) < 1e-14


def test_tensor_basis_ordering_direction1_fastest():
    p = 2
    knots = [splines.open_uniform_knots(n, p, p - 1) for n in (2, 3, 4)]
    nb = [splines.n_basis(k, p) for k in knots]
    X = np.random.default_rng(2).random((7, 3))
    T = splines.tensor_basis(knots, p, X)
    one = [splines.bspline_basis(knots[j], p, X[:, j]) for j in range(3)]
    for (k1, k2, k3) in [(0, 0, 0), (1, 2, 3), (3, 0, 5), (2, 4, 1)]:
        col = k1 + nb[0] * (k2 + nb[1] * k3)
        assert np.allclose(T[:, col], one[0][:, k1] * one[1][:, k2] * one[2][:, k3], atol=1e-15)
    G = splines.tensor_grid([np.arange(2), np.arange(3) * 10, np.arange(2) * 100])
    assert G[1].tolist() == [1, 0, 0] and G[2].tolist() == [0, 10, 0] and G[6].tolist() == [0, 0, 100]


def test_tensor_basis_grad_matches_finite_differences():
    p = 3
    knots = [splines.open_uniform_knots(n, p, p - 1) for n in (2, 2, 3)]
    X = 0.05 + 0.9 * np.random.default_rng(3).random((5, 3))
    G = splines.tensor_basis_grad(knots, p, X)
    eps = 1e-6
    for e in range(3):
        dX = np.zeros(3)
        dX[e] = eps
        fd = (splines.tensor_basis(knots, p, X + dX) - splines.tensor_basis(knots, p, X - dX)) / (2 * eps)
        assert np.max(np.abs(fd - G[:, :, e])) < 1e-7


# --- geometry -------------------------------------------------------------

def test_annulus_exact_circle_and_corners():
    g = geometry.QuarterAnnulus(1.0, 2.0, 1.0)
    X = np.random.default_rng(4).random((300, 3))
    P = g.F(X)
    r = np.hypot(P[:, 0], P[:, 1])
    assert np.max(np.abs(r - (1.0 + X[:, 1]))) < 1e-14       # exact circles, linear in radius
    assert np.max(np.abs(P[:, 2] - X[:, 2])) < 1e-15
    assert P[:, :2].min() >= -1e-15
    C = g.F(np.array([[0, 0, 0], [1, 0, 0], [0, 1, 1], [1, 1, 0.5], [0.5, 0, 0]], dtype=float))
    s = np.sqrt(0.5)
    assert np.allclose(C, [[1, 0, 0], [0, 1, 0], [2, 0, 1], [0, 2, 0.5], [s, s, 0]], atol=1e-15)


def test_annulus_jacobian_and_volume():
    g = geometry.QuarterAnnulus(1.0, 2.0, 1.0)
    X = 0.02 + 0.96 * np.random.default_rng(5).random((20, 3))
    J = g.DF(X)
    eps = 1e-6
    for e in range(3):
        dX = np.zeros(3)
        dX[e] = eps
        fd = (g.F(X + dX) - g.F(X - dX)) / (2 * eps)
        assert np.max(np.abs(fd - J[:, :, e])) < 1e-8
    # integral of |det DF| over the parameter cube = (pi/4)(r_out^2 - r_in^2) h
    x40, w40 = np.polynomial.legendre.leggauss(40)
    x4, w4 = np.polynomial.legendre.leggauss(4)
    Xq = splines.tensor_grid([0.5 + 0.5 * x40, 0.5 + 0.5 * x4, 0.5 + 0.5 * x4])
    Wq = splines.tensor_weights([0.5 * w40, 0.5 * w4, 0.5 * w4])
    vol = np.sum(Wq * g.detDF(Xq))
    assert abs(vol - 0.75 * np.pi) < 1e-13


# --- dof counts printed in the paper -------------------------------------

def _two_patch_knots(n_half, p, cont, join_mult):
    """Knot vector of two patches of n_half elements joined with a knot of
    multiplicity join_mult (p: C^0 join, p+1: C^-1 join)."""
    a = splines.open_uniform_knots(n_half, p, cont)
    inner_a = a[p + 1:-(p + 1)] * 0.5
    inner_b = 0.5 + a[p + 1:-(p + 1)] * 0.5
    return np.concatenate([np.zeros(p + 1), inner_a, np.full(join_mult, 0.5), inner_b, np.ones(p + 1)])


def _load(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(v) for v in line.split()])
    return rows


def test_table2_dof_counts():
    """Table 2: 1 x 8 x 32 elements (radial, axial, angular) on the half
    cylinder, the angular direction made of two 16-element patches joined C^0
    in the solution space and C^-1 in the interpolation space (the reading of
    Sec. 4.1/4.2 for the geometry's C^0 interface); both spaces C^{p-1}."""
    for p, N, Nt in _load("table2_dof_counts.txt"):
        rad = splines.n_basis(splines.open_uniform_knots(1, p, p - 1), p)
        ax = splines.n_basis(splines.open_uniform_knots(8, p, p - 1), p)
        ang = splines.n_basis(_two_patch_knots(16, p, p - 1, p), p)
        ang_t = splines.n_basis(_two_patch_knots(16, p, p - 1, p + 1), p)
        assert rad * ax * ang == N
        assert rad * ax * ang_t == Nt


def test_table1_dof_counts_cases_2_to_5():
    """Table 1 cases 2-5 (p = 2, C^0 interpolation, C^-1 at the geometry's
    C^0 interface). The meshes (radial, axial, angular) are this project's
    reading: the paper prints only h, N and Ntilde. Case 1 is inconsistent
    with the stated continuity rule and is not checked."""
    meshes = {2: (2, 15, 28), 3: (2, 18, 32), 4: (2, 21, 38), 5: (3, 23, 42)}
    p = 2
    for case, N, Nt in _load("table1_dof_counts.txt"):
        if case == 1:
            continue
        a, b, c = meshes[case]
        n = [splines.n_basis(splines.open_uniform_knots(m, p, p - 1), p) for m in (a, b)]
        ang = splines.n_basis(_two_patch_knots(c // 2, p, p - 1, p), p)
        nt = [splines.n_basis(splines.open_uniform_knots(m, p, 0), p) for m in (a, b)]
        ang_t = splines.n_basis(_two_patch_knots(c // 2, p, 0, p + 1), p)
        assert n[0] * n[1] * ang == N
        assert nt[0] * nt[1] * ang_t == Nt
