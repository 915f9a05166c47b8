"""Sampling the truncated K-L expansion (oracle; test infrastructure).

Sec. 2: the random field is expanded as alpha(x, xi) = mean(x) + sum_m
sqrt(lambda_m) xi_m phi_m(x) with independent standard normal xi_m; the
truncated expansion keeps M terms. Here the centred part is evaluated at the
tensor Gauss grid of the parametric domain (p + 1 points per element and
direction, direction 1 fastest), with phi_m = sum_j V[j, m] N_j in the
method's trial basis: N_j = B_j / sqrt(det DF) for the Galerkin method
(Sec. 3.1) and the rational basis R_j for collocation (Sec. 3.2). The 3D
basis functions are evaluated directly at the 3D points (no Kronecker or
sum-factorisation shortcut).

Only tests/, the package's smoke check and bench.py's CPU legs use this.
"""
import numpy as np

from . import collocation, splines
from .problem import Problem


def grid(prob: Problem):
    """Parametric Gauss grid X^ (Q x 3), its weights, and physical points F(X^)."""
    X, W = prob.quadrature()
    return X, W, prob.geom.F(X)


def trial_basis(prob: Problem, method, X):
    """N_j at the parametric points X (rows: points, columns: j)."""
    if method == "galerkin":
        B = splines.tensor_basis(prob.trial_knots(), prob.p, X)
        return B / np.sqrt(np.abs(prob.geom.detDF(X)))[:, None]
    return collocation.rational_basis(prob, X, collocation.nurbs_weights(prob))


def modes(prob: Problem, method, V):
    """phi_m at the grid (Q x M)."""
    X, _, _ = grid(prob)
    return trial_basis(prob, method, X) @ V


def samples(prob: Problem, method, lam, V, xi):
    """Realisations of the centred truncated expansion at the grid: Q x ns for
    xi of shape M x ns (negative eigenvalues count as zero)."""
    scale = np.sqrt(np.maximum(np.asarray(lam, dtype=float), 0.0))
    return modes(prob, method, V) @ (scale[:, None] * xi)


def variance_integral(prob: Problem, method, lam, V):
    """integral over D of the pointwise variance sum_m lambda_m phi_m(x)^2
    (Gauss rule on the grid, |det DF| dx^)."""
    X, W, _ = grid(prob)
    Phi = trial_basis(prob, method, X) @ V
    var = Phi ** 2 @ np.maximum(np.asarray(lam, dtype=float), 0.0)
    return float(np.sum(W * np.abs(prob.geom.detDF(X)) * var))
