"""Standard Gauss–Legendre Galerkin matrices (oracle; test infrastructure).

Sec. 1 (footnote) and Sec. 3.1 describe the standard Galerkin method that the
matrix-free method replaces: A_ij = integral integral N_i(x) Gamma(x, x')
N_j(x') dx dx' evaluated with a Gauss–Legendre rule on every pair of elements.
Here it is a brute-force double quadrature with ``nq`` points per direction
per element, for tiny meshes only. With a kernel that lies in the
interpolation space it reproduces the IBQ matrix exactly; otherwise the IBQ
matrix converges to it under refinement.

``solve`` / ``standard_form`` with ``nq = p + 1`` are the reference for the
library's KL_GALERKIN_STD method (the same rule: p + 1 Gauss points per
direction per element on both sides).
"""
import numpy as np
import scipy.linalg as sla

from . import splines
from .problem import Problem


def matrices(prob: Problem, nq):
    U = prob.trial_knots()
    Xq, Wq = prob.quadrature(nq)
    Bq = splines.tensor_basis(U, prob.p, Xq)
    detq = prob.geom.detDF(Xq)
    Nq = Bq / np.sqrt(detq)[:, None]                      # N_i = B_i / sqrt(det DF)
    Pq = prob.geom.F(Xq)
    G = prob.gamma(Pq, Pq)
    WN = (Wq * detq)[:, None] * Nq
    A = WN.T @ G @ WN
    Z = Nq.T @ WN
    return 0.5 * (A + A.T), Z


def dims(prob: Problem, nq=None):
    """(N trial dofs, number of Gauss points)."""
    U = prob.trial_knots()
    N = int(np.prod([splines.n_basis(k, prob.p) for k in U]))
    Xq, _ = prob.quadrature(nq if nq is not None else prob.p + 1)
    return N, Xq.shape[0]


def apply_A(prob: Problem, X, nq=None):
    A, _ = matrices(prob, nq if nq is not None else prob.p + 1)
    return A @ X


def standard_form(prob: Problem, nq=None):
    """A' = L^-1 A L^-T with Z = L L^T (Cholesky standard form, as Sec. 3.1)."""
    A, Z = matrices(prob, nq if nq is not None else prob.p + 1)
    L = np.linalg.cholesky(Z)
    T = sla.solve_triangular(L, A, lower=True)
    Ap = sla.solve_triangular(L, T.T, lower=True).T
    return 0.5 * (Ap + Ap.T), L


def solve(prob: Problem, M=None, nq=None):
    """Largest M eigenpairs of A v = lambda Z v (descending, Z-orthonormal,
    largest-magnitude component positive)."""
    A, Z = matrices(prob, nq if nq is not None else prob.p + 1)
    lam, V = sla.eigh(A, Z)
    lam, V = lam[::-1], V[:, ::-1]
    if M is not None:
        lam, V = lam[:M], V[:, :M]
    V = V.copy()
    for j in range(V.shape[1]):
        i = np.argmax(np.abs(V[:, j]))
        if V[i, j] < 0:
            V[:, j] = -V[:, j]
    return lam, V, dict(A=A, Z=Z)
