"""IBQ-Galerkin matrices and dense eigensolve (oracle; test infrastructure).

Sec. 3.1. The trial functions are N_i(x) = B_i(x^) / sqrt(det DF(x^))
(Eq. trialspace), so the mass matrix of Eq. (galerkin system matrices, Z part)
is Z_ij = integral_D N_i N_j dx. The covariance matrix A is computed through
interpolation-based quadrature: the paper gives the factorisation

    A = M^T  B~^-1  J  Gamma  J  B~^-T  M

with Gamma_ab = Gamma(F(x~_a), F(x~_b)) over the Greville points x~ of the
interpolation space, J = diag(sqrt(det DF(x~_a))), B~_ak = B~_k(x~_a) the
collocation matrix of the interpolation basis at its own Greville points and
M_ki = integral B~_k(x^) B_i(x^) dx^ the mixed mass matrix (Ñ x N).

Everything is assembled as full dense matrices, point by point, with no
Kronecker or sum-factorisation shortcut: the 3D basis functions are evaluated
at 3D points, integrals use the tensor Gauss rule with p+1 points per
direction per element (exact for the degree-2p products), and the linear
solves with B~ are dense library solves. The generalized symmetric eigenproblem
A v = lambda Z v is solved by scipy.linalg.eigh.
"""
import numpy as np
import scipy.linalg as sla

from . import splines
from .problem import Problem


def matrices(prob: Problem, with_parts=False):
    p = prob.p
    U = prob.trial_knots()
    Ut = prob.interp_knots()

    # Greville points of the interpolation space (tensor grid, direction 1 fastest)
    Xg = splines.tensor_grid([splines.greville(k, p) for k in Ut])
    # at a C^-1 breakpoint (the half cylinder's join) two Greville points
    # coincide; the left one belongs to the left patch's last function
    Lg = splines.tensor_grid([splines.greville_left(k, p).astype(float) for k in Ut]) > 0.5
    Bt = splines.tensor_basis(Ut, p, Xg, Lg)              # B~[a, k] = B~_k(x~_a)

    # Gauss rule on the (shared) mesh
    Xq, Wq = prob.quadrature()
    Bq = splines.tensor_basis(U, p, Xq)                   # B_i at quadrature points
    Btq = splines.tensor_basis(Ut, p, Xq)                 # B~_k at quadrature points
    detq = prob.geom.detDF(Xq)

    M = Btq.T @ (Wq[:, None] * Bq)                        # M[k, i] = int B~_k B_i dx^

    # Z_ij = int_D N_i N_j dx = sum_q w_q detDF_q N_i(x_q) N_j(x_q)
    Nq = Bq / np.sqrt(detq)[:, None]
    Z = Nq.T @ ((Wq * detq)[:, None] * Nq)

    Jg = np.sqrt(prob.geom.detDF(Xg))                     # J = sqrt(det DF) at x~
    Pg = prob.geom.F(Xg)
    G = prob.gamma(Pg, Pg)                                # Gamma(x_a, x_b)

    K = Jg[:, None] * G * Jg[None, :]                     # J Gamma J
    C = sla.solve(Bt, K)                                  # B~^-1 J Gamma J
    C = sla.solve(Bt, C.T).T                              # ... B~^-T
    A = M.T @ C @ M
    A = 0.5 * (A + A.T)                                   # exact symmetry of the congruence
    if with_parts:
        return A, Z, dict(M=M, Bt=Bt, J=Jg, Gamma=G, Xg=Xg, Pg=Pg)
    return A, Z


def dims(prob: Problem):
    p = prob.p
    N = int(np.prod([splines.n_basis(k, p) for k in prob.trial_knots()]))
    Nt = int(np.prod([splines.n_basis(k, p) for k in prob.interp_knots()]))
    return N, Nt


def apply_A(prob: Problem, X):
    """Y = A X with the dense IBQ-Galerkin A (coefficient basis)."""
    A, _ = matrices(prob)
    return A @ X


def apply_Zinv(prob: Problem, X):
    _, Z = matrices(prob)
    return sla.solve(Z, X, assume_a="pos")


def standard_form(prob: Problem):
    """A' = L^-1 A L^-T with Z = L L^T (Sec. 3.1, Cholesky standard form)."""
    A, Z = matrices(prob)
    L = np.linalg.cholesky(Z)
    T = sla.solve_triangular(L, A, lower=True)
    Ap = sla.solve_triangular(L, T.T, lower=True).T
    return 0.5 * (Ap + Ap.T), L


def solve(prob: Problem, M=None):
    """Largest M eigenpairs of A v = lambda Z v, eigenvalues descending.

    Eigenvectors are Z-orthonormal (v^T Z v = 1, i.e. unit L2 norm of the
    eigenfunction) with the largest-magnitude component made positive.
    """
    A, Z = matrices(prob)
    lam, V = sla.eigh(A, Z)
    lam = lam[::-1]
    V = V[:, ::-1]
    if M is not None:
        lam, V = lam[:M], V[:, :M]
    V = _fix_signs(V)
    return lam, V, dict(A=A, Z=Z)


def _fix_signs(V):
    V = V.copy()
    for j in range(V.shape[1]):
        i = np.argmax(np.abs(V[:, j]))
        if V[i, j] < 0:
            V[:, j] = -V[:, j]
    return V
