"""Isogeometric collocation matrices and dense eigensolve (oracle).

Test infrastructure only. Sec. 3.2: the trial space is spanned by NURBS
R_j (isoparametric), the residual of the Fredholm equation is collocated at
the Greville abscissae x_i, and the system matrices are

    A_ij = integral_D Gamma(x_i, x') R_j(x') dx',     Z_ij = R_j(x_i)

(Eq. colloc system matrices). The integral is evaluated with the tensor
Gauss–Legendre rule with (p+1) points per direction per element used in
Sec. 4.1, i.e. A_ij = sum_q w_q det DF(x^_q) Gamma(x_i, F(x^_q)) R_j(x^_q),
which is the operator of Algorithm 1 (before its final Z^-1) written as a
dense matrix. The generalized
eigenproblem is not symmetric; it is solved with the QZ algorithm
(scipy.linalg.eig).

NURBS weights. On the cube all weights are 1 (plain B-splines). On the
quarter annulus the geometry's NURBS denominator W(xh_1) is a quadratic
polynomial of the angle parameter, so the refined, degree-raised trial space
carries weights w_j = coefficients of W in the degree-p spline basis of
direction 1; they are obtained here by L2 projection of W onto that space
(exact, because W lies in it). The 3D weight of multi-index (j1, j2, j3) is
w_{j1}, and R_j(x^) = w_j B_j(x^) / sum_l w_l B_l(x^).

On the projective cube the denominator W(x^) = 1 + c . x^ is trilinear and
not a product of one-parameter functions; its coefficients in the 3D trial
space are found by interpolation at the trial Greville points with the dense
3D collocation matrix of the B-splines (exact, because W lies in the space).
The 3D weights are then not a tensor product and neither is Z, the case
Sec. 3.2 factors with a full pivoted LU.
"""
import numpy as np
import scipy.linalg as sla

from . import splines
from .problem import Problem


def nurbs_weights(prob: Problem):
    """Per-multi-index NURBS weights of the trial space (direction 1 fastest)."""
    U = prob.trial_knots()
    p = prob.p
    n = [splines.n_basis(k, p) for k in U]
    if prob.geometry == "projective_cube":
        Xc = collocation_points(prob)
        Bc = splines.tensor_basis(U, p, Xc)
        return np.linalg.solve(Bc, prob.geom.weight_function_3d(Xc))
    if prob.geometry not in ("annulus", "half_annulus"):
        return np.ones(int(np.prod(n)))
    # L2 projection of W onto the 1D space of direction 1 (exact: W is
    # quadratic, piecewise with a C^0 join at 1/2 for the half annulus, where
    # the trial space is C^0 too)
    xq, wq = splines.element_gauss(U[0], p + 2)
    B = splines.bspline_basis(U[0], p, xq)
    Wv = prob.geom.weight_function(xq)
    mass = B.T @ (wq[:, None] * B)
    rhs = B.T @ (wq * Wv)
    w1 = sla.solve(mass, rhs, assume_a="pos")
    idx = np.arange(int(np.prod(n)))
    return w1[idx % n[0]]


def rational_basis(prob: Problem, X, w):
    """R_j(x) = w_j B_j(x) / sum_l w_l B_l(x) at the points X."""
    B = splines.tensor_basis(prob.trial_knots(), prob.p, X)
    num = B * w[None, :]
    return num / num.sum(axis=1, keepdims=True)


def collocation_points(prob: Problem):
    return splines.tensor_grid([splines.greville(k, prob.p) for k in prob.trial_knots()])


def matrices(prob: Problem, with_parts=False, chunk=1024):
    w = nurbs_weights(prob)
    Xc = collocation_points(prob)
    Z = rational_basis(prob, Xc, w)                       # Z_ij = R_j(x_i)
    Xq, Wq = prob.quadrature()
    Rq = rational_basis(prob, Xq, w)                      # R_j(x^_q)
    detq = prob.geom.detDF(Xq)
    Pc = prob.geom.F(Xc)
    Pq = prob.geom.F(Xq)
    WR = (Wq * detq)[:, None] * Rq                        # w_q det DF_q R_j(x^_q)
    A = np.empty((Pc.shape[0], Rq.shape[1]))
    for s in range(0, Pc.shape[0], chunk):
        A[s:s + chunk] = prob.gamma(Pc[s:s + chunk], Pq) @ WR
    if with_parts:
        return A, Z, dict(Xc=Xc, Xq=Xq, Wq=Wq, detq=detq, Rq=Rq, w=w, Pc=Pc, Pq=Pq)
    return A, Z


def dims(prob: Problem):
    N = int(np.prod([splines.n_basis(k, prob.p) for k in prob.trial_knots()]))
    NeNq = int(np.prod(prob.elems)) * (prob.p + 1) ** prob.d
    return N, NeNq


def apply_A(prob: Problem, X):
    A, _ = matrices(prob)
    return A @ X


def apply_Zinv(prob: Problem, X):
    _, Z = matrices(prob)
    return sla.solve(Z, X)


def l2_norms(prob: Problem, V, parts=None):
    """||phi_h||_L2 of the fields sum_j V_j R_j, by the same Gauss rule."""
    if parts is None:
        _, _, parts = matrices(prob, with_parts=True)
    vals = parts["Rq"] @ V
    return np.sqrt(np.sum((parts["Wq"] * parts["detq"])[:, None] * vals ** 2, axis=0))


def solve(prob: Problem, M=None, imag_tol=1e-8):
    """Largest-real-part M eigenpairs of A v = lambda Z v (QZ).

    Returns real parts (descending) and real eigenvectors normalised to unit
    L2 norm of the field with the largest-magnitude component positive; the
    info dict reports the largest relative imaginary part seen among them.
    """
    A, Z, parts = matrices(prob, with_parts=True)
    lam, V = sla.eig(A, Z)
    order = np.argsort(-lam.real)
    lam, V = lam[order], V[:, order]
    if M is not None:
        lam, V = lam[:M], V[:, :M]
    scale = np.max(np.abs(lam.real)) if lam.size else 1.0
    max_imag = float(np.max(np.abs(lam.imag)) / scale) if lam.size else 0.0
    Vr = np.real(V)
    nrm = l2_norms(prob, Vr, parts)
    Vr = Vr / nrm[None, :]
    for j in range(Vr.shape[1]):
        i = np.argmax(np.abs(Vr[:, j]))
        if Vr[i, j] < 0:
            Vr[:, j] = -Vr[:, j]
    return lam.real, Vr, dict(A=A, Z=Z, max_imag=max_imag, complex=max_imag > imag_tol)
