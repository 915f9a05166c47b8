"""Standard Gauss–Legendre Galerkin matrices (oracle; test infrastructure).

Sec. 1 (footnote) and Sec. 3.1 describe the standard Galerkin method that the
matrix-free method replaces: A_ij = integral integral N_i(x) Gamma(x, x')
N_j(x') dx dx' evaluated with a Gauss–Legendre rule on every pair of elements.
Here it is a brute-force double quadrature with ``nq`` points per direction
per element, for tiny meshes only. With a kernel that lies in the
interpolation space it reproduces the IBQ matrix exactly; otherwise the IBQ
matrix converges to it under refinement.
"""
import numpy as np

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
