"""Entry-by-entry comparison of a GPU block with the oracle's (test helper).

Every entry of Y = op(X) is checked on its own against the oracle's value:
    |Y_ij - ref_ij| <= tol * s_ij,   s = |op| |X|,
with |op| a dense matrix of absolute values built from the oracle's factors
of the operator in the order the method applies them (for the IBQ-Galerkin
A = Q^T (J Gamma J) Q with Q = B~^-T M: |Q|^T (J Gamma J) |Q|; the kernel
matrix and J are non-negative). That is the size of the rounding error of
each entry, so a wrong entry anywhere (a ragged tile tail, a last target
tile, a dropped split) fails even when it is small against the norm of the
whole block. A failure names the worst entry.
"""
import numpy as np
import scipy.linalg as sla


def assert_entrywise(Y, ref, scale, tol, label=""):
    """Y, ref, scale: arrays of one shape (k, n): vector c, entry i."""
    Y = np.asarray(Y)
    ref = np.asarray(ref)
    assert Y.shape == ref.shape == scale.shape, (Y.shape, ref.shape, scale.shape)
    if not np.all(np.isfinite(Y)):
        c, i = np.argwhere(~np.isfinite(Y))[0]
        raise AssertionError(f"{label}: non-finite entry ({c}, {i}) = {Y[c, i]}")
    tiny = np.finfo(np.float64).tiny
    r = np.abs(Y - ref) / np.maximum(scale, tiny)
    c, i = np.unravel_index(int(np.argmax(r)), r.shape)
    if r[c, i] > tol:
        raise AssertionError(f"{label}: worst entry (vector {c}, row {i}) Y={Y[c, i]!r} ref={ref[c, i]!r} "
                             f"|err|/scale={r[c, i]:.3e} > {tol:.1e} (scale {scale[c, i]:.3e}); "
                             f"{int(np.sum(r > tol))} entries over")
    return float(r[c, i])


def bound(absop, X):
    """s = |op| |X| for a block X of shape (k, n)."""
    return (absop @ np.abs(X).T).T


def galerkin_abs(parts, Z):
    """|op| for the IBQ-Galerkin A, A' = L^-1 A L^-T and Z^-1 from the
    oracle's dense parts (Sec. 3.1 factorisation)."""
    Q = sla.solve(parts["Bt"].T, parts["M"])                # B~^-T M
    K = parts["J"][:, None] * parts["Gamma"] * parts["J"][None, :]
    absA = np.abs(Q).T @ np.abs(K) @ np.abs(Q)
    return _with_standard_form(absA, Z)


def dense_abs(A, Z):
    """|op| when the operator's factors have no sign changes (collocation:
    Gamma (J W R) with R >= 0; standard Galerkin: N^T W Gamma W N)."""
    return _with_standard_form(np.abs(A), Z)


def collocation_abs(A, Z):
    absA = np.abs(A)
    absZi = np.abs(np.linalg.inv(Z))
    return dict(A=absA, Zinv=absZi, Aprime=absZi @ absA)


def _with_standard_form(absA, Z):
    L = np.linalg.cholesky(Z)
    absLi = np.abs(sla.solve_triangular(L, np.eye(L.shape[0]), lower=True))
    return dict(A=absA, Zinv=np.abs(np.linalg.inv(Z)), Aprime=absLi @ absA @ absLi.T)
