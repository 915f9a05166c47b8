"""Covariance functions Gamma(x, x') for the oracle (test infrastructure).

The paper never writes its kernels out (they are defined in its reference
[mika 2020]); the formulas used here are the ones the workloads are specified
with:

* ``gauss``     sigma^2 exp(-|x-x'|^2 / L^2)
* ``exp_sep``   sigma^2 exp(-sum_d |x_d-x'_d| / L)       (separable exponential)
* ``exp``       sigma^2 exp(-|x-x'| / L)                 (Euclidean exponential)
* ``matern32``  sigma^2 (1 + sqrt(3) r / L) exp(-sqrt(3) r / L)
* ``const``     sigma^2                                   (rank-one test kernel)

All evaluate in float64 on broadcastable arrays of points with the coordinate
axis last.
"""
import numpy as np

KERNELS = ("gauss", "exp_sep", "exp", "matern32", "const")


def evaluate(name, sigma, L, x, y):
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    diff = x - y
    s2 = sigma * sigma
    if name == "gauss":
        r2 = np.sum(diff * diff, axis=-1)
        return s2 * np.exp(-r2 / (L * L))
    if name == "exp_sep":
        return s2 * np.exp(-np.sum(np.abs(diff), axis=-1) / L)
    if name == "exp":
        r = np.sqrt(np.sum(diff * diff, axis=-1))
        return s2 * np.exp(-r / L)
    if name == "matern32":
        a = np.sqrt(3.0) * np.sqrt(np.sum(diff * diff, axis=-1)) / L
        return s2 * (1.0 + a) * np.exp(-a)
    if name == "const":
        return s2 * np.ones(np.broadcast(x[..., 0], y[..., 0]).shape)
    raise ValueError(f"unknown kernel {name!r}")


def matrix(name, sigma, L, P, Q, chunk=2048):
    """Dense Gamma(P_i, Q_j) for point sets P (n x d) and Q (m x d)."""
    P = np.atleast_2d(P)
    Q = np.atleast_2d(Q)
    out = np.empty((P.shape[0], Q.shape[0]))
    for s in range(0, P.shape[0], chunk):
        out[s:s + chunk] = evaluate(name, sigma, L, P[s:s + chunk, None, :], Q[None, :, :])
    return out


def interp_continuity(name, p):
    """Continuity of the IBQ interpolation space (Sec. 4.1 and Sec. 4.2).

    Rough (C^0) exponential kernels use C^0 interpolation splines; smooth
    kernels use maximal C^{p-1} smoothness, as the trial space.
    """
    return 0 if name in ("exp", "exp_sep") else p - 1
