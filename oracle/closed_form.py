"""Closed-form and independent reference spectra (oracle; test infrastructure).

* ``exp1d_eigenvalues``: the textbook solution of the Fredholm problem of
  Sec. 2 (Eq. fredholm) for the 1D exponential kernel exp(-|x-y|/L) on an
  interval of length 2a (Ghanem and Spanos, the paper's reference on
  stochastic finite elements). With c = 1/L the even modes solve
  c - omega tan(omega a) = 0, the odd modes omega + c tan(omega a) = 0, and
  lambda = 2c / (omega^2 + c^2).
* ``nystrom_1d``: Gauss–Legendre Nystrom discretisation of a 1D kernel on
  [0, 1], W^1/2 K W^1/2, whose spectrum converges exponentially fast for
  smooth kernels; used as the converged continuous reference.
* ``legendre_orthonormal``: tensor-product Legendre polynomials orthonormal
  on the unit cube, for degenerate kernels sum_m mu_m P_m(x) P_m(x') whose
  nonzero eigenvalues are exactly the mu_m.
"""
import itertools

import numpy as np
from scipy.optimize import brentq


def exp1d_eigenvalues(L, n, length=1.0):
    """Largest n eigenvalues of exp(-|x-y|/L) on an interval of given length."""
    a = 0.5 * length
    c = 1.0 / L
    lams = []
    k = 0
    eps = 1e-14
    while len(lams) < 2 * n + 4:
        # even: c - w tan(w a) = 0, w a in (k pi, k pi + pi/2)
        lo, hi = (k * np.pi + eps) / a, (k * np.pi + 0.5 * np.pi - eps) / a
        w = brentq(lambda w: c * np.cos(w * a) - w * np.sin(w * a), lo, hi, xtol=1e-15, rtol=1e-15)
        lams.append(2 * c / (w * w + c * c))
        # odd: w + c tan(w a) = 0, w a in (k pi + pi/2, (k+1) pi)
        lo, hi = (k * np.pi + 0.5 * np.pi + eps) / a, ((k + 1) * np.pi - eps) / a
        w = brentq(lambda w: w * np.cos(w * a) + c * np.sin(w * a), lo, hi, xtol=1e-15, rtol=1e-15)
        lams.append(2 * c / (w * w + c * c))
        k += 1
    return np.sort(np.array(lams))[::-1][:n]


def product_spectrum(lams_1d, n):
    """Largest n products lambda_a lambda_b lambda_c of 1D spectra (one per axis)."""
    prods = np.array([np.prod(t) for t in itertools.product(*lams_1d)])
    return np.sort(prods)[::-1][:n]


def nystrom_1d(kfun, n=400):
    x, w = np.polynomial.legendre.leggauss(n)
    x = 0.5 * (x + 1.0)
    w = 0.5 * w
    K = kfun(x[:, None], x[None, :])
    sw = np.sqrt(w)
    S = sw[:, None] * K * sw[None, :]
    return np.sort(np.linalg.eigvalsh(0.5 * (S + S.T)))[::-1]


def legendre_1d(deg, x):
    """Legendre polynomial of degree deg, orthonormal on [0, 1]."""
    c = np.zeros(deg + 1)
    c[deg] = 1.0
    return np.sqrt(2 * deg + 1) * np.polynomial.legendre.legval(2 * np.asarray(x) - 1, c)


def legendre_orthonormal(degs, X):
    """prod_d P_{degs[d]}(X[..., d]) on the unit cube (orthonormal in L2)."""
    out = 1.0
    for j, k in enumerate(degs):
        out = out * legendre_1d(k, X[..., j])
    return out


def degenerate_kernel(terms):
    """Kernel sum_m mu_m P_m(x) P_m(y) from a list of (mu, degs)."""
    def k(x, y):
        out = 0.0
        for mu, degs in terms:
            out = out + mu * legendre_orthonormal(degs, x) * legendre_orthonormal(degs, y)
        return out
    return k
