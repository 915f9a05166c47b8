"""Problem description shared by the oracle's Galerkin and collocation modules.

A problem is a geometry (unit cube in d = 1, 2 or 3 dimensions, or the quarter
annular cylinder), a polynomial degree p, the number of elements per
parametric direction, a covariance kernel with sigma and correlation length L.
The kernel may also be given as a Python callable k(x, y) on broadcastable
point arrays, which the pins use for polynomial (degenerate) kernels.
"""
from dataclasses import dataclass, field

import numpy as np

from . import geometry, kernels, splines


@dataclass
class Problem:
    geometry: str
    p: int
    elems: tuple
    kernel: object = "gauss"
    sigma: float = 1.0
    L: float = 1.0
    geo: tuple = (1.0, 2.0, 1.0)
    interp_cont: object = None   # None: rule of Sec. 4; int: explicit continuity

    def __post_init__(self):
        self.elems = tuple(int(n) for n in self.elems)
        self.d = len(self.elems)
        self.geom = geometry.make_geometry(self.geometry, self.d, self.geo)

    # -- kernel -----------------------------------------------------------
    def gamma(self, P, Q):
        if callable(self.kernel):
            P = np.atleast_2d(P)
            Q = np.atleast_2d(Q)
            return self.kernel(P[:, None, :], Q[None, :, :])
        return kernels.matrix(self.kernel, self.sigma, self.L, P, Q)

    def interpolation_continuity(self):
        if self.interp_cont is not None:
            return int(self.interp_cont)
        if callable(self.kernel):
            return self.p - 1
        return kernels.interp_continuity(self.kernel, self.p)

    # -- spaces -----------------------------------------------------------
    def trial_knots(self):
        return [splines.open_uniform_knots(n, self.p, self.p - 1) for n in self.elems]

    def interp_knots(self):
        r = self.interpolation_continuity()
        return [splines.open_uniform_knots(n, self.p, r) for n in self.elems]

    def quadrature(self, nq=None):
        """Tensor Gauss rule with nq (default p+1) points per direction per element."""
        nq = self.p + 1 if nq is None else nq
        rules = [splines.element_gauss(k, nq) for k in self.trial_knots()]
        X = splines.tensor_grid([r[0] for r in rules])
        W = splines.tensor_weights([r[1] for r in rules])
        return X, W
