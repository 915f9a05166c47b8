"""Problem description shared by the oracle's Galerkin and collocation modules.

A problem is a geometry (unit cube in d = 1, 2 or 3 dimensions, the quarter
or half annular cylinder, or the projective image of the cube), a polynomial
degree p, the number of elements per
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
    geo: tuple = None           # geometry parameters; None: the geometry's default
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
    def _joined(self, j):
        # the half annulus's angle direction has a C^0 geometry join at 1/2
        return self.geometry == "half_annulus" and j == 0

    def trial_knots(self):
        """C^{p-1} splines; C^0 at a geometry join (the trial space follows the
        geometry's continuity)."""
        return [splines.joined_knots(n, self.p, self.p - 1, 0) if self._joined(j)
                else splines.open_uniform_knots(n, self.p, self.p - 1) for j, n in enumerate(self.elems)]

    def interp_knots(self):
        """Continuity of the rule of Sec. 4; C^-1 at a geometry join (Sec. 4.1)."""
        r = self.interpolation_continuity()
        return [splines.joined_knots(n, self.p, r, -1) if self._joined(j)
                else splines.open_uniform_knots(n, self.p, r) for j, n in enumerate(self.elems)]

    def quadrature(self, nq=None):
        """Tensor Gauss rule with nq (default p+1) points per direction per element."""
        nq = self.p + 1 if nq is None else nq
        rules = [splines.element_gauss(k, nq) for k in self.trial_knots()]
        X = splines.tensor_grid([r[0] for r in rules])
        W = splines.tensor_weights([r[1] for r in rules])
        return X, W
