"""Geometry maps F : D^ -> D and det DF for the oracle (test infrastructure).

Sec. 3.1 uses the geometric mapping F from the reference domain to the
physical domain, its Jacobian determinant det DF(x^) in the trial space
(Eq. trialspace) and J = sqrt(det DF) at the Greville points; Sec. 3.2 uses
det DF at the quadrature points (the weights of Algorithm 1).

Two domains are provided:

* ``Cube``: the unit cube (or unit interval/square for d < 3); F is the
  identity and det DF = 1.
* ``QuarterAnnulus``: the quarter annular cylinder with inner radius r_in,
  outer radius r_out and height h, written as the coarsest exact NURBS volume:
  quadratic in direction 1 (the angle) with control points (1,0), (1,1), (0,1)
  scaled by the radius and weights 1, sqrt(2)/2, 1; linear in direction 2
  (radius r_in -> r_out) and direction 3 (height 0 -> h). F and DF are
  evaluated from that NURBS definition (rational basis and quotient rule),
  point by point.
* ``HalfAnnulus``: the half annular cylinder (the shape of the paper's Sec. 4
  benchmark), two such quarter arcs joined C^0 at the parameter 1/2: angle
  knots 0,0,0,1/2,1/2,1,1,1, control points (1,0), (1,1), (0,1), (-1,1),
  (-1,0) and weights 1, sqrt(2)/2, 1, sqrt(2)/2, 1.
* ``ProjectiveCube``: the image of the unit cube under the projective map
  x = x^ / (1 + c . x^), a hexahedron with planar faces. As a NURBS volume it
  is trilinear with corner weights 1 + c . v and control points v / (1 + c . v)
  (v the cube's corners); its weight function 1 + c . x^ is a sum, not a
  product, of functions of one parameter each, so the NURBS basis is not a
  tensor product once two entries of c are nonzero (Sec. 3.2: the collocation
  matrix is then not a Kronecker product).

The annuli and the projective cube share one NURBS-volume evaluator: F and DF
from the definition (rational basis, quotient rule), point by point.
"""
import numpy as np

from . import splines


class Cube:
    name = "cube"

    def __init__(self, d=3):
        self.d = d

    def F(self, Xh):
        return np.array(Xh, dtype=np.float64, copy=True)

    def detDF(self, Xh):
        return np.ones(np.atleast_2d(Xh).shape[0])

    def volume(self):
        return 1.0


class NurbsVolume:
    """A single-patch NURBS volume: knots[j], degrees[j], control points
    P[i1, i2, i3, :] and weights w[i1, i2, i3]."""
    d = 3

    def _basis(self, Xh):
        Xh = np.atleast_2d(np.asarray(Xh, dtype=np.float64))
        B = [splines.bspline_basis(self.knots[j], self.degrees[j], Xh[:, j]) for j in range(3)]
        dB = [splines.bspline_basis_deriv(self.knots[j], self.degrees[j], Xh[:, j]) for j in range(3)]
        return B, dB

    def _num_den(self, B):
        # N(x) = sum w P B1 B2 B3, W(x) = sum w B1 B2 B3
        wB = np.einsum("ijk,ai,aj,ak->a", self.w, B[0], B[1], B[2])
        num = np.einsum("ijk,ijkc,ai,aj,ak->ac", self.w, self.P, B[0], B[1], B[2])
        return num, wB

    def F(self, Xh):
        B, _ = self._basis(Xh)
        num, den = self._num_den(B)
        return num / den[:, None]

    def DF(self, Xh):
        """Jacobian matrix dF_c/dxh_e by the quotient rule, shape (npts, 3, 3)."""
        B, dB = self._basis(Xh)
        num, den = self._num_den(B)
        J = np.zeros((num.shape[0], 3, 3))
        for e in range(3):
            Bs = [dB[j] if j == e else B[j] for j in range(3)]
            dnum, dden = self._num_den(Bs)
            J[:, :, e] = (dnum * den[:, None] - num * dden[:, None]) / (den ** 2)[:, None]
        return J

    def detDF(self, Xh):
        """|det DF|, the change-of-variables factor (the annuli's
        parametrisation is left-handed: det DF itself is negative there)."""
        return np.abs(np.linalg.det(self.DF(Xh)))

    def weight_function_3d(self, Xh):
        """The NURBS denominator W(x^) = sum_v w_v B_v(x^) at the points Xh."""
        B, _ = self._basis(Xh)
        return self._num_den(B)[1]


class QuarterAnnulus(NurbsVolume):
    name = "annulus"
    quarters = 1

    def __init__(self, r_in=1.0, r_out=2.0, height=1.0):
        self.r_in, self.r_out, self.h = float(r_in), float(r_out), float(height)
        s = np.sqrt(2.0) / 2.0
        if self.quarters == 1:
            angle_knots = np.array([0, 0, 0, 1, 1, 1.0])
            arc = np.array([[1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
            warc = np.array([1.0, s, 1.0])
        else:
            angle_knots = np.array([0, 0, 0, 0.5, 0.5, 1, 1, 1.0])
            arc = np.array([[1.0, 0.0], [1.0, 1.0], [0.0, 1.0], [-1.0, 1.0], [-1.0, 0.0]])
            warc = np.array([1.0, s, 1.0, s, 1.0])
        self.warc = warc
        self.knots = [angle_knots, np.array([0, 0, 1, 1.0]), np.array([0, 0, 1, 1.0])]
        self.degrees = [2, 1, 1]
        na = len(warc)
        radii = [self.r_in, self.r_out]
        zs = [0.0, self.h]
        # control points P[i1, i2, i3] and weights w[i1, i2, i3]
        self.P = np.zeros((na, 2, 2, 3))
        self.w = np.zeros((na, 2, 2))
        for i1 in range(na):
            for i2 in range(2):
                for i3 in range(2):
                    self.P[i1, i2, i3, 0] = radii[i2] * arc[i1, 0]
                    self.P[i1, i2, i3, 1] = radii[i2] * arc[i1, 1]
                    self.P[i1, i2, i3, 2] = zs[i3]
                    self.w[i1, i2, i3] = warc[i1]

    def weight_function(self, t):
        """The NURBS denominator W(xh_1), a quadratic polynomial in the angle
        parameter (piecewise, C^0 at 1/2, for the half annulus; the radial and
        axial weights are all 1)."""
        b = splines.bspline_basis(self.knots[0], 2, t)
        return b @ self.warc

    def volume(self):
        return 0.25 * self.quarters * np.pi * (self.r_out ** 2 - self.r_in ** 2) * self.h


class HalfAnnulus(QuarterAnnulus):
    name = "half_annulus"
    quarters = 2


class ProjectiveCube(NurbsVolume):
    """The unit cube mapped by x = x^ / (1 + c . x^) (1 + c . x^ > 0 on the
    cube), written as the trilinear NURBS volume with corner weights
    w_v = 1 + c . v and control points v / w_v, v in {0, 1}^3; F and DF come
    from that NURBS definition like the annuli's."""
    name = "projective_cube"

    def __init__(self, c1=0.5, c2=0.25, c3=-0.2):
        self.c = np.array([c1, c2, c3], dtype=np.float64)
        if 1.0 + np.minimum(self.c, 0.0).sum() <= 0.0:
            raise ValueError("1 + c . x^ must stay positive on the unit cube")
        self.knots = [np.array([0, 0, 1, 1.0])] * 3
        self.degrees = [1, 1, 1]
        self.P = np.zeros((2, 2, 2, 3))
        self.w = np.zeros((2, 2, 2))
        for i1 in range(2):
            for i2 in range(2):
                for i3 in range(2):
                    v = np.array([i1, i2, i3], dtype=np.float64)
                    wv = 1.0 + self.c @ v
                    self.w[i1, i2, i3] = wv
                    self.P[i1, i2, i3] = v / wv

    def corners(self):
        """The hexahedron's eight corners F(v), indexed like P."""
        return self.P.copy()

    def volume(self):
        """Volume of the image: the cube's six Kuhn simplices (0 -> e_a ->
        e_a + e_b -> 1 for each order a, b, c of the axes) map to the six
        tetrahedra of the hexahedron (a projective map keeps segments straight
        and faces planar where 1 + c . x^ > 0), each of volume |det| / 6."""
        import itertools
        Pc = self.corners()
        vol = 0.0
        for order in itertools.permutations(range(3)):
            idx = np.zeros(3, dtype=int)
            verts = [Pc[tuple(idx)]]
            for a in order:
                idx[a] = 1
                verts.append(Pc[tuple(idx)])
            E = np.array([verts[j + 1] - verts[0] for j in range(3)])
            vol += abs(np.linalg.det(E)) / 6.0
        return vol


def make_geometry(name, d=3, geo=None):
    if name == "cube":
        return Cube(d)
    if name == "annulus":
        if d != 3:
            raise ValueError("the annulus is three-dimensional")
        geo = geo or (1.0, 2.0, 1.0)
        return QuarterAnnulus(*geo)
    if name == "half_annulus":
        if d != 3:
            raise ValueError("the half annulus is three-dimensional")
        geo = geo or (1.0, 2.0, 1.0)
        return HalfAnnulus(*geo)
    if name == "projective_cube":
        if d != 3:
            raise ValueError("the projective cube is three-dimensional")
        return ProjectiveCube(*(geo if geo is not None else (0.5, 0.25, -0.2)))
    raise ValueError(f"unknown geometry {name!r}")
