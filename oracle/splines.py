"""B-spline spaces for the oracle (test infrastructure only; see package doc).

Sec. 3.1 builds the trial space from tensor-product B-splines of degree p and
the interpolation-based quadrature from a second tensor-product B-spline
space on the same mesh (Sec. 4: "the interpolation space ... is defined on the
same mesh as the solution space, but its continuity is adapted"). Sec. 3.2
collocates at the Greville abscissae. Everything below is the textbook
definition, evaluated point by point in float64.
"""
import numpy as np


def open_uniform_knots(n_elem, p, cont):
    """Open knot vector on [0, 1] with ``n_elem`` equal elements, degree p.

    Interior breakpoints get multiplicity ``p - cont`` so that the splines are
    C^cont there (cont = p-1: maximal smoothness, cont = 0: C^0 as used for
    the exponential kernel in Sec. 4.1).
    """
    if n_elem < 1 or p < 1 or not (-1 <= cont <= p - 1):
        raise ValueError("bad knot parameters")
    mult = p - cont
    interior = np.repeat(np.arange(1, n_elem) / n_elem, mult)
    return np.concatenate([np.zeros(p + 1), interior, np.ones(p + 1)])


def joined_knots(n_elem, p, cont, join_cont):
    """Open knot vector like ``open_uniform_knots`` (n_elem even) whose middle
    breakpoint 1/2 gets multiplicity p - join_cont: a C^join_cont join of two
    patches inside one parameter domain (Sec. 4.1: the half cylinder's
    geometry is C^0 there, its interpolation space C^-1)."""
    if n_elem < 2 or n_elem % 2 or p < 1 or not (-1 <= cont <= p - 1) or not (-1 <= join_cont <= cont):
        raise ValueError("bad knot parameters")
    interior = []
    for e in range(1, n_elem):
        mult = p - join_cont if 2 * e == n_elem else p - cont
        interior += [e / n_elem] * mult
    return np.concatenate([np.zeros(p + 1), np.array(interior), np.ones(p + 1)])


def greville_left(knots, p):
    """Which Greville points lie at the right end of their basis function's
    support inside the domain (a C^-1 breakpoint): there the function is
    evaluated as the limit from the left."""
    t = np.asarray(knots, dtype=np.float64)
    g = greville(t, p)
    return np.array([g[i] == t[i + p + 1] and g[i] < t[-1] for i in range(len(g))])


def n_basis(knots, p):
    return len(knots) - p - 1


def greville(knots, p):
    """Greville abscissae xi*_i = (t_{i+1} + ... + t_{i+p}) / p (Sec. 3.2)."""
    n = n_basis(knots, p)
    return np.array([np.sum(knots[i + 1:i + p + 1]) / p for i in range(n)])


def _last_nonempty_span(t):
    return max(i for i in range(len(t) - 1) if t[i] < t[i + 1])


def bspline_basis(knots, p, x, left=None):
    """All degree-p B-splines at the points x by the Cox–de Boor recursion.

    Returns an array of shape (len(x), n_basis). Degree 0 splines are the
    indicator functions of the half-open knot spans [t_i, t_i+1); the right
    end of the parameter domain belongs to the last non-empty span. Points
    flagged in ``left`` use the spans (t_i, t_i+1] instead (limits from the
    left). Terms with a zero denominator (repeated knots) are dropped (the
    0/0 := 0 convention).
    """
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    t = np.asarray(knots, dtype=np.float64)
    lf = np.zeros(x.size, dtype=bool) if left is None else np.asarray(left, dtype=bool)
    m = len(t) - 1
    last = _last_nonempty_span(t)
    B = np.zeros((x.size, m))
    for i in range(m):
        if t[i] < t[i + 1]:
            inside = (x >= t[i]) & (x < t[i + 1])
            if i == last:
                inside |= x == t[i + 1]
            inside_l = (x > t[i]) & (x <= t[i + 1])
            B[:, i] = np.where(lf, inside_l, inside)
    for d in range(1, p + 1):
        Bn = np.zeros((x.size, m - d))
        for i in range(m - d):
            den_l = t[i + d] - t[i]
            den_r = t[i + d + 1] - t[i + 1]
            if den_l > 0:
                Bn[:, i] += (x - t[i]) / den_l * B[:, i]
            if den_r > 0:
                Bn[:, i] += (t[i + d + 1] - x) / den_r * B[:, i + 1]
        B = Bn
    return B


def bspline_basis_deriv(knots, p, x):
    """First derivatives of all degree-p B-splines at x.

    Uses the standard identity
    B'_{i,p} = p/(t_{i+p}-t_i) B_{i,p-1} - p/(t_{i+p+1}-t_{i+1}) B_{i+1,p-1}.
    """
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    t = np.asarray(knots, dtype=np.float64)
    n = n_basis(t, p)
    Bm = bspline_basis(t, p - 1, x) if p >= 1 else None  # n+1 functions of degree p-1
    D = np.zeros((x.size, n))
    for i in range(n):
        den_l = t[i + p] - t[i]
        den_r = t[i + p + 1] - t[i + 1]
        if den_l > 0:
            D[:, i] += p / den_l * Bm[:, i]
        if den_r > 0:
            D[:, i] -= p / den_r * Bm[:, i + 1]
    return D


def element_gauss(knots, nq):
    """Gauss–Legendre rule with ``nq`` points on every non-empty knot span.

    Returns (points, weights) in the parameter domain, element by element in
    increasing order. Sec. 4.1 uses (p+1) points per direction per element.
    """
    xg, wg = np.polynomial.legendre.leggauss(nq)
    brk = np.unique(np.asarray(knots, dtype=np.float64))
    pts, wts = [], []
    for a, b in zip(brk[:-1], brk[1:]):
        pts.append(0.5 * (a + b) + 0.5 * (b - a) * xg)
        wts.append(0.5 * (b - a) * wg)
    return np.concatenate(pts), np.concatenate(wts)


# ---------------------------------------------------------------------------
# Tensor-product helpers. Multi-indices and point grids are ordered
# lexicographically with direction 1 varying fastest, matching the Kronecker
# ordering Z = Z_d x ... x Z_1 of Sec. 3.1.
# ---------------------------------------------------------------------------

def tensor_grid(axes):
    """Cartesian product of 1D point sets; row r has direction 1 fastest."""
    grids = np.meshgrid(*axes[::-1], indexing="ij")
    cols = [g.reshape(-1) for g in grids[::-1]]
    return np.stack(cols, axis=1)


def tensor_weights(wts):
    grids = np.meshgrid(*wts[::-1], indexing="ij")
    out = np.ones(grids[0].size)
    for g in grids:
        out = out * g.reshape(-1)
    return out


def tensor_basis(knot_list, p, X, left=None):
    """Tensor-product B-splines evaluated at the d-dimensional points X.

    Row a of the result holds B_k(X[a]) = prod_d B_{k_d}(X[a, d]) for every
    multi-index k (direction 1 fastest). Each point is evaluated on its own;
    no Kronecker factorisation of the resulting matrix is used. ``left``
    (optional, shape of X) flags coordinates evaluated as limits from the left.
    """
    X = np.atleast_2d(X)
    d = X.shape[1]
    vals = [bspline_basis(knot_list[j], p, X[:, j], None if left is None else left[:, j]) for j in range(d)]
    out = vals[0]
    for j in range(1, d):
        # new index = k_prev + n_prev * k_j  (previous directions vary faster)
        out = (vals[j][:, :, None] * out[:, None, :]).reshape(X.shape[0], -1)
    return out


def tensor_basis_grad(knot_list, p, X):
    """Gradient of the tensor-product B-splines: shape (npts, nbasis, d)."""
    X = np.atleast_2d(X)
    d = X.shape[1]
    vals = [bspline_basis(knot_list[j], p, X[:, j]) for j in range(d)]
    ders = [bspline_basis_deriv(knot_list[j], p, X[:, j]) for j in range(d)]
    grads = []
    for e in range(d):
        out = ders[0] if e == 0 else vals[0]
        for j in range(1, d):
            f = ders[j] if j == e else vals[j]
            out = (f[:, :, None] * out[:, None, :]).reshape(X.shape[0], -1)
        grads.append(out)
    return np.stack(grads, axis=2)
