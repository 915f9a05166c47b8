"""Pins of the oracle on the half annular cylinder (two quarter arcs joined C^0
at the angle parameter 1/2; the interpolation space is C^-1 there, Sec. 4.1)."""
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import collocation, galerkin, splines, standard
from oracle.problem import Problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "half_cylinder_dofs.txt")


def _rel(a, b):
    return np.max(np.abs(np.asarray(a) - np.asarray(b)) / np.abs(np.asarray(b)))


def _golden():
    rows = []
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            ex, case, kern, p, ea, er, ez, N, Nt = line.split()
            rows.append((int(ex), int(case), kern, int(p), (int(ea), int(er), int(ez)), int(N),
                         None if Nt == "-" else int(Nt)))
    return rows


@pytest.mark.parametrize("row", _golden(), ids=lambda r: f"ex{r[0]}case{r[1]}")
def test_dof_counts_of_the_paper_tables(row):
    ex, case, kern, p, elems, N, Nt = row
    prob = Problem("half_annulus", p, elems, kern)
    n, nt = galerkin.dims(prob)
    assert n == N
    if Nt is not None:
        assert nt == Nt
    assert collocation.dims(prob)[0] == N


def test_c_minus_one_interpolation_reproduces_its_space():
    """Interpolation at the Greville points of the C^-1 space (the point at the
    join counted twice, the left one as a limit from the left) reproduces
    every function of the space; without the left limit the two rows of the
    collocation matrix coincide."""
    for p in (2, 3):
        Ut = splines.joined_knots(6, p, 0, -1)
        g = splines.greville(Ut, p)
        left = splines.greville_left(Ut, p)
        assert left.sum() == 1 and np.sum(g == 0.5) == 2
        B = splines.bspline_basis(Ut, p, g, left)
        c = np.random.default_rng(p).standard_normal(B.shape[1])
        assert np.allclose(np.linalg.solve(B, B @ c), c, atol=1e-12)
        assert np.linalg.matrix_rank(splines.bspline_basis(Ut, p, g)) == B.shape[1] - 1


def test_nurbs_weights_reproduce_the_half_arc_weight():
    prob = Problem("half_annulus", 3, (6, 2, 2), "gauss")
    w = collocation.nurbs_weights(prob)
    U = prob.trial_knots()
    n1 = splines.n_basis(U[0], 3)
    t = np.linspace(0, 1, 81)
    Wt = splines.bspline_basis(U[0], 3, t) @ w[:n1]
    assert np.max(np.abs(Wt - prob.geom.weight_function(t))) < 1e-14


def test_constant_kernel_gives_the_volume():
    """sigma^2 |D| with |D| = pi/2 (r_out^2 - r_in^2) h: collocation up to the
    Gauss rule's error on the rational det DF; IBQ-Galerkin converges to it."""
    vol = 0.5 * np.pi * 3.0
    lc, _, _ = collocation.solve(Problem("half_annulus", 2, (4, 2, 1), "const", 1.0, 1.0), 2)
    assert abs(lc[0] - vol) / vol < 1e-6 and abs(lc[1]) < 1e-12
    errs = []
    for n in (2, 4, 8, 16):
        lg, _, _ = galerkin.solve(Problem("half_annulus", 2, (n, n, 1), "const", 1.0, 1.0), 1)
        errs.append(abs(lg[0] - vol) / vol)
    # measured: 2.5e-3, 7.4e-4, 4.4e-5, 2.6e-6
    assert errs[1] < errs[0] and errs[2] < errs[1] / 8 and errs[3] < errs[2] / 8 and errs[3] < 1e-5


def test_ibq_converges_to_standard_galerkin():
    diffs = []
    for n in (2, 4, 8):
        prob = Problem("half_annulus", 2, (n, 2, 2), "gauss", 1.0, 1.5)
        lam, _, _ = galerkin.solve(prob, 4)
        As, Zs = standard.matrices(prob, nq=4)
        ls = sla.eigh(As, Zs, eigvals_only=True)[::-1][:4]
        diffs.append(_rel(lam, ls))
    # measured: 0.38, 0.094, 0.018 (refined in the angle direction only)
    assert diffs[1] < diffs[0] / 3 and diffs[2] < diffs[1] / 3 and diffs[2] < 0.03


def test_galerkin_and_collocation_agree_under_refinement():
    d = []
    for n in (2, 4, 8):
        prob = Problem("half_annulus", 2, (n, 2, 2), "gauss", 1.0, 1.5)
        lg, _, _ = galerkin.solve(prob, 4)
        lc, _, info = collocation.solve(prob, 4)
        assert not info["complex"]
        d.append(_rel(lc, lg))
    # measured: 0.36, 0.066, 0.011
    assert d[1] < d[0] / 3 and d[2] < d[1] / 3 and d[2] < 0.02
