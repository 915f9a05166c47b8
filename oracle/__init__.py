"""Plain FP64 CPU oracle for the matrix-free Karhunen–Loève methods.

This package is TEST INFRASTRUCTURE. It is the independent checker of the GPU
library and nothing else: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it. The
product path (``paper_2101_00629_gb300``) never imports, calls or links it, and
it never imports the product.

Everything here is dense and direct, in float64, written so that each line
can be read against the paper (Mika, Hiemstra, Hughes, Schillinger,
"A comparison of matrix-free isogeometric Galerkin and collocation methods for
Karhunen–Loève expansion"):

* ``splines``     – knot vectors, Cox–de Boor B-splines, Greville abscissae,
                    element Gauss rules (Sec. 3.1, Sec. 3.2).
* ``geometry``    – the geometry map F and det DF for the unit cube and the
                    quarter annular cylinder (exact quadratic NURBS arc).
* ``kernels``     – covariance functions Gamma(x, x').
* ``galerkin``    – the IBQ-Galerkin matrices A = M^T B~^-1 J Gamma J B~^-T M
                    and Z, assembled densely without Kronecker shortcuts
                    (Sec. 3.1, Eq. galerkin_system_matrices, trial space
                    Eq. trialspace and the unnumbered IBQ factorisation), and
                    the dense generalized symmetric eigensolve.
* ``collocation`` – the collocation matrices of Eq. colloc_system_matrices with
                    (p+1)^3 Gauss points per element (Sec. 3.2, Sec. 4.1) and
                    the dense QZ eigensolve.
* ``standard``    – standard Gauss–Legendre Galerkin (Sec. 3.1, footnote of
                    Sec. 1) used only as an independent brute-force
                    cross-check on tiny meshes.
* ``closed_form`` – textbook 1D exponential-kernel eigenpairs and a Gauss–
                    Legendre Nystrom reference for smooth 1D kernels.

Pins: every function here is checked by ``tests/test_oracle_*.py`` against
closed forms, invariants, special cases and brute force.
"""
