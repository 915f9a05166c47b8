"""Seeded synthetic inputs shared by the oracle side and the GPU side.

This module holds workload descriptions and seeded random blocks only; it
contains none of the method's arithmetic, so that the oracle and the CUDA
library stay independent of each other while seeing identical inputs.

Blocks of k vectors of length n are returned as float64 arrays of shape
(k, n), C-contiguous; read as an n x k matrix this is column-major with
leading dimension n, the layout the C ABI takes.
"""
import numpy as np

# The workloads of the benchmark suite (unit cube and quarter annular cylinder
# with r_in = 1, r_out = 2, height 1). "methods" lists the discretisations run.
WORKLOADS = {
    "cube_p2_e4_gauss": dict(geometry="cube", p=2, elems=(4, 4, 4), kernel="gauss",
                              sigma=1.0, L=0.5, M=10, k=8, methods=("galerkin",)),
    "cube_p2_e16_expsep": dict(geometry="cube", p=2, elems=(16, 16, 16), kernel="exp_sep",
                                sigma=1.0, L=1.0, M=20, k=8, methods=("galerkin", "collocation")),
    "annulus_p3_e32x32x16_gauss": dict(geometry="annulus", p=3, elems=(32, 32, 16), kernel="gauss",
                                        sigma=1.0, L=0.5, M=50, k=16,
                                        methods=("galerkin", "collocation")),
    "annulus_p2_e64x32x16_exp": dict(geometry="annulus", p=2, elems=(64, 32, 16), kernel="exp",
                                      sigma=1.0, L=1.0, M=100, k=32,
                                      methods=("galerkin", "collocation")),
    "annulus_p4_e64x32x16_exp": dict(geometry="annulus", p=4, elems=(64, 32, 16), kernel="exp",
                                      sigma=1.0, L=1.0, M=100, k=32,
                                      methods=("galerkin", "collocation")),
    # the 16^3 cube workload on the projective cube x = x^ / (1 + c . x^):
    # collocation with NURBS weights that are not a tensor product
    "projective_p2_e16_expsep": dict(geometry="projective_cube", p=2, elems=(16, 16, 16), kernel="exp_sep",
                                     sigma=1.0, L=1.0, M=20, k=8, geo=(0.5, 0.25, -0.2),
                                     methods=("galerkin", "collocation")),
}

# Small parity cases: several 128-point tiles with ragged tails, sizes the
# dense oracle finishes in seconds.
PARITY_CASES = {
    "cube_p2_e3x4x5_gauss": dict(geometry="cube", p=2, elems=(3, 4, 5), kernel="gauss", sigma=1.3, L=0.6),
    "cube_p2_e6x5x7_expsep": dict(geometry="cube", p=2, elems=(6, 5, 7), kernel="exp_sep", sigma=1.0, L=1.0),
    "cube_p3_e4x3x3_matern": dict(geometry="cube", p=3, elems=(4, 3, 3), kernel="matern32", sigma=0.8, L=0.7),
    "cube_p2_e5x4x4_exp": dict(geometry="cube", p=2, elems=(5, 4, 4), kernel="exp", sigma=1.0, L=0.9),
    "annulus_p2_e4x4x2_gauss": dict(geometry="annulus", p=2, elems=(4, 4, 2), kernel="gauss", sigma=1.0, L=0.5),
    "annulus_p3_e4x3x2_exp": dict(geometry="annulus", p=3, elems=(4, 3, 2), kernel="exp", sigma=1.0, L=1.0),
    # half annular cylinder (C^0 geometry join at the angle parameter 1/2)
    "half_annulus_p2_e4x3x2_gauss": dict(geometry="half_annulus", p=2, elems=(4, 3, 2), kernel="gauss", sigma=1.0,
                                         L=0.6),
    "half_annulus_p2_e6x2x2_exp": dict(geometry="half_annulus", p=2, elems=(6, 2, 2), kernel="exp", sigma=1.0, L=1.0),
    # projective cube x = x^ / (1 + c . x^): NURBS weights that are not a tensor product
    "projective_p2_e4x3x3_gauss": dict(geometry="projective_cube", p=2, elems=(4, 3, 3), kernel="gauss", sigma=1.0,
                                       L=0.6, geo=(0.5, 0.25, -0.2)),
    "projective_p3_e3x3x2_exp": dict(geometry="projective_cube", p=3, elems=(3, 3, 2), kernel="exp", sigma=1.2,
                                     L=0.8, geo=(-0.3, 0.4, 0.6)),
}


def random_block(n, k, seed):
    """k standard-normal vectors of length n (PCG64 stream from ``seed``)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.ascontiguousarray(rng.standard_normal((k, n)))


def problem_args(spec):
    """The geometry/discretisation fields of a workload (no M, k, methods);
    "geo" (geometry parameters) only where the workload sets it."""
    keys = ("geometry", "p", "elems", "kernel", "sigma", "L") + (("geo",) if "geo" in spec else ())
    return {key: spec[key] for key in keys}


def serving_requests(n=500, seed=2101, max_elems=48, mean_interarrival_s=0.05):
    """A seeded stream of K-L requests with Poisson arrivals: geometry cube or
    quarter annulus, degree 2..4, per-axis elements from {8, 16, 24, 32, 40, 48}
    (n^3 for the cube, (2n, n, n/2) for the annulus) capped at max_elems,
    kernel Gaussian / Euclidean exponential / Matern-3/2, L log-uniform in
    [0.1, 2], M uniform in 10..100, Galerkin or collocation with equal
    probability. Returns a list of dicts with an arrival time "t" (seconds
    from the first arrival) and the fields of problem_args plus M, method."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = [e for e in (8, 16, 24, 32, 40, 48) if e <= max_elems] or [max_elems]
    out, t = [], 0.0
    for i in range(n):
        geometry = ("cube", "annulus")[int(rng.integers(2))]
        e = int(sizes[int(rng.integers(len(sizes)))])
        elems = (e, e, e) if geometry == "cube" else (2 * e, e, max(1, e // 2))
        req = dict(id=i, t=t, geometry=geometry, p=int(rng.integers(2, 5)), elems=elems,
                   kernel=("gauss", "exp", "matern32")[int(rng.integers(3))], sigma=1.0,
                   L=float(np.exp(rng.uniform(np.log(0.1), np.log(2.0)))), M=int(rng.integers(10, 101)),
                   method=("galerkin", "collocation")[int(rng.integers(2))])
        out.append(req)
        t += float(rng.exponential(mean_interarrival_s))
    return out
