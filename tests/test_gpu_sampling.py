"""K-L field sampling on the GPU against the oracle (same eigenpairs, same
seeded standard normal variables): realisations at the tensor Gauss grid and
the grid's physical points, elementwise."""
import numpy as np
import pytest

from _entrywise import assert_entrywise
from kl_inputs import PARITY_CASES
from oracle import collocation, galerkin, sampling, standard
from oracle.problem import Problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kl():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_00629_gb300 import _build
    _build.build()
    import paper_2101_00629_gb300 as mod
    return mod


@pytest.mark.parametrize("case,method", [("cube_p2_e3x4x5_gauss", "galerkin"),
                                         ("annulus_p2_e4x4x2_gauss", "galerkin"),
                                         ("annulus_p3_e4x3x2_exp", "collocation"),
                                         ("cube_p2_e6x5x7_expsep", "collocation"),
                                         ("half_annulus_p2_e4x3x2_gauss", "galerkin"),
                                         ("half_annulus_p2_e6x2x2_exp", "collocation"),
                                         ("half_annulus_p2_e4x3x2_gauss", "galerkin_std"),
                                         ("projective_p2_e4x3x3_gauss", "collocation"),
                                         ("projective_p3_e3x3x2_exp", "galerkin")])
def test_samples_match_oracle(kl, case, method):
    import torch
    c = PARITY_CASES[case]
    prob = Problem(c["geometry"], c["p"], c["elems"], c["kernel"], c["sigma"], c["L"], geo=c.get("geo"))
    M, ns = 9, 37
    if method == "galerkin_std":
        lam, V, _ = standard.solve(prob, M)   # the IBQ trial space, standard quadrature
        basis = "galerkin"
    else:
        lam, V, _ = (galerkin if method == "galerkin" else collocation).solve(prob, M)
        basis = method
    xi = np.random.Generator(np.random.PCG64(2101)).standard_normal((M, ns))
    ref = sampling.samples(prob, basis, lam, V, xi)              # Q x ns
    X, W, P = sampling.grid(prob)
    p = kl.params(geometry=c["geometry"], degree=c["p"], elems=c["elems"], kernel=c["kernel"], sigma=c["sigma"],
                  L=c["L"], method=method, precision="fp64", geo=c.get("geo", (1.0, 2.0, 1.0)))
    h = kl.kl_create(p, torch.cuda.current_stream())
    try:
        N = kl.kl_dims(h)[0]
        Q = kl.kl_sample_size(h)
        assert N == V.shape[0] and Q == ref.shape[0]
        Vd = torch.from_numpy(np.ascontiguousarray(V.T)).cuda()       # M x N: column-major N x M
        xid = torch.from_numpy(np.ascontiguousarray(xi.T)).cuda()     # ns x M: column-major M x ns
        out = torch.full((ns, Q + 3), float("nan"), dtype=torch.float64, device="cuda")
        kl.kl_sample(h, M, lam, Vd, N, xid, M, ns, out, Q + 3)
        xyz = torch.empty(3 * Q, dtype=torch.float64, device="cuda")
        kl.kl_sample_points(h, xyz)
        torch.cuda.synchronize()
        got = out[:, :Q].cpu().numpy().T
        err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
        perr = np.max(np.abs(xyz.cpu().numpy().reshape(3, Q).T - P))
        # entry by entry: the trial functions are non-negative, so the same
        # expansion with |V| and |xi| bounds each sample's rounding error
        scale = sampling.samples(prob, basis, lam, np.abs(V), np.abs(xi))
        r = assert_entrywise(got.T, ref.T, scale.T, 1e-12, f"{case} {method} samples")
        print(f"{case} {method}: samples {err:.2e} (worst entry {r:.2e} of its bound), points {perr:.2e}")
        assert perr < 1e-13
        assert np.isnan(out[:, Q:].cpu().numpy()).all()   # nothing written past the grid (ldo)
    finally:
        kl.kl_destroy(h)


def test_sample_argument_checks(kl):
    import torch
    p = kl.params(elems=(3, 3, 3))
    h = kl.kl_create(p, torch.cuda.current_stream())
    try:
        N = kl.kl_dims(h)[0]
        Q = kl.kl_sample_size(h)
        V = torch.zeros((2, N), dtype=torch.float64, device="cuda")
        xi = torch.zeros((4, 2), dtype=torch.float64, device="cuda")
        out = torch.zeros((4, Q), dtype=torch.float64, device="cuda")
        for args in [(0, N, 2, Q), (2, N - 1, 2, Q), (2, N, 1, Q), (2, N, 2, Q - 1)]:
            M, ldv, ldxi, ldo = args
            with pytest.raises(kl.KLError):
                kl.kl_sample(h, M, np.ones(2), V, ldv, xi, ldxi, 4, out, ldo)
    finally:
        kl.kl_destroy(h)
