"""GPU parity of the symmetric split-BF16 Galerkin product.

Gamma over one point set is symmetric (Sec. 3.1), so the tensor-core
product evaluates each pair of 128-point tile and 64-point chunk above the
diagonal once and applies it twice (W_I += Gamma_Ic X_c, W_c += Gamma_Ic^T
X_I). Checked here, through the C ABI:
  * entry by entry against the FP64 oracle (the bound of the other
    split-BF16 tests: 5e-5 (|A||X|));
  * against the dense form of the same product (every pair evaluated,
    KL_DEBUG_PAIR_DENSE): both use bit-identical kernel values and splits and
    differ only in the order of the FP32 accumulations, so they agree to
    1e-6 of |A||X| entry by entry; a wrong transposed operand (layout,
    row-to-lane map, X of the wrong tile) breaks this by orders of
    magnitude;
  * bitwise repeatability (fixed reduction order);
  * the multi-band path (transposed partial sums above the per-band cap) on
    a 24x24x24 cube with 16 vectors;
  * that the symmetric form is the one that ran (profile class).
"""
import numpy as np
import pytest

from _entrywise import assert_entrywise, bound, galerkin_abs
from kl_inputs import PARITY_CASES, WORKLOADS, problem_args, random_block
from oracle import galerkin
from oracle.problem import Problem

pytestmark = pytest.mark.gpu

BF16_TOL = 5e-5      # split-BF16 product against the FP64 oracle
ORDER_TOL = 1e-6     # symmetric against dense form: accumulation order only


@pytest.fixture(scope="module")
def kl():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_00629_gb300 import _build
    _build.build()
    import paper_2101_00629_gb300 as mod
    return mod


def _create(kl, spec, **kw):
    import torch
    if "geo" in spec:
        kw = dict(kw, geo=spec["geo"])
    p = kl.params(geometry=spec["geometry"], degree=spec["p"], elems=spec["elems"], kernel=spec["kernel"],
                  sigma=spec["sigma"], L=spec["L"], method="galerkin", precision="bf16", **kw)
    return kl.kl_create(p, torch.cuda.current_stream())


def _apply(kl, h, X, ldx=None):
    import torch
    k, n = X.shape
    ldx = n if ldx is None else ldx
    Xd = torch.zeros((k, ldx), dtype=torch.float64, device="cuda")
    Xd[:, :n] = torch.from_numpy(X)
    Yd = torch.full((k, ldx), float("nan"), dtype=torch.float64, device="cuda")
    kl.kl_apply_A(h, Xd, ldx, Yd, ldx, k)
    torch.cuda.synchronize()
    return Yd[:, :n].cpu().numpy()


def _profiled_apply(kl, h, X, ldx=None):
    kl.kl_profile_enable(h, True)
    Y = _apply(kl, h, X, ldx)
    prof = kl.kl_profile_read(h)
    kl.kl_profile_enable(h, False)
    return Y, prof


def _oracle(case):
    spec = PARITY_CASES[case]
    prob = Problem(spec["geometry"], spec["p"], spec["elems"], spec["kernel"], spec["sigma"], spec["L"],
                   geo=spec.get("geo"))
    A, Z, parts = galerkin.matrices(prob, with_parts=True)
    return A, galerkin_abs(parts, Z)["A"]


@pytest.mark.parametrize("k", [1, 5, 8, 16])
@pytest.mark.parametrize("case", ["cube_p2_e6x5x7_expsep", "cube_p2_e3x4x5_gauss", "annulus_p2_e4x4x2_gauss",
                                  "cube_p3_e4x3x3_matern", "cube_p2_e5x4x4_exp"])
def test_symmetric_against_oracle_and_dense(kl, case, k):
    A, absA = _oracle(case)
    h = _create(kl, PARITY_CASES[case])
    try:
        N, S, T = kl.kl_dims(h)
        X = random_block(N, k, seed=300 + k)
        Ys, prof = _profiled_apply(kl, h, X, ldx=N + 5)
        assert "pair_tc_bf16_sym" in prof and "pair_tc_bf16" not in prof, sorted(prof)
        kl.kl_debug_set(h, kl.KL_DEBUG_PAIR_DENSE, 1)
        Yd, prof_d = _profiled_apply(kl, h, X, ldx=N + 5)
        assert "pair_tc_bf16" in prof_d and "pair_tc_bf16_sym" not in prof_d, sorted(prof_d)
        kl.kl_debug_set(h, kl.KL_DEBUG_PAIR_DENSE, 0)
        ref = (A @ X.T).T
        sc = bound(absA, X)
        r = assert_entrywise(Ys, ref, sc, BF16_TOL, f"{case} k={k} symmetric vs oracle")
        rd = assert_entrywise(Ys, Yd, sc, ORDER_TOL, f"{case} k={k} symmetric vs dense")
        print(f"{case} k={k} (T={T}): symmetric vs oracle {r:.2e}, vs dense {rd:.2e} of the bounds")
        # the same handle gives the same bits again
        Ys2 = _apply(kl, h, X, ldx=N + 5)
        assert np.array_equal(Ys, Ys2)
    finally:
        kl.kl_destroy(h)


def _kron3_apply(F, X):
    k = X.shape[0]
    n = [f.shape[1] for f in F]
    T = X.reshape(k, n[2], n[1], n[0])
    T = np.einsum("ia,cdba->cdbi", F[0], T)
    T = np.einsum("ib,cdba->cdia", F[1], T)
    T = np.einsum("id,cdba->ciba", F[2], T)
    return T.reshape(k, -1)


@pytest.mark.parametrize("elems,k", [(16, 8), (16, 16), (24, 16)])
def test_symmetric_full_size_cube(kl, elems, k):
    """The 16x16x16 cube of the benchmark (N~ = 35 937 points; one band) and
    a 24x24x24 cube (N~ = 117 649; 16 vectors make seven bands, the running
    sums carried between the bands' reductions). Against the exact Kronecker
    form of the separable kernel and the dense form."""
    w = WORKLOADS["cube_p2_e16_expsep"]
    args = dict(problem_args(w), elems=(elems, elems, elems))
    one_d = []
    for n in args["elems"]:
        prob = Problem("cube", 2, (n,), args["kernel"], 1.0, args["L"])
        A, Z, parts = galerkin.matrices(prob, with_parts=True)
        one_d.append((A, galerkin_abs(parts, Z)["A"]))
    h = _create(kl, dict(args), block_k=k)
    try:
        N, S, T = kl.kl_dims(h)
        X = random_block(N, k, seed=41 + k)
        Ys, prof = _profiled_apply(kl, h, X)
        assert "pair_tc_bf16_sym" in prof, sorted(prof)
        kl.kl_debug_set(h, kl.KL_DEBUG_PAIR_DENSE, 1)
        Yd = _apply(kl, h, X)
        kl.kl_debug_set(h, kl.KL_DEBUG_PAIR_DENSE, 0)
        s2 = args["sigma"] ** 2
        ref = _kron3_apply([o[0] for o in one_d], X) * s2
        sc = _kron3_apply([o[1] for o in one_d], np.abs(X)) * s2
        r = assert_entrywise(Ys, ref, sc, BF16_TOL, f"{elems}^3 symmetric k={k} vs Kronecker form")
        rd = assert_entrywise(Ys, Yd, sc, ORDER_TOL, f"{elems}^3 symmetric k={k} vs dense")
        print(f"{elems}^3 k={k}: vs Kronecker form {r:.2e}, vs dense {rd:.2e} of the bounds; "
              f"symmetric {prof['pair_tc_bf16_sym']['ms']:.3f} ms")
    finally:
        kl.kl_destroy(h)


@pytest.mark.parametrize("method", ["galerkin", "collocation"])
def test_shared_sms_same_bits(kl, method):
    """A pairwise grid that leaves SMs free for other streams
    (kl_set_shared_sms) gives the same bits: the work units and the order of
    their reduction do not depend on the grid. Out-of-range counts are
    refused."""
    import torch
    w = WORKLOADS["cube_p2_e16_expsep"]
    args = problem_args(w)
    p = kl.params(geometry=args["geometry"], degree=args["p"], elems=args["elems"], kernel=args["kernel"],
                  sigma=args["sigma"], L=args["L"], method=method, precision="bf16")
    h = kl.kl_create(p, torch.cuda.current_stream())
    try:
        N, _, _ = kl.kl_dims(h)
        X = random_block(N, 8, seed=77)
        Y0 = _apply(kl, h, X)
        for n in (8, 37, 0):
            kl.kl_set_shared_sms(h, n)
            assert np.array_equal(_apply(kl, h, X), Y0), n
        for bad in (-1, 100000):
            with pytest.raises(kl.KLError):
                kl.kl_set_shared_sms(h, bad)
    finally:
        kl.kl_destroy(h)
