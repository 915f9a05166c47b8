"""The allocation-free pairwise entry point against the library's regular
entry points (GPU).

For callers that cannot allocate device memory, kl_pairwise_noalloc computes
Y = sigma^2 Gamma(targets, sources) X with its scratch in a static device
array. It is checked here against kl_apply_Zinv / kl_apply_A: on the unit
interval with linear splines (p = 1) the IBQ interpolation space equals the
trial space, B~ is the identity at the nodes and M is the mass matrix Z, so
Z^-1 A Z^-1 = Gamma at the nodes. Two calls in a row must both match.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12   # the FP64 normwise tolerance of the parity tests


@pytest.fixture(scope="module")
def kl():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_00629_gb300 import _build
    _build.build()
    import paper_2101_00629_gb300 as mod
    return mod


def _via_existing_entry_points(kl, n, sigma, L, X):
    import torch
    h = kl.kl_create(kl.params(geometry="cube", degree=1, elems=(n,), kernel="gauss", sigma=sigma, L=L,
                               method="galerkin", precision="fp64"), torch.cuda.current_stream())
    try:
        N, _, _ = kl.kl_dims(h)
        k = X.shape[0]
        Xd = torch.from_numpy(X).cuda()
        T1 = torch.empty_like(Xd)
        T2 = torch.empty_like(Xd)
        kl.kl_apply_Zinv(h, Xd, N, T1, N, k)
        kl.kl_apply_A(h, T1, N, T2, N, k)
        kl.kl_apply_Zinv(h, T2, N, T1, N, k)
        torch.cuda.synchronize()
        return T1.cpu().numpy()
    finally:
        kl.kl_destroy(h)


def test_noalloc_matches_existing_entry_points_twice(kl):
    import torch
    n, sigma, L, k = 40, 1.3, 0.3, 5
    nodes = np.arange(n + 1) / n
    pts = np.concatenate([nodes, np.zeros(n + 1), np.zeros(n + 1)])   # x, then y, then z
    P = torch.from_numpy(pts).cuda()
    rng = np.random.default_rng(2021)
    stream = torch.cuda.current_stream()
    for call in range(2):
        X = rng.standard_normal((k, n + 1))
        ref = _via_existing_entry_points(kl, n, sigma, L, X)
        Xd = torch.from_numpy(X).cuda()
        Yd = torch.full_like(Xd, float("nan"))
        kl.kl_pairwise_noalloc("gauss", sigma, L, P, n + 1, P, n + 1, Xd, n + 1, Yd, n + 1, k, stream)
        torch.cuda.synchronize()
        Y = Yd.cpu().numpy()
        err = np.linalg.norm(Y - ref) / np.linalg.norm(ref)
        print(f"call {call}: normwise difference {err:.2e}")
        assert err < FP64_TOL


def test_noalloc_rejects_sizes_beyond_its_scratch(kl):
    import torch
    T = (1 << 21) // 4 + 1
    P = torch.zeros(3 * T, dtype=torch.float64, device="cuda")
    X = torch.zeros((4, T), dtype=torch.float64, device="cuda")
    with pytest.raises(kl.KLError) as ei:
        kl.kl_pairwise_noalloc("gauss", 1.0, 1.0, P, T, P, T, X, T, X, T, 4, torch.cuda.current_stream())
    assert ei.value.status == -1 and "static scratch" in str(ei.value)
