"""The allocation-free pairwise entry point against the library's regular
entry points (GPU).

For callers that cannot allocate device memory, kl_pairwise_noalloc computes
Y = sigma^2 Gamma(targets, sources) X with its scratch in a static device
array. It is checked against kl_apply_Zinv / kl_apply_A: on the unit interval with
linear splines (p = 1) the IBQ interpolation space equals the trial space, B~
is the identity at the nodes and M is the mass matrix Z, so Z^-1 A Z^-1 =
Gamma at the nodes (two calls in a row must both match); and against the
oracle's dense kernel matrix on sampled rows, for calls with many source
splits, with the split count cut by the array's size, and a small call after
a large one.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12   # the FP64 tolerance of the parity tests


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
        # entry by entry against the size of the entry (the operators
        # applied are dense and their reference's rounding is at that scale)
        r = np.abs(Y - ref) / np.maximum(np.abs(ref).max(axis=1, keepdims=True), 1e-300)
        print(f"call {call}: worst entry difference {r.max():.2e} of its vector's largest entry")
        assert r.max() < FP64_TOL


def _oracle_rows(kernel, sigma, L, tgt, src, X, rows):
    """sigma^2 Gamma(tgt[rows], src) X by the oracle's dense kernel matrix."""
    from oracle import kernels
    G = kernels.matrix(kernel, sigma, L, tgt[rows], src)
    return (G @ X.T).T


def _call(kl, kernel, sigma, L, tgt, src, X):
    import torch
    T, S, k = tgt.shape[0], src.shape[0], X.shape[0]
    Pt = torch.from_numpy(np.ascontiguousarray(tgt.T.reshape(-1))).cuda()   # all x, then y, then z
    Ps = torch.from_numpy(np.ascontiguousarray(src.T.reshape(-1))).cuda()
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.full((k, T), float("nan"), dtype=torch.float64, device="cuda")
    kl.kl_pairwise_noalloc(kernel, sigma, L, Pt, T, Ps, S, Xd, S, Yd, T, k, torch.cuda.current_stream())
    torch.cuda.synchronize()
    return Yd.cpu().numpy()


def _check_rows(Y, ref, absref, rows, label):
    """Entry by entry: |Y - ref| <= 1e-12 (|Gamma| |X|) (Gamma >= 0)."""
    r = np.abs(Y[:, rows] - ref) / absref
    c, i = np.unravel_index(int(np.argmax(r)), r.shape)
    print(f"{label}: worst entry {r[c, i]:.2e} of its bound (vector {c}, target {rows[i]})")
    assert r[c, i] < FP64_TOL, (label, c, rows[i], r[c, i])


def test_noalloc_split_paths_large_then_small(kl):
    """Several source splits (T = S = 8192, k = 8: 16 splits), then the size
    at which the scratch limit cuts the splits down (k = 32, T = S = 65536:
    k T = 2^21, one split), then the small call again: every call must match
    the oracle's dense kernel rows, whatever the earlier call left in the
    shared array. Rows: a random sample, the first and the last (ragged)
    target tile."""
    rng = np.random.default_rng(2101)
    cases = [("gauss", 1.2, 0.4, 8192, 8), ("exp", 0.9, 0.7, 65536, 32), ("gauss", 1.2, 0.4, 8192, 8)]
    for call, (kernel, sigma, L, n, k) in enumerate(cases):
        tgt = rng.random((n, 3))
        src = rng.random((n, 3))
        X = rng.standard_normal((k, n))
        Y = _call(kl, kernel, sigma, L, tgt, src, X)
        rows = np.unique(np.concatenate([rng.integers(0, n, 96), np.arange(128), np.arange(n - 100, n)]))
        ref = _oracle_rows(kernel, sigma, L, tgt, src, X, rows)
        absref = _oracle_rows(kernel, sigma, L, tgt, src, np.abs(X), rows)
        _check_rows(Y, ref, absref, rows, f"call {call} {kernel} T=S={n} k={k}")
        assert np.all(np.isfinite(Y))


def test_noalloc_rejects_sizes_beyond_its_scratch(kl):
    import torch
    T = (1 << 21) // 4 + 1
    P = torch.zeros(3 * T, dtype=torch.float64, device="cuda")
    X = torch.zeros((4, T), dtype=torch.float64, device="cuda")
    with pytest.raises(kl.KLError) as ei:
        kl.kl_pairwise_noalloc("gauss", 1.0, 1.0, P, T, P, T, X, T, X, T, 4, torch.cuda.current_stream())
    assert ei.value.status == -1 and "static scratch" in str(ei.value)
    # a target count whose product with k would overflow a 64-bit integer
    # is refused before any arithmetic on it
    huge = (1 << 62)
    with pytest.raises(kl.KLError) as ei:
        kl.kl_pairwise_noalloc("gauss", 1.0, 1.0, P, huge, P, T, X, T, X, huge, 4, torch.cuda.current_stream())
    assert ei.value.status == -1 and "static scratch" in str(ei.value)
