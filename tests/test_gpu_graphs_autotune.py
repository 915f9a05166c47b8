"""CUDA-graph replay of operator applications and the block-size autotuner
(GPU): replayed applications and solves are bitwise identical to eager ones;
the autotuner returns the fastest timed block size and handles created with
block_k = 0 take it from the cache."""
import os

import numpy as np
import pytest

from kl_inputs import PARITY_CASES, random_block

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


def _params(kl, case, method, precision, block_k=8):
    c = PARITY_CASES[case]
    return kl.params(geometry=c["geometry"], degree=c["p"], elems=c["elems"], kernel=c["kernel"],
                     sigma=c["sigma"], L=c["L"], method=method, precision=precision, block_k=block_k, seed=11)


@pytest.mark.parametrize("precision", ["fp64", "bf16"])
@pytest.mark.parametrize("method", ["galerkin", "collocation"])
def test_graph_replay_matches_eager(kl, method, precision):
    import torch
    stream = torch.cuda.current_stream()
    p = _params(kl, "annulus_p2_e4x4x2_gauss", method, precision)
    outs = {}
    for graphs in (False, True):
        h = kl.kl_create(p, stream)
        try:
            kl.kl_set_graphs(h, graphs)
            N = kl.kl_dims(h)[0]
            X = torch.from_numpy(random_block(N, 8, 5)).cuda()
            res = []
            l0 = kl.kl_launch_count(h)
            for rep in range(3):  # eager, captured, replayed
                Y = torch.empty_like(X)
                kl.kl_apply_Aprime(h, X, N, Y, N, 8)
                torch.cuda.synchronize()
                res.append(Y.cpu().numpy())
            launches = kl.kl_launch_count(h) - l0
            lam = np.zeros(6)
            kl.kl_eigs(h, 6, 0.0, lam, None, 0, 0)
            lam2 = np.zeros(6)
            kl.kl_eigs(h, 6, 0.0, lam2, None, 0, 0)  # second solve replays the graphs
        finally:
            kl.kl_destroy(h)
        outs[graphs] = (res, launches, lam, lam2)
    (r0, l_eager, lam0, lam0b), (r1, l_graph, lam1, lam1b) = outs[False], outs[True]
    for a, b in zip(r0, r1):
        assert np.array_equal(a, b)
    assert l_eager == l_graph  # the count includes the kernels inside replayed graphs
    assert np.array_equal(lam0, lam1) and np.array_equal(lam0b, lam1b) and np.array_equal(lam0, lam0b)


def test_autotune_picks_fastest_and_cache_is_used(kl, tmp_path, monkeypatch):
    import torch
    stream = torch.cuda.current_stream()
    p = _params(kl, "cube_p2_e6x5x7_expsep", "galerkin", "bf16", block_k=0)
    cache = str(tmp_path / "tune.txt")
    M = 8
    best, secs = kl.kl_autotune(p, M, 0.0, stream, cache)
    assert best in (8, 16, 32)
    timed = {k: s for k, s in zip((8, 16, 32), secs) if s > 0}
    assert best in timed and timed[best] == min(timed.values())
    lines = open(cache).read().strip().splitlines()
    assert len(lines) == 1 and lines[0].split()[1] == str(best)
    # a handle with block_k = 0 takes the cached size at kl_eigs
    monkeypatch.setenv("KL_TUNE_CACHE", cache)
    h = kl.kl_create(p, stream)
    try:
        lam = np.zeros(M)
        kl.kl_eigs(h, M, 0.0, lam, None, 0, 0)
        assert kl.kl_block_size(h) == best
        # and solves to the same eigenvalues as a handle with that size fixed
        h2 = kl.kl_create(_params(kl, "cube_p2_e6x5x7_expsep", "galerkin", "bf16", block_k=best), stream)
        lam2 = np.zeros(M)
        kl.kl_eigs(h2, M, 0.0, lam2, None, 0, 0)
        kl.kl_destroy(h2)
        assert np.array_equal(lam, lam2)
    finally:
        kl.kl_destroy(h)
    # other M: no cache entry, the default size
    monkeypatch.setenv("KL_TUNE_CACHE", cache)
    h = kl.kl_create(p, stream)
    try:
        lam = np.zeros(M + 1)
        kl.kl_eigs(h, M + 1, 0.0, lam, None, 0, 0)
        assert kl.kl_block_size(h) == 8
    finally:
        kl.kl_destroy(h)
