"""Failure detection (GPU): every error path is driven from the host, and
nothing here faults, traps or hangs the GPU.

* a bounded wait of the tcgen05 kernel that gives up (the pipeline wait limit
  set to a few hundred clock cycles through kl_debug_set): the kernel records
  the timeout, lets its issued MMAs and copies finish, frees its tensor memory
  and returns; kl_eigs reports KL_ERR_TIMEOUT and the same handle solves
  normally afterwards;
* a NaN planted in the eigensolver's start block: KL_ERR_NUMERIC;
* the restart limit: KL_ERR_NOCONV with the best pairs still returned;
* a device allocation that fails (injected on the host): KL_ERR_OOM from
  kl_create and from kl_eigs, nothing leaked, the handle still usable; in a
  server, exactly the request that met it fails and the others complete;
* with the bounds-checking build, a launch whose range runs past its buffer
  is refused before it runs.
"""
import numpy as np
import pytest

from kl_inputs import PARITY_CASES

pytestmark = pytest.mark.gpu

CASE = "cube_p2_e6x5x7_expsep"
M = 8


@pytest.fixture(scope="module")
def kl():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_00629_gb300 import _build
    _build.build()
    import paper_2101_00629_gb300 as mod
    return mod


def _params(kl, precision, method="galerkin", **kw):
    c = PARITY_CASES[CASE]
    return kl.params(geometry=c["geometry"], degree=c["p"], elems=c["elems"], kernel=c["kernel"],
                     sigma=c["sigma"], L=c["L"], method=method, precision=precision, block_k=8, **kw)


def _create(kl, p):
    import torch
    return kl.kl_create(p, torch.cuda.current_stream())


def _eigs(kl, h):
    lam = np.zeros(M)
    rc = kl.kl_eigs(h, M, 0.0, lam, None, 0, 0)
    return rc, lam


@pytest.mark.parametrize("precision", ["bf16", "tf32"])
def test_wait_limit_gives_up_with_timeout(kl, precision):
    ref_h = _create(kl, _params(kl, precision))
    try:
        rc, ref = _eigs(kl, ref_h)
        assert rc == kl.KL_OK
    finally:
        kl.kl_destroy(ref_h)
    h = _create(kl, _params(kl, precision))
    try:
        kl.kl_debug_set(h, kl.KL_DEBUG_WAIT_LIMIT, 200)
        with pytest.raises(kl.KLError) as ei:
            _eigs(kl, h)
        assert ei.value.status == kl.KL_ERR_TIMEOUT, str(ei.value)
        # the context and the handle are still usable: the default limit
        # gives the same eigenvalues as a fresh handle
        kl.kl_debug_set(h, kl.KL_DEBUG_WAIT_LIMIT, 0)
        rc, lam = _eigs(kl, h)
        assert rc == kl.KL_OK
        assert np.max(np.abs(lam - ref) / np.abs(ref)) <= 1e-12
    finally:
        kl.kl_destroy(h)


def test_nan_in_start_block_is_numeric_error(kl):
    h = _create(kl, _params(kl, "fp64"))
    try:
        kl.kl_debug_set(h, kl.KL_DEBUG_NAN_START, 1)
        with pytest.raises(kl.KLError) as ei:
            _eigs(kl, h)
        assert ei.value.status == kl.KL_ERR_NUMERIC, str(ei.value)
        kl.kl_debug_set(h, kl.KL_DEBUG_NAN_START, 0)
        rc, lam = _eigs(kl, h)
        assert rc == kl.KL_OK and np.all(np.isfinite(lam))
    finally:
        kl.kl_destroy(h)


@pytest.mark.parametrize("method", ["galerkin", "collocation"])
def test_restart_limit_is_noconv_with_pairs(kl, method):
    h = _create(kl, _params(kl, "fp64", method=method, max_restarts=1))
    try:
        lam = np.zeros(M)
        res = np.zeros(M)
        info = kl.kl_solve_info()
        # a tolerance below FP64 roundoff cannot be met: the loop stops at
        # its one restart and still returns its best pairs
        rc = kl.kl_eigs(h, M, 1e-17, lam, None, 0, 0, res, info)
        assert rc == kl.KL_ERR_NOCONV
        assert info.restarts == 1
        assert np.all(np.isfinite(lam)) and np.all(np.diff(lam) <= 0)
        assert np.all(np.isfinite(res)) and np.all(res < 1e-2)
    finally:
        kl.kl_destroy(h)


def _free_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_allocation_failure_in_create_and_eigs(kl):
    before = _free_bytes()
    for nth in (1, 2, 3, 4):
        kl.kl_debug_set(None, kl.KL_DEBUG_FAIL_ALLOC, nth)
        with pytest.raises(kl.KLError) as ei:
            _create(kl, _params(kl, "bf16"))
        assert ei.value.status == kl.KL_ERR_OOM, (nth, str(ei.value))
    kl.kl_debug_set(None, kl.KL_DEBUG_FAIL_ALLOC, 0)
    # every partial handle was freed
    assert abs(_free_bytes() - before) < (64 << 20)
    h = _create(kl, _params(kl, "bf16"))
    try:
        rc, ref = _eigs(kl, h)
        assert rc == kl.KL_OK
    finally:
        kl.kl_destroy(h)
    h = _create(kl, _params(kl, "bf16"))
    try:
        # the eigensolver workspace is the next allocation of this handle
        kl.kl_debug_set(None, kl.KL_DEBUG_FAIL_ALLOC, 1)
        with pytest.raises(kl.KLError) as ei:
            _eigs(kl, h)
        assert ei.value.status == kl.KL_ERR_OOM, str(ei.value)
        kl.kl_debug_set(None, kl.KL_DEBUG_FAIL_ALLOC, 0)
        rc, lam = _eigs(kl, h)
        assert rc == kl.KL_OK and np.max(np.abs(lam - ref) / np.abs(ref)) <= 1e-12
    finally:
        kl.kl_debug_set(None, kl.KL_DEBUG_FAIL_ALLOC, 0)
        kl.kl_destroy(h)


def test_allocation_failure_inside_a_server(kl):
    """One allocation fails while four requests are served: exactly one
    request reports KL_ERR_OOM, the other three complete, and the server
    keeps serving (a fifth request submitted afterwards completes)."""
    plist = []
    for seed in range(4):
        p = _params(kl, "bf16")
        p.seed = 200 + seed
        plist.append(p)
    s = kl.kl_serve_open(0, 4, 0)
    lams = [np.zeros(M) for _ in range(5)]
    results = {}
    try:
        kl.kl_debug_set(None, kl.KL_DEBUG_FAIL_ALLOC, 1)
        for i, p in enumerate(plist):
            kl.kl_serve_submit(s, p, M, 0.0, i, lams[i])
        while len(results) < 4:
            for r in kl.kl_serve_poll(s, 16, 500):
                results[r["request_id"]] = r
        kl.kl_debug_set(None, kl.KL_DEBUG_FAIL_ALLOC, 0)
        kl.kl_serve_submit(s, plist[0], M, 0.0, 4, lams[4])
        while len(results) < 5:
            for r in kl.kl_serve_poll(s, 16, 500):
                results[r["request_id"]] = r
    finally:
        kl.kl_debug_set(None, kl.KL_DEBUG_FAIL_ALLOC, 0)
        kl.kl_serve_close(s)
    status = [results[i]["status"] for i in range(4)]
    assert sorted(status) == [kl.KL_ERR_OOM, 0, 0, 0], status
    assert results[4]["status"] == 0


def test_bounds_build_refuses_a_range_past_its_buffer(kl):
    """Only in the bounds-checking build (KL_CHECK_BOUNDS=1): a leading
    dimension far beyond the buffer is refused on the host before the launch.
    The regular build would launch it, so the test is skipped there."""
    import torch
    if not kl.kl_bounds_checked():
        pytest.skip("regular build (KL_CHECK_BOUNDS not set)")
    h = _create(kl, _params(kl, "fp64"))
    try:
        N = kl.kl_dims(h)[0]
        X = torch.zeros((2, N), dtype=torch.float64, device="cuda")
        Y = torch.zeros((2, N), dtype=torch.float64, device="cuda")
        with pytest.raises(kl.KLError) as ei:
            kl.kl_apply_A(h, X, N + (100 << 20), Y, N, 2)
        assert ei.value.status == kl.KL_ERR_CUDA
    finally:
        kl.kl_destroy(h)
