"""CPU-side checks of the C ABI library: it loads, exports every entry point
declared in include/kl.h, its struct layouts match the binding, and argument
validation runs on the host without touching a GPU."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "kl.h")


@pytest.fixture(scope="module")
def kl():
    from paper_2101_00629_gb300 import _build
    _build.build()
    import paper_2101_00629_gb300 as mod
    return mod


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(kl_[a-z_A-Z0-9]+)\s*\(", text)))


def test_header_declarations_match_binding(kl):
    assert _declared() == sorted(kl.EXPORTED_SYMBOLS)


def test_library_exports_every_declared_symbol(kl):
    lib = ctypes.CDLL(kl.library_path())
    for name in _declared():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", kl.library_path()], capture_output=True, text=True)
    if out.returncode == 0:
        exported = set(re.findall(r" T (kl_\w+)", out.stdout))
        assert set(_declared()) <= exported


def test_struct_layout_matches_c(kl):
    src = r"""
    #include <stdio.h>
    #include <stddef.h>
    #include "kl.h"
    int main(void) {
      printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(kl_params), offsetof(kl_params, sigma),
             offsetof(kl_params, seed), sizeof(kl_solve_info), sizeof(kl_kernel_stats),
             offsetof(kl_params, precision), sizeof(kl_serve_config), sizeof(kl_serve_result),
             offsetof(kl_serve_result, max_resid), sizeof(kl_serve_stats),
             offsetof(kl_serve_stats, peak_est_bytes));
      return 0;
    }
    """
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        r = subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    assert vals == [ctypes.sizeof(kl.kl_params), kl.kl_params.sigma.offset, kl.kl_params.seed.offset,
                    ctypes.sizeof(kl.kl_solve_info), ctypes.sizeof(kl.kl_kernel_stats),
                    kl.kl_params.precision.offset, ctypes.sizeof(kl.kl_serve_config),
                    ctypes.sizeof(kl.kl_serve_result), kl.kl_serve_result.max_resid.offset,
                    ctypes.sizeof(kl.kl_serve_stats), kl.kl_serve_stats.peak_est_bytes.offset]


def test_default_params_and_status_strings(kl):
    p = kl.kl_default_params()
    assert (p.dim, p.degree, p.elems[0], p.kernel, p.method, p.precision, p.block_k) == (3, 2, 4, 0, 0, 0, 8)
    assert p.seed == 2101 and p.interp_continuity == -2
    assert kl.kl_status_string(0) == "ok"
    assert kl.kl_status_string(-4) == "eigensolver did not converge"
    assert kl.kl_status_string(1) == "complex eigenvalues met"


@pytest.mark.parametrize("field,value,msg", [
    ("degree", 0, "degree"), ("degree", 9, "degree"), ("dim", 4, "dim"), ("sigma", -1.0, "sigma"),
    ("L", 0.0, "L must"), ("kernel", 9, "kernel"), ("method", 5, "method"), ("precision", 7, "precision"),
    ("block_k", 65, "block_k"), ("interp_continuity", 2, "interp_continuity"), ("refine", 3, "refine"),
])
def test_create_rejects_bad_params_on_host(kl, field, value, msg):
    p = kl.params()
    setattr(p, field, value)
    with pytest.raises(kl.KLError) as ei:
        kl.kl_create(p)
    assert ei.value.status == -1
    assert msg in str(ei.value)


def test_create_rejects_bad_geometry(kl):
    p = kl.params(geometry="annulus", elems=(2, 2, 2), geo=(2.0, 1.0, 1.0))
    with pytest.raises(kl.KLError) as ei:
        kl.kl_create(p)
    assert ei.value.status == -1
    p = kl.params(geometry="annulus", elems=(2, 2))
    with pytest.raises(kl.KLError):
        kl.kl_create(p)


@pytest.mark.parametrize("geo,elems,msg", [((-0.6, -0.5, 0.0), (2, 2, 2), "positive"),
                                           ((float("nan"), 0.0, 0.0), (2, 2, 2), "finite"),
                                           ((0.5, 0.25, -0.2), (2, 2), "dim = 3")])
def test_create_rejects_bad_projective_cube(kl, geo, elems, msg):
    p = kl.params(geometry="projective_cube", elems=elems, geo=geo)
    with pytest.raises(kl.KLError) as ei:
        kl.kl_create(p)
    assert ei.value.status == -1
    assert msg in str(ei.value)


def test_null_arguments(kl):
    lib = kl._load()
    assert lib.kl_create(None, None, None) == -1
    assert lib.kl_destroy(None) == 0
    assert lib.kl_dims(None, None, None, None) == -1
    assert lib.kl_apply_A(None, None, 0, None, 0, 1) == -1
    assert lib.kl_eigs(None, 1, 0.0, None, None, 0, 0, None, None) == -1
    assert lib.kl_launch_count(None) == 0
    assert lib.kl_serve_submit(None, None, 1, 0.0, 0, None, None, 0) == -1
    assert lib.kl_serve_close(None) == 0


def _est(kl, **kw):
    args = dict(geometry="cube", degree=2, elems=(8, 8, 8), kernel="gauss", sigma=1.0, L=0.5,
                method="galerkin", precision="bf16", block_k=8)
    M = kw.pop("M", 10)
    args.update(kw)
    return kl.kl_estimate_bytes(kl.params(**args), M)


def test_estimate_bytes_on_host(kl):
    """The admission estimate needs no GPU and grows with what the handle holds:
    the mesh (tables, points, operator workspaces), the basis (M, block size)
    and, for collocation, the quadrature point set."""
    base = _est(kl)
    assert base > 0
    assert _est(kl, elems=(16, 8, 8)) > base
    assert _est(kl, M=40) > base
    assert _est(kl, block_k=32) > base
    assert _est(kl, method="collocation") > base
    # non-tensor NURBS weights add the weight arrays (3 N + 2 N_e N_q values)
    assert _est(kl, method="collocation", geometry="projective_cube", geo=(0.5, 0.25, -0.2)) > \
        _est(kl, method="collocation")
    # C0 interpolation of the exponential kernels has about 5x the points
    # (17^3 vs 10^3 here); the basis and its workspaces do not grow with them
    assert _est(kl, kernel="exp") > 1.5 * base
    # lower bound: the Krylov basis and its image alone (2 N mcap doubles)
    p = kl.params(geometry="cube", degree=2, elems=(16, 16, 16), kernel="exp_sep", method="galerkin",
                  precision="bf16", block_k=8)
    N = 18 ** 3
    assert kl.kl_estimate_bytes(p, 20) > 2 * N * 72 * 8
    with pytest.raises(kl.KLError):
        kl.kl_estimate_bytes(p, 0)
    bad = kl.params(geometry="cube", degree=0)
    with pytest.raises(kl.KLError):
        kl.kl_estimate_bytes(bad, 10)
