"""The half annular cylinder through the C ABI: the library's spaces have the
dof counts printed in the paper's Tables 1 and 2 (Sec. 4), on the mesh
reading recorded beside them in tests/golden/half_cylinder_dofs.txt."""
import os

import pytest

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "half_cylinder_dofs.txt")


def _golden():
    rows = []
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            ex, case, kern, p, ea, er, ez, N, Nt = line.split()
            rows.append((int(ex), int(case), kern, int(p), (int(ea), int(er), int(ez)), int(N),
                         None if Nt == "-" else int(Nt)))
    return rows


@pytest.fixture(scope="module")
def kl():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_00629_gb300 import _build
    _build.build()
    import paper_2101_00629_gb300 as mod
    return mod


@pytest.mark.parametrize("row", _golden(), ids=lambda r: f"ex{r[0]}case{r[1]}")
def test_library_dims_match_paper_tables(kl, row):
    import torch
    ex, case, kern, p, elems, N, Nt = row
    for method in ("galerkin", "collocation"):
        prm = kl.params(geometry="half_annulus", degree=p, elems=elems, kernel=kern, sigma=1.0, L=1.0,
                        method=method, precision="fp64", block_k=8)
        h = kl.kl_create(prm, torch.cuda.current_stream())
        try:
            n, s, t = kl.kl_dims(h)
        finally:
            kl.kl_destroy(h)
        assert n == N
        if method == "galerkin" and Nt is not None:
            assert s == Nt
