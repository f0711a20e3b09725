"""h2_matvec_static (the matvec entry point that allocates no device memory, for callers
that may not allocate while it runs) against h2_matvec, through the C-ABI.

Collected last on purpose: it runs after every other test, and it must also pass on
its own in a fresh process.
"""
import numpy as np
import pytest
import torch

from conftest import problem

pytestmark = pytest.mark.gpu

TOL = 1e-13          # the matvec tolerance of the other GPU tests


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_11152_b300 import build
    build.build()
    import paper_2509_11152_b300 as h2
    return h2


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def test_static_scratch_matvec_matches_allocating_matvec(h):
    pb = problem("cov2d", n=1024, leaf=32)
    M = h.h2_matrix_create(pb.A)
    g = torch.Generator(device="cpu").manual_seed(11)
    for call in range(2):                                    # two calls in a row
        x = h.colmajor(torch.randn(pb.A.n, 3, generator=g, dtype=torch.float64).cuda())
        y_ref = h.colmajor(torch.zeros_like(x))
        y_st = h.colmajor(torch.zeros_like(x))
        h.h2_matvec(M, x, y_ref)
        h.h2_matvec_static(M, x, y_st)
        assert _rel(y_st, y_ref) <= TOL, call


def test_static_scratch_rejects_oversize(h):
    pb = problem("cov2d", n=1024, leaf=32)
    M = h.h2_matrix_create(pb.A)
    words = 1 << 22
    nrhs = words // (2 * int(np.sum(pb.A.rank))) + 1          # just above the array
    x = h.colmajor(torch.zeros(pb.A.n, nrhs, dtype=torch.float64, device="cuda"))
    y = h.colmajor(torch.zeros_like(x))
    with pytest.raises(h.H2Error) as e:
        h.h2_matvec_static(M, x, y)
    assert e.value.code == -1 and "static scratch" in str(e.value)
    # the library is still usable afterwards
    x1 = h.colmajor(torch.ones(pb.A.n, 1, dtype=torch.float64, device="cuda"))
    y1 = h.colmajor(torch.zeros_like(x1))
    y2 = h.colmajor(torch.zeros_like(x1))
    h.h2_matvec_static(M, x1, y1)
    h.h2_matvec(M, x1, y2)
    assert _rel(y1, y2) <= TOL
