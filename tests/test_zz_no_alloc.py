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


def _pool_used(dev):
    """(used bytes now, used-bytes high watermark) of the device's default memory pool,
    the pool the library's stream-ordered allocations come from."""
    from cuda.bindings import runtime as rt
    err, pool = rt.cudaDeviceGetDefaultMemPool(dev)
    assert err == rt.cudaError_t.cudaSuccess
    err, cur = rt.cudaMemPoolGetAttribute(pool, rt.cudaMemPoolAttr.cudaMemPoolAttrUsedMemCurrent)
    assert err == rt.cudaError_t.cudaSuccess
    err, high = rt.cudaMemPoolGetAttribute(pool, rt.cudaMemPoolAttr.cudaMemPoolAttrUsedMemHigh)
    assert err == rt.cudaError_t.cudaSuccess
    return int(cur), int(high)


def _pool_reset_high(dev):
    from cuda.bindings import driver
    from cuda.bindings import runtime as rt
    err, pool = rt.cudaDeviceGetDefaultMemPool(dev)
    assert err == rt.cudaError_t.cudaSuccess
    (err,) = rt.cudaMemPoolSetAttribute(pool, rt.cudaMemPoolAttr.cudaMemPoolAttrUsedMemHigh, driver.cuuint64_t(0))
    assert err == rt.cudaError_t.cudaSuccess


def test_static_scratch_takes_nothing_from_the_pool(h):
    """The point of the entry point: no device allocation during the call.  The
    allocating h2_matvec raises the pool's used-memory high watermark above the memory
    in use before the call (this shows the check can see an allocation);
    h2_matvec_static leaves it there."""
    pb = problem("cov2d", n=1024, leaf=32)
    M = h.h2_matrix_create(pb.A)
    dev = torch.cuda.current_device()
    x = h.colmajor(torch.randn(pb.A.n, 2, dtype=torch.float64, device="cuda"))
    y = h.colmajor(torch.zeros_like(x))
    h.h2_matvec_static(M, x, y)                              # first call: address look-up
    torch.cuda.synchronize()
    for fn, allocates in ((h.h2_matvec, True), (h.h2_matvec_static, False), (h.h2_matvec_static, False)):
        torch.cuda.synchronize()
        _pool_reset_high(dev)
        before, _ = _pool_used(dev)
        fn(M, x, y)
        torch.cuda.synchronize()
        _, high = _pool_used(dev)
        if allocates:
            assert high > before, (fn.__name__, high, before)
        else:
            assert high <= before, (fn.__name__, high, before)


def test_static_scratch_rejects_host_vectors(h):
    """Host memory given to the C entry point is refused before any kernel runs."""
    import ctypes
    from paper_2509_11152_b300 import binding
    pb = problem("cov2d", n=1024, leaf=32)
    M = h.h2_matrix_create(pb.A)
    xh = np.zeros((pb.A.n, 1))
    yh = np.zeros((pb.A.n, 1))
    rc = binding.lib().h2_matvec_static(M.handle, 1, ctypes.c_void_p(xh.ctypes.data), pb.A.n,
                                        ctypes.c_void_p(yh.ctypes.data), pb.A.n)
    assert rc == -1
    assert b"device memory" in binding.lib().h2_last_error() or b"CUDA pointer" in binding.lib().h2_last_error()


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
