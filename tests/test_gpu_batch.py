"""GPU parity of the uneven batch (independent systems factorised as one forest, one
launch per level and kernel over all systems' boxes) against the CPU oracle run on
each system separately, through the C-ABI."""
import functools

import numpy as np
import pytest
import torch

from h2gen import make_batch, rhs
from oracle import dense, rs

from conftest import problem

pytestmark = pytest.mark.gpu

EPS = 1e-6
NRHS = 4


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_11152_b300 import build
    build.build()
    import paper_2509_11152_b300 as h2
    return h2


@functools.lru_cache(maxsize=None)
def batch():
    pbs = make_batch("gauss3d", nsys=4, nmin=300, nmax=3000, leaf=32)
    pbs.append(problem("cov2d", n=256, leaf=16, eta=1e-6))     # nothing admissible
    pbs.append(problem("cov2d", n=1024, leaf=32))              # another kernel family
    return pbs


@functools.lru_cache(maxsize=None)
def oracle():
    out = []
    for z, pb in enumerate(batch()):
        A = pb.A.numpy()
        b = rhs(A.n, NRHS, seed=100 + z)
        Z = rs.factorize(A, EPS, pb.norm_a)
        out.append((A, b, Z, rs.solve(Z, b)))
    return out


def _stacked_rhs():
    return np.concatenate([o[1] for o in oracle()], axis=0)


def _split(x):
    off = np.cumsum([0] + [pb.A.n for pb in batch()])
    return [x[off[z]:off[z + 1]] for z in range(len(batch()))]


def test_batch_offsets(h):
    M = h.h2_matrix_create_batch([pb.A for pb in batch()])
    off = h.h2_matrix_batch_info(M)
    assert np.array_equal(off, np.cumsum([0] + [pb.A.n for pb in batch()]))


def test_batch_matvec_matches_oracle(h):
    M = h.h2_matrix_create_batch([pb.A for pb in batch()])
    x = np.concatenate([rhs(pb.A.n, 3, seed=7 + z) for z, pb in enumerate(batch())])
    xt = h.colmajor(torch.from_numpy(x).cuda())
    yt = h.colmajor(torch.zeros_like(xt))
    h.h2_matvec(M, xt, yt)
    for (A, _, _, _), xs, ys in zip(oracle(), _split(x), _split(yt.cpu().numpy())):
        y0 = dense.matvec(A, xs)
        assert np.linalg.norm(ys - y0) / np.linalg.norm(y0) <= 1e-13


def test_batch_fp64_factor_solve_matches_oracle_per_system(h):
    pbs = batch()
    M = h.h2_matrix_create_batch([pb.A for pb in pbs])
    Z = h.h2_factor_create(M, EPS, [pb.norm_a for pb in pbs], h.H2_PREC_FP64)
    x = h.colmajor(torch.from_numpy(_stacked_rhs()).cuda())
    h.h2_solve(Z, x)
    for z, ((A, b, Z0, x0), xs) in enumerate(zip(oracle(), _split(x.cpu().numpy()))):
        rel = np.linalg.norm(xs - x0) / np.linalg.norm(x0)
        assert rel <= 1e-10, (z, rel)


def test_batch_equals_separate_factorisations(h):
    """Same ranks as each system factorised alone, and the same solution up to
    rounding (the batch only regroups the launches)."""
    pbs = batch()
    M = h.h2_matrix_create_batch([pb.A for pb in pbs])
    Z = h.h2_factor_create(M, EPS, [pb.norm_a for pb in pbs], h.H2_PREC_FP64)
    xb = h.colmajor(torch.from_numpy(_stacked_rhs()).cuda())
    h.h2_solve(Z, xb)
    xs = _split(xb.cpu().numpy())
    nl = h.h2_factor_stats_get(Z)["nlevels"]
    lays = [h.h2_layout_get(Z, a) for a in range(nl)]
    for z, pb in enumerate(pbs):
        M1 = h.h2_matrix_create(pb.A)
        Z1 = h.h2_factor_create(M1, EPS, pb.norm_a, h.H2_PREC_FP64)
        x1 = h.colmajor(torch.from_numpy(oracle()[z][1]).cuda())
        h.h2_solve(Z1, x1)
        x1 = x1.cpu().numpy()
        assert np.linalg.norm(xs[z] - x1) / np.linalg.norm(x1) <= 1e-13
        for a in range(h.h2_factor_stats_get(Z1)["nlevels"]):
            qa = h.h2_plan_query_batch([p.A for p in pbs], a)
            boxes = np.flatnonzero(qa["system"] == z)
            assert np.array_equal(lays[a]["ranks"][boxes], h.h2_layout_get(Z1, a)["ranks"])


@pytest.mark.parametrize("prec", ["fp32", "tf32x3"])
def test_batch_fp32_refinement_reaches_backward_error_per_system(h, prec):
    pbs = batch()
    M = h.h2_matrix_create_batch([pb.A for pb in pbs])
    Z = h.h2_factor_create(M, EPS, [pb.norm_a for pb in pbs],
                           h.H2_PREC_FP32 if prec == "fp32" else h.H2_PREC_TF32X3)
    b = _stacked_rhs()
    bt = h.colmajor(torch.from_numpy(b).cuda())
    xt = h.colmajor(torch.zeros_like(bt))
    it, berr, ok = h.h2_refine_solve(Z, M, bt, xt, 1e-10, 60)
    assert ok and berr <= 1e-10
    for z, ((A, bz, _, _), xz, pb) in enumerate(zip(oracle(), _split(xt.cpu().numpy()), pbs)):
        nw, _ = dense.backward_error(A, xz, bz, pb.norm_a)
        assert nw <= 1e-10, (z, nw)
