"""GPU parity: the CUDA library (through its C-ABI) against the CPU oracle.

Bars (stated by the method's specification for this build):
  * float64 factor + solve at the same eps_lu: relative solution difference <= 1e-10,
    identical augmented ranks, colours, block pattern and prefix-sum offsets;
  * float32 factor + float64 refinement: backward error ||Ax-b||/(||A|| ||x||) <= 1e-10,
    measured with the oracle's own H^2 matvec;
  * float64 H^2 matvec: relative difference <= 1e-13.
"""
import functools

import numpy as np
import pytest
import torch

from h2gen import rhs
from oracle import dense, rs

from conftest import problem

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
BERR_TOL = 1e-10


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_11152_b300 import build
    build.build()
    import paper_2509_11152_b300 as h2
    return h2


@functools.lru_cache(maxsize=None)
def dense_solution(name, nrhs, seed, **over):
    """A^-1 b of the expanded H^2 matrix (float64 LAPACK): the exact solution the
    refined results are compared with."""
    pb = problem(name, **over)
    A = pb.A.numpy()
    return np.linalg.solve(dense.expand(A), rhs(A.n, nrhs, seed=seed))


@functools.lru_cache(maxsize=None)
def oracle_solution(name, eps, nrhs, seed, **over):
    pb = problem(name, **over)
    A = pb.A.numpy()
    b = rhs(A.n, nrhs, seed=seed)
    Z = rs.factorize(A, eps, pb.norm_a)
    return pb, A, b, Z, rs.solve(Z, b)


CASES = [
    ("cov2d", dict(n=1024, leaf=32), 1e-8),
    ("cov2d", {}, 1e-8),                                  # the 4,096-point workload itself
    ("laplace2d", dict(n=4096, leaf=32, eta=0.7), 1e-6),
    ("matern3d", dict(n=2048, leaf=32), 1e-6),
    ("sphere", dict(n=4096, leaf=64), 1e-5),
    ("gauss3d", dict(n=1500, leaf=32), 1e-6),            # ragged leaves (46/47 points)
    ("helmholtz3d", dict(n=4096, leaf=64), 1e-6),         # indefinite oscillatory IE, 16^3 lattice
    ("lru3d", dict(n=4096, leaf=64), 1e-7),               # covariance + rank-32 update
    ("sphere", dict(n=8192), 1e-5),                       # the benchmark's leaf size (128)
    ("lru3d", dict(n=8192, leaf=128), 1e-7),              # level-2 boxes of up to 200 points
]
IDS = [f"{c[0]}-{c[1].get('n', 'full')}" for c in CASES]


def _gpu_solve(h, pb, b, eps, prec):
    M = h.h2_matrix_create(pb.A)
    Z = h.h2_factor_create(M, eps, pb.norm_a, prec)
    x = h.colmajor(torch.from_numpy(b).cuda())
    h.h2_solve(Z, x)
    return M, Z, x.cpu().numpy()


@pytest.mark.parametrize("name,over,eps", CASES, ids=IDS)
def test_fp64_factor_solve_matches_oracle(h, name, over, eps):
    pb, A, b, Z0, x0 = oracle_solution(name, eps, 2, 1, **over)
    M, Z, x = _gpu_solve(h, pb, b, eps, h.H2_PREC_FP64)
    rel = np.linalg.norm(x - x0) / np.linalg.norm(x0)
    assert rel <= FP64_TOL, rel
    st = h.h2_factor_stats_get(Z)
    assert st["nlevels"] == len(Z0.levels)
    assert st["top_size"] == sum(Z0.top_sizes)
    for li, lv in enumerate(Z0.levels):
        lay = h.h2_layout_get(Z, li)
        assert np.array_equal(lay["sizes"], np.asarray(lv.sizes))
        assert np.array_equal(lay["ranks"], np.asarray([bx.kt for bx in lv.boxes]))
        assert np.array_equal(lay["colour"], np.asarray(lv.colour, np.int32))
        assert np.array_equal(lay["row_ptr"], lv.layout["row_ptr"])
        assert np.array_equal(lay["col"], lv.layout["col"])
        assert np.array_equal(lay["kind"], lv.layout["kind"].astype(np.int32))
        assert np.array_equal(lay["offset"], lv.layout["offset"])


@pytest.mark.parametrize("prec", ["fp32", "tf32x3"])
@pytest.mark.parametrize("name,over,eps", CASES, ids=IDS)
def test_fp32_factor_with_refinement(h, name, over, eps, prec):
    pb, A, b, Z0, x0 = oracle_solution(name, eps, 2, 1, **over)
    M = h.h2_matrix_create(pb.A)
    Z = h.h2_factor_create(M, eps, pb.norm_a, h.H2_PREC_FP32 if prec == "fp32" else h.H2_PREC_TF32X3)
    bt = h.colmajor(torch.from_numpy(b).cuda())
    xt = h.colmajor(torch.zeros_like(bt))
    it, berr, ok = h.h2_refine_solve(Z, M, bt, xt, BERR_TOL, 30)
    x = xt.cpu().numpy()
    # the error against the float64 oracle, stated for every result: the unrefined
    # solve against the oracle's (same algorithm and eps_lu, float64), the refined
    # solution against the exact solve of the H^2 matrix
    x1 = h.colmajor(torch.from_numpy(b).cuda())
    h.h2_solve(Z, x1)
    e_solve = np.linalg.norm(x1.cpu().numpy() - x0) / np.linalg.norm(x0)
    xd = dense_solution(name, 2, 1, **over)
    e_ref = np.linalg.norm(x - xd) / np.linalg.norm(xd)
    msg = (f"{name} {prec}: {it} corrections, berr {berr:.2e}; solve vs oracle solve {e_solve:.2e}, "
           f"refined vs exact {e_ref:.2e}")
    print(msg)
    assert ok and berr <= BERR_TOL, msg
    nw, _ = dense.backward_error(A, x, b, pb.norm_a)       # the oracle's own matvec
    assert nw <= BERR_TOL, (nw, msg)
    # ranks of the float32 factor stay those of the float64 oracle almost everywhere
    lay = h.h2_layout_get(Z, 0)
    r0 = np.asarray([bx.kt for bx in Z0.levels[0].boxes])
    assert np.mean(lay["ranks"] == r0) > 0.9


W_CASES = [CASES[0], CASES[4], CASES[5], CASES[9]]       # cov2d, sphere, gauss3d (ragged), lru3d (200-point boxes)


@pytest.mark.parametrize("prec,flag", [("fp64", "inverse"), ("fp32", "inverse"), ("tf32x3", "triangular")])
@pytest.mark.parametrize("name,over,eps", W_CASES, ids=[f"{c[0]}-{c[1].get('n', 'full')}" for c in W_CASES])
def test_w_step_override_matches_oracle(h, name, over, eps, prec, flag):
    """The non-default application of D_RR^-1 (explicit inverse for FP64 / FP32,
    triangular solves for TF32X3): same bars as the default paths."""
    from paper_2509_11152_b300 import binding
    pb, A, b, Z0, x0 = oracle_solution(name, eps, 2, 1, **over)
    M = h.h2_matrix_create(pb.A)
    fl = binding.H2_FLAG_W_INVERSE if flag == "inverse" else binding.H2_FLAG_W_TRIANGULAR
    p = {"fp64": h.H2_PREC_FP64, "fp32": h.H2_PREC_FP32, "tf32x3": h.H2_PREC_TF32X3}[prec]
    Z = h.h2_factor_create(M, eps, pb.norm_a, p, flags=fl)
    if prec == "fp64":
        x = h.colmajor(torch.from_numpy(b).cuda())
        h.h2_solve(Z, x)
        rel = np.linalg.norm(x.cpu().numpy() - x0) / np.linalg.norm(x0)
        assert rel <= FP64_TOL, rel
        lay = h.h2_layout_get(Z, 0)
        assert np.array_equal(lay["ranks"], np.asarray([bx.kt for bx in Z0.levels[0].boxes]))
        return
    bt = h.colmajor(torch.from_numpy(b).cuda())
    xt = h.colmajor(torch.zeros_like(bt))
    it, berr, ok = h.h2_refine_solve(Z, M, bt, xt, BERR_TOL, 30)
    x = xt.cpu().numpy()
    xd = dense_solution(name, 2, 1, **over)
    e_ref = np.linalg.norm(x - xd) / np.linalg.norm(xd)
    msg = f"{name} {prec} {flag}: {it} corrections, berr {berr:.2e}, refined vs exact {e_ref:.2e}"
    print(msg)
    assert ok and berr <= BERR_TOL, msg
    nw, _ = dense.backward_error(A, x, b, pb.norm_a)
    assert nw <= BERR_TOL, (nw, msg)


def test_w_step_flags_exclude_each_other(h):
    from paper_2509_11152_b300 import binding
    pb = problem("cov2d", n=1024, leaf=32)
    M = h.h2_matrix_create(pb.A)
    with pytest.raises(Exception):
        h.h2_factor_create(M, 1e-8, pb.norm_a, h.H2_PREC_FP32,
                           flags=binding.H2_FLAG_W_INVERSE | binding.H2_FLAG_W_TRIANGULAR)


@pytest.mark.parametrize("name,over", [("cov2d", dict(n=1024, leaf=32)), ("sphere", dict(n=4096, leaf=64)),
                                       ("gauss3d", dict(n=1500, leaf=32))])
def test_matvec_matches_oracle(h, name, over):
    pb = problem(name, **over)
    A = pb.A.numpy()
    x = rhs(A.n, 3, seed=5)
    y0 = dense.matvec(A, x)
    M = h.h2_matrix_create(pb.A)
    xt = h.colmajor(torch.from_numpy(x).cuda())
    yt = h.colmajor(torch.zeros_like(xt))
    h.h2_matvec(M, xt, yt)
    y = yt.cpu().numpy()
    assert np.linalg.norm(y - y0) / np.linalg.norm(y0) <= 1e-13


def test_zero_truncation_matches_dense_solve(h):
    pb = problem("cov2d", n=1024, leaf=32)
    A = pb.A.numpy()
    b = rhs(A.n, 2, seed=3)
    xd = np.linalg.solve(dense.expand(A), b)
    _, _, x = _gpu_solve(h, pb, b, 1e-13, h.H2_PREC_FP64)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 1e-11


def test_no_admissible_block_is_dense_lu(h):
    pb = problem("cov2d", n=256, leaf=16, eta=1e-6)
    A = pb.A.numpy()
    assert A.top_level() is None
    b = rhs(A.n, 2, seed=4)
    xd = np.linalg.solve(dense.expand(A), b)
    M, Z, x = _gpu_solve(h, pb, b, 1e-6, h.H2_PREC_FP64)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 1e-13
    assert h.h2_factor_stats_get(Z)["nlevels"] == 0


def test_single_box_depth_zero(h):
    pb = problem("cov2d", n=50, leaf=64)
    assert pb.A.depth == 0
    A = pb.A.numpy()
    b = rhs(A.n, 1, seed=6)
    xd = np.linalg.solve(dense.expand(A), b)
    _, _, x = _gpu_solve(h, pb, b, 1e-8, h.H2_PREC_FP64)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 1e-13


def test_many_rhs_and_host_pointers(h):
    name, over, eps = "laplace2d", dict(n=4096, leaf=32, eta=0.7), 1e-6
    pb, A, b, Z0, x0 = oracle_solution(name, eps, 8, 2, **over)
    M = h.h2_matrix_create(pb.A)
    Z = h.h2_factor_create(M, eps, pb.norm_a, h.H2_PREC_FP64)
    xh = h.colmajor(torch.from_numpy(b))              # host memory: copied by the library
    h.h2_solve(Z, xh)
    xd = h.colmajor(torch.from_numpy(b).cuda())
    h.h2_solve(Z, xd)
    assert np.array_equal(xh.numpy(), xd.cpu().numpy())
    assert np.linalg.norm(xh.numpy() - x0) / np.linalg.norm(x0) <= FP64_TOL


def test_refinement_without_corrections_reports_no_convergence(h):
    pb = problem("cov2d", n=1024, leaf=32)
    M = h.h2_matrix_create(pb.A)
    Z = h.h2_factor_create(M, 1e-4, pb.norm_a, h.H2_PREC_FP32)
    b = torch.from_numpy(rhs(pb.A.n, 1, seed=7)).cuda()
    x = torch.zeros_like(b)
    it, berr, ok = h.h2_refine_solve(Z, M, b, x, 1e-14, 0)
    assert not ok and it == 0 and 1e-12 < berr < 1e-2


def test_singular_matrix_reports_error_and_context_survives(h):
    pb = problem("cov2d", n=512, leaf=32)
    Azero = pb.A.to("cpu")
    Azero.D = torch.zeros_like(Azero.D)
    Azero.S = torch.zeros_like(Azero.S)
    M = h.h2_matrix_create(Azero)
    with pytest.raises(h.H2Error) as e:
        h.h2_factor_create(M, 1e-8, pb.norm_a, h.H2_PREC_FP64)
    assert e.value.code == -3                       # H2_ERR_SINGULAR
    # the CUDA context is still usable
    b = rhs(pb.A.n, 1, seed=8)
    _, _, x = _gpu_solve(h, pb, b, 1e-8, h.H2_PREC_FP64)
    assert np.isfinite(x).all()


def test_rank_cap_reports_and_a_sufficient_cap_factorises(h):
    """h2_factor_opts.k_cap: a cap below the largest augmented rank fails with
    H2_ERR_RANK_CAP (the context stays usable), the largest rank itself passes and gives
    the uncapped factor's solution (same ranks, same arithmetic)."""
    pb = problem("sphere", n=4096, leaf=64)
    M = h.h2_matrix_create(pb.A)
    Z0 = h.h2_factor_create(M, 1e-5, pb.norm_a, h.H2_PREC_FP64)
    kmax = max(int(h.h2_layout_get(Z0, lv)["ranks"].max()) for lv in range(h.h2_factor_stats_get(Z0)["nlevels"]))
    assert kmax > 1
    with pytest.raises(h.H2Error) as e:
        h.h2_factor_create(M, 1e-5, pb.norm_a, h.H2_PREC_FP64, k_cap=kmax - 1)
    assert e.value.code == -4                       # H2_ERR_RANK_CAP
    Z = h.h2_factor_create(M, 1e-5, pb.norm_a, h.H2_PREC_FP64, k_cap=kmax)
    b = rhs(pb.A.n, 1, seed=13)
    x0 = h.colmajor(torch.from_numpy(b).cuda())
    x1 = h.colmajor(torch.from_numpy(b).cuda())
    h.h2_solve(Z0, x0)
    h.h2_solve(Z, x1)
    assert (torch.linalg.norm(x0 - x1) / torch.linalg.norm(x0)).item() <= 1e-12


def test_gmres_refinement_when_plain_corrections_stall(h):
    """A loose eps_lu on an ill-conditioned Gaussian-kernel matrix: plain corrections
    stop contracting and the refinement continues with preconditioned GMRES cycles;
    the backward error is checked with the oracle's own matvec."""
    pb = problem("gauss3d", n=4096, leaf=32)
    A = pb.A.numpy()
    M = h.h2_matrix_create(pb.A)
    Z = h.h2_factor_create(M, 1e-2, pb.norm_a, h.H2_PREC_TF32X3)
    b = rhs(A.n, 2, seed=9)
    bt = h.colmajor(torch.from_numpy(b).cuda())
    xt = h.colmajor(torch.zeros_like(bt))
    it, berr, ok = h.h2_refine_solve(Z, M, bt, xt, BERR_TOL, 60)
    assert ok and berr <= BERR_TOL and it > 3
    nw, _ = dense.backward_error(A, xt.cpu().numpy(), b, pb.norm_a)
    assert nw <= BERR_TOL


def test_schur_pipeline_timeout_is_reported_and_context_survives(h):
    """The tensor-core Schur kernel's bounded waits: with H2_FLAG_DEBUG_SHORT_WAIT every
    pipeline wait gives up after one cycle (the wait for the MMAs already issued keeps
    its full budget), so the factorisation fails with H2_ERR_TIMEOUT instead of hanging,
    and the library and the CUDA context stay usable."""
    name, over, eps = "sphere", dict(n=4096, leaf=64), 1e-5
    pb, A, b, Z0, x0 = oracle_solution(name, eps, 2, 1, **over)
    M = h.h2_matrix_create(pb.A)
    from paper_2509_11152_b300 import binding
    with pytest.raises(h.H2Error) as e:
        h.h2_factor_create(M, eps, pb.norm_a, h.H2_PREC_TF32X3, flags=binding.H2_FLAG_DEBUG_SHORT_WAIT)
    assert e.value.code == -7                       # H2_ERR_TIMEOUT
    Z = h.h2_factor_create(M, eps, pb.norm_a, h.H2_PREC_TF32X3)
    bt = h.colmajor(torch.from_numpy(b).cuda())
    xt = h.colmajor(torch.zeros_like(bt))
    it, berr, ok = h.h2_refine_solve(Z, M, bt, xt, BERR_TOL, 30)
    assert ok and berr <= BERR_TOL


@pytest.mark.parametrize("prec", ["fp32", "tf32x3"])
@pytest.mark.parametrize("name,over,eps", [CASES[4], CASES[5], CASES[9]], ids=[IDS[4], IDS[5], IDS[9]])
def test_reduced_precision_layout_matches_oracle_under_forced_ranks(h, name, over, eps, prec):
    """With the oracle's augmented ranks forced (opts.force_ranks), a float32 factor's
    level sizes, ranks, colours, block pattern and prefix-sum offsets equal the
    oracle's entry by entry, and the factor still refines to the float64 target."""
    pb, A, b, Z0, x0 = oracle_solution(name, eps, 2, 1, **over)
    ranks = [np.asarray([bx.kt for bx in lv.boxes], np.int32) for lv in Z0.levels]
    M = h.h2_matrix_create(pb.A)
    Z = h.h2_factor_create(M, eps, pb.norm_a, h.H2_PREC_FP32 if prec == "fp32" else h.H2_PREC_TF32X3,
                           force_ranks=ranks)
    st = h.h2_factor_stats_get(Z)
    assert st["nlevels"] == len(Z0.levels) and st["top_size"] == sum(Z0.top_sizes)
    for li, lv in enumerate(Z0.levels):
        lay = h.h2_layout_get(Z, li)
        assert np.array_equal(lay["sizes"], np.asarray(lv.sizes)), li
        assert np.array_equal(lay["ranks"], ranks[li]), li
        assert np.array_equal(lay["colour"], np.asarray(lv.colour, np.int32)), li
        assert np.array_equal(lay["row_ptr"], lv.layout["row_ptr"]), li
        assert np.array_equal(lay["col"], lv.layout["col"]), li
        assert np.array_equal(lay["kind"], lv.layout["kind"].astype(np.int32)), li
        assert np.array_equal(lay["offset"], lv.layout["offset"]), li
    bt = h.colmajor(torch.from_numpy(b).cuda())
    xt = h.colmajor(torch.zeros_like(bt))
    it, berr, ok = h.h2_refine_solve(Z, M, bt, xt, BERR_TOL, 30)
    assert ok and berr <= BERR_TOL, (it, berr)
