"""How the partial factorisation's redundant-block solves behave in float32 (a study
on the oracle; run it as a script, it takes a few minutes: `python
tests/study_partial_lu_precision.py`).

The float32 factor of the library forms D_RR^-1 explicitly (one inverse per box, then
W_U = D_RR^-1 D_{R,N}, W_L = D_{N,R} D_RR^-1 and the diagonal solve step as GEMMs).
Here the oracle's partial factorisation (Sec. 2.1, Eq. 2.1) is replaced by float32
variants, with the rest of the factor stored in float32 as in
tests/test_precision_study.py, and plain float64 refinement is run on the largest
member of the uneven Gaussian batch (N = 8192, leaf 64, eps_lu 1e-6):

  inv32    explicit inverse computed in float32, products in float32
  inv64    the float64 inverse rounded to float32, products in float32
  inv32ns  inv32 plus one Newton-Schulz step X + X (I - D_RR X) with the residual in float64
  lu32     float32 LU with partial pivoting and triangular solves (no inverse)

Result (recorded with this script): inv32 stalls at a backward error of 1.7e-6 (no
convergence in 40 corrections), inv64 and inv32ns need 18 corrections, lu32 needs 9
(as many as float32 storage with float64 arithmetic).  Multiplying by a rounded
inverse costs about cond(D_RR) * u, triangular solves do not; this is the float32
path's weak step on ill-conditioned problems.
"""
import os
import sys

import numpy as np
import pytest
import scipy.linalg as sla

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

from h2gen import rhs  # noqa: E402
from oracle import dense, rs  # noqa: E402

from conftest import problem  # noqa: E402
import test_precision_study as ps  # noqa: E402


def partial_lu_variant(variant):
    """The oracle's partial LU (pivot "lu") with the redundant-block solves in float32."""
    def partial_lu(i, n, r, nbrs, sizes, D, F, pivot="lu"):
        WL, WU = {}, {}
        lu = None
        if r == 0:
            return lu, WL, WU

        def rows_of(j):
            return slice(r, n) if j == i else slice(0, sizes[j])
        DRR = D[(i, i)][:r, :r]
        f32 = lambda a: np.asarray(a, np.float32)
        if variant == "lu32":
            lu32 = sla.lu_factor(f32(DRR))
            lu = sla.lu_factor(f32(DRR).astype(np.float64))          # the solve's diagonal step
            for j in nbrs[i]:
                WU[j] = sla.lu_solve(lu32, f32(D[(i, j)][:r, rows_of(j)])).astype(np.float64)
                WL[j] = sla.lu_solve(lu32, f32(D[(j, i)][rows_of(j), :r].T), trans=1).T.astype(np.float64)
        else:
            if variant == "inv32":
                X = np.linalg.inv(f32(DRR))
            elif variant == "inv64":
                X = f32(np.linalg.inv(DRR))
            elif variant == "inv32ns":
                X0 = np.linalg.inv(f32(DRR)).astype(np.float64)
                X = f32(X0 + X0 @ (np.eye(r) - DRR @ X0))
            else:
                raise ValueError(variant)
            lu = sla.lu_factor(np.linalg.inv(X.astype(np.float64)))  # applies X in the solve
            for j in nbrs[i]:
                WU[j] = (X @ f32(D[(i, j)][:r, rows_of(j)])).astype(np.float64)
                WL[j] = (f32(D[(j, i)][rows_of(j), :r]) @ X).astype(np.float64)
        for j in nbrs[i]:
            Dj = f32(D[(j, i)][rows_of(j), :r])
            for kk in nbrs[i]:
                upd = (Dj @ f32(WU[kk])).astype(np.float64)
                if (j, kk) in D:
                    D[(j, kk)][rows_of(j), rows_of(kk)] -= upd
                else:
                    F[(j, kk)][rows_of(j), rows_of(kk)] -= upd
        for j in nbrs[i]:
            D[(i, j)][:r, :] = 0.0
            D[(j, i)][:, :r] = 0.0
        return lu, WL, WU
    return partial_lu


def refine(variant, name="gauss3d", over=None, eps=1e-6, maxit=40):
    pb = problem(name, **(over or dict(n=8192)))
    A = pb.A.numpy()
    b = rhs(A.n, 1, seed=0)
    mp = pytest.MonkeyPatch()
    mp.setattr(rs, "_partial_lu", partial_lu_variant(variant))
    try:
        Z = ps._factor_in("fp32", A, eps, pb.norm_a, mp)
    finally:
        mp.undo()
    x = rs.solve(Z, b)
    for it in range(maxit + 1):
        r = b - dense.matvec(A, x)
        berr = float(np.linalg.norm(r) / (pb.norm_a * np.linalg.norm(x)))
        if berr <= 1e-10 or not np.isfinite(berr) or it == maxit:
            return it, berr
        x = x + rs.solve(Z, r)


if __name__ == "__main__":
    for v in ("inv32", "inv64", "inv32ns", "lu32"):
        it, berr = refine(v)
        print(f"{v:8s} corrections {it:2d}  backward error {berr:.1e}", flush=True)
