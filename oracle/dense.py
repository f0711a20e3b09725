"""Oracle: dense reference operations on an H^2 matrix (plain float64 numpy).

Test infrastructure only.  ``expand`` writes out the matrix the H^2 format defines
(Sec. 1.1): ``U_s S_st U_t^T`` on admissible pairs, with the nested bases
``U_p = diag(U_c1, U_c2) [E_c1; E_c2]``, and the dense near-field blocks on the
inadmissible leaf pairs.  ``matvec`` applies the same matrix without expanding it
(upsweep, couplings, downsweep, near field).  ``backward_error`` gives the two
error measures used for the solver: ``||Ax-b|| / (||A|| ||x||)`` and the paper's
``||Ax-b|| / ||b||`` (Sec. 3, "Solve").
"""
from __future__ import annotations

import numpy as np

from .rs import _blk


def _bases(A):
    d = A.depth
    nn = A.nnodes
    first_leaf = (1 << d) - 1
    U = [None] * nn
    for g in range(nn - 1, -1, -1):
        sz = int(A.node_size[g])
        k = int(A.rank[g])
        if g >= first_leaf:
            U[g] = _blk(A.U, A.U_off, g - first_leaf, sz, k)
        else:
            parts = []
            for c in (2 * g + 1, 2 * g + 2):
                Ec = _blk(A.E, A.E_off, c, int(A.rank[c]), k)
                parts.append(U[c] @ Ec)
            U[g] = np.vstack(parts)
    return U


def expand(A) -> np.ndarray:
    """Dense n x n matrix (tree order) defined by the H^2 representation."""
    n = A.n
    M = np.zeros((n, n))
    U = _bases(A)
    first_leaf = (1 << A.depth) - 1
    for g in range(A.nnodes):
        s0, ss = int(A.node_start[g]), int(A.node_size[g])
        for e in range(A.adm_ptr[g], A.adm_ptr[g + 1]):
            t = int(A.adm_col[e])
            t0, ts = int(A.node_start[t]), int(A.node_size[t])
            S = _blk(A.S, A.S_off, e, int(A.rank[g]), int(A.rank[t]))
            M[s0:s0 + ss, t0:t0 + ts] = U[g] @ S @ U[t].T
        if g >= first_leaf:
            base = A.inad_ptr[first_leaf]
            for e in range(A.inad_ptr[g], A.inad_ptr[g + 1]):
                t = int(A.inad_col[e])
                t0, ts = int(A.node_start[t]), int(A.node_size[t])
                M[s0:s0 + ss, t0:t0 + ts] = _blk(A.D, A.D_off, e - base, ss, ts)
    return M


def matvec(A, x: np.ndarray) -> np.ndarray:
    """``y = A x`` for x of shape (n, nrhs), tree order, float64."""
    x = np.asarray(x, dtype=np.float64).reshape(A.n, -1)
    nn = A.nnodes
    first_leaf = (1 << A.depth) - 1
    xh = [None] * nn
    for g in range(nn - 1, -1, -1):                          # upsweep
        k = int(A.rank[g])
        if g >= first_leaf:
            s0, ss = int(A.node_start[g]), int(A.node_size[g])
            xh[g] = _blk(A.U, A.U_off, g - first_leaf, ss, k).T @ x[s0:s0 + ss]
        else:
            xh[g] = sum(_blk(A.E, A.E_off, c, int(A.rank[c]), k).T @ xh[c]
                        for c in (2 * g + 1, 2 * g + 2))
    yh = [None] * nn
    for g in range(nn):                                      # couplings + downsweep
        k = int(A.rank[g])
        acc = np.zeros((k, x.shape[1]))
        for e in range(A.adm_ptr[g], A.adm_ptr[g + 1]):
            t = int(A.adm_col[e])
            acc += _blk(A.S, A.S_off, e, k, int(A.rank[t])) @ xh[t]
        if g > 0:
            p = (g - 1) // 2
            acc += _blk(A.E, A.E_off, g, k, int(A.rank[p])) @ yh[p]
        yh[g] = acc
    y = np.zeros_like(x)
    base = A.inad_ptr[first_leaf]
    for g in range(first_leaf, nn):                          # leaves + near field
        s0, ss = int(A.node_start[g]), int(A.node_size[g])
        y[s0:s0 + ss] += _blk(A.U, A.U_off, g - first_leaf, ss, int(A.rank[g])) @ yh[g]
        for e in range(A.inad_ptr[g], A.inad_ptr[g + 1]):
            t = int(A.inad_col[e])
            t0, ts = int(A.node_start[t]), int(A.node_size[t])
            y[s0:s0 + ss] += _blk(A.D, A.D_off, e - base, ss, ts) @ x[t0:t0 + ts]
    return y


def backward_error(A, x, b, norm_a: float) -> tuple[float, float]:
    """Max over right-hand sides of ``||Ax-b||/(||A|| ||x||)`` and ``||Ax-b||/||b||``."""
    x = np.asarray(x).reshape(A.n, -1)
    b = np.asarray(b).reshape(A.n, -1)
    r = matvec(A, x) - b
    rn = np.linalg.norm(r, axis=0)
    nw = rn / (norm_a * np.linalg.norm(x, axis=0))
    rel = rn / np.linalg.norm(b, axis=0)
    return float(nw.max()), float(rel.max())
