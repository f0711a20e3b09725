"""H^2 matrix construction for the test problems (Sec. 3): Chebyshev interpolation
on the bounding boxes of the clusters, then algebraic compression to a tolerance
with orthonormal nested bases.

Steps (the construction the paper takes from Borm & Garcke, ref. borm07):

1. Interpolation.  Order ``p_l = p0 + floor((d-l)/2)`` at level ``l`` (raised every
   other level going up).  Leaf basis = tensor Lagrange polynomials of the leaf box
   evaluated at its points; transfer ``E_c`` = parent's Lagrange polynomials at the
   child's Chebyshev nodes; coupling ``S_st = K(xi_s, xi_t)``.
2. Orthogonalisation, leaves to root: ``U = QR``; inner nodes QR the stacked
   ``[R_c1 E_c1; R_c2 E_c2]``; couplings become ``R_s S R_t^T``.
3. Compression: total far-field weights top-down (``W_t`` = R-factor of
   ``[E_t W_parent, S_t,s ...]``), then truncated SVDs leaves to root keeping
   ``sigma_j > eps * sigma_1`` per cluster, with the new bases nested in the new
   child bases; couplings are projected onto the new bases.

A global low-rank update ``W W^T`` (the paper's LRU problem, Sec. 3) enters at step 1
as ``q`` extra basis columns per cluster (identity transfers and couplings) and in
the near-field blocks, and is compressed together with the kernel part.

The result is a symmetric H^2 matrix with orthonormal nested bases:
``A_st = U_s S_st U_t^T`` on admissible pairs and dense near-field blocks on the
inadmissible leaf pairs.  Everything is float64 torch on a chosen device.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import torch

from .kernels import Kernel, near_block
from .tree import BlockPartition, ClusterTree


# ---------------------------------------------------------------- interpolation
def _cheb_nodes(p: int, dev) -> torch.Tensor:
    a = torch.arange(p, dtype=torch.float64, device=dev)
    return torch.cos((2.0 * a + 1.0) * math.pi / (2.0 * p))


def _lagrange_1d(xhat: torch.Tensor, nodes: torch.Tensor) -> torch.Tensor:
    """``l_a(xhat)`` for all nodes ``a``: shape ``xhat.shape + (p,)``."""
    p = nodes.numel()
    diff = xhat.unsqueeze(-1) - nodes            # (..., p)
    out = []
    for a in range(p):
        num = torch.ones_like(xhat)
        for b in range(p):
            if b != a:
                num = num * diff[..., b] / (nodes[a] - nodes[b])
        out.append(num)
    return torch.stack(out, dim=-1)


def _multi_index(p: int, dim: int) -> np.ndarray:
    return np.array(list(itertools.product(range(p), repeat=dim)), dtype=np.int64)


def _box_map(lo: torch.Tensor, hi: torch.Tensor):
    """Centre and half-width of boxes, with degenerate sides widened."""
    c = 0.5 * (lo + hi)
    h = 0.5 * (hi - lo)
    scale = torch.clamp(h.max(), min=1e-300)
    h = torch.clamp(h, min=1e-9 * float(scale))
    return c, h


def _lagrange_nd(x: torch.Tensor, c: torch.Tensor, h: torch.Tensor, p: int) -> torch.Tensor:
    """Tensor Lagrange basis of order ``p`` on boxes (c, h) at points ``x``.
    ``x``: (B, n, dim), ``c``/``h``: (B, dim)  ->  (B, n, p^dim)."""
    dim = x.shape[-1]
    nodes = _cheb_nodes(p, x.device)
    xhat = (x - c.unsqueeze(1)) / h.unsqueeze(1)
    l1 = [_lagrange_1d(xhat[..., k], nodes) for k in range(dim)]   # each (B, n, p)
    mi = torch.as_tensor(_multi_index(p, dim), device=x.device)
    out = l1[0][..., mi[:, 0]]
    for k in range(1, dim):
        out = out * l1[k][..., mi[:, k]]
    return out


def _cheb_points(c: torch.Tensor, h: torch.Tensor, p: int) -> torch.Tensor:
    """Tensor Chebyshev grid on boxes: (B, dim) -> (B, p^dim, dim)."""
    dim = c.shape[-1]
    nodes = _cheb_nodes(p, c.device)
    mi = torch.as_tensor(_multi_index(p, dim), device=c.device)
    ref = torch.stack([nodes[mi[:, k]] for k in range(dim)], dim=-1)  # (k0, dim)
    return c.unsqueeze(1) + h.unsqueeze(1) * ref.unsqueeze(0)


# ---------------------------------------------------------------- helpers
def _qr(x: torch.Tensor, mode: str = "reduced"):
    """Batched QR; small dense factorisations run on the host (batched CUDA QR of
    many small matrices is far slower than LAPACK on the CPU)."""
    q, r = torch.linalg.qr(x.cpu(), mode=mode)
    return q.to(x.device), r.to(x.device)


def _svd(x: torch.Tensor):
    u, s, vh = torch.linalg.svd(x.cpu(), full_matrices=False)
    return u.to(x.device), s.to(x.device), vh.to(x.device)


def _level_ids(l: int) -> np.ndarray:
    return np.arange((1 << l) - 1, (1 << (l + 1)) - 1)


def _pad_points(pts: torch.Tensor, tree: ClusterTree, ids: np.ndarray, mmax: int):
    """Points of nodes ``ids`` gathered to (B, mmax, dim), zero padded, + sizes."""
    dev = pts.device
    st = torch.as_tensor(tree.start[ids], device=dev)
    sz = torch.as_tensor(tree.size[ids], device=dev)
    ar = torch.arange(mmax, device=dev)
    idx = st.unsqueeze(1) + ar.unsqueeze(0)
    valid = ar.unsqueeze(0) < sz.unsqueeze(1)
    idx = torch.where(valid, idx, torch.zeros_like(idx))
    out = pts[idx]
    out = out * valid.unsqueeze(-1)
    return out, valid


class _Pairs:
    """Admissible pairs of one level, grouped by row for padded batching."""

    def __init__(self, pairs: np.ndarray, first: int, cnt: int):
        self.pairs = pairs
        rows = pairs[:, 0] - first if len(pairs) else np.zeros(0, np.int64)
        self.deg = np.bincount(rows, minlength=cnt) if len(pairs) else np.zeros(cnt, np.int64)
        self.ptr = np.concatenate([[0], np.cumsum(self.deg)])
        self.maxdeg = int(self.deg.max()) if cnt else 0


class _Clock:
    """Wall-clock per construction phase (synchronising the device)."""

    def __init__(self, dev):
        self.dev = dev
        self.t = {}
        self.t0 = self._now()

    def _now(self):
        if self.dev.type == "cuda":
            torch.cuda.synchronize(self.dev)
        import time
        return time.perf_counter()

    def lap(self, name):
        now = self._now()
        self.t[name] = self.t.get(name, 0.0) + now - self.t0
        self.t0 = now


def construct_h2(points: np.ndarray, tree: ClusterTree, part: BlockPartition, kern: Kernel,
                 p0: int, eps: float, device="cpu", chunk: int = 2048, lowrank: np.ndarray | None = None):
    """Build the H^2 matrix; returns a dict of per-level padded tensors (see
    ``h2matrix.H2Matrix.from_levels``).

    ``lowrank`` (n x q, original point order) adds the update ``W W^T`` to the whole
    matrix.  Every cluster's interpolation basis is extended by its rows of ``W``
    (``[L_t, W_t]``), so transfers become ``diag(E, I_q)`` and couplings
    ``diag(S, I_q)``, and the near-field blocks get ``W_s W_t^T``; the
    orthogonalisation and compression below then treat it like any other basis."""
    dev = torch.device(device)
    clock = _Clock(dev)
    d = tree.depth
    dim = points.shape[1]
    pts = torch.as_tensor(points[tree.perm], dtype=torch.float64, device=dev)
    lo = torch.as_tensor(tree.lo, dtype=torch.float64, device=dev)
    hi = torch.as_tensor(tree.hi, dtype=torch.float64, device=dev)
    order = [p0 + (d - l) // 2 for l in range(d + 1)]
    k0 = [p ** dim for p in order]
    centre, half = _box_map(lo, hi)
    leaf_ids = _level_ids(d)
    mmax = int(tree.size[leaf_ids].max())

    # ---- 1+2: interpolation and orthogonalisation, leaves to root
    xl, _ = _pad_points(pts, tree, leaf_ids, mmax)
    L0 = _lagrange_nd(xl, centre[leaf_ids], half[leaf_ids], order[d])   # (nl, mmax, k0)
    _, valid = _pad_points(pts, tree, leaf_ids, mmax)
    L0 = L0 * valid.unsqueeze(-1)
    q = 0
    if lowrank is not None:
        Wt = torch.as_tensor(lowrank[tree.perm], dtype=torch.float64, device=dev)   # tree order
        q = Wt.shape[1]
        Wl, _ = _pad_points(Wt, tree, leaf_ids, mmax)                              # zero padded
        L0 = torch.cat([L0, Wl], dim=2)

    def with_identity(X):
        """``diag(X, I_q)`` for a batch of matrices (X itself when q = 0)."""
        if q == 0:
            return X
        out = torch.zeros(X.shape[:-2] + (X.shape[-2] + q, X.shape[-1] + q), dtype=X.dtype, device=dev)
        out[..., :X.shape[-2], :X.shape[-1]] = X
        out[..., X.shape[-2]:, X.shape[-1]:] = torch.eye(q, dtype=X.dtype, device=dev)
        return out
    Uq, Rr = _qr(L0)
    U = {d: Uq}                   # orthonormal leaf basis (nl, mmax, r_d)
    R = {d: Rr}                   # (cnt, r_l, k0_l)
    E = {}                        # E[l]: (cnt_l, r_l, r_{l-1}) orthonormal transfers
    for l in range(d, 0, -1):
        ids = _level_ids(l)
        par = _level_ids(l - 1)
        # parent Lagrange polynomials at child Chebyshev nodes
        xi = _cheb_points(centre[ids], half[ids], order[l])             # (cnt, k0_l, dim)
        pidx = torch.as_tensor((ids - 1) // 2, device=dev)
        E0 = with_identity(_lagrange_nd(xi, centre[pidx], half[pidx], order[l - 1]))   # (cnt, k0_l, k0_{l-1})
        RE = R[l] @ E0                                                  # (cnt, r_l, k0_{l-1})
        stacked = torch.cat([RE[0::2], RE[1::2]], dim=1)                # (cntp, 2 r_l, k0_{l-1})
        Qp, Rp = _qr(stacked)
        r_l = RE.shape[1]
        E[l] = torch.stack([Qp[:, :r_l], Qp[:, r_l:]], dim=1).reshape(len(ids), r_l, Qp.shape[2])
        R[l - 1] = Rp

    def coupling(l, pr):
        """Orthogonalised couplings ``R_s S0 R_t^T`` for pairs ``pr`` (global ids)."""
        s = torch.as_tensor(pr[:, 0], device=dev)
        t = torch.as_tensor(pr[:, 1], device=dev)
        xs = _cheb_points(centre[s], half[s], order[l])
        xt = _cheb_points(centre[t], half[t], order[l])
        S0 = with_identity(kern(torch.cdist(xs, xt, compute_mode="donot_use_mm_for_euclid_dist")))
        first = (1 << l) - 1
        Rs = R[l][s - first]
        Rt = R[l][t - first]
        return Rs @ S0 @ Rt.transpose(1, 2)

    clock.lap("orthogonalise")
    # ---- 3a: total far-field weights, root to leaves
    W = {0: torch.zeros((1, R[0].shape[1], R[0].shape[1]), dtype=torch.float64, device=dev)}
    for l in range(1, d + 1):
        ids = _level_ids(l)
        first = ids[0]
        cnt = len(ids)
        pa = _Pairs(part.adm[l], first, cnt)
        r_l = R[l].shape[1]
        Wl = torch.zeros((cnt, r_l, r_l), dtype=torch.float64, device=dev)
        step = max(1, min(chunk, (1 << 28) // max(1, (pa.maxdeg + 1) * r_l * r_l)))
        for c0 in range(0, cnt, step):
            c1 = min(cnt, c0 + step)
            rows = np.arange(c0, c1)
            inherit = E[l][rows] @ W[l - 1][torch.as_tensor(rows // 2, device=dev)]
            cols = [inherit]
            md = int(pa.deg[c0:c1].max()) if c1 > c0 else 0
            if md:
                sel = np.concatenate([np.arange(pa.ptr[r], pa.ptr[r + 1]) for r in rows])
                Sx = coupling(l, pa.pairs[sel])
                slot = np.concatenate([np.arange(pa.deg[r]) for r in rows])
                rloc = np.concatenate([np.full(pa.deg[r], r - c0) for r in rows])
                G = torch.zeros((c1 - c0, md, r_l, r_l), dtype=torch.float64, device=dev)
                G[torch.as_tensor(rloc, device=dev), torch.as_tensor(slot, device=dev)] = Sx
                cols.append(G.permute(0, 2, 1, 3).reshape(c1 - c0, r_l, md * r_l))
            Gt = torch.cat(cols, dim=2).transpose(1, 2)                  # (B, q, r_l)
            if Gt.shape[1] < r_l:
                Gt = torch.cat([Gt, torch.zeros((Gt.shape[0], r_l - Gt.shape[1], r_l),
                                                dtype=Gt.dtype, device=dev)], dim=1)
            Rg = torch.linalg.qr(Gt.cpu(), mode="r")[1].to(dev)          # (B, r_l, r_l)
            Wl[c0:c1] = Rg.transpose(1, 2)
        W[l] = Wl

    clock.lap("weights")
    # ---- 3b: truncation, leaves to root
    rank = {}
    P = {}                       # P[l]: (cnt, rows_l, kpad_l) new basis in child coords
    B = {}                       # B[l]: (cnt, r_l, kpad_l) = U_old^T U_new
    for l in range(d, -1, -1):
        ids = _level_ids(l)
        cnt = len(ids)
        if l == d:
            M = W[d]
        else:
            Bc = B[l + 1]                                                 # (2cnt, r_c, kpc)
            Ehat = Bc.transpose(1, 2) @ E[l + 1]                          # (2cnt, kpc, r_l)
            Ehat = Ehat.reshape(cnt, 2 * Ehat.shape[1], Ehat.shape[2])
            M = Ehat @ W[l]
        Ul, sv, _ = _svd(M)
        keep = sv > eps * sv[:, :1]
        kk = keep.sum(dim=1)
        kpad = max(1, int(kk.max()))
        Pl = Ul[:, :, :kpad] * keep[:, :kpad].unsqueeze(1)
        rank[l] = kk.cpu().numpy().astype(np.int64)
        P[l] = Pl
        if l == d:
            B[l] = Pl
        else:
            Ec = E[l + 1].reshape(cnt, 2, E[l + 1].shape[1], E[l + 1].shape[2])
            Bc = B[l + 1].reshape(cnt, 2, B[l + 1].shape[1], B[l + 1].shape[2])
            kpc = Bc.shape[3]
            B[l] = (Ec[:, 0].transpose(1, 2) @ Bc[:, 0] @ Pl[:, :kpc]
                    + Ec[:, 1].transpose(1, 2) @ Bc[:, 1] @ Pl[:, kpc:])

    clock.lap("truncate")
    # ---- outputs: new leaf bases, transfers and couplings (padded per level)
    Unew = U[d] @ P[d]                                                   # (nl, mmax, kpad_d)
    Enew = {}
    for l in range(d, 0, -1):
        kpc = P[l].shape[2]
        Pp = P[l - 1]                                                    # (cntp, 2 kpc, kpp)
        Enew[l] = torch.stack([Pp[:, :kpc], Pp[:, kpc:]], dim=1).reshape(
            2 * Pp.shape[0], kpc, Pp.shape[2])
    Snew = {}
    for l in range(1, d + 1):
        pr = part.adm[l]
        if not len(pr):
            continue
        first = (1 << l) - 1
        outs = []
        for c0 in range(0, len(pr), chunk * 8):
            sub = pr[c0:c0 + chunk * 8]
            S = coupling(l, sub)
            Bs = B[l][torch.as_tensor(sub[:, 0] - first, device=dev)]
            Bt = B[l][torch.as_tensor(sub[:, 1] - first, device=dev)]
            outs.append(Bs.transpose(1, 2) @ S @ Bt)
        Snew[l] = torch.cat(outs, dim=0)

    clock.lap("couplings")
    # dense near field on inadmissible leaf pairs
    inad = part.inad[d]
    Dn = []
    for c0 in range(0, len(inad), chunk * 4):
        sub = inad[c0:c0 + chunk * 4]
        xs, vs = _pad_points(pts, tree, sub[:, 0], mmax)
        xt, vt = _pad_points(pts, tree, sub[:, 1], mmax)
        same = torch.as_tensor(sub[:, 0] == sub[:, 1], device=dev)
        blk = near_block(kern, xs, xt, same=False)
        blk_same = near_block(kern, xs, xt, same=True)
        blk = torch.where(same.view(-1, 1, 1), blk_same, blk)
        if q:
            Ws, _ = _pad_points(Wt, tree, sub[:, 0], mmax)
            Wu, _ = _pad_points(Wt, tree, sub[:, 1], mmax)
            blk = blk + Ws @ Wu.transpose(1, 2)
        blk = blk * (vs.unsqueeze(2) & vt.unsqueeze(1))
        Dn.append(blk)
    Dnear = torch.cat(Dn, dim=0) if Dn else torch.zeros((0, mmax, mmax), dtype=torch.float64, device=dev)
    clock.lap("near_field")
    return dict(rank=rank, U=Unew, E=Enew, S=Snew, D=Dnear, mmax=mmax, seconds=clock.t)


def matvec_levels(tree: ClusterTree, part: BlockPartition, lev: dict, x: torch.Tensor) -> torch.Tensor:
    """``y = A x`` on the padded per-level representation returned by
    :func:`construct_h2` (x in tree order, shape (n, nrhs)); batched over every
    level so it stays fast at a million unknowns."""
    d = tree.depth
    dev = x.device
    leaf_ids = _level_ids(d)
    mmax = lev["mmax"]
    nrhs = x.shape[1]
    st = torch.as_tensor(tree.start[leaf_ids], device=dev)
    sz = torch.as_tensor(tree.size[leaf_ids], device=dev)
    ar = torch.arange(mmax, device=dev)
    idx = st.unsqueeze(1) + ar.unsqueeze(0)
    valid = ar.unsqueeze(0) < sz.unsqueeze(1)
    idx = torch.where(valid, idx, torch.zeros_like(idx))
    xl = x[idx] * valid.unsqueeze(-1)                                   # (nl, mmax, nrhs)
    xh = {d: lev["U"].transpose(1, 2) @ xl}
    for l in range(d, 0, -1):
        up = lev["E"][l].transpose(1, 2) @ xh[l]                        # (cnt_l, kp_{l-1}, nrhs)
        xh[l - 1] = up[0::2] + up[1::2]
    yh = {}
    for l in range(d + 1):
        first = (1 << l) - 1
        acc = torch.zeros_like(xh[l])
        if l in lev["S"]:
            pr = part.adm[l]
            s = torch.as_tensor(pr[:, 0] - first, device=dev)
            t = torch.as_tensor(pr[:, 1] - first, device=dev)
            acc.index_add_(0, s, lev["S"][l] @ xh[l][t])
        if l > 0:
            acc += lev["E"][l] @ yh[l - 1].repeat_interleave(2, dim=0)
        yh[l] = acc
    yl = lev["U"] @ yh[d]
    near = part.inad[d]
    first = (1 << d) - 1
    s = torch.as_tensor(near[:, 0] - first, device=dev)
    t = torch.as_tensor(near[:, 1] - first, device=dev)
    yl.index_add_(0, s, lev["D"] @ xl[t])
    y = torch.zeros((x.shape[0], nrhs), dtype=x.dtype, device=dev)
    y.index_put_((idx[valid],), yl[valid], accumulate=True)
    return y


def spectral_norm(tree: ClusterTree, part: BlockPartition, lev: dict, iters: int = 50,
                  seed: int = 0) -> float:
    """``||A||_2`` of the (symmetric) H^2 matrix by power iteration from a seeded
    N(0,1) start vector."""
    dev = lev["U"].device
    g = torch.Generator(device="cpu").manual_seed(seed)
    v = torch.randn((int(tree.size[0]), 1), generator=g, dtype=torch.float64).to(dev)
    v /= torch.linalg.norm(v)
    lam = 0.0
    for _ in range(iters):
        w = matvec_levels(tree, part, lev, v)
        lam = float(torch.linalg.norm(w))
        if lam == 0.0:
            break
        v = w / lam
    return lam
