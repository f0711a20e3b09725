"""Flat, pointer-friendly storage of a symmetric H^2 matrix.

This is the interchange format between the input generator, the CPU oracle and
the CUDA library's C-ABI (``h2_matrix_desc``).  Nodes use heap numbering (level
``l`` = ids ``2^l-1 .. 2^(l+1)-2``); all dense blocks are column-major float64.

  node_start/node_size  tree-order index range of every node
  rank[g]               number of basis columns of node g
  U_off[leaf]           leaf basis U_i  (size_i x rank_i)
  E_off[g], g >= 1      transfer E_g    (rank_g x rank_parent(g)),  U_p|_g = U_g E_g
  adm_ptr/adm_col       admissible pairs per node (CSR over all nodes, same level)
  S_off[e]              coupling S_st   (rank_s x rank_t) of admissible entry e
  inad_ptr/inad_col     inadmissible pairs per node (CSR over all nodes, incl. self)
  D_off[e]              dense block     (size_s x size_t) of the e-th inadmissible
                        entry of a leaf row (leaf rows only, CSR order)
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch


def _flatten_blocks(blocks: torch.Tensor, rows, cols):
    """Concatenate the valid ``rows[b] x cols[b]`` top-left parts of padded blocks
    in column-major order.  Returns (data, offsets) with offsets of length B+1."""
    nb = blocks.shape[0]
    rows = torch.as_tensor(rows, device=blocks.device)
    cols = torch.as_tensor(cols, device=blocks.device)
    sizes = rows * cols
    off = torch.zeros(nb + 1, dtype=torch.int64, device=blocks.device)
    if nb:
        off[1:] = torch.cumsum(sizes, 0)
    if nb == 0:
        return blocks.new_zeros(0), off
    t = blocks.transpose(1, 2)                         # (B, cols, rows): col-major walk
    if bool((rows == blocks.shape[1]).all()) and bool((cols == blocks.shape[2]).all()):
        return t.reshape(-1).clone(), off
    ri = torch.arange(blocks.shape[1], device=blocks.device)
    ci = torch.arange(blocks.shape[2], device=blocks.device)
    mask = (ci.view(1, -1, 1) < cols.view(-1, 1, 1)) & (ri.view(1, 1, -1) < rows.view(-1, 1, 1))
    return t[mask], off


@dataclass
class H2Matrix:
    n: int
    depth: int
    node_start: np.ndarray
    node_size: np.ndarray
    rank: np.ndarray
    U_off: np.ndarray
    U: torch.Tensor
    E_off: np.ndarray
    E: torch.Tensor
    adm_ptr: np.ndarray
    adm_col: np.ndarray
    S_off: np.ndarray
    S: torch.Tensor
    inad_ptr: np.ndarray
    inad_col: np.ndarray
    D_off: np.ndarray
    D: torch.Tensor
    perm: np.ndarray = None
    meta: dict = field(default_factory=dict)

    # ------------------------------------------------------------ construction
    @classmethod
    def from_levels(cls, tree, part, lev) -> "H2Matrix":
        d = tree.depth
        nn = tree.nnodes
        rank = np.zeros(nn, dtype=np.int64)
        for l in range(d + 1):
            rank[(1 << l) - 1:(1 << (l + 1)) - 1] = lev["rank"][l]
        leaves = np.arange((1 << d) - 1, nn)
        U, U_off = _flatten_blocks(lev["U"], tree.size[leaves], rank[leaves])
        # transfers, level by level, node order
        Es, E_sz = [], [0]
        for l in range(1, d + 1):
            ids = np.arange((1 << l) - 1, (1 << (l + 1)) - 1)
            data, off = _flatten_blocks(lev["E"][l], rank[ids], rank[(ids - 1) // 2])
            Es.append(data)
            E_sz.extend((off[1:] - off[:-1]).cpu().tolist())
        E = torch.cat(Es) if Es else U.new_zeros(0)
        E_off = np.concatenate([[0], np.cumsum(E_sz)]).astype(np.int64)
        # admissible CSR over all nodes + couplings
        adm_all = [part.adm[l] for l in range(d + 1)]
        adm = np.concatenate(adm_all, axis=0) if adm_all else np.zeros((0, 2), np.int64)
        adm_ptr = np.concatenate([[0], np.cumsum(np.bincount(adm[:, 0], minlength=nn))]).astype(np.int64)
        Ss, S_sz = [], []
        for l in range(d + 1):
            pr = part.adm[l]
            if not len(pr):
                continue
            data, off = _flatten_blocks(lev["S"][l], rank[pr[:, 0]], rank[pr[:, 1]])
            Ss.append(data)
            S_sz.extend((off[1:] - off[:-1]).cpu().tolist())
        S = torch.cat(Ss) if Ss else U.new_zeros(0)
        S_off = np.concatenate([[0], np.cumsum(S_sz)]).astype(np.int64)
        inad = np.concatenate([part.inad[l] for l in range(d + 1)], axis=0)
        inad_ptr = np.concatenate([[0], np.cumsum(np.bincount(inad[:, 0], minlength=nn))]).astype(np.int64)
        near = part.inad[d]
        D, D_off = _flatten_blocks(lev["D"], tree.size[near[:, 0]], tree.size[near[:, 1]])
        return cls(n=int(tree.size[0]), depth=d, node_start=tree.start.copy(),
                   node_size=tree.size.copy(), rank=rank,
                   U_off=U_off.cpu().numpy(), U=U, E_off=E_off, E=E,
                   adm_ptr=adm_ptr, adm_col=adm[:, 1].copy(), S_off=S_off, S=S,
                   inad_ptr=inad_ptr, inad_col=inad[:, 1].copy(),
                   D_off=D_off.cpu().numpy(), D=D, perm=tree.perm.copy())

    # ------------------------------------------------------------ utilities
    @property
    def nnodes(self) -> int:
        return (1 << (self.depth + 1)) - 1

    def level_ids(self, l: int) -> np.ndarray:
        return np.arange((1 << l) - 1, (1 << (l + 1)) - 1)

    def to(self, device) -> "H2Matrix":
        out = H2Matrix(**{k: getattr(self, k) for k in self.__dataclass_fields__})
        out.U = self.U.to(device)
        out.E = self.E.to(device)
        out.S = self.S.to(device)
        out.D = self.D.to(device)
        return out

    def numpy(self) -> "H2Matrix":
        out = self.to("cpu")
        out.U = out.U.numpy()
        out.E = out.E.numpy()
        out.S = out.S.numpy()
        out.D = out.D.numpy()
        return out

    def top_level(self) -> int | None:
        """Coarsest level that holds an admissible block (``None`` when none)."""
        for l in range(self.depth + 1):
            ids = self.level_ids(l)
            if self.adm_ptr[ids[-1] + 1] - self.adm_ptr[ids[0]] > 0:
                return l
        return None

    def nbytes(self) -> int:
        return int(8 * (self.U.numel() + self.E.numel() + self.S.numel() + self.D.numel()))

    def save(self, path: str) -> None:
        arrs = {k: getattr(self, k) for k in self.__dataclass_fields__ if k != "meta"}
        arrs = {k: (v.cpu().numpy() if torch.is_tensor(v) else np.asarray(v)) for k, v in arrs.items()}
        with open(path, "wb") as f:
            np.savez(f, **arrs)

    @classmethod
    def load(cls, path: str) -> "H2Matrix":
        z = np.load(path)
        kw = {k: z[k] for k in z.files}
        for k in ("U", "E", "S", "D"):
            kw[k] = torch.from_numpy(kw[k])
        kw["n"] = int(kw["n"])
        kw["depth"] = int(kw["depth"])
        return cls(**kw)


def h2_matvec_torch(A: H2Matrix, x: torch.Tensor) -> torch.Tensor:
    """``y = A x`` in float64 (x in tree order, shape (n, nrhs)); used by the input
    generator for the spectral-norm estimate only.  Loops over nodes — intended for
    inputs up to a few tens of thousands of nodes."""
    d = A.depth
    dev = A.U.device
    nn = A.nnodes
    xh = [None] * nn
    yh = [None] * nn
    nrhs = x.shape[1]
    first_leaf = (1 << d) - 1
    for g in range(nn - 1, -1, -1):
        k = int(A.rank[g])
        if g >= first_leaf:
            i = g - first_leaf
            st, sz = int(A.node_start[g]), int(A.node_size[g])
            Ub = A.U[A.U_off[i]:A.U_off[i + 1]].view(k, sz).T
            xh[g] = Ub.T @ x[st:st + sz]
        else:
            acc = torch.zeros((k, nrhs), dtype=torch.float64, device=dev)
            for c in (2 * g + 1, 2 * g + 2):
                kc = int(A.rank[c])
                Ec = A.E[A.E_off[c]:A.E_off[c + 1]].view(k, kc).T
                acc += Ec.T @ xh[c]
            xh[g] = acc
    for g in range(nn):
        k = int(A.rank[g])
        acc = torch.zeros((k, nrhs), dtype=torch.float64, device=dev)
        for e in range(A.adm_ptr[g], A.adm_ptr[g + 1]):
            t = int(A.adm_col[e])
            S = A.S[A.S_off[e]:A.S_off[e + 1]].view(int(A.rank[t]), k).T
            acc += S @ xh[t]
        if g > 0:
            p = (g - 1) // 2
            kp = int(A.rank[p])
            Eg = A.E[A.E_off[g]:A.E_off[g + 1]].view(kp, k).T
            acc += Eg @ yh[p]
        yh[g] = acc
    y = torch.zeros_like(x)
    for g in range(first_leaf, nn):
        i = g - first_leaf
        st, sz = int(A.node_start[g]), int(A.node_size[g])
        k = int(A.rank[g])
        Ub = A.U[A.U_off[i]:A.U_off[i + 1]].view(k, sz).T
        y[st:st + sz] += Ub @ yh[g]
        for e in range(A.inad_ptr[g], A.inad_ptr[g + 1]):
            t = int(A.inad_col[e])
            j = e - A.inad_ptr[first_leaf]
            szt, stt = int(A.node_size[t]), int(A.node_start[t])
            Db = A.D[A.D_off[j]:A.D_off[j + 1]].view(szt, sz).T
            y[st:st + sz] += Db @ x[stt:stt + szt]
    return y
