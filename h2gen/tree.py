"""Cluster tree and block partition of the H^2 matrix (Sec. 1.1, Eq. 1.1).

* KD-tree: a complete binary tree of depth ``d = ceil(log2(N/m))``; every node
  splits its points at the median of the widest side of its bounding box
  (sizes ``floor(n/2)`` and ``ceil(n/2)``; ties broken by original index).
* Admissibility (Eq. 1.1): ``(D(s)+D(t))/2 <= eta * Dist(s,t)`` with ``D`` the
  diagonal of the axis-aligned bounding box and ``Dist`` the Euclidean distance
  between the two boxes (0 when they touch or overlap).
* Dual traversal from (root, root): admissible pairs become admissible leaves of
  the matrix tree, inadmissible pairs are refined into their four child pairs
  until the leaf level, where they are stored densely.

Nodes use heap numbering: level ``l`` holds ids ``2^l-1 .. 2^(l+1)-2``; the
children of ``g`` are ``2g+1`` and ``2g+2``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class ClusterTree:
    depth: int
    perm: np.ndarray        # tree order -> original point index
    start: np.ndarray       # (nnodes,) first tree-order index of each node
    size: np.ndarray        # (nnodes,) number of points of each node
    lo: np.ndarray          # (nnodes, dim) bounding box lower corner
    hi: np.ndarray          # (nnodes, dim) bounding box upper corner

    @property
    def nnodes(self) -> int:
        return (1 << (self.depth + 1)) - 1


def tree_depth(n: int, leaf: int) -> int:
    return max(0, int(math.ceil(math.log2(n / leaf)))) if n > leaf else 0


def build_kdtree(points: np.ndarray, leaf: int) -> ClusterTree:
    n, dim = points.shape
    d = tree_depth(n, leaf)
    nnodes = (1 << (d + 1)) - 1
    start = np.zeros(nnodes, dtype=np.int64)
    size = np.zeros(nnodes, dtype=np.int64)
    lo = np.zeros((nnodes, dim))
    hi = np.zeros((nnodes, dim))
    size[0] = n
    perm = np.arange(n, dtype=np.int64)
    for l in range(d + 1):
        first = (1 << l) - 1
        cnt = 1 << l
        ids = np.arange(first, first + cnt)
        st = start[ids]
        sz = size[ids]
        # bounding boxes of this level's nodes (points are contiguous per node)
        p = points[perm]
        nonempty = sz > 0
        bmin = np.full((cnt, dim), np.inf)
        bmax = np.full((cnt, dim), -np.inf)
        if nonempty.any():
            bmin[nonempty] = np.minimum.reduceat(p, st[nonempty], axis=0)
            bmax[nonempty] = np.maximum.reduceat(p, st[nonempty], axis=0)
        lo[ids] = bmin
        hi[ids] = bmax
        if l == d:
            break
        # split along the widest dimension of every node at this level
        widest = np.argmax(bmax - bmin, axis=1)
        owner = np.repeat(np.arange(cnt), sz)
        coord = p[np.arange(n), widest[owner]]
        # sort within each node by (coordinate, original index)
        order = np.lexsort((perm, coord, owner))
        perm = perm[order]
        left = sz // 2
        ch_l = 2 * ids + 1
        ch_r = 2 * ids + 2
        start[ch_l] = st
        size[ch_l] = left
        start[ch_r] = st + left
        size[ch_r] = sz - left
    return ClusterTree(d, perm, start, size, lo, hi)


def admissible(tree: ClusterTree, s: np.ndarray, t: np.ndarray, eta: float) -> np.ndarray:
    """Vectorised Eq. 1.1 for node-id arrays ``s`` and ``t``."""
    diam_s = np.linalg.norm(tree.hi[s] - tree.lo[s], axis=1)
    diam_t = np.linalg.norm(tree.hi[t] - tree.lo[t], axis=1)
    gap = np.maximum(0.0, np.maximum(tree.lo[t] - tree.hi[s], tree.lo[s] - tree.hi[t]))
    dist = np.linalg.norm(gap, axis=1)
    return 0.5 * (diam_s + diam_t) <= eta * dist


@dataclass
class BlockPartition:
    """Per level, the admissible and inadmissible node pairs (global node ids),
    each sorted by (row, col)."""
    adm: list          # adm[l]: (npairs, 2) int64
    inad: list         # inad[l]: (npairs, 2) int64

    def top_level(self) -> int | None:
        """Coarsest level holding an admissible pair (``None`` if there is none)."""
        for l, a in enumerate(self.adm):
            if len(a):
                return l
        return None


def dual_traversal(tree: ClusterTree, eta: float) -> BlockPartition:
    d = tree.depth
    adm, inad = [], []
    pairs = np.array([[0, 0]], dtype=np.int64)
    for l in range(d + 1):
        if len(pairs):
            ok = admissible(tree, pairs[:, 0], pairs[:, 1], eta)
        else:
            ok = np.zeros(0, dtype=bool)
        a = pairs[ok]
        b = pairs[~ok]
        adm.append(a[np.lexsort((a[:, 1], a[:, 0]))] if len(a) else a.reshape(0, 2))
        b = b[np.lexsort((b[:, 1], b[:, 0]))] if len(b) else b.reshape(0, 2)
        inad.append(b)
        if l == d:
            break
        # refine inadmissible pairs into their four child pairs
        s = b[:, 0]
        t = b[:, 1]
        kids = []
        for cs in (1, 2):
            for ct in (1, 2):
                kids.append(np.stack([2 * s + cs, 2 * t + ct], axis=1))
        pairs = np.concatenate(kids, axis=0) if kids else np.zeros((0, 2), np.int64)
    return BlockPartition(adm, inad)
