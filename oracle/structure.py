"""Oracle: level structure of the strong recursive skeletonisation (integer work).

Test infrastructure only: nothing in the product path imports this module.

* ``neighbours``: the inadmissible (near-field) graph of a level, ``N(i)`` including
  ``i`` itself (Sec. 1.1; the block-sparse matrix ``D`` of Alg. 1).
* ``greedy_colouring``: first-fit colouring in ascending box index of that graph
  without self loops (Sec. 2.2: same-coloured boxes share no near-field block, so
  they can be skeletonised independently).
* ``fill_pattern``: the blocks that can receive fill-in at a level (Sec. 2.1 step 3
  and the level close): pairs ``(j,k)`` outside the near field with a common
  near-field neighbour, plus fill carried from the level below whose parent pair
  is not in the near field.
* ``level_layout``: canonical block list (near field and fill merged, rows then
  columns ascending) with offsets = exclusive prefix sum of ``n_j*n_k`` (the
  prefix-sum placement of Sec. 2.2).
"""
from __future__ import annotations

import numpy as np


def level_range(l: int) -> tuple[int, int]:
    return (1 << l) - 1, 1 << l


def neighbours(A, l: int) -> list[list[int]]:
    """``N(i)`` as sorted local indices for every box of level ``l``."""
    first, cnt = level_range(l)
    out = []
    for i in range(cnt):
        g = first + i
        cols = A.inad_col[A.inad_ptr[g]:A.inad_ptr[g + 1]]
        out.append(sorted(int(c) - first for c in cols))
    return out


def admissible_pairs(A, l: int) -> dict:
    """``{(s, t): entry index}`` of admissible pairs at level ``l`` (local indices)."""
    first, cnt = level_range(l)
    out = {}
    for i in range(cnt):
        g = first + i
        for e in range(A.adm_ptr[g], A.adm_ptr[g + 1]):
            out[(i, int(A.adm_col[e]) - first)] = e
    return out


def greedy_colouring(nbrs: list[list[int]]) -> list[int]:
    colour = [-1] * len(nbrs)
    for i in range(len(nbrs)):
        used = {colour[j] for j in nbrs[i] if j != i and colour[j] >= 0}
        c = 0
        while c in used:
            c += 1
        colour[i] = c
    return colour


def fill_pattern(nbrs: list[list[int]], carried: set) -> set:
    near = {(i, j) for i in range(len(nbrs)) for j in nbrs[i]}
    fill = set()
    for i in range(len(nbrs)):
        for j in nbrs[i]:
            for k in nbrs[i]:
                if (j, k) not in near:
                    fill.add((j, k))
    fill |= {p for p in carried if p not in near}
    return fill


def carried_to_parent(fill: set, parent_near: set) -> set:
    """Fill pairs of a level mapped to their parent pairs, minus the parent near field
    (those are merged into the parent's near-field blocks instead)."""
    return {(j // 2, k // 2) for (j, k) in fill if (j // 2, k // 2) not in parent_near}


def level_layout(nbrs, fill, sizes):
    """Canonical merged block list and prefix-sum offsets of one level."""
    near = {(i, j) for i in range(len(nbrs)) for j in nbrs[i]}
    blocks = sorted(near | fill)
    kind = np.array([0 if b in near else 1 for b in blocks], dtype=np.int64)
    rows = np.array([b[0] for b in blocks], dtype=np.int64)
    cols = np.array([b[1] for b in blocks], dtype=np.int64)
    words = np.array([sizes[b[0]] * sizes[b[1]] for b in blocks], dtype=np.int64)
    off = np.zeros(len(blocks) + 1, dtype=np.int64)
    off[1:] = np.cumsum(words)
    ptr = np.zeros(len(nbrs) + 1, dtype=np.int64)
    np.add.at(ptr, rows + 1, 1)
    ptr = np.cumsum(ptr)
    return dict(row_ptr=ptr, col=cols, kind=kind, offset=off)
