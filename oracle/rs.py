"""Oracle: strong recursive skeletonisation factorisation and solve of a symmetric
H^2 matrix, plain float64 numpy/scipy, one box at a time.

Test infrastructure only: used by the tests, by the entry point's smoke check and by
the timed CPU baseline; the CUDA library never imports it and shares no code with it.

Factorisation (Alg. 1 and Alg. 2; Sec. 2.1 steps 1-4; level close and Eq. 2.1):
levels from the leaves (d) up to the top level t; at each level the colours of
``greedy_colouring`` in order; within a colour, as in Alg. 2, every box is augmented
from the same fill matrix, then every box is projected, then every box gets its
partial LU (boxes in ascending index; their Schur updates commute).  For box i:

  1. fill row  F_i* of the working fill-in matrix, ``Y = (I - V V^T) F_i*``;
  2. truncSVD option 2 (Sec. 2.1): QR of ``Y^T``, SVD of R; the left singular
     vectors of Y (right singular vectors of R) with ``sigma > eps_fill`` form
     ``Vbar``, ``eps_fill = eps_lu * ||A||``, capped so ``k~ <= n_i``;
  3. ``V~ = [V, Vbar]``; complement from a full Householder QR of ``V~``;
     ``Q~ = [V~perp, V~]`` (redundant indices first);
  4. projection: ``Q~^T D_i*``, ``D_*i Q~``; ``Q~^T F_i*`` and ``F_*i Q~`` with the
     redundant rows/columns of F dropped (the truncation);
  5. partial LU: ``D_RR = P L U`` (partial pivoting); ``W_U = D_RR^-1 D_R*``,
     ``W_L = D_*R D_RR^-1``; Schur update ``A_** -= D_*R W_U`` on all block pairs of
     ``N(i)``, into the near field where the pair is inadmissible and into the
     fill-in matrix otherwise; the redundant rows/columns are then zero.

Level close: skeleton parts of the blocks plus the zero-padded couplings
``S~ = [[S,0],[0,0]]`` form the parent level's blocks, fill under an admissible
ancestor is carried up, and the parent basis is ``[T~_c1; T~_c2]`` with
``T~_c = [E_c; 0]``.  The top level's remaining dense matrix gets a dense LU.

Solve (Alg. 3): Eq. 2.1 inverted exactly: forward in elimination order (Q~^T, then
the L update), diagonal L solves, upsweep; dense top solve; downsweep, diagonal U
solves, backward in reverse elimination order (U update, then Q~).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

from . import structure as st


def _blk(arr, off, e, rows, cols):
    """Column-major block ``e`` of a flat array as a (rows, cols) ndarray copy."""
    return np.array(arr[off[e]:off[e + 1]]).reshape(cols, rows).T.copy()


@dataclass
class BoxFactor:
    n: int                      # size of the box at its level
    k: int                      # basis rank before augmentation
    kt: int                     # augmented (skeleton) rank k~
    Q: np.ndarray               # n x n, [V~perp, V~]
    lu: tuple | None            # scipy lu_factor of D_RR (r x r)
    nb: list                    # neighbours N(i) in the order used below
    WL: dict                    # j -> (rows of j) x r   (j = i: skeleton rows only)
    WU: dict                    # j -> r x (cols of j)   (j = i: skeleton cols only)

    @property
    def r(self) -> int:
        return self.n - self.kt


@dataclass
class LevelFactor:
    level: int
    sizes: list
    colour: list
    order: list                 # elimination order (local box indices)
    boxes: list                 # BoxFactor per local index
    layout: dict


@dataclass
class Factor:
    depth: int
    top: int | None
    levels: list = field(default_factory=list)     # leaves first
    top_sizes: list = field(default_factory=list)
    top_lu: tuple | None = None
    n: int = 0

    def ranks(self, level: int) -> np.ndarray:
        lv = next(x for x in self.levels if x.level == level)
        return np.array([b.kt for b in lv.boxes], dtype=np.int64)


# ------------------------------------------------------------------ leaf input
def _leaf_state(A):
    d = A.depth
    first, cnt = st.level_range(d)
    sizes = [int(A.node_size[first + i]) for i in range(cnt)]
    V = []
    for i in range(cnt):
        V.append(_blk(A.U, A.U_off, i, sizes[i], int(A.rank[first + i])))
    D = {}
    base = A.inad_ptr[first]
    for i in range(cnt):
        g = first + i
        for e in range(A.inad_ptr[g], A.inad_ptr[g + 1]):
            j = int(A.inad_col[e]) - first
            D[(i, j)] = _blk(A.D, A.D_off, e - base, sizes[i], sizes[j])
    return sizes, V, D


def _coupling(A, e, ks, kt):
    return _blk(A.S, A.S_off, e, ks, kt)


def _transfer(A, g):
    p = (g - 1) // 2
    return _blk(A.E, A.E_off, g, int(A.rank[g]), int(A.rank[p]))


# ------------------------------------------------------------------ one box
def _svd(R):
    """Thin SVD of R by LAPACK's divide-and-conquer driver; on the rare strongly graded
    R where that driver does not converge, by its QR-iteration driver (the same
    decomposition, computed another way)."""
    try:
        return np.linalg.svd(R, full_matrices=False)
    except np.linalg.LinAlgError:
        return sla.svd(R, full_matrices=False, lapack_driver="gesvd")


def _augment(V, Frow, eps_fill, method="qr"):
    """Alg. 2 truncSVD + augment: returns V~ = [V, Vbar].

    method "qr" (Sec. 2.1, the second approach, the one the paper uses): QR of Y^T,
    SVD of R, keep sigma > eps_fill.
    method "gram" (Sec. 2.1, the first approach; named again in Sec. 3's scaling discussion as
    trading accuracy for speed): the eigendecomposition of the Gram matrix Y Y^T, keep
    lambda > eps_fill^2.  The same subspace as "qr" while the kept sigma are well above
    sqrt(machine eps) * sigma_max; below that the squared values sink into rounding.
    method "cholqr" (Sec. 3's Cholesky QR in place of the Householder QR): the
    R-factor of Y^T from the Cholesky factor of Y Y^T + s I, then the SVD of R as in
    "qr".  The shift s = 11 (m n + n (n + 1)) u ||Y||_F^2 (Y^T is m x n; the shifted
    Cholesky QR of Fukaya, Kannan, Nakatsukasa, Yamamoto and Yanagisawa, 2020, with the
    Frobenius norm bounding the 2-norm) keeps the factorisation defined for the
    rank-deficient fill; it lifts
    every squared singular value by about s, so the kept count compares sigma_R^2 - s
    with eps_fill^2.  Same accuracy limit as "gram"."""
    n, k = V.shape
    if Frow is None or Frow.shape[1] == 0 or k >= n:
        return V
    Y = Frow - V @ (V.T @ Frow)
    if method == "gram":
        lam, W = np.linalg.eigh(Y @ Y.T)                 # ascending eigenvalues
        lam, W = lam[::-1], W[:, ::-1]                   # largest first
        keep = min(int(np.count_nonzero(lam > eps_fill * eps_fill)), n - k)
        Vbar = W[:, :keep]
    elif method == "cholqr":
        m = Y.shape[1]
        y2 = float(np.sum(Y * Y))
        if y2 == 0.0:
            return V
        shift = 11.0 * (m * n + n * (n + 1)) * np.finfo(float).eps * y2
        R = np.linalg.cholesky(Y @ Y.T + shift * np.eye(n)).T          # R^T R = Y Y^T + s I
        _, s, Wt = _svd(R)
        keep = min(int(np.count_nonzero(s * s - shift > eps_fill * eps_fill)), n - k)
        Vbar = Wt[:keep].T
    elif method == "qr":
        R = np.linalg.qr(Y.T, mode="r")                  # QR of Y^T
        _, s, Wt = _svd(R)                               # R = U_R diag(s) W_R^T
        keep = int(np.count_nonzero(s > eps_fill))
        keep = min(keep, n - k)
        Vbar = Wt[:keep].T                               # right sing. vectors of R
    else:
        raise ValueError(f"unknown augmentation method {method!r}")
    if keep:
        # they lie in range(Y), orthogonal to V in exact arithmetic; one pass of
        # block Gram-Schmidt + QR restores that in floating point
        Vbar = Vbar - V @ (V.T @ Vbar)
        Vbar = np.linalg.qr(Vbar)[0]
    return np.hstack([V, Vbar])


def _complete(Vt):
    """Q~ = [V~perp, V~] with V~perp from a full Householder QR of V~."""
    n, kt = Vt.shape
    if kt == 0:
        return np.eye(n)
    Qh, _ = np.linalg.qr(Vt, mode="complete")
    return np.hstack([Qh[:, kt:], Vt])


def _augment_box(i, sizes, V, F, frow, eps_fill, hook=None, method="qr"):
    """Alg. 2, first parallel loop: V~_i = [V_i, truncSVD((I - V V^T) F_i*)]."""
    frow_keys = [(i, j) for j in frow.get(i, [])]
    Frow = np.hstack([F[key] for key in frow_keys]) if frow_keys else None
    Vt = _augment(V[i], Frow, eps_fill, method)
    if hook is not None:
        hook("augment", i=i, V=V[i], Vt=Vt, Frow=Frow)
    return Vt


def _project_box(i, Q, r, nbrs, D, F, frow, fcol):
    """Alg. 2: D <- Q^T D Q and F <- Q^T F Q on the block row and column of box i,
    with the redundant rows/columns of F dropped (the truncation)."""
    for j in nbrs[i]:
        D[(i, j)] = Q.T @ D[(i, j)]
    for j in nbrs[i]:
        D[(j, i)] = D[(j, i)] @ Q
    for key in [(i, j) for j in frow.get(i, [])]:
        B = Q.T @ F[key]
        B[:r, :] = 0.0
        F[key] = B
    for key in [(j, i) for j in fcol.get(i, [])]:
        B = F[key] @ Q
        B[:, :r] = 0.0
        F[key] = B


def _partial_lu(i, n, r, nbrs, sizes, D, F, pivot="lu"):
    """Alg. 2 partialLU for box i: LU of D_RR, elementary factors, Schur update of
    N(i) x N(i) (fill outside the near field goes to F), eliminated rows/cols zeroed.

    pivot "lu": partial pivoting (the paper's dense LU).  pivot "cholesky" (a symmetric
    variant for SPD matrices; the paper notes that the method keeps symmetry): D_RR =
    L L^T and W_L = W_U^T, so only one of the two elementary factors needs storing."""
    WL, WU = {}, {}
    lu = None
    if r > 0:
        DRR = D[(i, i)][:r, :r].copy()

        def rows_of(j):                   # coordinates of j still in the matrix
            return slice(r, n) if j == i else slice(0, sizes[j])

        if pivot == "cholesky":
            ch = sla.cho_factor(DRR, lower=True, check_finite=True)
            lu = ("chol", ch[0])
            for j in nbrs[i]:
                WU[j] = sla.cho_solve(ch, D[(i, j)][:r, rows_of(j)])
                WL[j] = WU[j].T
        else:
            lu = sla.lu_factor(DRR, check_finite=True)
            for j in nbrs[i]:
                WU[j] = sla.lu_solve(lu, D[(i, j)][:r, rows_of(j)])
                WL[j] = sla.lu_solve(lu, D[(j, i)][rows_of(j), :r].T, trans=1).T
        for j in nbrs[i]:
            Dj = D[(j, i)][rows_of(j), :r]
            for kk in nbrs[i]:
                upd = Dj @ WU[kk]
                if (j, kk) in D:
                    D[(j, kk)][rows_of(j), rows_of(kk)] -= upd
                else:
                    F[(j, kk)][rows_of(j), rows_of(kk)] -= upd
        for j in nbrs[i]:
            D[(i, j)][:r, :] = 0.0
            D[(j, i)][:, :r] = 0.0
    return lu, WL, WU


def _skeletonise_colour(C, nbrs, sizes, V, D, F, frow, fcol, eps_fill, hook=None, method="qr", pivot="lu"):
    """Alg. 2 for one colour: augment every box from the same fill matrix, then
    project every box, then the partial LU of every box.  (Boxes of one colour share
    no near-field block, but two of them can share a fill block, so augmenting one
    after projecting the other would not be Alg. 2.)"""
    Vt = {i: _augment_box(i, sizes, V, F, frow, eps_fill, hook, method) for i in C}
    Qs = {i: _complete(Vt[i]) for i in C}
    for i in C:
        _project_box(i, Qs[i], sizes[i] - Vt[i].shape[1], nbrs, D, F, frow, fcol)
    out = {}
    for i in C:
        n, kt = sizes[i], Vt[i].shape[1]
        lu, WL, WU = _partial_lu(i, n, n - kt, nbrs, sizes, D, F, pivot)
        out[i] = BoxFactor(n=n, k=V[i].shape[1], kt=kt, Q=Qs[i], lu=lu, nb=list(nbrs[i]), WL=WL, WU=WU)
    return out


# ------------------------------------------------------------------ driver
def factorize(A, eps_lu: float, norm_a: float, hook=None, augment: str = "qr", lu: str = "lu") -> Factor:
    """Alg. 1: factorise the H^2 matrix ``A`` (flat numpy storage) with threshold
    ``eps_lu``; ``norm_a`` is ``||A||_2`` (so ``eps_fill = eps_lu * norm_a``).
    ``hook(event, **state)``, if given, observes intermediate states (tests only).
    ``augment``: "qr" (truncSVD option 2), "gram" (Gram matrix + eigendecomposition) or
    "cholqr" (shifted Cholesky QR of Y^T + SVD of R).
    ``lu``: "lu" (partial pivoting) or "cholesky" (SPD matrices; W_L = W_U^T)."""
    if augment not in ("qr", "gram", "cholqr") or lu not in ("lu", "cholesky"):
        raise ValueError((augment, lu))
    eps_fill = eps_lu * norm_a
    d = A.depth
    t = A.top_level()
    Z = Factor(depth=d, top=t, n=A.n)
    sizes, V, D = _leaf_state(A)
    F = {}
    carried = set()
    last = t if t is not None else d + 1          # no admissible block: no level
    for l in range(d, last - 1, -1):
        first, cnt = st.level_range(l)
        nbrs = st.neighbours(A, l)
        colour = st.greedy_colouring(nbrs)
        fill = st.fill_pattern(nbrs, carried)
        for key in fill:
            if key not in F:
                F[key] = np.zeros((sizes[key[0]], sizes[key[1]]))
        layout = st.level_layout(nbrs, fill, sizes)
        order = [i for c in range(max(colour) + 1) for i in range(cnt) if colour[i] == c]
        frow, fcol = {}, {}
        for (a, b) in sorted(fill):
            frow.setdefault(a, []).append(b)
            fcol.setdefault(b, []).append(a)
        boxes = [None] * cnt
        if hook is not None:
            hook("level_start", l=l, D=D, F=F, V=V, sizes=sizes)
        for c in range(max(colour) + 1):
            C = [i for i in range(cnt) if colour[i] == c]
            done = _skeletonise_colour(C, nbrs, sizes, V, D, F, frow, fcol, eps_fill, hook, augment, lu)
            for i in C:
                boxes[i] = done[i]
                if hook is not None:
                    hook("box", l=l, i=i, box=boxes[i], V=V[i])
        Z.levels.append(LevelFactor(l, list(sizes), colour, order, boxes, layout))
        if hook is not None:
            hook("level_end", l=l, D=D, F=F, boxes=boxes)
        sizes, V, D, F, carried = _close_level(A, l, boxes, D, F, fill)
    # top: dense LU of the remaining matrix
    lt = (last - 1) if t is not None else d
    first, cnt = st.level_range(lt)
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(int)
    Dt = np.zeros((offs[-1], offs[-1]))
    for (i, j), B in D.items():
        Dt[offs[i]:offs[i + 1], offs[j]:offs[j + 1]] = B
    Z.top_sizes = list(sizes)
    Z.top_lu = sla.lu_factor(Dt) if offs[-1] > 0 else None
    return Z


def _close_level(A, l, boxes, D, F, fill):
    """Level close: build the parent level's near-field blocks, fill and basis."""
    first, cnt = st.level_range(l)
    pfirst, pcnt = st.level_range(l - 1)
    adm = st.admissible_pairs(A, l)
    kt = [b.kt for b in boxes]
    r = [b.r for b in boxes]
    psizes = [kt[2 * p] + kt[2 * p + 1] for p in range(pcnt)]
    pnbrs = st.neighbours(A, l - 1)
    pnear = {(p, q) for p in range(pcnt) for q in pnbrs[p]}

    def skel(c, e):
        """Skeleton x skeleton part of child pair (c, e), or None if empty."""
        out = None
        if (c, e) in D:
            out = D[(c, e)][r[c]:, r[e]:].copy()
        if (c, e) in adm:
            kc, ke = boxes[c].k, boxes[e].k
            Sx = np.zeros((kt[c], kt[e]))
            Sx[:kc, :ke] = _coupling(A, adm[(c, e)], kc, ke)
            out = Sx if out is None else out + Sx
        if (c, e) in F:
            Fs = F[(c, e)][r[c]:, r[e]:]
            out = Fs.copy() if out is None else out + Fs
        return out

    pD, pF = {}, {}
    targets = [(pq, pD) for pq in sorted(pnear)]
    pfill_keys = {(c // 2, e // 2) for (c, e) in fill} - pnear
    targets += [(pq, pF) for pq in sorted(pfill_keys)]
    for (p, q), dst in targets:
        B = np.zeros((psizes[p], psizes[q]))
        for a, c in enumerate((2 * p, 2 * p + 1)):
            for b, e in enumerate((2 * q, 2 * q + 1)):
                blk = skel(c, e)
                if blk is None:
                    continue
                ro = 0 if a == 0 else kt[2 * p]
                co = 0 if b == 0 else kt[2 * q]
                B[ro:ro + kt[c], co:co + kt[e]] = blk
        dst[(p, q)] = B
    # parent basis [T~_c1; T~_c2], T~_c = [E_c; 0]
    pV = []
    for p in range(pcnt):
        g = pfirst + p
        kp = int(A.rank[g])
        Vp = np.zeros((psizes[p], kp))
        ro = 0
        for c in (2 * p, 2 * p + 1):
            kc = boxes[c].k
            Vp[ro:ro + kc, :] = _transfer(A, first + c)
            ro += kt[c]
        pV.append(Vp)
    carried = set(pF.keys())
    return psizes, pV, pD, pF, carried


# ------------------------------------------------------------------ solve
def solve(Z: Factor, b: np.ndarray) -> np.ndarray:
    """Alg. 3: ``x = A^-1 b`` for ``b`` of shape (n, nrhs) in tree order."""
    b = np.array(b, dtype=np.float64).reshape(Z.n, -1)
    lv0 = Z.levels[0] if Z.levels else None
    sizes = lv0.sizes if lv0 else Z.top_sizes
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(int)
    vec = [b[offs[i]:offs[i + 1]].copy() for i in range(len(sizes))]
    stack = []
    for lv in Z.levels:                               # forward, leaves up
        for i in lv.order:
            bx = lv.boxes[i]
            vec[i] = bx.Q.T @ vec[i]
            r = bx.r
            if r == 0:
                continue
            for j in bx.nb:
                if j == i:
                    vec[i][r:] -= bx.WL[j] @ vec[i][:r]
                else:
                    vec[j] -= bx.WL[j] @ vec[i][:r]
        for i, bx in enumerate(lv.boxes):             # diagonal forward (P, L)
            if bx.r:
                if isinstance(bx.lu[0], str):
                    vec[i][:bx.r] = sla.solve_triangular(bx.lu[1], vec[i][:bx.r], lower=True)
                    continue
                lu, piv = bx.lu
                y = vec[i][:bx.r].copy()
                for a, p in enumerate(piv):
                    y[[a, p]] = y[[p, a]]
                vec[i][:bx.r] = sla.solve_triangular(lu, y, lower=True, unit_diagonal=True)
        stack.append(vec)
        vec = [np.vstack([vec[2 * p][lv.boxes[2 * p].r:], vec[2 * p + 1][lv.boxes[2 * p + 1].r:]])
               for p in range(len(vec) // 2)]
    xt = np.vstack(vec) if vec else np.zeros((0, b.shape[1]))
    if Z.top_lu is not None:
        xt = sla.lu_solve(Z.top_lu, xt)
    to = np.concatenate([[0], np.cumsum(Z.top_sizes)]).astype(int)
    vec = [xt[to[p]:to[p + 1]] for p in range(len(Z.top_sizes))]
    for lv in reversed(Z.levels):                     # backward, top down
        low = stack.pop()
        for p in range(len(vec)):                     # downsweep
            c1, c2 = 2 * p, 2 * p + 1
            r1, r2 = lv.boxes[c1].r, lv.boxes[c2].r
            k1 = lv.boxes[c1].kt
            low[c1][r1:] = vec[p][:k1]
            low[c2][r2:] = vec[p][k1:]
        vec = low
        for i, bx in enumerate(lv.boxes):             # diagonal backward (U)
            if bx.r:
                if isinstance(bx.lu[0], str):
                    vec[i][:bx.r] = sla.solve_triangular(bx.lu[1], vec[i][:bx.r], lower=True, trans=1)
                    continue
                lu, _ = bx.lu
                vec[i][:bx.r] = sla.solve_triangular(lu, vec[i][:bx.r], lower=False)
        for i in reversed(lv.order):
            bx = lv.boxes[i]
            r = bx.r
            if r:
                for j in bx.nb:
                    src = vec[i][r:] if j == i else vec[j]
                    vec[i][:r] -= bx.WU[j] @ src
            vec[i] = bx.Q @ vec[i]
    return np.vstack(vec)


def slogdet(Z: Factor) -> float:
    """``log|det A|`` from the factors: the Q~ are orthogonal and the elementary
    factors unit triangular, so only the redundant blocks and the top remain."""
    s = 0.0
    for lv in Z.levels:
        for bx in lv.boxes:
            if bx.r and isinstance(bx.lu[0], str):               # D_RR = L L^T
                s += 2.0 * float(np.sum(np.log(np.abs(np.diag(bx.lu[1])))))
            elif bx.r:
                s += float(np.sum(np.log(np.abs(np.diag(bx.lu[0])))))
    if Z.top_lu is not None:
        s += float(np.sum(np.log(np.abs(np.diag(Z.top_lu[0])))))
    return s
