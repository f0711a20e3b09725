"""The workloads: point set + kernel + tree/admissibility parameters + tolerance.

``WORKLOADS`` holds the problem families at their full sizes; tests build
smaller members of the same families through :func:`make_problem` overrides.
Construction tolerance is one tenth of the factorisation tolerance, as in the
paper's Table 1 (``eps = eps_lu / 10``).
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, replace

import numpy as np
import torch

from . import points as P
from .construct import construct_h2, spectral_norm
from .h2matrix import H2Matrix
from .kernels import Kernel, helmholtz3d_cell_average, laplace2d_cell_average
from .tree import build_kdtree, dual_traversal


@dataclass(frozen=True)
class Workload:
    name: str
    n: int
    family: str          # point/kernel family
    leaf: int
    eta: float
    tol: float           # factorisation tolerance eps_lu
    nrhs: int
    p0: int              # leaf Chebyshev order
    seed: int = 0


WORKLOADS = {
    # 2D exponential covariance, uniform points in the unit square
    "cov2d": Workload("cov2d", 4096, "cov2d", 64, 1.0, 1e-8, 1, 8),
    # 3D Matern-3/2 covariance, uniform points in the unit cube
    "matern3d": Workload("matern3d", 65536, "matern3d", 64, 1.0, 1e-6, 1, 5),
    # 2D Laplace volume IE on a jittered 512x512 grid
    "laplace2d": Workload("laplace2d", 262144, "laplace2d", 64, 0.7, 1e-6, 8, 8),
    # 3D Laplace single layer 1/(4 pi r) on a Fibonacci sphere
    "sphere": Workload("sphere", 1 << 20, "sphere", 128, 1.0, 1e-5, 1, 4),
    # one system of the uneven batch of Gaussian-kernel problems
    "gauss3d": Workload("gauss3d", 8192, "gauss3d", 64, 1.0, 1e-6, 4, 4),
    # 3D Helmholtz volume IE cos(3r)/r on a 32^3 cubic lattice (Table 1 parameters)
    "helmholtz3d": Workload("helmholtz3d", 32768, "helmholtz3d", 64, 0.7, 1e-6, 1, 4),
    # 3D exponential covariance plus a random rank-32 update (Table 1 "LRU" parameters)
    "lru3d": Workload("lru3d", 32768, "lru3d", 128, 0.9, 1e-7, 1, 4),
}

HELMHOLTZ_KAPPA = 3.0     # wavenumber of the Helmholtz IE, fixed as the lattice is refined
LRU_RANK = 32             # rank of the global update of the LRU problem


def family_points_kernel(w: Workload):
    """Points (original order) and kernel (with its diagonal) of a workload."""
    n = w.n
    if w.family == "cov2d":
        return P.uniform_box(n, 2, w.seed), Kernel("exp", 0.1, 1.0 + 1e-2)
    if w.family == "matern3d":
        return P.uniform_box(n, 3, w.seed), Kernel("matern32", 0.2, 1.0 + 1e-3)
    if w.family == "gauss3d":
        return P.uniform_box(n, 3, w.seed), Kernel("gauss", 0.3, 1.0 + 1e-2)
    if w.family == "laplace2d":
        side = int(round(math.sqrt(n)))
        assert side * side == n, "laplace2d needs a square number of points"
        h = 1.0 / side
        return (P.jittered_grid_2d(side, 0.25, w.seed),
                Kernel("laplace2d", 1.0, laplace2d_cell_average(h) + 1e-4))
    if w.family == "helmholtz3d":
        side = int(round(n ** (1.0 / 3.0)))
        assert side ** 3 == n, "helmholtz3d needs a cubic number of points"
        h = 1.0 / side
        diag = helmholtz3d_cell_average(h, HELMHOLTZ_KAPPA) + 1e-2
        return P.cubic_lattice(side), Kernel("helmholtz3d", 1.0, diag, HELMHOLTZ_KAPPA)
    if w.family == "lru3d":
        return P.uniform_box(n, 3, w.seed), Kernel("exp", 0.2, 1.0 + 1e-2)
    if w.family == "sphere":
        # regularised diagonal 1/(4 pi h): h = rho/2 with rho the radius of a disk of
        # area 4 pi/n (one point's share of the sphere), so the diagonal equals the
        # mean of 1/(4 pi r) over that disk and the matrix is SPD
        h = 1.0 / math.sqrt(n)
        return P.fibonacci_sphere(n, 1e-3, w.seed), Kernel("laplace3d", 1.0, 1.0 / (4.0 * math.pi * h))
    raise ValueError(w.family)


def family_lowrank(w: Workload):
    """Factor ``W`` (original point order) of the global update ``W W^T`` of a
    workload, or None."""
    if w.family == "lru3d":
        return P.low_rank_factor(w.n, LRU_RANK, w.seed)
    return None


@dataclass
class Problem:
    workload: Workload
    A: H2Matrix
    norm_a: float
    build_seconds: float
    stats: dict


def make_problem(name: str, device="cpu", **over) -> Problem:
    """Build the H^2 matrix of workload ``name`` (fields overridable, e.g. ``n=``)."""
    w = replace(WORKLOADS[name], **over)
    t0 = time.perf_counter()
    pts, kern = family_points_kernel(w)
    tree = build_kdtree(pts, w.leaf)
    part = dual_traversal(tree, w.eta)
    t_tree = time.perf_counter() - t0
    lev = construct_h2(pts, tree, part, kern, w.p0, w.tol / 10.0, device=device, lowrank=family_lowrank(w))
    t1 = time.perf_counter()
    norm_a = spectral_norm(tree, part, lev)
    t_norm = time.perf_counter() - t1
    t2 = time.perf_counter()
    A = H2Matrix.from_levels(tree, part, lev)
    seconds = dict(tree=t_tree, **lev["seconds"], norm=t_norm, flatten=time.perf_counter() - t2)
    del lev
    if torch.cuda.is_available() and str(device).startswith("cuda"):
        torch.cuda.synchronize()
    t1 = time.perf_counter()
    csp = 0
    for l in range(tree.depth + 1):
        ids = A.level_ids(l)
        deg = A.inad_ptr[ids + 1] - A.inad_ptr[ids]
        csp = max(csp, int(deg.max()))
    stats = dict(depth=tree.depth, top_level=part.top_level(), csp=csp,
                 kmax=int(A.rank.max()), nbytes=A.nbytes(),
                 seconds={k: round(v, 2) for k, v in seconds.items()})
    A.meta = dict(workload=w.name, norm_a=norm_a)
    return Problem(w, A, norm_a, t1 - t0, stats)


def uneven_sizes(nsys: int = 64, nmin: int = 2048, nmax: int = 131072) -> list[int]:
    """System sizes of the uneven batch: N_s = round(exp(U(ln nmin, ln nmax))), the
    uniform draw seeded by s."""
    out = []
    for s in range(nsys):
        u = np.random.default_rng(s).uniform(math.log(nmin), math.log(nmax))
        out.append(int(round(math.exp(u))))
    return out


def make_batch(name: str = "gauss3d", nsys: int = 64, nmin: int = 2048, nmax: int = 131072,
               device="cpu", **over) -> list[Problem]:
    """The uneven batch: system s is workload ``name`` with N_s points drawn with seed s."""
    return [make_problem(name, device=device, n=n, seed=s, **over)
            for s, n in enumerate(uneven_sizes(nsys, nmin, nmax))]


def rhs(n: int, nrhs: int, seed: int = 0) -> np.ndarray:
    """Right-hand sides: N(0,1) entries, seeded (tree order = generation order)."""
    return P.standard_normal((n, nrhs), seed)


def save_problem(pb: Problem, path: str) -> None:
    """Write a built problem (matrix arrays + workload + norm) to an .npz file."""
    import json
    pb.A.save(path)
    with open(path + ".json", "w") as f:
        json.dump({"workload": pb.workload.__dict__, "norm_a": pb.norm_a, "stats": pb.stats}, f)


def load_problem(path: str, device="cpu") -> Problem:
    """Read a problem written by :func:`save_problem` (values moved to ``device``)."""
    import json
    with open(path + ".json") as f:
        meta = json.load(f)
    A = H2Matrix.load(path).to(device)
    w = Workload(**meta["workload"])
    A.meta = dict(workload=w.name, norm_a=meta["norm_a"])
    return Problem(w, A, meta["norm_a"], 0.0, meta["stats"])
