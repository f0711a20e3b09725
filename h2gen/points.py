"""Seeded synthetic point sets for the solver's test problems.

The paper's experiments (Sec. 3, "Test Problems") discretise kernels on point
sets in 2D/3D.  These generators produce the point clouds used by the workloads:
i.i.d. uniform points in the unit square / cube, a jittered 2D grid, a cubic
lattice and a jittered Fibonacci lattice on the unit sphere, plus the random factor
of a low-rank update.  Every generator is a pure function of its arguments and seed.
"""
from __future__ import annotations

import math

import numpy as np


def uniform_box(n: int, dim: int, seed: int = 0) -> np.ndarray:
    """``n`` i.i.d. points uniform in ``[0,1]^dim`` (float64, shape (n, dim))."""
    rng = np.random.default_rng(seed)
    return rng.random((n, dim))


def jittered_grid_2d(side: int, jitter: float = 0.25, seed: int = 0) -> np.ndarray:
    """Cell centres ``((i+1/2)h, (j+1/2)h)`` of a ``side x side`` grid on the unit
    square, ``h = 1/side``, each coordinate moved by ``U(-jitter*h, +jitter*h)``."""
    rng = np.random.default_rng(seed)
    h = 1.0 / side
    g = (np.arange(side) + 0.5) * h
    xx, yy = np.meshgrid(g, g, indexing="ij")
    pts = np.stack([xx.ravel(), yy.ravel()], axis=1)
    pts += rng.uniform(-jitter * h, jitter * h, size=pts.shape)
    return pts


def cubic_lattice(side: int) -> np.ndarray:
    """Cell centres ``((i+1/2)h, (j+1/2)h, (k+1/2)h)`` of a ``side^3`` lattice on the
    unit cube, ``h = 1/side`` (float64, shape (side^3, 3))."""
    h = 1.0 / side
    g = (np.arange(side) + 0.5) * h
    xx, yy, zz = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)


def fibonacci_sphere(n: int, jitter: float = 1e-3, seed: int = 0) -> np.ndarray:
    """Quasi-uniform points on the unit sphere: a Fibonacci lattice
    ``z_i = 1-(2i+1)/n``, ``phi_i = i*pi*(3-sqrt 5)``, moved by ``U(-jitter, jitter)``
    in each coordinate and projected back onto ``|x| = 1``."""
    rng = np.random.default_rng(seed)
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    phi = i * math.pi * (3.0 - math.sqrt(5.0))
    rad = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    pts = np.stack([rad * np.cos(phi), rad * np.sin(phi), z], axis=1)
    pts += rng.uniform(-jitter, jitter, size=pts.shape)
    pts /= np.linalg.norm(pts, axis=1, keepdims=True)
    return pts


def log_uniform_sizes(count: int, lo: int, hi: int) -> list[int]:
    """System sizes of the uneven batch: ``N_s = round(exp(U(ln lo, ln hi)))`` with the
    uniform draw of system ``s`` seeded by ``s``."""
    out = []
    for s in range(count):
        rng = np.random.default_rng(s)
        out.append(int(round(math.exp(rng.uniform(math.log(lo), math.log(hi))))))
    return out


def low_rank_factor(n: int, rank: int, seed: int = 0) -> np.ndarray:
    """The factor ``W`` (n x rank, N(0, 1/rank) entries) of a random positive
    semi-definite update ``W W^T`` whose diagonal is 1 on average; seeded by
    ``seed`` on a stream separate from the point sets'."""
    rng = np.random.default_rng([seed, 7919])
    return rng.standard_normal((n, rank)) / np.sqrt(rank)


def standard_normal(shape, seed: int = 0) -> np.ndarray:
    """Seeded N(0,1) draws (right-hand sides and test solutions)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape)
