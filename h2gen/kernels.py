"""Kernel functions of the test problems (Sec. 3, "Test Problems") and the
diagonal values used for their discretisations.

Each kernel maps a tensor of pairwise distances ``r > 0`` to matrix entries; the
diagonal of the discrete matrix is given separately by ``diag_value`` because
several kernels are singular at ``r = 0``.  All functions work on torch tensors
(any device, float64).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch


@dataclass(frozen=True)
class Kernel:
    name: str
    length: float = 1.0      # correlation length (covariance kernels)
    diag: float = 1.0        # value placed on the matrix diagonal
    kappa: float = 0.0       # wavenumber (oscillatory kernel)

    def __call__(self, r: torch.Tensor) -> torch.Tensor:
        if self.name == "exp":            # exponential covariance e^{-r/l}
            return torch.exp(-r / self.length)
        if self.name == "matern32":       # Matern nu=3/2 covariance
            s = math.sqrt(3.0) * r / self.length
            return (1.0 + s) * torch.exp(-s)
        if self.name == "gauss":          # Gaussian covariance e^{-r^2/(2 l^2)}
            return torch.exp(-(r * r) / (2.0 * self.length * self.length))
        if self.name == "laplace2d":      # 2D Laplace free-space Green's function
            return -torch.log(r) / (2.0 * math.pi)
        if self.name == "laplace3d":      # 3D Laplace free-space Green's function
            return 1.0 / (4.0 * math.pi * r)
        if self.name == "helmholtz3d":    # oscillatory volume IE kernel cos(kappa r)/r
            return torch.cos(self.kappa * r) / r
        raise ValueError(f"unknown kernel {self.name}")


def laplace2d_cell_average(h: float) -> float:
    """Mean of ``-log|x|/(2 pi)`` over an ``h x h`` cell centred at the origin.

    Uses the closed form ``int_0^a int_0^a log(x^2+y^2) dx dy = a^2 (2 log a - 3 +
    pi/2 + log 2)`` with ``a = h/2`` and the four-fold symmetry of the cell, which
    gives ``-(log h - log(2)/2 - 3/2 + pi/4) / (2 pi)``."""
    return -(math.log(h) - 0.5 * math.log(2.0) - 1.5 + math.pi / 4.0) / (2.0 * math.pi)


def helmholtz3d_cell_average(h: float, kappa: float, order: int = 24) -> float:
    """Mean of ``cos(kappa r)/r`` over an ``h x h x h`` cell centred at the origin.

    For a radial ``f`` the field ``x F(r)`` with ``F(r) = r^-3 int_0^r s^2 f(s) ds`` has
    divergence ``f``, so the volume integral is the flux ``sum over faces of
    (h/2) int_face F(r) dS``.  For ``f = cos(kappa s)/s``,
    ``F(r) = (cos(kappa r) + kappa r sin(kappa r) - 1) / (kappa^2 r^3)`` (``1/(2r)`` at
    ``kappa = 0``; its Taylor series where ``kappa r < 0.2``), which is smooth on the
    faces (``r >= h/2``), so an ``order^2`` Gauss-Legendre rule on one face (times six,
    by symmetry) is accurate to rounding."""
    a = 0.5 * h
    t, w = np.polynomial.legendre.leggauss(order)
    u = a * t
    U, V = np.meshgrid(u, u, indexing="ij")
    W = np.outer(a * w, a * w)
    r = np.sqrt(U * U + V * V + a * a)
    x = kappa * r
    x2 = x * x
    # Taylor series of r F(r) in x = kappa r where the closed form cancels (x < 0.2)
    series = 0.5 - x2 / 8.0 + x2 * x2 / 144.0 - x2 ** 3 / 5760.0 + x2 ** 4 / 403200.0
    with np.errstate(divide="ignore", invalid="ignore"):
        closed = (np.cos(x) + x * np.sin(x) - 1.0) / (x2 if kappa != 0.0 else 1.0)
    F = np.where(x < 0.2, series, closed) / r
    return float(6.0 * a * np.sum(W * F) / h ** 3)


def kernel_matrix(kern: Kernel, x: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
    """Dense ``K(x_i, y_j)`` for point sets that share no point (off-diagonal use)."""
    r = torch.cdist(x, y)
    return kern(r)


def _pairwise_dist(x: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
    """Distances computed coordinate by coordinate (exactly zero for equal points,
    unlike the matmul-based ``cdist``)."""
    d2 = torch.zeros(x.shape[:-1] + (y.shape[-2],), dtype=x.dtype, device=x.device)
    for c in range(x.shape[-1]):
        diff = x[..., :, c:c + 1] - y[..., c:c + 1].transpose(-1, -2)
        d2 += diff * diff
    return torch.sqrt(d2)


def near_block(kern: Kernel, x: torch.Tensor, y: torch.Tensor, same: bool) -> torch.Tensor:
    """Dense near-field block between point sets ``x`` and ``y``.  When ``same`` is
    true the two sets are the same cluster and the diagonal gets ``kern.diag``."""
    r = _pairwise_dist(x, y)
    if same:
        n = x.shape[-2]
        eye = torch.eye(n, dtype=torch.bool, device=x.device)
        r = torch.where(eye, torch.ones_like(r), r)
        v = kern(r)
        return torch.where(eye, torch.full_like(v, kern.diag), v)
    return kern(r)
