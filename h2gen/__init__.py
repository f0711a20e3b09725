"""Seeded synthetic inputs: point sets, kernels, cluster trees and H^2 matrices.

This package generates the inputs that both the CPU oracle and the CUDA library
consume; it contains none of the factorisation's arithmetic.
"""
from .h2matrix import H2Matrix
from .problems import WORKLOADS, Problem, Workload, make_batch, make_problem, rhs, uneven_sizes

__all__ = ["H2Matrix", "WORKLOADS", "Problem", "Workload", "make_batch", "make_problem", "rhs", "uneven_sizes"]
