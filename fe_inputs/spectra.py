"""Known spectra of the synthetic tensor-grid workloads (workload metadata).

The Dirichlet boxes and squares of this package use lumped first-order elements
on the Kuhn split, for which M^{-1} S is the finite-difference Laplacian; its
eigenvalues omega^2 are the sums over the axes of (2 / h_a)^2 sin^2(k_a pi / (2 n_a)),
k_a = 1 .. n_a - 1. bench.py uses them to count the eigenvalues an interval holds
and to report how far accepted pairs lie from them. The test oracle has its own
copy of this closed form; a CPU test checks that the two agree.
"""
from __future__ import annotations

import numpy as np

__all__ = ["grid_omega2", "omega2_in", "cluster"]


def grid_omega2(cells, h) -> np.ndarray:
    """Every omega^2 of the grid with n_a = cells[a] cells of width h[a], ascending."""
    total = np.zeros(1)
    for n, ha in zip(cells, h):
        axis = (2.0 / ha) ** 2 * np.sin(np.arange(1, n) * np.pi / (2.0 * n)) ** 2
        total = np.add.outer(total, axis).ravel()
    return np.sort(total)


def omega2_in(cells, h, omega_min: float, omega_max: float) -> np.ndarray:
    """The omega^2 of the grid whose omega lies in [omega_min, omega_max]."""
    w2 = grid_omega2(cells, h)
    return w2[(w2 >= omega_min * omega_min) & (w2 <= omega_max * omega_max)]


def cluster(w2, rel: float = 1e-8):
    """Distinct values of w2 (agreeing to rel counts as one) and how often each occurs."""
    w2 = np.sort(np.asarray(w2, dtype=np.float64))
    if w2.size == 0:
        return w2, np.zeros(0, dtype=np.int64)
    new = np.concatenate([[True], np.diff(w2) > rel * np.abs(w2[1:])])
    starts = np.flatnonzero(new)
    return w2[starts], np.diff(np.append(starts, w2.size)).astype(np.int64)
