"""Exact spectra of the pencils built on tensor grids (TEST INFRASTRUCTURE ONLY).

For first-order elements on the Kuhn split of a box of n_a x h_a cells per
axis, with the mass lumped (Remark rmk:mass_lumping) and homogeneous
Dirichlet conditions on every face, the element sums reduce M^{-1} S to the
finite-difference Laplacian: every simplex edge that is not parallel to an
axis carries a zero coupling, and each axis edge carries vol/h_a^2 from every
simplex that contains it. Its eigenvalues (the omega^2 of eq.
def:basisMatrixEVP) are therefore

    omega^2(k) = sum_a (4 / h_a^2) sin^2(k_a pi / (2 n_a)),  k_a = 1 .. n_a - 1,

with eigenvectors prod_a sin(k_a pi x_a / (n_a h_a)) sampled at the nodes.
This is the "plain definition" of the result the eigensolver reaches on
those grids; the tests pin it against dense LAPACK on small grids.
"""
from __future__ import annotations

import itertools

import numpy as np

__all__ = ["box_spectrum", "eigenvalues_in", "distinct", "box_eigenvector"]


def box_spectrum(cells, h) -> np.ndarray:
    """All omega^2 of the Dirichlet box, ascending (with multiplicity)."""
    per_axis = []
    for n, ha in zip(cells, h):
        k = np.arange(1, n, dtype=np.float64)
        per_axis.append(4.0 / (ha * ha) * np.sin(k * np.pi / (2.0 * n)) ** 2)
    lam = per_axis[0]
    for pa in per_axis[1:]:
        lam = (lam[:, None] + pa[None, :]).ravel()
    return np.sort(lam)


def eigenvalues_in(cells, h, omega_min: float, omega_max: float) -> np.ndarray:
    """omega^2 with omega in the closed interval [omega_min, omega_max]."""
    lam = box_spectrum(cells, h)
    w = np.sqrt(lam)
    return lam[(w >= omega_min) & (w <= omega_max)]


def distinct(lam: np.ndarray, rel: float = 1e-8):
    """Cluster sorted eigenvalues that agree to ``rel``; returns (values, multiplicities)."""
    lam = np.sort(np.asarray(lam, dtype=np.float64))
    if lam.size == 0:
        return lam, np.zeros(0, dtype=np.int64)
    vals, mult = [lam[0]], [1]
    for x in lam[1:]:
        if abs(x - vals[-1]) <= rel * abs(x):
            mult[-1] += 1
        else:
            vals.append(x)
            mult.append(1)
    return np.array(vals), np.array(mult, dtype=np.int64)


def box_eigenvector(cells, k) -> np.ndarray:
    """Closed-form eigenvector for mode k (x-fastest dof order, interior nodes)."""
    parts = []
    for n, ka in zip(cells, k):
        i = np.arange(1, n, dtype=np.float64)
        parts.append(np.sin(ka * np.pi * i / n))
    v = parts[0]
    for p in parts[1:]:
        v = (p[:, None] * v[None, :]).ravel()
    return v
