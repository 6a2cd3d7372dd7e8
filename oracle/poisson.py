"""Finite-difference Poisson operator of the self-consistent loop (the paper
motivates the diagonal of G^< by the electron density that enters Poisson's
equation, Sec. 1).  TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Reading (the paper gives no electrostatics): on the L (transport) x W grid of
a device, site (x, y) = x*W + y, the potential energy U of the electrons obeys
    (K U)_j = sum_{k neighbour of j} (U_j - U_k) = lam (n_j - nD_j),
the five-point Laplacian with U = 0 on the ghost columns x = -1 and x = L
(the leads' potential, Dirichlet) and no ghost rows in y (no field across
the hard-wall edges, Neumann).  K is symmetric positive definite.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def operator(L: int, W: int) -> sp.csr_matrix:
    """K as a sparse matrix of order L*W, assembled neighbour by neighbour."""
    n = L * W
    rows, cols, vals = [], [], []
    for x in range(L):
        for y in range(W):
            j = x * W + y
            diag = 0.0
            for dx, dy in ((-1, 0), (1, 0), (0, -1), (0, 1)):
                xx, yy = x + dx, y + dy
                if yy < 0 or yy >= W:
                    continue  # Neumann: no neighbour across the edge
                diag += 1.0
                if 0 <= xx < L:
                    rows.append(j)
                    cols.append(xx * W + yy)
                    vals.append(-1.0)
                # xx outside: ghost with U = 0, only the diagonal term remains
            rows.append(j)
            cols.append(j)
            vals.append(diag)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def apply(L: int, W: int, u: np.ndarray) -> np.ndarray:
    return operator(L, W) @ u


def solve(L: int, W: int, rhs: np.ndarray) -> np.ndarray:
    """U with K U = rhs (sparse LU)."""
    return spla.spsolve(operator(L, W).tocsc(), rhs)
