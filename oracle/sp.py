"""Newton iteration of the self-consistent Schroedinger-Poisson problem
(the paper's motivation, Sec. 1: the density from the diagonal of G^< feeds
Poisson's equation).  TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Unknown: the electrostatic potential energy U (eV) on the device sites,
added to the diagonal of H.  With the Poisson operator K of ``poisson``
(Dirichlet at the ends, Neumann at the edges), the coupling lam (eV per
electron) and the background charge nD (electrons per site),
    F(U) = K U - lam (n(U) - nD) = 0,
    J(U) = K - lam chi(U),            chi = dn/dU (``response.jacobian``),
    U <- U - J^{-1} F(U)              (one Newton step, a dense solve here).
"""
from __future__ import annotations

import numpy as np

from . import poisson, response


def residual(dev, tr, L: int, W: int, lam: float, nD, U) -> np.ndarray:
    return poisson.apply(L, W, U) - lam * (response.density(dev, tr, U) - nD)


def newton(dev, tr, L: int, W: int, lam: float, nD, steps: int, U0=None):
    """Returns (iterates [steps + 1, n] with U0 first, |F| max norm of each iterate)."""
    U = np.zeros(dev.n) if U0 is None else np.array(U0, dtype=np.float64)
    K = poisson.operator(L, W).toarray()
    its, res = [U.copy()], []
    for _ in range(steps):
        F = K @ U - lam * (response.density(dev, tr, U) - nD)
        res.append(float(np.abs(F).max()))
        J = K - lam * response.jacobian(dev, tr, U)
        U = U - np.linalg.solve(J, F)
        its.append(U.copy())
    res.append(float(np.abs(residual(dev, tr, L, W, lam, nD, U)).max()))
    return np.array(its), np.array(res)
