"""Transmission of a 1D tight-binding chain by 2x2 transfer matrices.

An independent textbook method (no Green's function) used to pin the oracle's
Landauer transmission.  Chain: on-site eps_j on device sites 1..N, eps0 in the
leads, hopping -t everywhere.  The Schroedinger equation at site j reads
psi_{j-1} = ((eps_j - E)/t) psi_j - psi_{j+1}.  Start on the right with a pure
transmitted wave psi_j = exp(i k j) (amplitude 1), propagate to the left lead
and split psi there into incoming and reflected waves A e^{ikj} + B e^{-ikj};
T = 1/|A|^2 (same velocity on both sides), where E = eps0 - 2 t cos k.
TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).
"""
from __future__ import annotations

import numpy as np


def chain_transmission(E: float, eps_device: np.ndarray, *, t: float = 1.0, eps0: float = 0.0) -> float:
    c = (eps0 - E) / (2.0 * t)
    if abs(c) >= 1.0:
        return 0.0
    k = np.arccos(c)
    N = len(eps_device)
    eps = lambda j: eps_device[j - 1] if 1 <= j <= N else eps0
    psi_next = np.exp(1j * k * (N + 2))  # psi_{j+1}
    psi = np.exp(1j * k * (N + 1))  # psi_j, j = N+1
    for j in range(N + 1, -1, -1):  # equation at site j gives psi_{j-1}
        psi_prev = ((eps(j) - E) / t) * psi - psi_next
        psi_next, psi = psi, psi_prev
    # now psi = psi_{-1}, psi_next = psi_0
    M = np.array([[1.0, 1.0], [np.exp(-1j * k), np.exp(1j * k)]])
    A, _ = np.linalg.solve(M, np.array([psi_next, psi]))
    return float(1.0 / abs(A) ** 2)
