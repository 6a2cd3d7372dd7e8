"""Lesser/greater self-energies (paper Eq. (1) and Sec. 3.1).

Gamma = i (Sigma - Sigma^dagger); Sigma^< = i f Gamma; Sigma^> = -i (1 - f) Gamma,
with f the Fermi function of the reservoir.  For a real-symmetric lead
Hamiltonian Gamma is real symmetric, so Sigma^< is purely imaginary and
skew-Hermitian, which is what the paper assumes (Sec. 3.1).

Phonon model (the paper only says Sigma_Phonon is diagonal at each grid point,
Sec. 2): a constant broadening Gamma_ph on every device site,
Sigma^r_ph = -i Gamma_ph / 2, Sigma^<_ph = i f(mu_ph) Gamma_ph,
Sigma^>_ph = -i (1 - f(mu_ph)) Gamma_ph.
TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).
"""
from __future__ import annotations

import numpy as np


def fermi(E: float, mu: float, kT: float) -> float:
    x = (E - mu) / kT
    if x > 0:
        ex = np.exp(-x)
        return ex / (1.0 + ex)
    return 1.0 / (1.0 + np.exp(x))


def broadening(sigma_r: np.ndarray) -> np.ndarray:
    return 1j * (sigma_r - sigma_r.conj().T)


def lesser(sigma_r: np.ndarray, f: float) -> np.ndarray:
    return 1j * f * broadening(sigma_r)


def greater(sigma_r: np.ndarray, f: float) -> np.ndarray:
    return -1j * (1.0 - f) * broadening(sigma_r)


def phonon(n: int, gamma_ph: float, f_ph: float) -> tuple:
    """Diagonals of (Sigma^r_ph, Sigma^<_ph, Sigma^>_ph) for the constant model."""
    r = np.full(n, -0.5j * gamma_ph)
    lt = np.full(n, 1j * f_ph * gamma_ph)
    gt = np.full(n, -1j * (1.0 - f_ph) * gamma_ph)
    return r, lt, gt
