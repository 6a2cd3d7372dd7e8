"""Observables computed from Green's functions (paper Sec. 1 and Sec. 4.2.1).

* electron density per site: n_j = 2 * sum_e w_e Im G^<_jj(E_e) / (2 pi)
  (spin 2, trapezoid weights w_e on the energy grid; -i G^<_jj = Im G^<_jj
  because the diagonal of the skew-Hermitian G^< is purely imaginary);
* terminal current spectrum (Meir-Wingreen):
  i_c(E) = Tr[Sigma^<_c G^>_cc - Sigma^>_c G^<_cc] on the contact block;
* transmission (Landauer): T(E) = Tr[Gamma_L G^r_LR Gamma_R G^a_RL];
* the error metric: max_j |x_j - y_j| / max_j |y_j|.
TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).
"""
from __future__ import annotations

import numpy as np

from .selfenergy import broadening


def trapezoid_weights(energies: np.ndarray) -> np.ndarray:
    E = np.asarray(energies, dtype=np.float64)
    w = np.zeros_like(E)
    if E.size > 1:
        d = np.diff(E)
        w[:-1] += 0.5 * d
        w[1:] += 0.5 * d
    return w


def density(Gl_diag: np.ndarray, energies: np.ndarray) -> np.ndarray:
    """Gl_diag is [n_e, n]; returns n_j (per site, energy-integrated)."""
    w = trapezoid_weights(energies)
    return 2.0 * (w[:, None] * Gl_diag.imag).sum(axis=0) / (2.0 * np.pi)


def current_spectrum(sigma_lesser_c, sigma_greater_c, Gl_cc, Gg_cc) -> complex:
    return np.trace(sigma_lesser_c @ Gg_cc - sigma_greater_c @ Gl_cc)


def transmission(sigma_L, sigma_R, G_LR) -> float:
    gL = broadening(sigma_L)
    gR = broadening(sigma_R)
    return float(np.real(np.trace(gL @ G_LR @ gR @ G_LR.conj().T)))


def rel_err(x, y) -> float:
    x = np.asarray(x)
    y = np.asarray(y)
    den = np.abs(y).max()
    return float(np.abs(x - y).max() / den) if den > 0 else float(np.abs(x - y).max())
