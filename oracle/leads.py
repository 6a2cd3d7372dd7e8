"""Surface Green's functions of semi-infinite leads and contact self-energies.

Paper Sec. 2: the semi-infinite leads are folded into the first and last layer
of the device, giving dense self-energy blocks Sigma_L, Sigma_R.  The paper does
not say how the surface Green's function is computed; two standard methods are
written here:

* ``surface_green_modes``: for a lead whose inter-layer hopping is a multiple
  of the identity (H01 = -hop * I), H00 = U diag(eps) U^T decouples the lead
  into independent 1D chains, one per transverse mode, each with the closed
  form surface Green's function g_n = lambda_n / hop, where lambda_n is the
  root of lambda^2 - x_n lambda + 1 = 0 (x_n = (z - eps_n)/hop) with
  |lambda_n| < 1.
* ``surface_green_decimation``: Lopez Sancho, Lopez Sancho and Rubio (J. Phys.
  F 15, 851 (1985)) renormalisation-decimation, for any H00, H01.

Both return g_s with z = E + i*eta; ``self_energy`` returns tau g_s tau^T.
TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).
"""
from __future__ import annotations

import numpy as np


def surface_green_modes(H00: np.ndarray, hop: float, z: complex) -> np.ndarray:
    """Closed-form surface Green's function of a lead with H01 = -hop * I."""
    eps, U = np.linalg.eigh(H00)
    x = (z - eps) / hop
    root = np.sqrt(x * x - 4.0 + 0j)
    lam1 = 0.5 * (x - root)
    lam2 = 0.5 * (x + root)
    lam = np.where(np.abs(lam1) < 1.0, lam1, lam2)
    g_modes = lam / hop
    return (U * g_modes) @ U.T


def surface_green_decimation(H00: np.ndarray, H01: np.ndarray, z: complex, *, tol: float = 1e-14,
                             max_iter: int = 200) -> np.ndarray:
    """Surface Green's function of the semi-infinite lead with layers 1, 2, ...
    where H_{k,k} = H00 and H_{k,k+1} = H01 (decimation of every other layer)."""
    m = H00.shape[0]
    I = np.eye(m)
    eps_s = H00.astype(complex).copy()
    eps = H00.astype(complex).copy()
    alpha = H01.astype(complex).copy()
    beta = H01.T.astype(complex).copy()
    scale = max(1.0, np.abs(H00).max(), np.abs(H01).max())
    for _ in range(max_iter):
        g = np.linalg.inv(z * I - eps)
        agb = alpha @ g @ beta
        bga = beta @ g @ alpha
        eps_s = eps_s + agb
        eps = eps + agb + bga
        alpha = alpha @ g @ alpha
        beta = beta @ g @ beta
        if max(np.abs(alpha).max(), np.abs(beta).max()) < tol * scale:
            break
    return np.linalg.inv(z * I - eps_s)


def surface_green(lead, z: complex, method: str = "auto") -> np.ndarray:
    if method == "auto":
        method = "modes" if lead.hop is not None else "decimation"
    if method == "modes":
        return surface_green_modes(lead.H00, lead.hop, z)
    return surface_green_decimation(lead.H00, lead.H01, z)


def self_energy(lead, E: float, eta: float, method: str = "auto") -> np.ndarray:
    """Retarded contact self-energy tau g_s tau^T on the device contact sites."""
    g = surface_green(lead, E + 1j * eta, method)
    return lead.tau @ g @ lead.tau.T
