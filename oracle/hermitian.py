"""The definition (paper Eq. (1)-(2)) for a general Hermitian H, which need
not be complex symmetric: a magnetic field (Peierls phases) or any complex
hopping.  TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper's elimination relies on A = A^T (Sec. 3.1, LDL^T); with complex
hoppings A is not symmetric, G^r is not symmetric, and every transposition of
the symmetric oracle becomes a conjugate transposition:
* the lead's hopping back towards the device is H10 = H01^dagger, so the
  renormalisation-decimation of Lopez Sancho, Lopez Sancho and Rubio (J. Phys.
  F 15, 851 (1985)) runs with alpha = H01, beta = H01^dagger;
* the contact self-energy is Sigma^r_c = tau g_s tau^dagger, tau the coupling
  from the device's contact sites to the lead layer next to them;
* Sigma^< = i f Gamma and Sigma^> = -i (1 - f) Gamma with Gamma = i (Sigma -
  Sigma^dagger) as before, G^r = A^{-1}, G^< = G^r Sigma^< G^r^dagger,
  G^> = G^r Sigma^> G^r^dagger.
For a real H these reduce to the symmetric oracle (``dense``), which a pin
checks.
"""
from __future__ import annotations

import numpy as np

from . import selfenergy


def surface_green(H00: np.ndarray, H01: np.ndarray, z: complex, *, tol: float = 1e-14,
                  max_iter: int = 200) -> np.ndarray:
    """Surface Green's function of the semi-infinite lead with layers 1, 2, ...,
    H_{k,k} = H00, H_{k,k+1} = H01 and H_{k+1,k} = H01^dagger (decimation of
    every other layer)."""
    m = H00.shape[0]
    I = np.eye(m)
    eps_s = H00.astype(complex).copy()
    eps = H00.astype(complex).copy()
    alpha = H01.astype(complex).copy()
    beta = H01.conj().T.astype(complex).copy()
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


def self_energy(lead, E: float, eta: float) -> np.ndarray:
    """Retarded contact self-energy tau g_s tau^dagger on the device contact sites."""
    g = surface_green(lead.H00, lead.H01, E + 1j * eta)
    return lead.tau @ g @ lead.tau.conj().T


def green_full(dev, tr, E: float) -> dict:
    """A, G^r, G^<, G^>, Sigma^<, Sigma^> (dense) and the per-contact Sigma^r
    at one energy."""
    H = dev.dense().astype(complex)
    A = -H
    A[np.diag_indices(dev.n)] += E + 1j * tr.eta
    sig = [self_energy(lead, E, tr.eta) for lead in dev.leads]
    Sl = np.zeros((dev.n, dev.n), dtype=complex)
    Sg = np.zeros_like(Sl)
    for idx, s, mu in zip(dev.contacts, sig, tr.mu):
        f = selfenergy.fermi(E, mu, tr.kT)
        A[np.ix_(idx, idx)] -= s
        Sl[np.ix_(idx, idx)] += selfenergy.lesser(s, f)
        Sg[np.ix_(idx, idx)] += selfenergy.greater(s, f)
    G = np.linalg.inv(A)
    Ga = G.conj().T
    return {"A": A, "Gr": G, "Gl": G @ Sl @ Ga, "Gg": G @ Sg @ Ga, "sigma_r": sig, "Sl": Sl, "Sg": Sg}


def green_diag(dev, tr, energies=None) -> dict:
    """Diagonals [n_e, n] of G^r, G^<, G^> in caller order."""
    energies = tr.energies if energies is None else np.asarray(energies)
    out = {k: np.zeros((len(energies), dev.n), dtype=complex) for k in ("Gr", "Gl", "Gg")}
    for e, E in enumerate(energies):
        full = green_full(dev, tr, float(E))
        for k in out:
            out[k][e] = np.diag(full[k])
    return out


def transmission(dev, tr, E: float) -> float:
    """Two-terminal transmission Tr[Gamma_L G_LR Gamma_R G_LR^dagger]."""
    full = green_full(dev, tr, E)
    (iL, iR), (sL, sR) = dev.contacts, full["sigma_r"]
    G_LR = full["Gr"][np.ix_(iL, iR)]
    return float(np.real(np.trace(selfenergy.broadening(sL) @ G_LR @ selfenergy.broadening(sR) @ G_LR.conj().T)))
