"""Per-energy terms of A(E) (paper Eq. (2)) shared by the oracle methods.

A(E) = (E + i eta) I - H - Sigma^r_L - Sigma^r_R - Sigma^r_Phonon.
eta is added to the whole device diagonal and to the lead energy z = E + i eta
(reading: the paper writes E I; a vanishing positive imaginary part is needed
for A to be invertible away from the contacts).
TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import leads, selfenergy


@dataclasses.dataclass
class EnergyTerms:
    E: float
    sigma_r: list  # per contact, m_c x m_c complex
    sigma_lesser: list
    sigma_greater: list
    ph_r: np.ndarray | None  # diagonal [n] or None
    ph_lesser: np.ndarray | None
    ph_greater: np.ndarray | None
    f: list  # Fermi occupation per contact


def energy_terms(dev, tr, E: float, lead_method: str = "auto") -> EnergyTerms:
    sig_r = [leads.self_energy(lead, E, tr.eta, lead_method) for lead in dev.leads]
    f = [selfenergy.fermi(E, mu, tr.kT) for mu in tr.mu]
    sig_l = [selfenergy.lesser(s, fc) for s, fc in zip(sig_r, f)]
    sig_g = [selfenergy.greater(s, fc) for s, fc in zip(sig_r, f)]
    ph_r = ph_l = ph_g = None
    if tr.gamma_ph > 0.0:
        mu_ph = tr.mu_ph if tr.mu_ph is not None else 0.5 * (tr.mu[0] + tr.mu[1])
        ph_r, ph_l, ph_g = selfenergy.phonon(dev.n, tr.gamma_ph, selfenergy.fermi(E, mu_ph, tr.kT))
    return EnergyTerms(E, sig_r, sig_l, sig_g, ph_r, ph_l, ph_g, f)


def dense_A(dev, tr, terms: EnergyTerms) -> np.ndarray:
    """Dense A(E), Eq. (2)."""
    A = -dev.dense().astype(complex)
    A[np.diag_indices(dev.n)] += terms.E + 1j * tr.eta
    for idx, s in zip(dev.contacts, terms.sigma_r):
        A[np.ix_(idx, idx)] -= s
    if terms.ph_r is not None:
        A[np.diag_indices(dev.n)] -= terms.ph_r
    return A


def dense_sigma(dev, terms: EnergyTerms, which: str) -> np.ndarray:
    """Full Sigma^< (which='lesser') or Sigma^> ('greater'), block diagonal."""
    S = np.zeros((dev.n, dev.n), dtype=complex)
    blocks = terms.sigma_lesser if which == "lesser" else terms.sigma_greater
    for idx, s in zip(dev.contacts, blocks):
        S[np.ix_(idx, idx)] += s
    ph = terms.ph_lesser if which == "lesser" else terms.ph_greater
    if ph is not None:
        S[np.diag_indices(dev.n)] += ph
    return S
