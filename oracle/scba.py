"""Self-consistent Born approximation of an elastic local phonon (dephasing)
self-energy, written densely per energy -- TEST INFRASTRUCTURE ONLY (see
``oracle/__init__``).

The paper leaves the phonon self-energy of Eq. (2) open (Sec. 2 names
non-diagonal and realistic scattering as future work).  The model here is the
standard elastic, local one (S. Datta, Superlattices Microstruct. 28, 253
(2000), Sec. 2): with a deformation-potential strength D (eV^2),

    Sigma^r_ph,jj(E) = D G^r_jj(E),  Sigma^<_ph,jj(E) = D G^<_jj(E),
    Sigma^>_ph,jj(E) = D G^>_jj(E),

iterated from a first guess (the constant broadening of the transport
parameters) until the self-energies stop changing; every energy iterates
alone because the scattering is elastic.  At the fixed point the scattering
current sum_j [Sigma^<_ph G^> - Sigma^>_ph G^<]_jj vanishes, so the terminal
currents balance (up to the eta leak).
"""
from __future__ import annotations

import numpy as np

from .problem import dense_A, dense_sigma, energy_terms


def _solve(dev, tr, terms):
    A = dense_A(dev, tr, terms)
    G = np.linalg.inv(A)
    Ga = G.conj().T
    Gl = G @ dense_sigma(dev, terms, "lesser") @ Ga
    Gg = G @ dense_sigma(dev, terms, "greater") @ Ga
    return G, Gl, Gg


def scba(dev, tr, E: float, D: float, *, updates: int | None = None, tol: float = 1e-13, max_updates: int = 2000,
         mix: float = 1.0) -> dict:
    """Diagonals of G^r, G^<, G^> after `updates` self-energy updates (or at
    convergence: relative change max|Sigma_new - Sigma| / max|Sigma_new| <= tol),
    each update Sigma <- (1 - mix) Sigma + mix D diag(G), followed by a solve.
    Also the terminal current spectra i_c = Tr[Sigma^<_c G^>_cc - Sigma^>_c G^<_cc],
    the scattering current and the last relative change."""
    terms = energy_terms(dev, tr, float(E))
    if terms.ph_r is None:
        raise ValueError("the first iterate needs a constant broadening (gamma_ph > 0)")
    G, Gl, Gg = _solve(dev, tr, terms)
    n_upd, change = 0, np.inf
    limit = updates if updates is not None else max_updates
    while n_upd < limit:
        new = [D * np.diag(G), D * np.diag(Gl), D * np.diag(Gg)]
        old = [terms.ph_r, terms.ph_lesser, terms.ph_greater]
        scale = max(np.abs(a).max() for a in new)
        diff = max(np.abs(a - b).max() for a, b in zip(new, old))
        change = diff / scale if scale > 0 else diff
        terms.ph_r, terms.ph_lesser, terms.ph_greater = [(1.0 - mix) * b + mix * a for a, b in zip(new, old)]
        G, Gl, Gg = _solve(dev, tr, terms)
        n_upd += 1
        if updates is None and change <= tol:
            break
    cur = []
    for idx, sl, sg in zip(dev.contacts, terms.sigma_lesser, terms.sigma_greater):
        cc = np.ix_(idx, idx)
        cur.append(np.trace(sl @ Gg[cc] - sg @ Gl[cc]))
    i_ph = np.sum(terms.ph_lesser * np.diag(Gg) - terms.ph_greater * np.diag(Gl))
    return {"Gr": np.diag(G), "Gl": np.diag(Gl), "Gg": np.diag(Gg), "updates": n_upd, "change": change,
            "currents": np.array(cur), "i_ph": i_ph,
            "ph_r": terms.ph_r, "ph_lesser": terms.ph_lesser, "ph_greater": terms.ph_greater}
