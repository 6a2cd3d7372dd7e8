"""The definition, written out densely (paper Eq. (1)-(2)).

G^r = A^{-1};  G^< = G^r Sigma^< (G^r)^dagger;  G^> = G^r Sigma^> (G^r)^dagger.
Only the diagonals are outputs of the method (Sec. 1), but the full matrices are
returned for the invariant checks.  Feasible for n up to a few thousand.
TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).
"""
from __future__ import annotations

import numpy as np

from .problem import dense_A, dense_sigma, energy_terms


def green_full(dev, tr, E: float, lead_method: str = "auto") -> dict:
    terms = energy_terms(dev, tr, E, lead_method)
    A = dense_A(dev, tr, terms)
    G = np.linalg.inv(A)
    Ga = G.conj().T
    Gl = G @ dense_sigma(dev, terms, "lesser") @ Ga
    Gg = G @ dense_sigma(dev, terms, "greater") @ Ga
    return {"A": A, "Gr": G, "Gl": Gl, "Gg": Gg, "terms": terms}


def green_diag(dev, tr, energies=None, lead_method: str = "auto") -> dict:
    """Diagonals [n_e, n] of G^r, G^<, G^> in caller order."""
    energies = tr.energies if energies is None else np.asarray(energies)
    out = {k: np.zeros((len(energies), dev.n), dtype=complex) for k in ("Gr", "Gl", "Gg")}
    for e, E in enumerate(energies):
        full = green_full(dev, tr, float(E), lead_method)
        for k in out:
            out[k][e] = np.diag(full[k])
    return out
