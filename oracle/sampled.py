"""Selected diagonal entries by the definition, one sparse solve per site.

For symmetric A (real-symmetric H and complex-symmetric self-energies), column
j of G^r = A^{-1} is x = A^{-1} e_j and equals row j, so (paper Eq. (1))
    G^r_jj = x_j,
    G^<_jj = sum_kl G^r_jk Sigma^<_kl conj(G^r_jl) = x^T Sigma^< conj(x),
and the same with Sigma^>.  One sparse LU of A per energy (scipy SuperLU) and
one solve per sampled site; usable at sizes where dense inversion is not.
TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .problem import energy_terms


def _sparse_A_and_sigmas(dev, tr, terms):
    H = sp.csr_matrix((dev.values, dev.colind, dev.rowptr), shape=(dev.n, dev.n))
    A = (-H).astype(complex).tolil()
    A.setdiag(A.diagonal() + terms.E + 1j * tr.eta)
    Sl = sp.lil_matrix((dev.n, dev.n), dtype=complex)
    Sg = sp.lil_matrix((dev.n, dev.n), dtype=complex)
    for idx, sr, sl, sg in zip(dev.contacts, terms.sigma_r, terms.sigma_lesser, terms.sigma_greater):
        for a, ia in enumerate(idx):
            for b, ib in enumerate(idx):
                A[ia, ib] = A[ia, ib] - sr[a, b]
                Sl[ia, ib] = Sl[ia, ib] + sl[a, b]
                Sg[ia, ib] = Sg[ia, ib] + sg[a, b]
    if terms.ph_r is not None:
        A.setdiag(A.diagonal() - terms.ph_r)
        Sl.setdiag(Sl.diagonal() + terms.ph_lesser)
        Sg.setdiag(Sg.diagonal() + terms.ph_greater)
    return A.tocsc(), Sl.tocsr(), Sg.tocsr()


def green_sites(dev, tr, E: float, sites, lead_method: str = "auto") -> dict:
    """G^r_jj, G^<_jj, G^>_jj for the given caller-order sites at energy E."""
    terms = energy_terms(dev, tr, E, lead_method)
    A, Sl, Sg = _sparse_A_and_sigmas(dev, tr, terms)
    lu = spla.splu(A)
    sites = np.asarray(sites)
    out = {k: np.zeros(len(sites), dtype=complex) for k in ("Gr", "Gl", "Gg")}
    for s, j in enumerate(sites):
        e = np.zeros(dev.n, dtype=complex)
        e[j] = 1.0
        x = lu.solve(e)
        out["Gr"][s] = x[j]
        out["Gl"][s] = x @ (Sl @ x.conj())
        out["Gg"][s] = x @ (Sg @ x.conj())
    return out
