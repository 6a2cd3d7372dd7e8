"""Density and its response to the on-site potential, from the dense
definition (paper Eq. (1)-(2)).  TEST INFRASTRUCTURE ONLY (see
``oracle/__init__``).

H(U) = H0 + diag(U), so dA/dU_k = -e_k e_k^T and
    dG^r/dU_k = G^r e_k e_k^T G^r,
    dG^</dU_k = G^r e_k e_k^T G^< + G^< e_k e_k^T G^a   (G^< = G^r Sigma^< G^a),
hence with n_j = (1/pi) sum_e w_e Im G^<_jj (spin 2, trapezoid weights):
    chi_jk = dn_j/dU_k = (1/pi) sum_e w_e Im[G_jk G^<_kj + G^<_jk conj(G_jk)].
The product chi v (forward) and c^T chi (adjoint) follow from it.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import dense, observables


def with_onsite(dev, U):
    """The device with H0 + diag(U) (U per site, eV); the diagonal must be in the pattern."""
    vals = dev.values.copy()
    for j in range(dev.n):
        row = slice(dev.rowptr[j], dev.rowptr[j + 1])
        hit = np.nonzero(dev.colind[row] == j)[0]
        vals[dev.rowptr[j] + hit[0]] += U[j]
    return dataclasses.replace(dev, values=vals)


def density(dev, tr, U=None) -> np.ndarray:
    d = dev if U is None else with_onsite(dev, U)
    return observables.density(dense.green_diag(d, tr)["Gl"], tr.energies)


def jacobian(dev, tr, U=None) -> np.ndarray:
    """chi_jk = dn_j / dU_k, dense [n, n]."""
    d = dev if U is None else with_onsite(dev, U)
    w = observables.trapezoid_weights(tr.energies)
    chi = np.zeros((dev.n, dev.n))
    for e, E in enumerate(tr.energies):
        f = dense.green_full(d, tr, float(E))
        G, Gl = f["Gr"], f["Gl"]
        chi += w[e] * np.imag(G * Gl.T + Gl * G.conj())
    return chi / np.pi


def _contact_blocks(dev, tr, d, E):
    f = dense.green_full(d, tr, float(E))
    cont = np.concatenate(dev.contacts)
    M = len(cont)
    S = np.zeros((M, M), complex)
    o = 0
    for ci, idx in enumerate(dev.contacts):
        m = len(idx)
        S[o:o + m, o:o + m] = f["terms"].sigma_lesser[ci]
        o += m
    return f["Gr"], f["Gr"][:, cont], S


def adjoint_terms(dev, tr, c, U=None) -> np.ndarray:
    """Per energy, t_k = sum_{a,b in contacts} Sigma^<_ab conj(U_kb) conj(Z_ka) with
    U = G^r[:, contacts] and Z = G^r diag(c) conj(U), [n_e, n]: the terms whose
    (2/pi) sum_e w_e Im t_k(E_e) is d(sum_j c_j n_j)/dU_k = (c^T chi)_k (contact
    Sigma^< only: G^< = U Sigma^<_CC U^dagger)."""
    d = dev if U is None else with_onsite(dev, U)
    out = []
    for E in tr.energies:
        G, Uc, S = _contact_blocks(dev, tr, d, E)
        Z = G @ (c[:, None] * Uc.conj())
        out.append(np.einsum("ab,kb,ka->k", S, Uc.conj(), Z.conj()))
    return np.array(out)


def forward_terms(dev, tr, v, U=None) -> np.ndarray:
    """Per energy, T_j = sum_{a,b in contacts} W_ja Sigma^<_ab conj(U_jb) with
    W = G^r diag(v) U and U = G^r[:, contacts], [n_e, n]: the terms whose
    (2/pi) sum_e w_e Im T_j(E_e) is (chi v)_j, the change of the density along
    v (dG^<_jj = T_j - conj(T_j) for a skew-Hermitian Sigma^<)."""
    d = dev if U is None else with_onsite(dev, U)
    out = []
    for E in tr.energies:
        G, Uc, S = _contact_blocks(dev, tr, d, E)
        Wm = G @ (v[:, None] * Uc)
        out.append(np.einsum("ja,ab,jb->j", Wm, S, Uc.conj()))
    return np.array(out)
