"""Recursive Green's function method (paper Sec. 2; Svizhenko et al. 2002,
Lake et al. 1997), for a device whose Hamiltonian only couples adjacent layers.

With tau_k = H[layer k, layer k+1] (so A_{k,k+1} = -tau_k) and A_kk the layer
block of A(E) (contact self-energy on the first and last layer):

forward ("fold" left to right)
    g_1 = A_11^{-1},               g_k = (A_kk - tau_{k-1}^T g_{k-1} tau_{k-1})^{-1}
    g<_1 = g_1 S<_11 g_1^dagger,   g<_k = g_k (S<_kk + tau_{k-1}^T g<_{k-1} tau_{k-1}) g_k^dagger
backward ("extract" right to left)
    G_NN = g_N,  G_kk = g_k + g_k tau_k G_{k+1} tau_k^T g_k
    G<_kk = g<_k + g_k tau_k G<_{k+1} tau_k^T g_k^dagger
            + g_k tau_k G_{k+1} tau_k^T g<_k + g<_k tau_k G_{k+1}^dagger tau_k^T g_k^dagger

The lesser recursion follows from G< = G^r S< G^a split at the cut between
layers k and k+1: rows of G^r in the left part factor as
(I + g_k tau_k G_{k+1} tau_k^T) g_left and G^r_{k,j>k} = g_k tau_k G^r_{k+1,j}.
Exact up to rounding; cost ~ 10 W^3 L complex multiply-adds for G^r (Sec. 2).
TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).
"""
from __future__ import annotations

import numpy as np

from .problem import energy_terms


def _layer_blocks(dev):
    """Dense layer blocks H_kk and couplings tau_k = H_{k,k+1}; checks that H
    only couples adjacent layers."""
    layer_of = np.full(dev.n, -1, dtype=np.int64)
    pos = np.zeros(dev.n, dtype=np.int64)
    for k, idx in enumerate(dev.layers):
        layer_of[idx] = k
        pos[idx] = np.arange(len(idx))
    if (layer_of < 0).any():
        raise ValueError("layers do not cover every site")
    nl = len(dev.layers)
    Hkk = [np.zeros((len(ix), len(ix))) for ix in dev.layers]
    tau = [np.zeros((len(dev.layers[k]), len(dev.layers[k + 1]))) for k in range(nl - 1)]
    for r in range(dev.n):
        for p in range(dev.rowptr[r], dev.rowptr[r + 1]):
            c = dev.colind[p]
            v = dev.values[p]
            kr, kc = layer_of[r], layer_of[c]
            if kr == kc:
                Hkk[kr][pos[r], pos[c]] = v
            elif kc == kr + 1:
                tau[kr][pos[r], pos[c]] = v
            elif kc != kr - 1:
                raise ValueError("H couples non-adjacent layers")
    return Hkk, tau


def _contact_slots(dev):
    """Map each contact to (layer index, positions of its sites in the layer)."""
    slots = []
    for idx in dev.contacts:
        for k, lay in enumerate(dev.layers):
            if np.isin(idx, lay).all():
                where = {int(s): i for i, s in enumerate(lay)}
                slots.append((k, np.array([where[int(s)] for s in idx])))
                break
        else:
            raise ValueError("contact not inside one layer")
    return slots


class RGF:
    """Block RGF over ``dev.layers``; ``solve(E)`` returns diag G^r, G^<, G^>."""

    def __init__(self, dev, tr):
        self.dev, self.tr = dev, tr
        self.Hkk, self.tau = _layer_blocks(dev)
        self.slots = _contact_slots(dev)

    def solve(self, E: float, lead_method: str = "auto") -> dict:
        dev, tr = self.dev, self.tr
        terms = energy_terms(dev, tr, E, lead_method)
        nl = len(dev.layers)
        A, Sl, Sg = [], [], []
        for k, idx in enumerate(dev.layers):
            m = len(idx)
            Akk = (E + 1j * tr.eta) * np.eye(m) - self.Hkk[k]
            Slk = np.zeros((m, m), dtype=complex)
            Sgk = np.zeros((m, m), dtype=complex)
            if terms.ph_r is not None:
                Akk = Akk - np.diag(terms.ph_r[idx])
                Slk += np.diag(terms.ph_lesser[idx])
                Sgk += np.diag(terms.ph_greater[idx])
            for c, (kc, p) in enumerate(self.slots):
                if kc == k:
                    Akk[np.ix_(p, p)] -= terms.sigma_r[c]
                    Slk[np.ix_(p, p)] += terms.sigma_lesser[c]
                    Sgk[np.ix_(p, p)] += terms.sigma_greater[c]
            A.append(Akk)
            Sl.append(Slk)
            Sg.append(Sgk)
        tau = self.tau
        g = [None] * nl
        gl = [None] * nl
        gg = [None] * nl
        for k in range(nl):
            if k == 0:
                g[k] = np.linalg.inv(A[k])
                Sk_l, Sk_g = Sl[k], Sg[k]
            else:
                g[k] = np.linalg.inv(A[k] - tau[k - 1].T @ g[k - 1] @ tau[k - 1])
                Sk_l = Sl[k] + tau[k - 1].T @ gl[k - 1] @ tau[k - 1]
                Sk_g = Sg[k] + tau[k - 1].T @ gg[k - 1] @ tau[k - 1]
            ga = g[k].conj().T
            gl[k] = g[k] @ Sk_l @ ga
            gg[k] = g[k] @ Sk_g @ ga
        out = {key: np.zeros(dev.n, dtype=complex) for key in ("Gr", "Gl", "Gg")}
        G = g[nl - 1]
        GL = gl[nl - 1]
        GG = gg[nl - 1]
        self._store(out, nl - 1, G, GL, GG)
        for k in range(nl - 2, -1, -1):
            t, tT = tau[k], tau[k].T
            gk, gka = g[k], g[k].conj().T
            X = gk @ t  # g_k tau_k
            Gn = gk + X @ G @ tT @ gk
            GLn = (gl[k] + X @ GL @ tT @ gka + X @ G @ tT @ gl[k] + gl[k] @ t @ G.conj().T @ tT @ gka)
            GGn = (gg[k] + X @ GG @ tT @ gka + X @ G @ tT @ gg[k] + gg[k] @ t @ G.conj().T @ tT @ gka)
            G, GL, GG = Gn, GLn, GGn
            self._store(out, k, G, GL, GG)
        return out

    def _store(self, out, k, G, GL, GG):
        idx = self.dev.layers[k]
        out["Gr"][idx] = np.diag(G)
        out["Gl"][idx] = np.diag(GL)
        out["Gg"][idx] = np.diag(GG)


def green_diag(dev, tr, energies=None, lead_method: str = "auto") -> dict:
    energies = tr.energies if energies is None else np.asarray(energies)
    solver = RGF(dev, tr)
    out = {k: np.zeros((len(energies), dev.n), dtype=complex) for k in ("Gr", "Gl", "Gg")}
    for e, E in enumerate(energies):
        r = solver.solve(float(E), lead_method)
        for k in out:
            out[k][e] = r[k]
    return out
