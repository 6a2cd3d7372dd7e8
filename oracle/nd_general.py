"""The multilevel algorithm of Sec. 3.2 for a general (not complex-symmetric)
A, block by block on a cluster tree: a block LU where the paper uses
LDL^T.  A test aid, like ``nd_reference``: it states the algorithm that a
general-Hermitian path of the kernels would run and checks it against the
definition (``hermitian``).  TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

With A_ij no longer equal to A_ji^T, every cluster i keeps two factors,
  right  PsiR_ij = -(A_ii)^{-1} A_ij,   left  PsiL_ji = -A_ji (A_ii)^{-1}
(j in P_i; for a symmetric A, PsiL_ji = PsiR_ij^T), and the steps become:
G^r:
  fold      A_jk += A_ji PsiR_ik   (j, k in P_i)   -- no symmetric copy
  root      G^(L-1) = (A^(L-1))^{-1}
  extract   G_ij  = sum_k PsiR_ik G_kj,  G_ji = sum_k G_jk PsiL_ki   (j in P_i)
            G_ii  = (A_ii)^{-1} + sum_j PsiR_ij G_ji
G^< = G^r Sigma^< G^a = A^{-1} N with N = Sigma^< G^a solved by the same
factorisation: the left factors eliminate the right-hand side, the right
factors substitute back, and the skew-Hermiticity of G^< gives the blocks
below the diagonal:
  N_ij = Sigma^<_ii (G^a)_ij = Sigma^<_ii (G_ji)^dagger   (on the pattern)
  fold      N_jk += PsiL_ji N_ik   (j, k in P_i)
  P^(L-1)   P_ij = (A_ii)^{-1} N_ij
  extract   P_ij += sum_k PsiR_ik P_kj,  P_ji = -(P_ij)^dagger,
            P_ii += sum_j PsiR_ij P_ji
For a symmetric A all of this reduces to ``nd_reference``.
"""
from __future__ import annotations

import numpy as np

from .nd_reference import ClusterTree


def _zero(ti, tj):
    return np.zeros((len(ti), len(tj)), dtype=complex)


class NDGeneral:
    def __init__(self, tree: ClusterTree, A: np.ndarray):
        self.t = tree
        self.A = A

    def green_retarded(self):
        t, A = self.t, self.A
        C = t.clusters
        nc = len(C)
        Ab = {(i, j): A[np.ix_(C[i], C[j])].astype(complex) for i in range(nc) for j in range(nc)}
        self.Ainv, self.PsiR, self.PsiL = {}, {}, {}
        for l in range(1, t.L):
            for i in t.by_level[l]:
                X = self.Ainv[i] = np.linalg.inv(Ab[i, i])
                for j in t.P[i]:
                    self.PsiR[i, j] = -X @ Ab[i, j]
                    self.PsiL[j, i] = -Ab[j, i] @ X
                for j in t.P[i]:
                    for k in t.P[i]:
                        Ab[j, k] = Ab[j, k] + Ab[j, i] @ self.PsiR[i, k]
                for j in t.P[i]:
                    Ab[i, j] = _zero(C[i], C[j])
                    Ab[j, i] = _zero(C[j], C[i])
        r = t.root
        self.Ainv[r] = np.linalg.inv(Ab[r, r])
        Gb = {(i, i): self.Ainv[i].copy() for i in range(nc)}
        for l in range(t.L - 2, -1, -1):
            for i in t.by_level[l + 1]:
                up, low = {}, {}
                for j in t.P[i]:
                    acc_u, acc_l = _zero(C[i], C[j]), _zero(C[j], C[i])
                    for k in t.P[i]:
                        acc_u = acc_u + self.PsiR[i, k] @ Gb.get((k, j), _zero(C[k], C[j]))
                        acc_l = acc_l + Gb.get((j, k), _zero(C[j], C[k])) @ self.PsiL[k, i]
                    up[j], low[j] = acc_u, acc_l
                for j in t.P[i]:
                    Gb[i, j], Gb[j, i] = up[j], low[j]
                acc = Gb[i, i]
                for j in t.P[i]:
                    acc = acc + self.PsiR[i, j] @ Gb[j, i]
                Gb[i, i] = acc
        self.G0 = Gb
        return Gb

    def green_lesser(self, S: np.ndarray):
        """P^(0) for a lesser (or greater) self-energy S, block diagonal over clusters."""
        t = self.t
        C = t.clusters
        nc = len(C)
        for i in range(nc):
            for j in range(nc):
                if i != j and np.abs(S[np.ix_(C[i], C[j])]).max(initial=0.0) > 0.0:
                    raise ValueError("Sigma^< must be block diagonal over the clusters")
        # N_ij = S_ii (G^a)_ij with (G^a)_ij = (G_ji)^dagger, on the pattern of G^(0)
        Nb = {(i, j): S[np.ix_(C[i], C[i])] @ self.G0[j, i].conj().T for (i, j) in self.G0}
        for l in range(1, t.L):
            for i in t.by_level[l]:
                for j in t.P[i]:
                    for k in t.P[i]:
                        Nb[j, k] = Nb.get((j, k), _zero(C[j], C[k])) + self.PsiL[j, i] @ Nb.get((i, k), _zero(C[i], C[k]))
        Pb = {(i, j): self.Ainv[i] @ nb for (i, j), nb in Nb.items()}
        for l in range(t.L - 2, -1, -1):
            for i in t.by_level[l + 1]:
                for j in t.P[i]:
                    acc = Pb.get((i, j), _zero(C[i], C[j]))
                    for k in t.P[i]:
                        acc = acc + self.PsiR[i, k] @ Pb.get((k, j), _zero(C[k], C[j]))
                    Pb[i, j] = acc
                for j in t.P[i]:
                    Pb[j, i] = -Pb[i, j].conj().T
                acc = Pb.get((i, i), _zero(C[i], C[i]))
                for j in t.P[i]:
                    acc = acc + self.PsiR[i, j] @ Pb[j, i]
                Pb[i, i] = acc
        return Pb

    def diag(self, blocks) -> np.ndarray:
        n = sum(len(c) for c in self.t.clusters)
        d = np.zeros(n, dtype=complex)
        for i, c in enumerate(self.t.clusters):
            d[c] = np.diag(blocks[i, i])
        return d
