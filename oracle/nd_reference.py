"""The paper's multilevel algorithm (Sec. 3.2), block by block, on a cluster tree.

A test aid: it follows the steps in the paper's order and notation on dense
cluster blocks, so that the block algebra (and the readings of the paper listed
below) can be checked against the definition (``oracle.dense``) on small
devices.  It is not the parity oracle of the CUDA path.

Notation (Sec. 3.2): clusters i with index sets I_i; P_i = ancestors of i;
level 1 = leaves, level L = the root separator (a cluster's level is one more
than the highest level of its children).

G^r (three steps):
  fold      for l = 1..L-1, clusters i on level l:
              Psi_ij = -(A_ii)^{-1} A_ij                 (j in P_i)
              A_jk  += Psi_ij^T A_ik,  A_kj = (A_jk)^T   (j, k in P_i)
              A_ij = A_ji = 0
  root      G^(L-1) = (A^(L-1))^{-1}   (block diagonal; only the root block is new)
  extract   for l = L-2..0, clusters i on level l+1:
              G_ij += sum_{k in P_i} Psi_ik G_kj,  G_ji = (G_ij)^T   (j in P_i)
              G_ii += sum_{j in P_i} Psi_ij G_ji
G^< (four steps):
  N = Sigma^< (G^(0))^dagger                  (Sigma^< block diagonal over clusters)
  fold      N_jk += Psi_ij^T N_ik              (j, k in P_i), levels 1..L-1
  P^(L-1) = G^(L-1) N^(L-1)
  extract   P_ij += sum_k Psi_ik P_kj,  P_ji = -(P_ij)^dagger,  P_ii += sum_j Psi_ij P_ji

Readings: (1) the extraction loops name "level l" for l = L-2..0; the appendix
(G^(1) updates the level-2 cluster, G^(0) the level-1 clusters) shows that
G^(l) is produced by the clusters on level l+1, which is what is done here.
(2) The appendix writes N = Sigma^< (G^<)^dagger; the general step (and the
block entries listed next to it) use G^(0), which is what is done here.
TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).
"""
from __future__ import annotations

import numpy as np


class ClusterTree:
    def __init__(self, clusters, parent):
        self.clusters = [np.asarray(c, dtype=np.int64) for c in clusters]
        self.parent = list(parent)
        nc = len(self.clusters)
        self.children = [[] for _ in range(nc)]
        roots = [i for i in range(nc) if self.parent[i] < 0]
        if len(roots) != 1:
            raise ValueError("tree must have exactly one root")
        self.root = roots[0]
        for i, p in enumerate(self.parent):
            if p >= 0:
                self.children[p].append(i)
        self.level = [0] * nc

        def lev(i):
            if self.level[i] == 0:
                self.level[i] = 1 + max((lev(c) for c in self.children[i]), default=0)
            return self.level[i]

        for i in range(nc):
            lev(i)
        self.L = self.level[self.root]
        self.P = []
        for i in range(nc):
            anc, p = [], self.parent[i]
            while p >= 0:
                anc.append(p)
                p = self.parent[p]
            self.P.append(anc)
        self.by_level = {l: [i for i in range(nc) if self.level[i] == l] for l in range(1, self.L + 1)}

    def check_partition(self, n):
        allidx = np.concatenate(self.clusters)
        if np.sort(allidx).tolist() != list(range(n)):
            raise ValueError("clusters must partition the sites")


def _zero(ti, tj):
    return np.zeros((len(ti), len(tj)), dtype=complex)


class NDReference:
    def __init__(self, tree: ClusterTree, A: np.ndarray, record: bool = False):
        self.t = tree
        self.A = A
        self.record = record
        self.trace = {}

    def _snapshot(self, name, blocks):
        if self.record:
            nc = len(self.t.clusters)
            pat = np.zeros((nc, nc), dtype=np.int64)
            for (i, j), b in blocks.items():
                if b is not None and np.abs(b).max() > 0.0:
                    pat[i, j] = 1
            self.trace[name] = pat

    def green_retarded(self):
        t, A = self.t, self.A
        C = t.clusters
        nc = len(C)
        Ab = {(i, j): A[np.ix_(C[i], C[j])].astype(complex) for i in range(nc) for j in range(nc)}
        self._snapshot("A0", Ab)
        self.Ainv, self.Psi = {}, {}
        for l in range(1, t.L):
            for i in t.by_level[l]:
                self.Ainv[i] = np.linalg.inv(Ab[i, i])
                for j in t.P[i]:
                    self.Psi[i, j] = -self.Ainv[i] @ Ab[i, j]
                for j in t.P[i]:
                    for k in t.P[i]:
                        Ab[j, k] = Ab[j, k] + self.Psi[i, j].T @ Ab[i, k]
                for j in t.P[i]:
                    for k in t.P[i]:
                        Ab[k, j] = Ab[j, k].T
                for j in t.P[i]:
                    Ab[i, j] = _zero(C[i], C[j])
                    Ab[j, i] = _zero(C[j], C[i])
            self._snapshot(f"A{l}", Ab)
        r = t.root
        self.Ainv[r] = np.linalg.inv(Ab[r, r])
        Gb = {(i, i): self.Ainv[i].copy() for i in range(nc)}
        self._snapshot(f"G{t.L - 1}", Gb)
        for l in range(t.L - 2, -1, -1):
            for i in t.by_level[l + 1]:
                for j in t.P[i]:
                    acc = Gb.get((i, j), _zero(C[i], C[j]))
                    for k in t.P[i]:
                        acc = acc + self.Psi[i, k] @ Gb.get((k, j), _zero(C[k], C[j]))
                    Gb[i, j] = acc
                for j in t.P[i]:
                    Gb[j, i] = Gb[i, j].T
                acc = Gb[i, i]
                for j in t.P[i]:
                    acc = acc + self.Psi[i, j] @ Gb[j, i]
                Gb[i, i] = acc
            self._snapshot(f"G{l}", Gb)
        self.G0 = Gb
        return Gb

    def green_lesser(self, S: np.ndarray, tag: str = ""):
        """P^(0) for a lesser (or greater) self-energy S, block diagonal over clusters."""
        t = self.t
        C = t.clusters
        nc = len(C)
        for i in range(nc):
            for j in range(nc):
                if i != j and np.abs(S[np.ix_(C[i], C[j])]).max(initial=0.0) > 0.0:
                    raise ValueError("Sigma^< must be block diagonal over the clusters")
        Nb = {(i, j): S[np.ix_(C[i], C[i])] @ g.conj() for (i, j), g in self.G0.items()}
        self._snapshot(f"N0{tag}", Nb)
        for l in range(1, t.L):
            for i in t.by_level[l]:
                for j in t.P[i]:
                    for k in t.P[i]:
                        Nb[j, k] = Nb.get((j, k), _zero(C[j], C[k])) + self.Psi[i, j].T @ Nb.get((i, k), _zero(C[i], C[k]))
            self._snapshot(f"N{l}{tag}", Nb)
        Pb = {(i, j): self.Ainv[i] @ nb for (i, j), nb in Nb.items()}
        self._snapshot(f"P{t.L - 1}{tag}", Pb)
        for l in range(t.L - 2, -1, -1):
            for i in t.by_level[l + 1]:
                for j in t.P[i]:
                    acc = Pb.get((i, j), _zero(C[i], C[j]))
                    for k in t.P[i]:
                        acc = acc + self.Psi[i, k] @ Pb.get((k, j), _zero(C[k], C[j]))
                    Pb[i, j] = acc
                for j in t.P[i]:
                    Pb[j, i] = -Pb[i, j].conj().T
                acc = Pb.get((i, i), _zero(C[i], C[i]))
                for j in t.P[i]:
                    acc = acc + self.Psi[i, j] @ Pb[j, i]
                Pb[i, i] = acc
            self._snapshot(f"P{l}{tag}", Pb)
        return Pb

    def diag(self, blocks) -> np.ndarray:
        n = sum(len(c) for c in self.t.clusters)
        d = np.zeros(n, dtype=complex)
        for i, c in enumerate(self.t.clusters):
            d[c] = np.diag(blocks[i, i])
        return d


def grid_bisection_tree(L: int, W: int, leaf: int, contacts: bool = True) -> ClusterTree:
    """A simple nested-dissection tree of an L x W grid (site x*W + y): cut the
    longer side in the middle with a width-1 line, recurse; when a piece that
    holds a whole contact column would be cut across, peel the contact column
    off with the neighbouring column as separator instead.  Independent of the
    CUDA path's partitioner."""
    clusters, parent = [], []

    def new(sites, par):
        clusters.append(np.array(sorted(sites), dtype=np.int64))
        parent.append(par)
        return len(clusters) - 1

    def rec(x0, x1, y0, y1, par):
        nx, ny = x1 - x0, y1 - y0
        if nx <= 0 or ny <= 0:
            return
        if nx * ny <= leaf:
            new([x * W + y for x in range(x0, x1) for y in range(y0, y1)], par)
            return
        has_left = contacts and x0 == 0 and y0 == 0 and y1 == W
        has_right = contacts and x1 == L and y0 == 0 and y1 == W
        if nx >= ny:
            c = x0 + nx // 2
            s = new([c * W + y for y in range(y0, y1)], par)
            rec(x0, c, y0, y1, s)
            rec(c + 1, x1, y0, y1, s)
        elif (has_left or has_right) and nx > 2:
            if has_left:
                s = new([1 * W + y for y in range(W)], par)
                new([y for y in range(W)], s)
                rec(2, x1, y0, y1, s)
            else:
                s = new([(L - 2) * W + y for y in range(W)], par)
                new([(L - 1) * W + y for y in range(W)], s)
                rec(x0, L - 2, y0, y1, s)
        elif (has_left or has_right):
            new([x * W + y for x in range(x0, x1) for y in range(y0, y1)], par)
        else:
            c = y0 + ny // 2
            s = new([x * W + c for x in range(x0, x1)], par)
            rec(x0, x1, y0, c, s)
            rec(x0, x1, c + 1, y1, s)

    rec(0, L, 0, W, -1)
    return ClusterTree(clusters, parent)


def layer_tree(layers) -> ClusterTree:
    """The partition that turns the algorithm into RGF (Sec. 3.2, Fig. 6): each
    transport layer is a cluster whose parent is the next layer."""
    nl = len(layers)
    return ClusterTree(list(layers), [k + 1 if k + 1 < nl else -1 for k in range(nl)])
